// Sharding one trace over ranks by its outer value.
//
// Algorithm 1 (Sec. 4.2) evaluates every binding on its own projection u^D
// (Sec. 2.4.3), and the bindings of one outer value d_0 form one subtree of the
// submonitor tree (Sec. 3.3): nothing of a subtree is shared with another
// before ApplyQuantifiers, whose per-level verdict counts (the vectors v of
// Sec. 3.4) are sums over the nodes of a level.  So a trace splits into
// independent parts by its outermost quantified value: each part is verified
// on its own, the parts' counts add up, and the root is valuated once on the
// sum (rv_combine_results).
//
// rv_shard_trace is the device half of that split: a stable multisplit of the
// events into `world` contiguous segments by a hash of the outer value (the
// key itself with one variable, its high 32 bits with two), keeping trace
// order inside every segment, ready for an all-to-all exchange.  The hash is
// independent of the mixing that picks key buckets inside the verifier, so a
// shard still spreads over all of its buckets.
#include <algorithm>
#include <cstring>

#include "profile.h"
#include "rv_device.cuh"

namespace {

constexpr int SH_WARPS = 8;
constexpr int SH_THREADS = SH_WARPS * 32;
constexpr int SH_MAX_WORLD = 256;
constexpr unsigned SH_FULL = 0xFFFFFFFFu;
constexpr int SH_BATCH = 8;           // rounds of 32 events whose loads are issued together

__host__ __device__ __forceinline__ uint32_t shard_rank(uint64_t outer, int world) {
  const uint64_t h = rvd::mix64(outer + 0x9E3779B97F4A7C15ull);
  return (uint32_t)(((h >> 32) * (uint64_t)world) >> 32);
}

// per warp slice: events per destination rank
template <typename K>
__global__ void __launch_bounds__(SH_THREADS)
k_shard_hist(const K* key, uint64_t n, uint64_t per_warp, int G_w, int shift, int world, uint32_t* hist) {
  __shared__ uint32_t cnt[SH_WARPS][SH_MAX_WORLD];
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * SH_WARPS + wl;
  for (int r = lane; r < world; r += 32) cnt[wl][r] = 0;
  __syncwarp();
  if (gw >= G_w) return;
  const uint64_t begin = (uint64_t)gw * per_warp, end = min(n, begin + per_warp);
  for (uint64_t base = begin; base < end; base += 32 * SH_BATCH) {
    K k[SH_BATCH];
#pragma unroll
    for (int j = 0; j < SH_BATCH; ++j) {       // all loads first, so that they are in flight together
      const uint64_t i = base + j * 32 + lane;
      k[j] = i < end ? key[i] : (K)0;
    }
#pragma unroll
    for (int j = 0; j < SH_BATCH; ++j)
      if (base + j * 32 + lane < end) atomicAdd(&cnt[wl][shard_rank((uint64_t)k[j] >> shift, world)], 1u);
  }
  __syncwarp();
  for (int r = lane; r < world; r += 32) hist[(uint64_t)gw * world + r] = cnt[wl][r];
}

// one CTA per destination rank r: exclusive prefix of column r over the warp
// slices (in place) and the rank's total
__global__ void __launch_bounds__(1024) k_shard_scan(uint32_t* hist, int G_w, int world, uint64_t* counts) {
  __shared__ uint64_t wsum[32];
  const int r = blockIdx.x;
  const int per = (G_w + blockDim.x - 1) / blockDim.x;
  const int j0 = threadIdx.x * per, j1 = min(G_w, j0 + per);
  uint64_t mine = 0;
  for (int j = j0; j < j1; j += 8) {            // eight loads in flight before their sums
    uint32_t x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = j + e < j1 ? hist[(uint64_t)(j + e) * world + r] : 0u;
#pragma unroll
    for (int e = 0; e < 8; ++e) mine += x[e];
  }
  // block-wide exclusive scan of the per-thread sums
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t incl = mine;
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t y = __shfl_up_sync(SH_FULL, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    uint64_t x = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t y = __shfl_up_sync(SH_FULL, x, d);
      if (lane >= d) x += y;
    }
    wsum[lane] = x;   // inclusive over warps
  }
  __syncthreads();
  uint64_t run = (w ? wsum[w - 1] : 0) + incl - mine;
  for (int j = j0; j < j1; j += 8) {
    uint32_t x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = j + e < j1 ? hist[(uint64_t)(j + e) * world + r] : 0u;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (j + e < j1) {
        hist[(uint64_t)(j + e) * world + r] = (uint32_t)run;
        run += x[e];
      }
  }
  if (threadIdx.x == blockDim.x - 1) counts[r] = run;
}

// per warp slice: stable placement, in trace order, behind the slice's
// exclusive prefix inside the destination rank's segment
template <typename K>
__global__ void __launch_bounds__(SH_THREADS)
k_shard_scatter(const K* key, const uint8_t* pred, const uint32_t* ts, const uint32_t* value, uint64_t n,
                uint64_t per_warp, int G_w, int shift, int world, const uint32_t* pre, const uint64_t* counts,
                K* key_out, uint8_t* pred_out, uint32_t* ts_out, uint32_t* value_out) {
  __shared__ uint64_t seg[SH_MAX_WORLD];
  __shared__ uint64_t cur[SH_WARPS][SH_MAX_WORLD];
  if (threadIdx.x == 0) {
    uint64_t s = 0;
    for (int r = 0; r < world; ++r) { seg[r] = s; s += counts[r]; }
  }
  __syncthreads();
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * SH_WARPS + wl;
  if (gw >= G_w) return;
  for (int r = lane; r < world; r += 32) cur[wl][r] = seg[r] + pre[(uint64_t)gw * world + r];
  __syncwarp();
  const uint64_t begin = (uint64_t)gw * per_warp, end = min(n, begin + per_warp);
  const uint32_t lt = (1u << lane) - 1u;
  for (uint64_t base0 = begin; base0 < end; base0 += 32 * SH_BATCH) {
    // the batch's fields are loaded before any of them is placed
    K k[SH_BATCH];
    uint8_t pr[SH_BATCH];
    uint32_t tv[SH_BATCH], vv[SH_BATCH];
#pragma unroll
    for (int j = 0; j < SH_BATCH; ++j) {
      const uint64_t i = base0 + j * 32 + lane;
      const bool v = i < end;
      k[j] = v ? key[i] : (K)0;
      pr[j] = v ? pred[i] : (uint8_t)0;
      tv[j] = v && ts_out ? ts[i] : 0u;
      vv[j] = v && value_out ? value[i] : 0u;
    }
#pragma unroll
    for (int j = 0; j < SH_BATCH; ++j) {
      const bool v = base0 + j * 32 + lane < end;
      const uint32_t r = v ? shard_rank((uint64_t)k[j] >> shift, world) : 0xFFFFFFFFu;
      const uint32_t peers = __match_any_sync(SH_FULL, r);
      uint64_t pos = 0;
      if (v) pos = cur[wl][r] + __popc(peers & lt);
      __syncwarp();
      if (v && lane == __ffs(peers) - 1) cur[wl][r] += __popc(peers);
      __syncwarp();
      if (v) {
        key_out[pos] = k[j];
        pred_out[pos] = pr[j];
        if (ts_out) ts_out[pos] = tv[j];
        if (value_out) value_out[pos] = vv[j];
      }
    }
  }
}

struct ShardPlan {
  uint64_t per_warp;
  int G_w;
  size_t o_hist, total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

ShardPlan shard_plan(uint64_t n, int world) {
  ShardPlan p{};
  const uint64_t max_w = (uint64_t)rv_num_sms() * 3 * SH_WARPS;
  uint64_t gw = std::max<uint64_t>(1, std::min<uint64_t>((n + 2047) / 2048, max_w));
  p.per_warp = std::max<uint64_t>(32, ((n + gw - 1) / gw + 31) / 32 * 32);
  p.G_w = (int)std::max<uint64_t>(1, (n + p.per_warp - 1) / p.per_warp);
  p.o_hist = 0;
  p.total = align256((size_t)p.G_w * world * 4);
  return p;
}

rv_status check_world(const rv_formula* f, int world) {
  if (!f) return rv_fail(RV_EINVAL, "null formula");
  if (world < 1 || world > SH_MAX_WORLD) return rv_fail(RV_EINVAL, "world size %d outside 1..%d", world, SH_MAX_WORLD);
  if (f->n_quant == 0 && world > 1)
    return rv_fail(RV_EINVAL, "an unquantified property has one binding, the whole trace: it cannot be sharded");
  return RV_OK;
}

template <typename K>
rv_status launch_shard(const rv_trace* t, int world, int shift, unsigned char* ws, const ShardPlan& p, K* key_out,
                       uint8_t* pred_out, uint32_t* ts_out, uint32_t* value_out, uint64_t* counts, cudaStream_t s) {
  uint32_t* hist = (uint32_t*)(ws + p.o_hist);
  const int grid = (p.G_w + SH_WARPS - 1) / SH_WARPS;
  const K* key = (const K*)t->key;
  RV_LAUNCH("k_shard_hist", k_shard_hist<K>, grid, SH_THREADS, 0, s, key, t->n, p.per_warp, p.G_w, shift, world, hist);
  RV_LAUNCH("k_shard_scan", k_shard_scan, world, 1024, 0, s, hist, p.G_w, world, counts);
  RV_LAUNCH("k_shard_scatter", k_shard_scatter<K>, grid, SH_THREADS, 0, s, key, t->pred, t->ts, t->value, t->n,
            p.per_warp, p.G_w, shift, world, hist, counts, key_out, pred_out, t->ts ? ts_out : nullptr,
            t->value ? value_out : nullptr);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rv_fail(RV_ECUDA, "shard launch: %s", cudaGetErrorString(e));
  return RV_OK;
}

}  // namespace

extern "C" size_t rv_shard_workspace_size(uint64_t n, int world) {
  if (world < 1 || world > SH_MAX_WORLD) return 0;
  return shard_plan(n, world).total;
}

extern "C" rv_status rv_shard_trace(const rv_formula* f, const rv_trace* t, int world, void* ws, size_t ws_bytes,
                                    void* key_out, uint8_t* pred_out, uint32_t* ts_out, uint32_t* value_out,
                                    uint64_t* counts_out, cudaStream_t s) {
  if (rv_status st = check_world(f, world)) return st;
  if (!t || !counts_out) return rv_fail(RV_EINVAL, "null trace or counts");
  if (t->n && (!t->key || !t->pred || !key_out || !pred_out || !ws))
    return rv_fail(RV_EINVAL, "null key, pred, output or workspace");
  if (t->n && t->ts && !ts_out) return rv_fail(RV_EINVAL, "the trace has timestamps: ts_out is needed");
  if (t->n && t->value && !value_out) return rv_fail(RV_EINVAL, "the trace has values: value_out is needed");
  if (t->n > 0xFFFFFFFFull) return rv_fail(RV_EINVAL, "traces are limited to 2^32-1 events");
  if (t->n == 0) {
    const cudaError_t e = cudaMemsetAsync(counts_out, 0, (size_t)world * 8, s);
    return e == cudaSuccess ? RV_OK : rv_fail(RV_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  }
  const ShardPlan p = shard_plan(t->n, world);
  if (ws_bytes < p.total) return rv_fail(RV_ENOMEM, "shard workspace of %zu bytes, need %zu", ws_bytes, p.total);
  const int shift = f->n_quant == 2 ? 32 : 0;
  if (f->key_bits == 64)
    return launch_shard<uint64_t>(t, world, shift, (unsigned char*)ws, p, (uint64_t*)key_out, pred_out, ts_out,
                                  value_out, counts_out, s);
  return launch_shard<uint32_t>(t, world, shift, (unsigned char*)ws, p, (uint32_t*)key_out, pred_out, ts_out,
                                value_out, counts_out, s);
}

extern "C" rv_status rv_shard_of(const rv_formula* f, const void* key, uint64_t n, int world, uint32_t* rank_out) {
  if (rv_status st = check_world(f, world)) return st;
  if (n && (!key || !rank_out)) return rv_fail(RV_EINVAL, "null key or output");
  const int shift = f->n_quant == 2 ? 32 : 0;
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t k = f->key_bits == 64 ? ((const uint64_t*)key)[i] : ((const uint32_t*)key)[i];
    rank_out[i] = shard_rank(k >> shift, world);
  }
  return RV_OK;
}

extern "C" rv_status rv_combine_results(const rv_formula* f, const rv_result* parts, int n_parts, rv_result* out) {
  if (!f || !out || n_parts < 1 || !parts) return rv_fail(RV_EINVAL, "null argument or no parts");
  if (f->n_quant == 0 && n_parts > 1)
    return rv_fail(RV_EINVAL, "an unquantified property has one binding: its result cannot come in parts");
  rv_result r;
  memset(&r, 0, sizeof r);
  r.status = RV_OK;
  for (int i = 0; i < n_parts; ++i) {
    const rv_result& p = parts[i];
    for (int v = 0; v < 6; ++v) {
      r.root_counts[v] += p.root_counts[v];
      r.level_counts[0][v] += p.level_counts[0][v];
      r.level_counts[1][v] += p.level_counts[1][v];
    }
    r.n_nodes[0] += p.n_nodes[0];
    r.n_nodes[1] += p.n_nodes[1];
    r.events += p.events;
    if (r.status == RV_OK && p.status != RV_OK) r.status = p.status;
  }
  if (f->n_quant == 0) {
    r.root = parts[0].root;
  } else {
    const rv_quant& q = f->q[0];
    r.root = rvv::valuate(q.kind, q.op, q.num, q.den, r.root_counts);
  }
  *out = r;
  return RV_OK;
}
