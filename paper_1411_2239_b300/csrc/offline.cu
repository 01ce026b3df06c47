// Offline verification of one trace against one LTL4-C formula on one GPU
// (Algorithm 1, Sec. 4.2: SortTrace -> SpawnMonitors -> Distribute ->
// ApplyQuantifiers), re-designed for B300.
//
// map      a stable two-level multisplit of the events by the mixed outer key.
//          Level 1 (k_hist_tile / column scans / k_scatter_tile): CTA tiles of
//          the trace are counting-sorted by the top 8 key bits in shared memory
//          and each bucket's run is written out contiguously.  Level 2
//          (k_hist2 / k_scan2 / k_scatter2 or k_scatter2_tile): tiles of every
//          first-level bucket are split again by the next B2 bits.  Trace order
//          is kept inside every bucket; a record is the letter plus the key
//          bits the bucket does not imply (4 or 8 bytes).  Heavy bindings of a
//          one-variable formula (found by k_hsample / k_hpick on a sample of
//          the trace) get second-level sub-buckets of their own.
// monitor  k_fold: one CTA folds a unit -- a piece of a large bucket, or whole
//          small buckets of one first-level bucket.  Each binding (key) takes a
//          slot in a shared-memory table; every record gets its rank among its
//          slot's records in its warp's slice; one scan and a placement group
//          the letters by binding in trace order; the runs are folded by the
//          LTL4 Moore monitor (plain state steps from q0, or 4-bit-per-state
//          transition maps composed by byte permutes where a run starts
//          elsewhere).  A binding that fills at least half of the unit (a Zipf
//          head) is folded in place instead of being sorted, and a heavy
//          binding's own sub-bucket is folded in place with no grouping at all.
// reduce   a bucket held by one unit is finalised in k_fold; buckets split
//          over several units pass (key, map) pairs to k_combine, which
//          composes them level by level in unit order (fan-in 16) and
//          finalises at the last level.  Finalising evaluates lambda(map[q0]),
//          counts verdicts per parent (per outer binding in a shared table
//          for two quantifiers, all bindings of an outer value share its
//          bucket), applies the quantifier constraint in integers, and adds
//          the counts of the root.  k_root valuates the root.
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <type_traits>
#include <vector>

#include "profile.h"
#include "rv_device.cuh"

using namespace rvd;

namespace {

constexpr int SC_WARPS = 8;
constexpr int FOLD_WARPS = 8;
constexpr int FOLD_THREADS = FOLD_WARPS * 32;
constexpr int SLOTS = 1024;
constexpr int HT_BITS = 11;
constexpr int HT_CAP = 1 << HT_BITS;
constexpr int UCAP = 256;
constexpr int GC = 16;      // items (units or groups) combined by one CTA per level
constexpr int COLCHUNK = 64;
constexpr uint16_t NO_SLOT = 0xFFFF;
constexpr uint16_t FULL_SLOT = 0xFFFE;
constexpr uint64_t EMPTY_KEY = ~0ull;
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int SPIN_LIMIT = 1 << 22;
constexpr int BATCH = 16;      // rounds of 32 events whose loads are issued together
constexpr int HVEC = 4;        // 16-byte loads in flight per lane in the level-2 histogram

struct Tile { uint32_t bucket, k, K, pad; uint64_t begin, end; };

// Bounds-checked builds (-DRV_CHECKED, for test runs): the global writes of
// the multisplit, tile and unit lists, fold and combine check their index
// against the array's size; a write outside is skipped and reported through
// the status word (ERR_BOUNDS, status RV_EINTERNAL) instead of faulting.
// The sizes of one verification are set before its kernels, so checked
// builds are for one verification at a time.
#ifdef RV_CHECKED
struct CheckCaps { unsigned long long n, tiles2, units, pool; };
__device__ CheckCaps g_caps;
__device__ unsigned int g_bounds_err;
#define RV_INB(i, cap) ((unsigned long long)(i) < (cap) ? true : (atomicOr(&g_bounds_err, 1u), false))
#else
#define RV_INB(i, cap) true
#endif
struct Item { uint64_t off; uint32_t cnt, pad; };
struct Group { uint32_t bucket, first, cnt, k, K, pad; };
struct Pair { uint64_t key, map; };

// record e of a 16-byte word (little-endian): four 32-bit or two 64-bit records
template <typename Rec>
__device__ __forceinline__ uint64_t word_rec(const uint4& x, int e) {
  if constexpr (sizeof(Rec) == 4) return e == 0 ? x.x : e == 1 ? x.y : e == 2 ? x.z : x.w;
  else return e == 0 ? ((uint64_t)x.y << 32 | x.x) : ((uint64_t)x.w << 32 | x.z);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Lanes of the warp whose `valid` flag and low BITS bits of v equal this
// lane's: one ballot per bit (full rate).
template <int BITS>
__device__ __forceinline__ uint32_t match_bits(uint32_t v, bool valid) {
  const uint32_t vb = __ballot_sync(FULL, valid);
  uint32_t m = valid ? vb : ~vb;
#pragma unroll
  for (int k = 0; k < BITS; ++k) {
    const uint32_t bk = __ballot_sync(FULL, (v >> k) & 1u);
    m &= ((v >> k) & 1u) ? bk : ~bk;
  }
  return m;
}

template <int F>
__device__ __forceinline__ uint64_t load_key(const void* p, uint64_t i) {
  if (F == FMT_K32) return ((const uint32_t*)p)[i];
  return ((const uint64_t*)p)[i];
}

// ------------------------------------------------------------------ level-1 multisplit
template <int F>
__global__ void __launch_bounds__(SC_WARPS * 32)
k_hist(const void* keyp, const uint32_t* ts, uint64_t n, uint64_t per_warp, int G_w, int B1, int nq,
       uint32_t* hist, Acc* acc) {
  extern __shared__ uint32_t sm_cnt[];
  const int P = 1 << B1;
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * SC_WARPS + wl;
  uint32_t* cnt = sm_cnt + wl * P;
  for (int b = lane; b < P; b += 32) cnt[b] = 0;
  __syncwarp();
  if (gw >= G_w) return;
  const uint64_t begin = (uint64_t)gw * per_warp, end = min(n, begin + per_warp);
  bool bad_ts = false;
  // BATCH rounds of 32 events: all loads of a batch are in flight together
  for (uint64_t base = begin; base < end; base += 32 * BATCH) {
    uint32_t b[BATCH];
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      const uint64_t i = base + j * 32 + lane;
      b[j] = i < end ? make_record<F>(load_key<F>(keyp, i), 0, B1, nq).bucket : 0xFFFFFFFFu;
    }
    if (ts) {
#pragma unroll
      for (int j = 0; j < BATCH; ++j) {
        const uint64_t i = base + j * 32 + lane;
        if (i < end && i > 0 && ts[i] < ts[i - 1]) bad_ts = true;
      }
    }
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      if (b[j] != 0xFFFFFFFFu) atomicAdd(&cnt[b[j]], 1u);
    }
  }
  if (__any_sync(FULL, bad_ts) && lane == 0) atomicOr(&acc->err, ERR_TS);
  for (int b = lane; b < P; b += 32) hist[(uint64_t)gw * P + b] = cnt[b];
}

// ------------------------------------------------------------------ level-1 multisplit, CTA tiles
// With 256 first-level buckets a CTA splits a tile of TILE events at a time:
// the tile is counting-sorted by bucket in shared memory (stable: per-warp
// counts over contiguous slices) and each bucket's run is written out
// contiguously, so the global writes are runs rather than scattered words.
template <int F> struct TileSize { static constexpr int v = 4096; };
template <> struct TileSize<FMT_K32> { static constexpr int v = 8192; };
constexpr int TB_THREADS = 256;
constexpr int TB_WARPS = TB_THREADS / 32;
// records of one level-2 tile (a piece of a first-level bucket)
template <int F> struct Tile2Len { static constexpr int v = 4096; };
template <> struct Tile2Len<FMT_K32> { static constexpr int v = 8192; };

template <int F>
__global__ void __launch_bounds__(TB_THREADS)
k_hist_tile(const void* keyp, const uint32_t* ts, uint64_t n, int nq, uint32_t* hist, Acc* acc) {
  constexpr int T = TileSize<F>::v;
  __shared__ uint32_t cnt[256];
  const uint64_t begin = (uint64_t)blockIdx.x * T;
  const int len = (int)min((uint64_t)T, n - begin);
  cnt[threadIdx.x] = 0;
  __syncthreads();
  bool bad_ts = false;
  for (int i0 = threadIdx.x; i0 < len; i0 += TB_THREADS * BATCH) {
    uint32_t b[BATCH];
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      const int i = i0 + j * TB_THREADS;
      b[j] = i < len ? make_record<F>(load_key<F>(keyp, begin + i), 0, 8, nq).bucket : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      const int i = i0 + j * TB_THREADS;
      if (b[j] != 0xFFFFFFFFu) {
        atomicAdd(&cnt[b[j]], 1u);
        if (ts && begin + i > 0 && ts[begin + i] < ts[begin + i - 1]) bad_ts = true;
      }
    }
  }
  if (__syncthreads_or(bad_ts) && threadIdx.x == 0) atomicOr(&acc->err, ERR_TS);
  hist[(uint64_t)blockIdx.x * 256 + threadIdx.x] = cnt[threadIdx.x];
}

template <int F>
struct TileShared {
  typename RecT<F>::type srec[TileSize<F>::v];   // the tile's records in trace order
  uint8_t sb[TileSize<F>::v];                    // bucket of srec[i]
  uint16_t perm[TileSize<F>::v];                 // perm[j]: record at position j of the bucket order
  uint32_t wcur[TB_WARPS][256];
  uint32_t loc[256];
  uint64_t gbase[256];
  uint32_t tsum[TB_WARPS];
};

template <int F>
__global__ void __launch_bounds__(TB_THREADS, 3)
k_scatter_tile(const void* keyp, const uint8_t* pred, uint64_t n, int nq, int n_letters, const uint32_t* pre,
               const uint64_t* bstart, typename RecT<F>::type* out, Acc* acc) {
  typedef typename RecT<F>::type Rec;
  constexpr int T = TileSize<F>::v;
  extern __shared__ __align__(16) unsigned char tile_smem[];
  TileShared<F>& S = *reinterpret_cast<TileShared<F>*>(tile_smem);
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  const uint64_t begin = (uint64_t)blockIdx.x * T;
  const int len = (int)min((uint64_t)T, n - begin);
  for (int i = threadIdx.x; i < TB_WARPS * 256; i += TB_THREADS) S.wcur[i / 256][i % 256] = 0;
  bool bad = false;
  // 1. records and buckets of the tile, in trace order
  for (int i0 = threadIdx.x; i0 < len; i0 += TB_THREADS * BATCH) {
    uint64_t k[BATCH];
    uint32_t l[BATCH];
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      const int i = i0 + j * TB_THREADS;
      k[j] = i < len ? load_key<F>(keyp, begin + i) : 0;
      l[j] = i < len ? pred[begin + i] : 0;
    }
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      const int i = i0 + j * TB_THREADS;
      if (i < len) {
        uint32_t letter = l[j];
        if (letter >= (uint32_t)n_letters) { bad = true; letter = 0; }
        const Bucketed r = make_record<F>(k[j], letter, 8, nq);
        S.srec[i] = (Rec)r.rec;
        S.sb[i] = (uint8_t)r.bucket;
      }
    }
  }
  __syncthreads();
  // 2. per-warp counts over contiguous slices
  const int per = (len + TB_WARPS - 1) / TB_WARPS;
  const int w0 = min(len, wl * per), w1 = min(len, w0 + per);
  for (int i = w0 + lane; i < w1; i += 32) atomicAdd(&S.wcur[wl][S.sb[i]], 1u);
  __syncthreads();
  // 3. thread b: offsets of bucket b inside the tile and in the output
  {
    const int b = threadIdx.x;
    uint32_t tot = 0;
    for (int w = 0; w < TB_WARPS; ++w) tot += S.wcur[w][b];
    uint32_t x = tot;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) S.tsum[wl] = x;
    __syncthreads();
    uint32_t run = x - tot;
    for (int w = 0; w < wl; ++w) run += S.tsum[w];
    S.loc[b] = run;
    S.gbase[b] = bstart[b] + pre[(uint64_t)blockIdx.x * 256 + b];
    for (int w = 0; w < TB_WARPS; ++w) { const uint32_t c = S.wcur[w][b]; S.wcur[w][b] = run; run += c; }
  }
  __syncthreads();
  // 4. stable placement by bucket
  for (int base = w0; base < w1; base += 32) {
    const int i = base + lane;
    const bool v = i < w1;
    const uint32_t b = v ? S.sb[i] : 0u;
    const uint32_t peers = match_bits<8>(b, v);
    uint32_t pos = 0;
    if (v) pos = S.wcur[wl][b] + __popc(peers & lt);
    __syncwarp();
    if (v && lane == __ffs(peers) - 1) S.wcur[wl][b] += __popc(peers);
    __syncwarp();
    if (v) S.perm[pos] = (uint16_t)i;
  }
  __syncthreads();
  // 5. runs of each bucket go out contiguously, gathered through perm
  for (int j = threadIdx.x; j < len; j += TB_THREADS) {
    const uint32_t i = S.perm[j], b = S.sb[i];
    const uint64_t o = S.gbase[b] + (j - S.loc[b]);
    if (RV_INB(o, g_caps.n)) out[o] = S.srec[i];
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&acc->err, ERR_LETTER);
}

// Rank of each lane's bucket b (< 256) among the records of its warp so far:
// lanes of equal buckets are matched (one ballot per bit: faster than the
// hardware match in this kernel, measured) and the lowest of them advances
// the warp's counter (equal buckets never share a leader, so no atomics).
__device__ __forceinline__ uint32_t warp_rank(uint32_t b, bool v, uint32_t* cnt, uint32_t lt) {
  const uint32_t peers = match_bits<8>(v ? b : 0u, v);   // b < 256
  const int ld = __ffs(peers) - 1;
  uint32_t old = 0;
  if (v && (int)(threadIdx.x & 31) == ld) {
    old = cnt[b];
    cnt[b] = old + __popc(peers);
  }
  old = __shfl_sync(FULL, old, ld);
  return old + __popc(peers & lt);
}

// Exclusive scan of a tile's per-warp bucket counts (thread b owns bucket b):
// loc[b] = start of bucket b in the tile, wcur[w][b] = cursor of warp w.
template <int NB>
__device__ __forceinline__ void tile_scan(uint32_t (*wcur)[NB], uint32_t* loc, uint32_t* tsum, int nb) {
  const int b = threadIdx.x, lane = b & 31, wl = b >> 5;
  uint32_t tot = 0;
  if (b < nb)
    for (int w = 0; w < TB_WARPS; ++w) tot += wcur[w][b];
  uint32_t x = tot;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tsum[wl] = x;
  __syncthreads();
  uint32_t run = x - tot;
  for (int w = 0; w < wl; ++w) run += tsum[w];
  if (b < nb) {
    loc[b] = run;
    for (int w = 0; w < TB_WARPS; ++w) { const uint32_t c = wcur[w][b]; wcur[w][b] = run; run += c; }
  }
}

// Sums and exclusive prefixes down a column p[0], p[s], p[2s], ...: the loads
// of COLB entries are issued before any of their stores, so a thread waits
// for one memory round trip per COLB entries rather than per entry.
constexpr int COLB = 16;
template <typename T>
__device__ __forceinline__ uint64_t col_sum(const T* p, uint64_t s, uint32_t n) {
  uint64_t sum = 0;
  for (uint32_t j0 = 0; j0 < n; j0 += COLB) {
    T x[COLB];
#pragma unroll
    for (int j = 0; j < COLB; ++j) x[j] = j0 + j < n ? p[(uint64_t)(j0 + j) * s] : (T)0;
#pragma unroll
    for (int j = 0; j < COLB; ++j) sum += x[j];
  }
  return sum;
}
// p[j s] <- run + p[0] + ... + p[(j-1) s] in place; returns run + the column's sum
template <typename T>
__device__ __forceinline__ uint64_t col_exscan(T* p, uint64_t s, uint32_t n, uint64_t run) {
  for (uint32_t j0 = 0; j0 < n; j0 += COLB) {
    T x[COLB];
#pragma unroll
    for (int j = 0; j < COLB; ++j) x[j] = j0 + j < n ? p[(uint64_t)(j0 + j) * s] : (T)0;
#pragma unroll
    for (int j = 0; j < COLB; ++j)
      if (j0 + j < n) {
        p[(uint64_t)(j0 + j) * s] = (T)run;
        run += x[j];
      }
  }
  return run;
}

// per (bucket, chunk of warps): chunk sums
__global__ void k_colscan_a(const uint32_t* hist, int G_w, int P, int nchunk, uint64_t* part) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P * nchunk) return;
  const int b = t % P, c = t / P;
  const int w0 = c * COLCHUNK, w1 = min(G_w, w0 + COLCHUNK);
  part[(uint64_t)c * P + b] = col_sum(hist + (uint64_t)w0 * P + b, (uint64_t)P, (uint32_t)(w1 - w0));
}
// per bucket: exclusive scan over chunks, bucket totals
__global__ void k_colscan_b(uint64_t* part, int P, int nchunk, uint64_t* tot) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= P) return;
  tot[b] = col_exscan(part + b, (uint64_t)P, (uint32_t)nchunk, 0);
}
// per (bucket, chunk): exclusive prefix over warps, in place
__global__ void k_colscan_c(uint32_t* hist, int G_w, int P, int nchunk, const uint64_t* part) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P * nchunk) return;
  const int b = t % P, c = t / P;
  const int w0 = c * COLCHUNK, w1 = min(G_w, w0 + COLCHUNK);
  col_exscan(hist + (uint64_t)w0 * P + b, (uint64_t)P, (uint32_t)(w1 - w0), part[(uint64_t)c * P + b]);
}


template <int F>
__global__ void __launch_bounds__(SC_WARPS * 32)
k_scatter(const void* keyp, const uint8_t* pred, uint64_t n, uint64_t per_warp, int G_w, int B1, int nq,
          int n_letters, const uint32_t* pre, const uint64_t* bstart, typename RecT<F>::type* out, Acc* acc) {
  extern __shared__ uint32_t sm_cur[];
  typedef typename RecT<F>::type Rec;
  const int P = 1 << B1;
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * SC_WARPS + wl;
  if (gw >= G_w) return;
  uint32_t* cur = sm_cur + wl * P;
  for (int b = lane; b < P; b += 32) cur[b] = (uint32_t)(bstart[b] + pre[(uint64_t)gw * P + b]);
  __syncwarp();
  const uint64_t begin = (uint64_t)gw * per_warp, end = min(n, begin + per_warp);
  bool bad = false;
  const uint32_t lt = lanemask_lt();
  for (uint64_t base = begin; base < end; base += 32 * BATCH) {
    uint32_t b[BATCH];
    Rec rec[BATCH];
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      const uint64_t i = base + j * 32 + lane;
      b[j] = 0xFFFFFFFFu;
      rec[j] = 0;
      if (i < end) {
        uint32_t letter = pred[i];
        if (letter >= (uint32_t)n_letters) { bad = true; letter = 0; }
        Bucketed r = make_record<F>(load_key<F>(keyp, i), letter, B1, nq);
        b[j] = r.bucket;
        rec[j] = (Rec)r.rec;
      }
    }
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      const bool v = b[j] != 0xFFFFFFFFu;
      const uint32_t peers = match_bits<11>(b[j], v);
      uint32_t pos = 0;
      if (v) pos = cur[b[j]] + __popc(peers & lt);
      __syncwarp();
      if (v && lane == __ffs(peers) - 1) cur[b[j]] += __popc(peers);
      __syncwarp();
      if (v && RV_INB(pos, g_caps.n)) out[pos] = rec[j];
    }
  }
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(&acc->err, ERR_LETTER);
}

// ------------------------------------------------------------------ tiles of buckets
// Every non-empty bucket b (bstart[b]..bstart[b+1]) is split into
// ceil(len / tile_len) tiles; first[b] / K[b] give its tile range.
__global__ void k_count_tiles(const uint64_t* bstart, int P, uint64_t tile_len, uint32_t* K) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= P) return;
  const uint64_t len = bstart[b + 1] - bstart[b];
  K[b] = (uint32_t)((len + tile_len - 1) / tile_len);
}

// single CTA: exclusive scan of in[0..P) into out[0..P), total into *total.
// Chunks are staged in shared memory with coalesced loads (padded by one word
// per 32 entries, so that a thread's contiguous run of 32 entries falls into
// 32 banks), each thread scans its run, and the results go back coalesced.
template <typename T> struct ScanChunk { static constexpr int v = 32768; };
template <> struct ScanChunk<uint64_t> { static constexpr int v = 16384; };
template <typename T> constexpr size_t scan_smem() { return (ScanChunk<T>::v + ScanChunk<T>::v / 32) * sizeof(T); }

template <typename T>
__global__ void __launch_bounds__(1024) k_scan(const T* in, int P, T* out, T* total, const unsigned int* Pdev = nullptr) {
  constexpr int CH = ScanChunk<T>::v, RUN = CH / 1024;
  if (Pdev) P = min(P, (int)*Pdev);
  extern __shared__ __align__(16) unsigned char scan_smem_raw[];
  T* sc = reinterpret_cast<T*>(scan_smem_raw);
  __shared__ T wsum[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  T carry = 0;
  for (int base = 0; base < P; base += CH) {
    const int len = min(CH, P - base);
    for (int i = t; i < len; i += 1024) sc[i + (i >> 5)] = in[base + i];
    __syncthreads();
    const int i0 = t * RUN;                      // this thread's run: entries i0 .. i0 + RUN - 1
    T s = 0;
#pragma unroll
    for (int j = 0; j < RUN; ++j) {
      const int i = i0 + j;
      s += i < len ? sc[i + (i >> 5)] : (T)0;
    }
    T x = s;
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      T z = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(FULL, z, o);
        if (lane >= o) z += y;
      }
      wsum[lane] = z;
    }
    __syncthreads();
    T run = carry + x - s + (w ? wsum[w - 1] : (T)0);
#pragma unroll
    for (int j = 0; j < RUN; ++j) {
      const int i = i0 + j;
      if (i < len) {
        const T v = sc[i + (i >> 5)];
        sc[i + (i >> 5)] = run;
        run += v;
      }
    }
    carry += wsum[31];
    __syncthreads();
    for (int i = t; i < len; i += 1024) out[base + i] = sc[i + (i >> 5)];
    __syncthreads();
  }
  if (t == 0) *total = carry;
}

// Units of the fold.  A bucket longer than half a unit is cut into
// ceil(len / unit) units; with `pack`, the shorter buckets of one first-level
// bucket whose starts fall into the same half-unit window share one unit,
// which is then at most one unit long and holds whole buckets only (a heavy
// key's own sub-bucket is never shared).  K[b] is the number of units
// starting at bucket b; uend[b] is the end of the unit a bucket of at most
// half a unit heads (its own end when it is not shared).
__global__ void k_count_units(const uint64_t* bstart, int P, int B2, uint64_t unit, int pack, uint32_t* K,
                              uint64_t* uend, int light) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= P) return;
  const uint64_t s = bstart[b], len = bstart[b + 1] - s, W = unit / 2;
  // sub-buckets light.. of every first-level bucket belong to single heavy keys
  const bool own = light && (b & ((1 << B2) - 1)) >= light;
  if (!pack || len > W || own) {
    K[b] = (uint32_t)((len + unit - 1) / unit);
    uend[b] = s + len;   // read for every bucket of at most half a unit, a heavy key's own included
    return;
  }
  const int first = (b >> B2) << B2, last = first + (light ? light : 1 << B2);
  const uint64_t base = bstart[first], g = (s - base) / W;
  const bool head = b == first || bstart[b] - bstart[b - 1] > W || (bstart[b - 1] - base) / W != g;
  if (!head) {
    K[b] = 0;
    return;
  }
  int e = b;
  while (e + 1 < last) {
    const uint64_t s1 = bstart[e + 1];
    if (bstart[e + 2] - s1 > W || (s1 - base) / W != g) break;
    ++e;
  }
  const uint64_t end = bstart[e + 1];
  K[b] = end > s ? 1u : 0u;
  uend[b] = end;
}

// one thread per tile: binary search of its bucket in first[]; with uend, a
// bucket of at most half a tile heads a shared tile that ends at uend[b]
__global__ void k_emit_tiles(const uint64_t* bstart, int P, uint64_t tile_len, const uint32_t* first, const uint32_t* K,
                             const unsigned int* n_tiles, Tile* tiles, uint64_t cap, const uint64_t* uend = nullptr) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= *n_tiles) return;
  int lo = 0, hi = P - 1;            // last bucket with first[b] <= t and K[b] > 0
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= t) lo = mid; else hi = mid - 1;
  }
  // the largest b with first[b] <= t has first[b] + K[b] = first[b+1] > t, so K[b] > 0
  const uint32_t j = t - first[lo];
  Tile tl;
  tl.bucket = (uint32_t)lo; tl.k = j; tl.K = K[lo]; tl.pad = 0;
  tl.begin = bstart[lo] + j * tile_len;
  tl.end = min(bstart[lo + 1], tl.begin + tile_len);
  if (uend && bstart[lo + 1] - bstart[lo] <= tile_len / 2) tl.end = uend[lo];
#ifdef RV_CHECKED
  // a unit lies inside the records and begins at its bucket's start or later
  if (tl.end < tl.begin || tl.end > g_caps.n || tl.begin < bstart[lo]) {
    atomicOr(&g_bounds_err, 1u);
    tl.end = tl.begin;
  }
#endif
  if (RV_INB(t, cap)) tiles[t] = tl;
}

// ------------------------------------------------------------------ heavy bindings
// A binding that holds a large share of the trace (a Zipf head) fills the
// units of its sub-bucket almost alone; giving it a sub-bucket of its own
// makes those units single-binding, folded without any grouping.  Heavy keys
// are found from a sample of the trace (every HSTRIDE-th event); a miss or a
// false hit changes only where a binding's records go, never the result.
constexpr int HSTRIDE = 256;           // at least; more for traces over 2^27 events
constexpr uint64_t HRECORDS = 8192;    // records that make a key heavy (about one unit)
constexpr int HTAB_BITS = 20;          // largest sample table; it holds at most half as many samples
constexpr int HMAXC = 64;              // heavy bindings per first-level bucket

struct HeavyDev {
  const uint32_t* cnt;                 // [P1] heavy bindings found per first-level bucket
  const uint64_t* list;                // [P1][hmax] their record keys
  int hmax;                            // 0: routing off
};

template <int F>
__device__ __forceinline__ uint64_t mixed_key(uint64_t key) {
  if (F == FMT_K32) return mix32((uint32_t)key);
  return mix64(key);
}

// Count sampled keys in a global open-addressing table (key 0: empty; a key
// whose mix is 0 is never counted).  The sample is HS_RUN consecutive events
// out of every HS_RUN * stride (the same rate as one event in stride, from
// far fewer scattered memory sectors).  A CTA first counts its HS_PER * 256
// samples in a table of its own in shared memory (at most half full), then
// adds one count per distinct key to the global table.
constexpr int HS_PER = 4;
constexpr int HS_TBITS = 11;
constexpr int HS_RUN = 8;

template <int F>
__global__ void __launch_bounds__(256)
k_hsample(const void* keyp, uint64_t n, uint64_t stride, int tbits, uint64_t* tk, uint32_t* tc) {
  constexpr int TAB = 1 << HS_TBITS;
  static_assert(TAB >= 2 * HS_PER * 256, "the CTA table holds every sample of the CTA at most half full");
  __shared__ unsigned long long sk[TAB];
  __shared__ uint32_t sc[TAB];
  for (int e = threadIdx.x; e < TAB; e += 256) { sk[e] = 0ull; sc[e] = 0u; }
  uint64_t m[HS_PER];
#pragma unroll
  for (int j = 0; j < HS_PER; ++j) {
    const uint64_t smp = ((uint64_t)blockIdx.x * HS_PER + j) * 256 + threadIdx.x;
    const uint64_t i = smp / HS_RUN * (HS_RUN * stride) + smp % HS_RUN;
    m[j] = i < n ? mixed_key<F>(load_key<F>(keyp, i)) : 0ull;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < HS_PER; ++j) {
    const uint32_t peers = __match_any_sync(FULL, m[j]);
    if (m[j] != 0ull && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
      uint32_t h = (uint32_t)((m[j] * 0x9E3779B97F4A7C15ull) >> (64 - HS_TBITS));
      for (int probe = 0; probe < TAB; ++probe) {
        const unsigned long long prev = atomicCAS(&sk[h], 0ull, (unsigned long long)m[j]);
        if (prev == 0ull || prev == m[j]) {
          atomicAdd(&sc[h], (uint32_t)__popc(peers));
          break;
        }
        h = (h + 1) & (TAB - 1);
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TAB; e += 256) {
    const unsigned long long key = sk[e];
    if (key == 0ull) continue;
    uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - tbits));
    for (int probe = 0; probe < (1 << tbits); ++probe) {
      const unsigned long long prev = atomicCAS((unsigned long long*)&tk[h], 0ull, key);
      if (prev == 0ull || prev == key) {
        atomicAdd(&tc[h], sc[e]);
        break;
      }
      h = (h + 1) & ((1u << tbits) - 1);
    }
  }
}

// keys sampled often enough become heavy: appended to their first-level
// bucket's list as record keys (the mixed bits a record keeps)
template <int F>
__global__ void k_hpick(const uint64_t* tk, const uint32_t* tc, int tbits, uint32_t thresh, int B1, int hmax,
                        uint32_t* hcnt, uint64_t* hlist) {
  const uint32_t h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= (1u << tbits) || tc[h] < thresh) return;
  const uint64_t m = tk[h];
  const int W = F == FMT_K32 ? 32 : 64;
  const uint32_t b1 = (uint32_t)(m >> (W - B1));
  const uint64_t local = m & (W == 32 ? (0xFFFFFFFFull >> B1) : (~0ull >> B1));
  const uint32_t j = atomicAdd(&hcnt[b1], 1u);
  if (j < (uint32_t)hmax) hlist[(uint64_t)b1 * hmax + j] = local;
}

// the first-level bucket's heavy record keys, staged for broadcast reads
__device__ __forceinline__ int load_heavy(const HeavyDev& hv, uint32_t b1, uint64_t* hl, int lane0, int step) {
  if (!hv.hmax) return 0;
  const int nh = (int)min(hv.cnt[b1], (uint32_t)hv.hmax);
  for (int j = lane0; j < nh; j += step) hl[j] = hv.list[(uint64_t)b1 * hv.hmax + j];
  return nh;
}

// A direct-mapped filter over the low HFILT_BITS bits of a record key: j + 1 for the
// heavy key j that has them, 0 for none, 0xFF when several share them.  Built
// by the 32 lanes of one warp together (all of them call it); nh <= HMAXC.
constexpr int HFILT_BITS = 10;         // 1024 entries: a few dozen heavy keys rarely share one
constexpr int HFILT = 1 << HFILT_BITS;
__device__ __forceinline__ void build_filter(uint8_t* filt, const uint64_t* hl, int nh, int lane) {
  static_assert(HMAXC % 32 == 0, "whole rounds of heavy keys");
  constexpr int R = HMAXC / 32;
  uint32_t* f4 = reinterpret_cast<uint32_t*>(filt);
  for (int i = lane; i < HFILT / 4; i += 32) f4[i] = 0u;
  __syncwarp();
  // every key writes its number at its entry (of several keys at one entry,
  // one write remains); a key that then finds another number there marks
  // the entry shared
  int h[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int j = r * 32 + lane;
    h[r] = j < nh ? (int)(hl[j] & (HFILT - 1)) : -1;
    if (h[r] >= 0) filt[h[r]] = (uint8_t)(j + 1);
  }
  __syncwarp();
  bool shared_entry[R];
#pragma unroll
  for (int r = 0; r < R; ++r) shared_entry[r] = h[r] >= 0 && filt[h[r]] != (uint8_t)(r * 32 + lane + 1);
  __syncwarp();
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (shared_entry[r]) filt[h[r]] = 0xFF;
  __syncwarp();
}

// second-level sub-bucket of a record: its own for a heavy key (P2L + j),
// else the next B2 bits of the mixed key
__device__ __forceinline__ uint32_t sub_of(uint64_t rec, int sh, uint32_t P2L, const uint64_t* hl, const uint8_t* filt,
                                           int nh) {
  uint32_t sb = (uint32_t)(rec >> sh) & (P2L - 1);
  if (nh == 0) return sb;
  const uint64_t lk = rec >> 8;
  const uint32_t f = filt[lk & (HFILT - 1)];
  // branch-free for the common cases (no heavy key, one heavy key behind the filter entry)
  const uint32_t j = (f - 1u) & (HMAXC - 1);
  sb = (f - 1u < (uint32_t)nh && hl[j] == lk) ? P2L + j : sb;
  if (f == 0xFF) {
    for (int q = 0; q < nh; ++q)
      if (hl[q] == lk) sb = P2L + q;
  }
  return sb;
}

// ------------------------------------------------------------------ level-2 multisplit
template <int F>
__global__ void __launch_bounds__(SC_WARPS * 32, 6)
k_hist2(const typename RecT<F>::type* recs, const Tile* tiles, const unsigned int* n_tiles, int B1, int B2,
        uint32_t* hist2, HeavyDev hv) {
  __shared__ uint32_t cnt_all[SC_WARPS][256];
  __shared__ uint64_t hl_all[SC_WARPS][HMAXC];
  __shared__ __align__(4) uint8_t filt_all[SC_WARPS][HFILT];
  const uint32_t P2L = 1u << B2;
  const int P2 = hv.hmax ? 2 << B2 : 1 << B2;    // light sub-buckets, then one per heavy key
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tile = blockIdx.x * SC_WARPS + wl;
  if (tile >= *n_tiles) return;
  uint32_t* cnt = cnt_all[wl];
  for (int b = lane; b < P2; b += 32) cnt[b] = 0;
  const Tile tl = tiles[tile];
  const int nh = load_heavy(hv, tl.bucket, hl_all[wl], lane, 32);
  __syncwarp();
  if (nh) build_filter(filt_all[wl], hl_all[wl], nh, lane);
  const uint64_t* hl = hl_all[wl];
  const uint8_t* filt = filt_all[wl];
  const int sh = sub_shift<F>(B1, B2);
  // Counts do not depend on the order, so the tile is read in 16-byte words
  // (HVEC in flight per lane); the records before the first 16-byte boundary
  // and after the last one are read one per lane.
  typedef typename RecT<F>::type Rec;
  constexpr int VEC = 16 / sizeof(Rec);
  const Rec* rb = recs + tl.begin;
  const uint64_t len = tl.end - tl.begin;
  const uint64_t head = min(len, (uint64_t)(((16u - ((uint32_t)(uintptr_t)rb & 15u)) & 15u) / sizeof(Rec)));
  const uint64_t nv = (len - head) / VEC, tail = head + nv * VEC;
  if ((uint64_t)lane < head) atomicAdd(&cnt[sub_of((uint64_t)rb[lane], sh, P2L, hl, filt, nh)], 1u);
  if ((uint64_t)lane < len - tail) atomicAdd(&cnt[sub_of((uint64_t)rb[tail + lane], sh, P2L, hl, filt, nh)], 1u);
  const uint4* v = reinterpret_cast<const uint4*>(rb + head);
  for (uint64_t q0 = 0; q0 < nv; q0 += 32 * HVEC) {
    uint4 x[HVEC];
#pragma unroll
    for (int j = 0; j < HVEC; ++j) {   // all loads first, so that they are in flight together
      const uint64_t q = q0 + j * 32 + lane;
      x[j] = q < nv ? v[q] : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int j = 0; j < HVEC; ++j) {
      if (q0 + j * 32 + lane >= nv) continue;
#pragma unroll
      for (int e = 0; e < VEC; ++e)
        atomicAdd(&cnt[sub_of(word_rec<Rec>(x[j], e), sh, P2L, hl, filt, nh)], 1u);
    }
  }
  __syncwarp();
  if (RV_INB(tile, g_caps.tiles2))
    for (int b = lane; b < P2; b += 32) hist2[(uint64_t)tile * P2 + b] = cnt[b];
}

// per (first-level bucket, sub-bucket): exclusive prefix over the bucket's
// tiles.  A bucket's tiles are cut into up to SCAN2_S slices of at least
// SCAN2_MIN tiles (a Zipf head's bucket holds over a thousand tiles, more than
// one SM moves quickly), one CTA per slice.  k_scan2_sums writes every slice's
// column sums when there are several; in k_scan2, rows of threads each take a
// contiguous share of the slice's tiles for every sub-bucket column (2^B2 <=
// 256 columns), the rows' sums are scanned in shared memory on top of the
// earlier slices' sums, then every row writes its share's prefixes.  The
// sub-buckets of a bucket fill exactly the bucket's range of the first-level
// output, so their starts are the bucket's start plus the totals of the
// columns before them, written by the last slice with the end sentinel.
constexpr int SCAN2_S = 8;
constexpr uint32_t SCAN2_MIN = 128;
__device__ __forceinline__ uint32_t scan2_slices(uint32_t k) {
  return min((uint32_t)SCAN2_S, max(1u, (k + SCAN2_MIN - 1) / SCAN2_MIN));
}
// tiles [j0, j1) of row `row` (of `rows`) in slice sl (of ns) of k tiles
__device__ __forceinline__ void scan2_share(uint32_t k, uint32_t sl, uint32_t ns, int row, int rows, uint32_t& j0,
                                            uint32_t& j1) {
  const uint32_t s0 = (uint32_t)((uint64_t)k * sl / ns), s1 = (uint32_t)((uint64_t)k * (sl + 1) / ns);
  const uint32_t share = (s1 - s0 + rows - 1) / rows;
  j0 = min(s1, s0 + row * share);
  j1 = min(s1, j0 + share);
}

__global__ void __launch_bounds__(1024)
k_scan2_sums(const uint32_t* hist2, const uint32_t* tfirst, const uint32_t* tK, int B2, uint32_t* ssum) {
  __shared__ uint64_t part[1024];
  const int P2 = 1 << B2, rows = 1024 >> B2;
  const int b1 = blockIdx.x / SCAN2_S;
  const uint32_t sl = blockIdx.x % SCAN2_S;
  const uint32_t f = tfirst[b1], k = tK[b1], ns = scan2_slices(k);
  if (ns == 1 || sl >= ns) return;
  const int col = threadIdx.x & (P2 - 1), row = threadIdx.x >> B2;
  uint32_t j0, j1;
  scan2_share(k, sl, ns, row, rows, j0, j1);
  part[threadIdx.x] = col_sum(hist2 + (uint64_t)(f + j0) * P2 + col, (uint64_t)P2, j1 - j0);
  __syncthreads();
  if (row == 0) {
    uint64_t sum = 0;
    for (int r = 0; r < rows; ++r) sum += part[(r << B2) + col];
    ssum[(uint64_t)blockIdx.x * P2 + col] = (uint32_t)sum;
  }
}

__global__ void __launch_bounds__(1024)
k_scan2(uint32_t* hist2, const uint32_t* tfirst, const uint32_t* tK, int P1, int B2, const uint32_t* ssum,
        const uint64_t* bstart1, uint64_t* bstart2) {
  __shared__ uint64_t part[1024];
  __shared__ uint64_t ctot[256];
  const int P2 = 1 << B2, rows = 1024 >> B2;
  const int b1 = blockIdx.x / SCAN2_S;
  const uint32_t sl = blockIdx.x % SCAN2_S;
  const uint32_t f = tfirst[b1], k = tK[b1], ns = scan2_slices(k);
  if (sl >= ns) return;
  const int col = threadIdx.x & (P2 - 1), row = threadIdx.x >> B2;
  uint32_t j0, j1;
  scan2_share(k, sl, ns, row, rows, j0, j1);
  uint32_t* colp = hist2 + (uint64_t)(f + j0) * P2 + col;
  part[threadIdx.x] = col_sum(colp, (uint64_t)P2, j1 - j0);
  __syncthreads();
  uint64_t run = 0;
  for (uint32_t q = 0; q < sl; ++q) run += ssum[((uint64_t)b1 * SCAN2_S + q) * P2 + col];
  for (int r = 0; r < row; ++r) run += part[(r << B2) + col];
  run = col_exscan(colp, (uint64_t)P2, j1 - j0, run);
  if (sl != ns - 1) return;           // uniform across the CTA
  if (row == rows - 1) ctot[col] = run;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x, per = (P2 + 31) / 32;
    const int c0 = min(P2, lane * per), c1 = min(P2, c0 + per);
    uint64_t sum = 0;
    for (int c = c0; c < c1; ++c) sum += ctot[c];
    uint64_t x = sum;
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    uint64_t st = bstart1[b1] + x - sum;
    for (int c = c0; c < c1; ++c) {
      bstart2[((uint64_t)b1 << B2) + c] = st;
      st += ctot[c];
    }
    if (b1 == P1 - 1 && lane == 31) bstart2[(uint64_t)P1 << B2] = bstart1[P1];
  }
}

template <int F>
__global__ void __launch_bounds__(SC_WARPS * 32)
k_scatter2(const typename RecT<F>::type* in, const Tile* tiles, const unsigned int* n_tiles, int B1, int B2,
           const uint32_t* pre2, const uint64_t* bstart2, typename RecT<F>::type* out, HeavyDev hv) {
  __shared__ uint32_t cur_all[SC_WARPS][256];
  __shared__ uint64_t hl_all[SC_WARPS][HMAXC];
  __shared__ __align__(4) uint8_t filt_all[SC_WARPS][HFILT];
  const uint32_t P2L = 1u << B2;
  const int B2e = hv.hmax ? B2 + 1 : B2;
  const int P2 = 1 << B2e;
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tile = blockIdx.x * SC_WARPS + wl;
  if (tile >= *n_tiles) return;
  const Tile tl = tiles[tile];
  uint32_t* cur = cur_all[wl];
  {
    // the tile's cursors (P2 <= 256: at most eight per lane), all loaded
    // before any is stored
    constexpr int CB = 8;
    uint64_t bs[CB];
    uint32_t po[CB];
#pragma unroll
    for (int j = 0; j < CB; ++j) {
      const int b = j * 32 + lane;
      bs[j] = b < P2 ? bstart2[((uint64_t)tl.bucket << B2e) + b] : 0ull;
      po[j] = b < P2 ? pre2[(uint64_t)tile * P2 + b] : 0u;
    }
#pragma unroll
    for (int j = 0; j < CB; ++j) {
      const int b = j * 32 + lane;
      if (b < P2) cur[b] = (uint32_t)(bs[j] + po[j]);
    }
  }
  const int nh = load_heavy(hv, tl.bucket, hl_all[wl], lane, 32);
  __syncwarp();
  if (nh) build_filter(filt_all[wl], hl_all[wl], nh, lane);
  const uint64_t* hl = hl_all[wl];
  const uint8_t* filt = filt_all[wl];
  const int sh = sub_shift<F>(B1, B2);
  const uint32_t lt = lanemask_lt();
  for (uint64_t base = tl.begin; base < tl.end; base += 32 * BATCH) {
    typename RecT<F>::type rec[BATCH];
    uint32_t b[BATCH];
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {   // all loads first, so that they are in flight together
      const uint64_t i = base + j * 32 + lane;
      rec[j] = i < tl.end ? in[i] : 0;
    }
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      const uint64_t i = base + j * 32 + lane;
      b[j] = i < tl.end ? sub_of((uint64_t)rec[j], sh, P2L, hl, filt, nh) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      const bool v = b[j] != 0xFFFFFFFFu;
      const uint32_t peers = __match_any_sync(FULL, v ? b[j] : 0xFFFFFFFFu);
      uint32_t pos = 0;
      if (v) pos = cur[b[j]] + __popc(peers & lt);
      __syncwarp();
      if (v && lane == __ffs(peers) - 1) cur[b[j]] += __popc(peers);
      __syncwarp();
      if (v && RV_INB(pos, g_caps.n)) out[pos] = rec[j];
    }
  }
}

// Level-2 split of 64-bit records, one CTA per tile of a first-level bucket:
// records stay in registers with their rank, are grouped by sub-bucket in
// shared memory, and every sub-bucket's run is written out contiguously
// (8-byte records scattered one by one from a warp waste most of each
// written sector).
template <int F>
struct Tile2Shared {
  typename RecT<F>::type orec[Tile2Len<F>::v];
  uint32_t ibr[Tile2Len<F>::v];
  uint8_t ob[Tile2Len<F>::v];
  uint32_t wcur[TB_WARPS][256];
  uint32_t loc[256];
  uint64_t gbase[256];
  uint64_t hl[HMAXC];
  alignas(4) uint8_t filt[HFILT];
  uint32_t tsum[TB_WARPS];
};

template <int F>
__global__ void __launch_bounds__(TB_THREADS, 2)
k_scatter2_tile(const typename RecT<F>::type* in, const Tile* tiles, const unsigned int* n_tiles, int B1, int B2,
                const uint32_t* pre2, const uint64_t* bstart2, typename RecT<F>::type* out, HeavyDev hv) {
  typedef typename RecT<F>::type Rec;
  constexpr int T = Tile2Len<F>::v, R = T / TB_THREADS, PER = T / TB_WARPS;
  extern __shared__ __align__(16) unsigned char tile2_smem[];
  Tile2Shared<F>& S = *reinterpret_cast<Tile2Shared<F>*>(tile2_smem);
  const uint32_t tile = blockIdx.x;
  if (tile >= *n_tiles) return;
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  const uint32_t P2L = 1u << B2;
  const int B2e = hv.hmax ? B2 + 1 : B2;
  const int P2 = 1 << B2e;
  const Tile tl = tiles[tile];
  const int len = (int)(tl.end - tl.begin);      // <= T by construction
  for (int i = threadIdx.x; i < TB_WARPS * 256; i += TB_THREADS) S.wcur[i / 256][i % 256] = 0;
  const int nh = load_heavy(hv, tl.bucket, S.hl, threadIdx.x, TB_THREADS);
  __syncthreads();
  if (nh && threadIdx.x < 32) build_filter(S.filt, S.hl, nh, (int)threadIdx.x);
  __syncthreads();
  const int sh = sub_shift<F>(B1, B2);
  const int w0 = wl * PER;
  const Rec* ip = in + tl.begin;
  Rec rec[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int i = w0 + j * 32 + lane;
    rec[j] = i < len ? ip[i] : (Rec)0;
  }
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int i = w0 + j * 32 + lane;
    const bool v = i < len;
    const uint32_t b = sub_of((uint64_t)rec[j], sh, P2L, S.hl, S.filt, nh);
    const uint32_t rank = warp_rank(b, v, S.wcur[wl], lt);
    if (v) S.ibr[i] = b | (rank << 8);
  }
  __syncthreads();
  tile_scan<256>(S.wcur, S.loc, S.tsum, P2);
  if ((int)threadIdx.x < P2)
    S.gbase[threadIdx.x] = bstart2[((uint64_t)tl.bucket << B2e) + threadIdx.x] + pre2[(uint64_t)tile * P2 + threadIdx.x];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int i = w0 + j * 32 + lane;
    if (i < len) {
      const uint32_t br = S.ibr[i], b = br & 0xFFu, pos = S.wcur[wl][b] + (br >> 8);
      S.orec[pos] = rec[j];
      S.ob[pos] = (uint8_t)b;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < len; i += TB_THREADS) {
    const uint32_t b = S.ob[i];
    const uint64_t o = S.gbase[b] + (i - S.loc[b]);
    if (RV_INB(o, g_caps.n)) out[o] = S.orec[i];
  }
}

// ------------------------------------------------------------------ fold / combine shared state
struct SlotTable {
  uint64_t tkey[HT_CAP];
  uint16_t tslot[HT_CAP];
  uint64_t skey[SLOTS];
  unsigned int nslots;
  unsigned int ovf;
};

struct OuterTable {
  uint32_t ukey[UCAP];
  uint32_t ucnt[UCAP][6];
  unsigned int nu;
  unsigned int ovf;
};

struct FinalCtx {              // per-thread tallies, reduced once per CTA
  uint32_t h0[6], h1[6];
  uint32_t nodes0, nodes1;
};

// h[v] += 1 with compile-time indices, so the tallies stay in registers
__device__ __forceinline__ void inc6(uint32_t* h, uint32_t v) {
#pragma unroll
  for (int k = 0; k < 6; ++k) h[k] += v == (uint32_t)k;
}

struct Params {
  MonitorTab tab;
  int B1, B2, nq;
  int light;           // heavy routing: sub-buckets light.. of a first-level bucket hold one binding each
  Acc* acc;
  rv_bindings out;
  int stream_mode;     // 1: fold the batch into StreamState instead of starting from q0
  StreamState ss;
};

__device__ __forceinline__ uint64_t key_mult(uint64_t key) { return key * 0x9E3779B97F4A7C15ull; }

__device__ __forceinline__ bool in_pass(uint64_t key, int bits, uint32_t value) {
  if (bits == 0) return true;
  return (uint32_t)((key_mult(key) >> 20) & ((1u << bits) - 1)) == value;
}

// Find the slot of key, inserting it if absent.  `init` runs once for a new
// slot before the slot becomes visible.  Returns -1 when the table is full.
template <typename Init>
__device__ __forceinline__ int find_or_insert(SlotTable& T, uint64_t key, Acc* acc, Init init) {
  uint32_t h = (uint32_t)(key_mult(key) >> (64 - HT_BITS));
  volatile uint64_t* vk = T.tkey;
  volatile uint16_t* vs = T.tslot;
  for (int probe = 0; probe < HT_CAP; ++probe) {
    uint64_t k = vk[h];
    if (k == EMPTY_KEY) {
      unsigned long long prev = atomicCAS((unsigned long long*)&T.tkey[h], (unsigned long long)EMPTY_KEY,
                                          (unsigned long long)key);
      if (prev == EMPTY_KEY) {
        unsigned int s = atomicAdd(&T.nslots, 1u);
        if (s >= SLOTS) {
          T.ovf = 1;
          __threadfence_block();
          vs[h] = FULL_SLOT;
          return -1;
        }
        T.skey[s] = key;
        init(s);
        __threadfence_block();
        vs[h] = (uint16_t)s;
        return (int)s;
      }
      k = prev;
    }
    if (k == key) {
      uint16_t s;
      int spins = 0;
      while ((s = vs[h]) == NO_SLOT) {
        if (++spins > SPIN_LIMIT) { atomicOr(&acc->err, ERR_SPIN); return -1; }
      }
      return s == FULL_SLOT ? -1 : (int)s;
    }
    h = (h + 1) & (HT_CAP - 1);
  }
  T.ovf = 1;
  return -1;
}

__device__ void reset_table(SlotTable& T) {
  for (int i = threadIdx.x; i < HT_CAP; i += blockDim.x) { T.tkey[i] = EMPTY_KEY; T.tslot[i] = NO_SLOT; }
  if (threadIdx.x == 0) { T.nslots = 0; T.ovf = 0; }
}

__device__ void reset_outer(OuterTable& U) {
  for (int i = threadIdx.x; i < UCAP; i += blockDim.x) {
    U.ukey[i] = 0xFFFFFFFFu;
    for (int v = 0; v < 6; ++v) U.ucnt[i][v] = 0;
  }
  if (threadIdx.x == 0) { U.nu = 0; U.ovf = 0; }
}

// linear search is enough: an outer table holds the few outer values of one bucket
__device__ int outer_slot(OuterTable& U, uint32_t u_local) {
  for (int attempt = 0; attempt < 2 * UCAP; ++attempt) {
    const unsigned int nu = min(*(volatile unsigned int*)&U.nu, (unsigned int)UCAP);
    for (unsigned int i = 0; i < nu; ++i) {
      uint32_t k;
      int spins = 0;
      while ((k = *(volatile uint32_t*)&U.ukey[i]) == 0xFFFFFFFFu) {
        if (++spins > SPIN_LIMIT) return -1;
      }
      if (k == (u_local | 0x80000000u)) return (int)i;
    }
    // claim the next entry; ukey holds u_local with the top bit set once valid
    unsigned int i = atomicCAS(&U.nu, nu, nu + 1);
    if (i == nu) {
      if (nu >= UCAP) { U.ovf = 1; return -1; }
      __threadfence_block();
      *(volatile uint32_t*)&U.ukey[nu] = u_local | 0x80000000u;
      return (int)nu;
    }
  }
  return -1;
}

// root counts of a stream move from verdict `from` (0xFF: new node) to `to`
__device__ __forceinline__ void root_delta(const Params& p, uint32_t stream, uint32_t from, uint32_t to) {
  if (from == to) return;
  if (from != 0xFFu) atomicAdd(&p.ss.root[stream * 6 + from], ~0ull);   // -1
  atomicAdd(&p.ss.root[stream * 6 + to], 1ull);
}

// Streaming: the binding continues from its stored state; a verdict change
// becomes count deltas (out of line: the plain offline fold never takes it).
template <int F>
__device__ __noinline__ void finalize_stream(const Params& p, OuterTable* U, uint64_t skey, uint64_t M, uint32_t b1) {
  const uint32_t b = p.nq == 2 ? (uint32_t)(skey & 0xFFFFFFFFull) : (uint32_t)original_key<F>(skey, b1, p.B1, p.nq);
  const uint32_t old = p.ss.bstate[b];
  const bool seen = old & 0x80u;
  const uint32_t st = seen ? (old & 15u) : (uint32_t)p.tab.q0;
  const uint32_t ns = (uint32_t)((M >> (4 * st)) & 15ull);
  const uint32_t v = p.tab.labels[ns];
  const uint32_t vold = seen ? p.ss.bverdict[b] : 0xFFu;
  p.ss.bstate[b] = (uint8_t)(0x80u | ns);
  p.ss.bverdict[b] = (uint8_t)v;
  if constexpr (F != FMT_K2) {
    root_delta(p, p.ss.bstream[b], vold, v);
  } else {
    const int ui = outer_slot(*U, (uint32_t)(skey >> 32));
    if (ui < 0) atomicOr(&p.acc->err, ERR_OUTER_FULL);
    else if (vold != v) {
      atomicAdd(&U->ucnt[ui][v], 1u);
      if (vold != 0xFFu) atomicAdd(&U->ucnt[ui][vold], 0xFFFFFFFFu);   // -1
    }
  }
}

// count verdict v under the binding's outer value (two quantifiers)
__device__ __noinline__ void count_outer(const Params& p, OuterTable* U, uint64_t skey, uint32_t v) {
  const int ui = outer_slot(*U, (uint32_t)(skey >> 32));
  if (ui < 0) atomicOr(&p.acc->err, ERR_OUTER_FULL);
  else atomicAdd(&U->ucnt[ui][v], 1u);
}

// per-binding output record
template <int F>
__device__ __noinline__ void emit_binding(const Params& p, uint64_t skey, uint32_t b1, uint32_t v) {
  unsigned long long idx = atomicAdd(&p.acc->n_out, 1ull);
  if (idx < p.out.capacity) {
    p.out.keys[idx] = original_key<F>(skey, b1, p.B1, p.nq);
    p.out.verdicts[idx] = (uint8_t)v;
  }
}

// verdict of one innermost binding whose composed map over its whole cluster is M
template <int F>
__device__ __forceinline__ void finalize_slot(const Params& p, FinalCtx& fc, OuterTable* U, uint64_t skey,
                                              uint64_t M, uint32_t bucket) {
  const uint32_t b1 = bucket >> p.B2;
  if (p.stream_mode) {
    finalize_stream<F>(p, U, skey, M, b1);
    return;
  }
  const uint32_t v = p.tab.labels[(uint32_t)((M >> (4 * p.tab.q0)) & 15ull)];
  if constexpr (F != FMT_K2) {
    inc6(fc.h0, v);
    fc.nodes0 += 1;
  } else {
    inc6(fc.h1, v);
    fc.nodes1 += 1;
    count_outer(p, U, skey, v);
  }
  if (p.out.keys) emit_binding<F>(p, skey, b1, v);
}

// after all innermost bindings of a bucket: valuate its outer nodes (level 1)
template <int F>
__device__ void finalize_outer(const Params& p, FinalCtx& fc, OuterTable* Up, uint32_t bucket) {
  if constexpr (F != FMT_K2) return;
  else {
  OuterTable& U = *Up;
  const unsigned int nu = min(U.nu, (unsigned int)UCAP);
  const uint32_t b1 = bucket >> p.B2;
  for (unsigned int i = threadIdx.x; i < nu; i += blockDim.x) {
    uint64_t v6[6];
    if (p.stream_mode) {
      // all bindings of an outer node share this bucket, so this CTA owns the node
      const uint32_t o = original_outer<F>(U.ukey[i] & 0x7FFFFFFFu, b1, p.B1);
      for (int v = 0; v < 6; ++v) {
        const uint32_t c = p.ss.ocounts[(uint64_t)o * 6 + v] + U.ucnt[i][v];
        p.ss.ocounts[(uint64_t)o * 6 + v] = c;
        v6[v] = c;
      }
      const uint32_t vd = (uint32_t)rvv::valuate(p.tab.q[1].kind, p.tab.q[1].op, p.tab.q[1].num, p.tab.q[1].den, v6);
      const uint32_t vold = p.ss.overdict[o];
      p.ss.overdict[o] = (uint8_t)vd;
      root_delta(p, p.ss.ostream[o], vold, vd);
      continue;
    }
    for (int v = 0; v < 6; ++v) v6[v] = U.ucnt[i][v];
    const int vd = rvv::valuate(p.tab.q[1].kind, p.tab.q[1].op, p.tab.q[1].num, p.tab.q[1].den, v6);
    inc6(fc.h0, (uint32_t)vd);
    fc.nodes0 += 1;
    if (p.out.outer_keys) {
      unsigned long long idx = atomicAdd(&p.acc->n_out_outer, 1ull);
      if (idx < p.out.outer_capacity) {
        p.out.outer_keys[idx] = original_outer<F>(U.ukey[i] & 0x7FFFFFFFu, b1, p.B1);
        p.out.outer_verdicts[idx] = (uint8_t)vd;
      }
    }
  }
  }
}

__device__ void flush_final(const Params& p, FinalCtx& fc) {
  uint32_t v[14];
  for (int i = 0; i < 6; ++i) { v[i] = fc.h0[i]; v[6 + i] = fc.h1[i]; }
  v[12] = fc.nodes0;
  v[13] = fc.nodes1;
  for (int i = 0; i < 14; ++i) {
    uint32_t x = __reduce_add_sync(FULL, v[i]);
    if ((threadIdx.x & 31) == 0 && x) {
      unsigned long long* dst = i < 6 ? &p.acc->level_counts[0][i]
                                : i < 12 ? &p.acc->level_counts[1][i - 6]
                                         : &p.acc->n_nodes[i - 12];
      atomicAdd(dst, (unsigned long long)x);
    }
  }
}

__device__ __forceinline__ void clear_final(FinalCtx& fc) {
  for (int i = 0; i < 6; ++i) { fc.h0[i] = 0; fc.h1[i] = 0; }
  fc.nodes0 = fc.nodes1 = 0;
}

// ------------------------------------------------------------------ fold
// Capacities of one fold CTA.  Records of one 32-bit key are small, so a unit
// holds more of them; a 64-bit or two-variable key brings larger binding
// tables (a nested trace has a few hundred innermost bindings per bucket).
template <int F> struct FoldCfg {
  static constexpr int UNIT = 8192, SL = 1024, HTB = 11, RB = 8, MINB = 2;
};
template <> struct FoldCfg<FMT_K32> {   // records come from shared memory: no load batching
  static constexpr int UNIT = 8192, SL = 512, HTB = 10, RB = 1, MINB = 3;
};

// A record's fold word: letter | slot << 8 | rank << 18, or letter | PK_OUT
// for a record outside the current pass.  The rank of a record is its index
// among the records of its slot in its warp's slice, so 10 bits suffice for
// slices of at most 1024 records.
constexpr uint32_t PK_OUT = 1u << 28;
constexpr uint16_t NO_POS = 0xFFFF;
static_assert(FoldCfg<FMT_K32>::UNIT / FOLD_WARPS <= 1024 && FoldCfg<FMT_K64>::UNIT / FOLD_WARPS <= 1024,
              "ranks are 10 bits");
static_assert(FoldCfg<FMT_K64>::SL <= 1024 && FoldCfg<FMT_K32>::SL <= 1024, "slots are 10 bits");

struct NoOuter {};

template <int F>
struct FoldShared {
  static constexpr int UNIT = FoldCfg<F>::UNIT, SL = FoldCfg<F>::SL, HT = 1 << FoldCfg<F>::HTB;
  static constexpr bool PACKED = F == FMT_K32;     // table entry = key << 32 | slot
  uint64_t lmap[RV_MAX_LETTERS];
  // fold word of every record of the unit; 32-bit records arrive here by one
  // bulk copy (16-byte aligned, so up to 4 extra records at either end)
  uint32_t pk[UNIT + 8];
  uint8_t sorted[UNIT];                // letters grouped by slot, trace order kept
  uint8_t vslot[SL];                   // verdict of every slot (two quantifiers: counted after the pass)
  uint64_t tkey[HT];
  uint16_t tslot[PACKED ? 2 : HT];     // slot of tkey[h] (64-bit keys)
  uint64_t skey[SL];                   // key of every slot
  uint16_t hpos[SL];                   // table position of every slot (NO_POS: none)
  uint16_t wc[FOLD_WARPS][SL];         // per-warp counts of every slot, then cursors
  uint32_t seg[SL + 1];                // run of every slot in `sorted`
  uint64_t firstmap[FOLD_THREADS];     // map of a piece's first run when that run began earlier
  uint64_t lastval[FOLD_THREADS];      // state or map of a piece's last run when it goes on
  uint64_t wmaps[FOLD_WARPS];
  uint32_t tsum[FOLD_WARPS];
  typename std::conditional<F == FMT_K2, OuterTable, NoOuter>::type U;
  Tile tile, ntile;                    // current and next unit
  unsigned int cur, ncur;
  uint64_t mbar;                       // completion of the bulk copy
  unsigned int bad;
  unsigned int nslots, ovf;
  int npass;
  uint32_t pass_bits[64], pass_val[64];
  uint64_t item_off;
  uint32_t item_cnt;
};

// MINB CTAs per SM must fit the SM's 228 KB of shared memory (1 KB of it reserved per CTA)
static_assert(FoldCfg<FMT_K32>::MINB * (sizeof(FoldShared<FMT_K32>) + 1024) <= 228 * 1024, "fold CTAs per SM");
static_assert(3 * (sizeof(TileShared<FMT_K32>) + 1024) <= 228 * 1024, "three level-1 tiles per SM");
static_assert(3 * (sizeof(TileShared<FMT_K64>) + 1024) <= 228 * 1024, "three level-1 tiles per SM");
static_assert(FoldCfg<FMT_K64>::MINB * (sizeof(FoldShared<FMT_K64>) + 1024) <= 228 * 1024, "fold CTAs per SM");
static_assert(FoldCfg<FMT_K2>::MINB * (sizeof(FoldShared<FMT_K2>) + 1024) <= 228 * 1024, "fold CTAs per SM");

template <int F>
__device__ __forceinline__ OuterTable* outer_of(FoldShared<F>& S) {
  if constexpr (F == FMT_K2) return &S.U;
  else return nullptr;
}

// a binding key inside a bucket: 24 bits for one 32-bit key, 56 otherwise
template <int F> using FKey = typename std::conditional<F == FMT_K32, uint32_t, uint64_t>::type;

template <int F>
__device__ __forceinline__ uint32_t fold_home(FKey<F> key) {
  // the low bits of a mixed key are uniform; a two-variable key carries the
  // raw inner value there, so it is hashed again
  if constexpr (F == FMT_K2) return (uint32_t)(key_mult(key) >> (64 - FoldCfg<F>::HTB));
  else return (uint32_t)key & ((1u << FoldCfg<F>::HTB) - 1);
}

constexpr int PROBE_NEED = -2;   // key absent: the probe ended at an empty entry
// low word of a 32-bit-key entry while its slot is being taken, and when the
// slot table was full
constexpr uint32_t E_PENDING = 0xFFFFFFFFu, E_FULL = 0xFFFFFFFEu;

// Slot stored with (or beside) the table entry at h whose key matched; waits,
// boundedly, while the inserting lane publishes it.  -1: no slot.
template <int F>
__device__ __forceinline__ int fold_entry_slot(FoldShared<F>& S, uint32_t h, uint64_t e, Acc* acc) {
  int spins = 0;
  if constexpr (FoldShared<F>::PACKED) {
    volatile uint64_t* vk = S.tkey;
    while ((uint32_t)e == E_PENDING) {
      if (++spins > SPIN_LIMIT) { atomicOr(&acc->err, ERR_SPIN); return -1; }
      e = vk[h];
    }
    return (uint32_t)e == E_FULL ? -1 : (int)(uint32_t)e;
  } else {
    volatile uint16_t* vs = S.tslot;
    uint16_t sl;
    while ((sl = vs[h]) == NO_SLOT) {
      if (++spins > SPIN_LIMIT) { atomicOr(&acc->err, ERR_SPIN); return -1; }
    }
    return sl == FULL_SLOT ? -1 : (int)sl;
  }
}

template <int F>
__device__ __forceinline__ bool fold_key_is(uint64_t e, FKey<F> key) {
  if constexpr (FoldShared<F>::PACKED) return (uint32_t)(e >> 32) == key;
  else return e == key;
}

// Lookup without insertion: the slot of key, PROBE_NEED, or -1 (table full or
// a bounded wait gave up).
template <int F>
__device__ __forceinline__ int fold_probe(FoldShared<F>& S, FKey<F> key, Acc* acc) {
  constexpr int HT = FoldShared<F>::HT;
  uint32_t h = fold_home<F>(key);
  volatile uint64_t* vk = S.tkey;
  for (int probe = 0; probe < HT; ++probe) {
    const uint64_t e = vk[h];
    if (e == EMPTY_KEY) return PROBE_NEED;
    if (fold_key_is<F>(e, key)) return fold_entry_slot<F>(S, h, e, acc);
    h = (h + 1) & (HT - 1);
  }
  S.ovf = 1;
  return -1;
}

// Insertion by one lane: the entry is claimed first, then a slot number is
// taken and published; lanes that meet the claimed entry wait for it.
// Returns -1 when the slot table is full (the pass then restarts split).
template <int F>
__device__ __noinline__ int fold_insert(FoldShared<F>& S, FKey<F> key, Acc* acc) {
  constexpr int HT = FoldShared<F>::HT, SL = FoldShared<F>::SL;
  constexpr bool PK = FoldShared<F>::PACKED;
  uint32_t h = fold_home<F>(key);
  volatile uint64_t* vk = S.tkey;
  for (int probe = 0; probe < HT; ++probe) {
    uint64_t e = vk[h];
    if (e == EMPTY_KEY) {
      const uint64_t claim = PK ? ((uint64_t)key << 32) | E_PENDING : (uint64_t)key;
      const unsigned long long prev = atomicCAS((unsigned long long*)&S.tkey[h], (unsigned long long)EMPTY_KEY,
                                                (unsigned long long)claim);
      if (prev == EMPTY_KEY) {
        const unsigned int s = atomicAdd(&S.nslots, 1u);
        const bool full = s >= (unsigned int)SL;
        if (full) S.ovf = 1;
        else { S.skey[s] = key; S.hpos[s] = (uint16_t)h; }
        __threadfence_block();
        if constexpr (PK) vk[h] = ((uint64_t)key << 32) | (full ? E_FULL : s);
        else *(volatile uint16_t*)&S.tslot[h] = full ? FULL_SLOT : (uint16_t)s;
        return full ? -1 : (int)s;
      }
      e = prev;
    }
    if (fold_key_is<F>(e, key)) return fold_entry_slot<F>(S, h, e, acc);
    h = (h + 1) & (HT - 1);
  }
  S.ovf = 1;
  return -1;
}

// Slot of every lane's key: a probe, then an insertion for keys not yet in
// the table.  Lanes insert in parallel; lanes holding the same new key meet
// at the entry the first of them claimed and wait for its slot.
template <int F>
__device__ __forceinline__ int warp_slot(FoldShared<F>& S, FKey<F> key, bool want, Acc* acc) {
  int slot = want ? fold_probe<F>(S, key, acc) : -1;
  if (slot == PROBE_NEED) slot = fold_insert<F>(S, key, acc);
  return slot;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// One-shot bulk copy global -> shared that completes on an mbarrier (the
// barrier expects `bytes`; both addresses and the size are multiples of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Wait for phase `parity` of the mbarrier, for at most about a second.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(a), "r"(parity)
                 : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

// A binding that a single unit holds whole: tallied now; for two quantifiers
// its verdict is counted under its outer binding after the pass, with equal
// (outer, verdict) pairs of a warp added at once.
template <int F>
__device__ __forceinline__ void fold_finalize(const Params& p, FinalCtx& fc, FoldShared<F>& S, int s, uint64_t skey,
                                              uint64_t M, uint32_t bucket) {
  if constexpr (F == FMT_K2) {
    if (!p.stream_mode) {
      const uint32_t v = p.tab.labels[(uint32_t)((M >> (4 * p.tab.q0)) & 15ull)];
      inc6(fc.h1, v);
      fc.nodes1 += 1;
      S.vslot[s] = (uint8_t)v;
      if (p.out.keys) emit_binding<F>(p, skey, bucket >> p.B2, v);
      return;
    }
  }
  finalize_slot<F>(p, fc, outer_of(S), skey, M, bucket);
}

// Fold of one unit (a contiguous range of one bucket's records):
// (1) every warp takes a contiguous slice and gives each record its slot and
//     its rank among the slot's records of the slice (ballot match per round);
// (2) one scan over (slot, warp) turns the per-warp counts into cursors;
// (3) each letter goes to cursor + rank, so the unit's letters are grouped by
//     binding with trace order kept;
// (4) each binding's run is folded: every thread an equal piece, runs that
//     cross pieces joined in order (plain state steps when the run starts at
//     the bucket's start, map composition otherwise).
// The key of the unit's first record is a candidate for a dominant binding
// (a Zipf head): when it holds at least half of the unit its records stay in
// place and are folded as contiguous pieces instead of being sorted.
template <int F>
__global__ void __launch_bounds__(FOLD_THREADS, FoldCfg<F>::MINB)
k_fold(const typename RecT<F>::type* recs, const Tile* units, const unsigned int* n_units, Params p,
       Item* items, Pair* pool) {
  typedef typename RecT<F>::type Rec;
  constexpr int SL = FoldCfg<F>::SL, HT = 1 << FoldCfg<F>::HTB, RB = FoldCfg<F>::RB;
  extern __shared__ __align__(16) unsigned char fold_smem[];
  FoldShared<F>& S = *reinterpret_cast<FoldShared<F>*>(fold_smem);
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31, nthr = FOLD_THREADS;
  const int ns = p.tab.n_states;
  const uint32_t lt = lanemask_lt();
  for (int i = threadIdx.x; i < RV_MAX_LETTERS; i += nthr) S.lmap[i] = p.tab.maps[i];
  for (int i = threadIdx.x; i < HT; i += nthr) {
    S.tkey[i] = EMPTY_KEY;
    if constexpr (!FoldShared<F>::PACKED) S.tslot[i] = NO_SLOT;
  }
  for (int i = threadIdx.x; i < FOLD_WARPS * SL; i += nthr) S.wc[i / SL][i % SL] = 0;
  FinalCtx fc;
  clear_final(fc);
  const unsigned int nun = *n_units;
  constexpr bool BULK = F == FMT_K32;   // records reach shared memory by a bulk copy
  uint32_t bulk_phase = 0;
  if (threadIdx.x == 0) {
    S.cur = atomicAdd(&p.acc->next_unit, 1u);
    if (S.cur < nun) S.tile = units[S.cur];
    S.bad = 0;
    if constexpr (BULK) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.mbar)) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  while (true) {
    __syncthreads();
    const unsigned int u = S.cur;
    if (u >= nun || S.bad) break;
    const Tile t = S.tile;
    unsigned int nxt = 0;
    Tile tn{};
    if (threadIdx.x == 0) nxt = atomicAdd(&p.acc->next_unit, 1u);   // claimed now, used at the end
    bool ahead = false;                                             // next unit looked up yet
    const bool single = t.K == 1;
    const bool use_state = single && !p.stream_mode;   // a single unit starting at q0: plain states
    const bool one_key = p.light && (int)(t.bucket & ((1u << p.B2) - 1)) >= p.light;
    const int len = (int)(t.end - t.begin);            // <= FoldCfg<F>::UNIT by construction
    if (threadIdx.x == 0) {
      S.npass = 1; S.pass_bits[0] = 0; S.pass_val[0] = 0;
      S.item_cnt = 0;
      S.item_off = single ? 0 : atomicAdd(&p.acc->pair_top[0], (unsigned long long)len);
    }
    if constexpr (F == FMT_K2) {
      if (t.k == 0) reset_outer(S.U);
    }
    const int per = (len + FOLD_WARPS - 1) / FOLD_WARPS;
    const int w0 = min(len, wl * per), w1 = min(len, w0 + per);
    // 32-bit records: the unit's records, copied in whole 16-byte words
    const char* ra = (const char*)(recs + t.begin);
    const char* ra16 = (const char*)((uintptr_t)ra & ~(uintptr_t)15);
    const uint32_t rbytes = (uint32_t)((((uintptr_t)(recs + t.end) + 15) & ~(uintptr_t)15) - (uintptr_t)ra16);
    uint32_t* P = S.pk + (BULK ? (ra - ra16) / 4 : 0);   // fold word of record i: P[i]
    FKey<F> cand = BULK ? 0 : (FKey<F>)((uint64_t)recs[t.begin] >> 8);
    while (true) {
      __syncthreads();
      if (S.npass == 0) break;
      const int bits = (int)S.pass_bits[S.npass - 1];
      const uint32_t val = S.pass_val[S.npass - 1];
      if constexpr (BULK) {
        // every pass reads the records afresh: the previous one overwrote them
        if (threadIdx.x == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          bulk_load(S.pk, ra16, rbytes, &S.mbar);
        }
        if (!mbar_wait(&S.mbar, bulk_phase)) atomicOr(&S.bad, 1u);
        bulk_phase ^= 1u;
        cand = (FKey<F>)(P[0] >> 8);
      }
      const bool cand_in = in_pass(cand, bits, val);
      if (threadIdx.x == 0) {
        // slot 0 belongs to the candidate; its records never touch the table
        S.nslots = cand_in ? 1u : 0u;
        S.ovf = 0;
        if (cand_in) { S.skey[0] = cand; S.hpos[0] = NO_POS; }
      }
      __syncthreads();
      if (S.bad) {
        // the copy never completed: report, give it another bounded wait, stop
        if (threadIdx.x == 0) {
          atomicOr(&p.acc->err, ERR_SPIN);
          mbar_wait(&S.mbar, bulk_phase ^ 1u);
        }
        break;
      }
      if (one_key) {
        // a heavy binding's own sub-bucket: fold the unit in place, in pieces
        const int c = ((len + nthr - 1) / nthr) | 1;   // odd: conflict-free reads across the warp
        const int a = min(len, (int)threadIdx.x * c), z = min(len, a + c);
        uint64_t M = IDENTITY_MAP;
        for (int i = a; i < z; ++i) {
          const uint32_t l = BULK ? P[i] & 0xFFu : (uint32_t)((uint64_t)recs[t.begin + i] & 0xFFu);
          M = apply_map(M, S.lmap[l], ns);
        }
        for (int off = 1; off < 32; off <<= 1) {
          const uint64_t o = __shfl_down_sync(FULL, M, off);
          if ((lane & (2 * off - 1)) == 0) M = apply_map(M, o, ns);
        }
        if (lane == 0) S.wmaps[wl] = M;
        __syncthreads();
        if (threadIdx.x == 0) {
          uint64_t T = S.wmaps[0];
          for (int w = 1; w < FOLD_WARPS; ++w) T = apply_map(T, S.wmaps[w], ns);
          if (single) fold_finalize<F>(p, fc, S, 0, (uint64_t)cand, T, t.bucket);
          else if (RV_INB(S.item_off, g_caps.pool)) pool[S.item_off] = Pair{(uint64_t)cand, T};
          S.item_cnt = 1;
          S.npass = 0;
        }
        continue;
      }
      // 1. slot and rank of every record of this warp's slice
#pragma unroll 1
      for (int base = w0; base < w1; base += 32 * RB) {
        Rec r[RB];
#pragma unroll
        for (int j = 0; j < RB; ++j) {
          const int i = base + j * 32 + lane;
          r[j] = i < w1 ? (BULK ? (Rec)P[i] : recs[t.begin + i]) : (Rec)0;
        }
#pragma unroll
        for (int j = 0; j < RB; ++j) {
          if (base + j * 32 >= w1) break;                  // warp-uniform
          const int i = base + j * 32 + lane;
          const bool valid = i < w1;
          const FKey<F> key = (FKey<F>)((uint64_t)r[j] >> 8);
          const uint32_t letter = (uint32_t)r[j] & 0xFFu;
          const bool in = valid && in_pass(key, bits, val);
          const bool is_cand = in && cand_in && key == cand;
          if (__all_sync(FULL, is_cand || !valid)) {
            // a round of the candidate only (the common case under a Zipf head)
            const uint32_t vm = __ballot_sync(FULL, valid);
            uint32_t old = 0;
            if (lane == 0) {
              old = S.wc[wl][0];
              S.wc[wl][0] = (uint16_t)(old + __popc(vm));
            }
            old = __shfl_sync(FULL, old, 0);
            if (valid) P[i] = letter | ((old + __popc(vm & lt)) << 18);
            continue;
          }
          int slot = warp_slot<F>(S, key, in && !is_cand, p.acc);
          if (is_cand) slot = 0;
          const bool v = slot >= 0;
          const uint32_t peers = __match_any_sync(FULL, v ? (uint32_t)slot : 0xFFFFFFFFu);
          const int ld = __ffs(peers) - 1;
          uint32_t old = 0;
          if (v && lane == ld) {
            old = S.wc[wl][slot];
            S.wc[wl][slot] = (uint16_t)(old + __popc(peers));
          }
          old = __shfl_sync(FULL, old, ld);
          if (valid) P[i] = v ? (letter | ((uint32_t)slot << 8) | ((old + __popc(peers & lt)) << 18)) : (letter | PK_OUT);
        }
      }
      __syncthreads();
      if (!ahead && threadIdx.x == 0) tn = units[nxt < nun ? nxt : nun - 1];   // completes during the scan and placement
      const unsigned int nsl_all = min(S.nslots, (unsigned int)SL);
      if (S.ovf) {
        // too many bindings: clear, then fold this unit in two passes split by a key bit
        for (int i = threadIdx.x; i < HT; i += nthr) {
          S.tkey[i] = EMPTY_KEY;
          if constexpr (!FoldShared<F>::PACKED) S.tslot[i] = NO_SLOT;
        }
        for (unsigned int s = threadIdx.x; s < nsl_all; s += nthr)
          for (int w = 0; w < FOLD_WARPS; ++w) S.wc[w][s] = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
          S.npass -= 1;
          if (bits >= 20 || S.npass + 2 > 64) {
            atomicOr(&p.acc->err, ERR_SPIN);
            S.npass = 0;
          } else {
            S.pass_bits[S.npass] = bits + 1; S.pass_val[S.npass] = val;
            S.pass_bits[S.npass + 1] = bits + 1; S.pass_val[S.npass + 1] = val | (1u << bits);
            S.npass += 2;
          }
        }
        continue;
      }
      const int nsl = (int)nsl_all;
      // 2. dominant candidate?  then the exclusive scan over (slot, warp)
      uint32_t c0 = 0;
      if (cand_in)
        for (int w = 0; w < FOLD_WARPS; ++w) c0 += S.wc[w][0];
      const bool dom = cand_in && 2 * c0 >= (uint32_t)len;
      {
        const int spt = (nsl + nthr - 1) / nthr;
        const int s0 = min(nsl, (int)threadIdx.x * spt), s1 = min(nsl, s0 + spt);
        uint32_t sum = 0;
        for (int s = s0; s < s1; ++s)
          if (!(dom && s == 0))
            for (int w = 0; w < FOLD_WARPS; ++w) sum += S.wc[w][s];
        uint32_t x = sum;
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(FULL, x, o);
          if (lane >= o) x += y;
        }
        if (lane == 31) S.tsum[wl] = x;
        __syncthreads();
        uint32_t run = x - sum;
        for (int w = 0; w < wl; ++w) run += S.tsum[w];
        for (int s = s0; s < s1; ++s) {
          S.seg[s] = run;
          const bool skip = dom && s == 0;
          for (int w = 0; w < FOLD_WARPS; ++w) {
            const uint32_t c = skip ? 0u : S.wc[w][s];
            S.wc[w][s] = (uint16_t)run;
            run += c;
          }
        }
        if (threadIdx.x == nthr - 1) S.seg[nsl] = run;   // records placed in this pass
      }
      __syncthreads();
      // 3. stable placement: cursor of (warp, slot) + rank
      for (int i = w0 + lane; i < w1; i += 32) {
        const uint32_t w = P[i];
        const uint32_t s = (w >> 8) & 1023u;
        if ((w & PK_OUT) || (dom && s == 0)) continue;
        S.sorted[S.wc[wl][s] + ((w >> 18) & 1023u)] = (uint8_t)w;
      }
      if (!ahead && threadIdx.x == 0) { S.ntile = tn; S.ncur = nxt; }
      __syncthreads();
      // 4. runs: every thread folds an equal piece of the sorted letters; a run
      // inside one piece is finished there, a run across pieces is joined below
      const uint32_t TOT = S.seg[nsl];
      const uint32_t C = ((TOT + nthr - 1) / nthr) | 1u;     // odd: the threads' pieces start in distinct banks
      const uint32_t pa = min(TOT, threadIdx.x * C), pz = min(TOT, pa + C);
      if (pa < pz) {
        int lo = 0, hi = nsl - 1;                 // last slot whose run starts at or before pa
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (S.seg[mid] <= pa) lo = mid; else hi = mid - 1;
        }
        int sl = lo;
        uint32_t pos = pa;
        while (pos < pz) {
          const uint32_t rs = S.seg[sl], re = S.seg[sl + 1];
          const uint32_t end = min(pz, re);
          if (end > pos) {
            const bool starts = pos == rs, ends = end == re;
            uint64_t V;
            if (use_state && starts) {
              uint32_t st = (uint32_t)p.tab.q0;
              for (uint32_t j = pos; j < end; ++j) st = step_state(st, S.lmap[S.sorted[j]]);
              V = (uint64_t)st << (4 * p.tab.q0);   // nibble q0 carries the state
            } else {
              V = IDENTITY_MAP;
              for (uint32_t j = pos; j < end; ++j) V = apply_map(V, S.lmap[S.sorted[j]], ns);
            }
            if (starts && ends) {
              if (single) fold_finalize<F>(p, fc, S, sl, S.skey[sl], V, t.bucket);
              else if (RV_INB(S.item_off + S.item_cnt + sl, g_caps.pool)) pool[S.item_off + S.item_cnt + sl] = Pair{S.skey[sl], V};
            } else if (!starts) {
              S.firstmap[threadIdx.x] = V;          // continues a run begun in an earlier piece
            } else {
              S.lastval[threadIdx.x] = V;           // begins a run that goes on
            }
          }
          pos = end;
          ++sl;
        }
      }
      __syncthreads();
      if (!ahead) {
        // the next unit's records go to L2 while this one is folded
        ahead = true;
        if (S.ncur < nun) {
          const Tile& x = S.ntile;
          const char* a = (const char*)(recs + x.begin);
          const char* z = (const char*)(recs + x.end);
          const char* line = (const char*)((uintptr_t)a & ~(uintptr_t)127) + 128 * (size_t)threadIdx.x;
          if (line < z) asm volatile("prefetch.L2 [%0];" ::"l"(line));
          if (line + 128 * nthr < z) asm volatile("prefetch.L2 [%0];" ::"l"(line + 128 * nthr));
        }
      }
      // join runs that cross pieces: the piece where a run begins composes the
      // first-run maps of the following pieces in order
      if (pa < pz) {
        int lo = 0, hi = nsl - 1;                 // slot of the run holding position pz - 1
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (S.seg[mid] <= pz - 1) lo = mid; else hi = mid - 1;
        }
        const int sl = lo;
        const uint32_t rs = S.seg[sl], re = S.seg[sl + 1];
        if (re > pz && rs >= pa) {                // my last run begins here and goes on
          uint64_t V = S.lastval[threadIdx.x];
          for (uint32_t q = threadIdx.x + 1; q < (uint32_t)nthr && q * C < re; ++q) {
            const uint64_t Mq = S.firstmap[q];
            if (use_state) {
              const uint32_t st = step_state((uint32_t)((V >> (4 * p.tab.q0)) & 15ull), Mq);
              V = (uint64_t)st << (4 * p.tab.q0);
            } else {
              V = apply_map(V, Mq, ns);
            }
          }
          if (single) fold_finalize<F>(p, fc, S, sl, S.skey[sl], V, t.bucket);
          else if (RV_INB(S.item_off + S.item_cnt + sl, g_caps.pool)) pool[S.item_off + S.item_cnt + sl] = Pair{S.skey[sl], V};
        }
      }
      // the dominant candidate: each thread folds its contiguous piece of the
      // unit in trace order, pieces are combined in order
      if (dom) {
        const int c = ((len + nthr - 1) / nthr) | 1;     // odd: conflict-free reads across the warp
        const int a = min(len, (int)threadIdx.x * c), z = min(len, a + c);
        uint64_t M = IDENTITY_MAP;
        for (int i = a; i < z; ++i) {
          const uint32_t w = P[i];
          if ((w & (PK_OUT | (1023u << 8))) == 0) M = apply_map(M, S.lmap[w & 0xFFu], ns);
        }
        for (int off = 1; off < 32; off <<= 1) {
          const uint64_t o = __shfl_down_sync(FULL, M, off);
          if ((lane & (2 * off - 1)) == 0) M = apply_map(M, o, ns);
        }
        if (lane == 0) S.wmaps[wl] = M;
        __syncthreads();
        if (threadIdx.x == 0) {
          uint64_t T = S.wmaps[0];
          for (int w = 1; w < FOLD_WARPS; ++w) T = apply_map(T, S.wmaps[w], ns);
          if (single) fold_finalize<F>(p, fc, S, 0, S.skey[0], T, t.bucket);
          else if (RV_INB(S.item_off + S.item_cnt, g_caps.pool)) pool[S.item_off + S.item_cnt + 0] = Pair{S.skey[0], T};
        }
      }
      if constexpr (F == FMT_K2) {
        if (single && !p.stream_mode) {
          __syncthreads();                   // every binding of this pass has its verdict
          for (int base = 0; base < nsl; base += nthr) {
            const int s = base + (int)threadIdx.x;
            uint32_t code = 0xFFFFFFFFu;
            if (s < nsl) {
              const int ui = outer_slot(S.U, (uint32_t)(S.skey[s] >> 32));
              if (ui < 0) atomicOr(&p.acc->err, ERR_OUTER_FULL);
              else code = ((uint32_t)ui << 3) | S.vslot[s];
            }
            const uint32_t peers = __match_any_sync(FULL, code);
            if (code != 0xFFFFFFFFu && lane == __ffs(peers) - 1)
              atomicAdd(&S.U.ucnt[code >> 3][code & 7u], (uint32_t)__popc(peers));
          }
        }
      }
      // clear the table entries and counters this pass used
      for (int s = threadIdx.x; s < nsl; s += nthr) {
        const uint16_t hp = S.hpos[s];
        if (hp != NO_POS) {
          S.tkey[hp] = EMPTY_KEY;
          if constexpr (!FoldShared<F>::PACKED) S.tslot[hp] = NO_SLOT;
        }
        for (int w = 0; w < FOLD_WARPS; ++w) S.wc[w][s] = 0;
      }
      __syncthreads();
      if (threadIdx.x == 0) { S.item_cnt += (uint32_t)nsl; S.npass -= 1; }
    }
    __syncthreads();
    if (single) finalize_outer<F>(p, fc, outer_of(S), t.bucket);
    else if (threadIdx.x == 0) items[u] = Item{S.item_off, S.item_cnt, 0};
    if (threadIdx.x == 0) {
      // a unit whose first pass overflowed never looked ahead: do it now
      if (!ahead) { S.ntile = units[nxt < nun ? nxt : nun - 1]; S.ncur = nxt; }
      S.cur = S.ncur;
      S.tile = S.ntile;
    }
  }
  __syncthreads();
  flush_final(p, fc);
}

// Groups of up to GC consecutive items of every bucket still holding K >= 2
// items are combined level by level; a bucket that ends up with one group is
// finalised by it.  The buckets that more than one unit folds, listed once after k_fold (in
// any order) with their unit counts and first units; the combine levels work
// on this short list instead of on every bucket.
__global__ void k_list_multi(const uint32_t* K, const uint32_t* first, int P, unsigned int* m, uint32_t* ids,
                             uint32_t* K0, uint32_t* F0) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= P || K[b] < 2) return;
  const unsigned int i = atomicAdd(m, 1u);
  ids[i] = (uint32_t)b;
  K0[i] = K[b];
  F0[i] = first[b];
}

// One CTA builds the next level's groups of every listed bucket: K_out[i] =
// ceil(K_in[i] / GC) groups for a bucket of K_in[i] >= 2 items (none for
// fewer), first_out[i] their exclusive prefix, the groups themselves and
// their number.  Chunks of GRP_CH entries are staged in shared memory (padded
// by one word per 32 entries) and every thread scans a run of GRP_RUN.
constexpr int GRP_RUN = 8;
constexpr int GRP_CH = GRP_RUN * 1024;
__global__ void __launch_bounds__(1024)
k_groups(const uint32_t* first_in, const uint32_t* K_in, const unsigned int* m, const uint32_t* ids, uint32_t* first_out,
         uint32_t* K_out, Group* groups, unsigned int* n_groups) {
  __shared__ uint32_t sg[GRP_CH + GRP_CH / 32];
  __shared__ uint32_t wsum[32];
  const unsigned int M = *m;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  uint32_t carry = 0;
  for (unsigned int base = 0; base < M; base += GRP_CH) {
    const int len = (int)min((unsigned int)GRP_CH, M - base);
    uint32_t kk[GRP_RUN];
#pragma unroll
    for (int r = 0; r < GRP_RUN; ++r) {
      const int i = t + r * 1024;
      kk[r] = i < len ? K_in[base + i] : 0u;
      if (i < len) sg[i + (i >> 5)] = kk[r] >= 2 ? (kk[r] + GC - 1) / GC : 0u;
    }
    __syncthreads();
    const int i0 = t * GRP_RUN;
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < GRP_RUN; ++j) {
      const int i = i0 + j;
      sum += i < len ? sg[i + (i >> 5)] : 0u;
    }
    uint32_t x = sum;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      uint32_t z = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, z, o);
        if (lane >= o) z += y;
      }
      wsum[lane] = z;
    }
    __syncthreads();
    uint32_t run = carry + x - sum + (w ? wsum[w - 1] : 0u);
#pragma unroll
    for (int j = 0; j < GRP_RUN; ++j) {
      const int i = i0 + j;
      if (i < len) {
        const uint32_t g = sg[i + (i >> 5)];
        sg[i + (i >> 5)] = run;
        run += g;
      }
    }
    carry += wsum[31];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < GRP_RUN; ++r) {
      const int i = t + r * 1024;
      if (i >= len) continue;
      const unsigned int e = base + i;
      const uint32_t k = kk[r], g = k >= 2 ? (k + GC - 1) / GC : 0u, first = sg[i + (i >> 5)];
      K_out[e] = g;
      first_out[e] = first;
      if (!g) continue;
      const uint32_t f0 = first_in[e], bucket = ids[e];
      for (uint32_t j = 0; j < g; ++j) {
        Group G;
        G.bucket = bucket;
        G.first = f0 + j * GC;
        G.cnt = min((uint32_t)GC, k - j * GC);
        G.k = j; G.K = g; G.pad = 0;
        groups[first + j] = G;
      }
    }
    __syncthreads();
  }
  if (t == 0) *n_groups = carry;
}

struct CombineShared {
  uint64_t smap[SLOTS];
  SlotTable T;
  OuterTable U;
  uint32_t pass_bits[64], pass_val[64];
  Item items[GC];            // the group's items
  int npass;
  uint64_t out_off;
  uint32_t out_cnt;
};

template <int F>
__global__ void __launch_bounds__(FOLD_THREADS)
k_combine(const Item* items_in, const Pair* pool_in, const Group* groups, const unsigned int* n_groups,
          unsigned int* next_group, Params p, Item* items_out, Pair* pool_out, int dst) {
  extern __shared__ __align__(16) unsigned char comb_smem[];
  CombineShared& S = *reinterpret_cast<CombineShared*>(comb_smem);
  const int ns = p.tab.n_states;
  FinalCtx fc;
  clear_final(fc);
  __shared__ unsigned int s_next;
  const unsigned int ng = *n_groups;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_next = atomicAdd(next_group, 1u);
    __syncthreads();
    const unsigned int g = s_next;
    if (g >= ng) break;
    const Group G = groups[g];
    const bool final_ = G.K == 1;
    if (threadIdx.x < G.cnt) S.items[threadIdx.x] = items_in[G.first + threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t total = 0;
      for (uint32_t j = 0; j < G.cnt; ++j) total += S.items[j].cnt;
      S.npass = 1; S.pass_bits[0] = 0; S.pass_val[0] = 0;
      S.out_cnt = 0;
      S.out_off = final_ ? 0 : atomicAdd(&p.acc->pair_top[dst], (unsigned long long)total);
    }
    reset_outer(S.U);
    __syncthreads();
    while (true) {
      __syncthreads();
      if (S.npass == 0) break;
      const int bits = (int)S.pass_bits[S.npass - 1];
      const uint32_t val = S.pass_val[S.npass - 1];
      reset_table(S.T);
      __syncthreads();
      // items in order (a key's maps compose in trace order); the first pair of
      // a thread in the next item is loaded while this item is inserted
      const uint32_t tid = threadIdx.x;
      Pair nx{0ull, 0ull};
      if (G.cnt && tid < S.items[0].cnt) nx = pool_in[S.items[0].off + tid];
      for (uint32_t j = 0; j < G.cnt; ++j) {
        const Item I = S.items[j];
        Pair pr = nx;
        if (j + 1 < G.cnt && tid < S.items[j + 1].cnt) nx = pool_in[S.items[j + 1].off + tid];
        for (uint32_t q = tid; q < I.cnt; q += blockDim.x) {
          if (q != tid) pr = pool_in[I.off + q];
          if (!in_pass(pr.key, bits, val)) continue;
          const int slot = find_or_insert(S.T, pr.key, p.acc, [&](unsigned int s) { S.smap[s] = IDENTITY_MAP; });
          if (slot >= 0) S.smap[slot] = apply_map(S.smap[slot], pr.map, ns);
        }
        __syncthreads();
      }
      if (S.T.ovf) {
        __syncthreads();
        if (threadIdx.x == 0) {
          S.npass -= 1;
          if (bits >= 20 || S.npass + 2 > 64) {
            atomicOr(&p.acc->err, ERR_SPIN);
            S.npass = 0;
          } else {
            S.pass_bits[S.npass] = bits + 1; S.pass_val[S.npass] = val;
            S.pass_bits[S.npass + 1] = bits + 1; S.pass_val[S.npass + 1] = val | (1u << bits);
            S.npass += 2;
          }
        }
        continue;
      }
      const unsigned int nsl = min(S.T.nslots, (unsigned int)SLOTS);
      for (unsigned int s = threadIdx.x; s < nsl; s += blockDim.x) {
        if (final_) finalize_slot<F>(p, fc, &S.U, S.T.skey[s], S.smap[s], G.bucket);
        else if (RV_INB(S.out_off + S.out_cnt + s, g_caps.pool)) pool_out[S.out_off + S.out_cnt + s] = Pair{S.T.skey[s], S.smap[s]};
      }
      __syncthreads();
      if (threadIdx.x == 0) { S.out_cnt += nsl; S.npass -= 1; }
    }
    __syncthreads();
    if (final_) finalize_outer<F>(p, fc, &S.U, G.bucket);
    else if (threadIdx.x == 0) items_out[g] = Item{S.out_off, S.out_cnt, 0};
  }
  __syncthreads();
  flush_final(p, fc);
}

#ifdef RV_CHECKED
// the bounds-check word of this verification, into its status word
__global__ void k_bounds(Acc* acc) {
  if (g_bounds_err) { atomicOr(&acc->err, (unsigned)ERR_BOUNDS); g_bounds_err = 0; }
}
#endif

__global__ void k_root(Acc* acc, Params p, uint64_t n, rv_result* out, int test_wait_polls) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (test_wait_polls > 0) {
    // a bounded wait on a flag that nothing sets: it gives up after the
    // given number of polls, reports ERR_SPIN and the kernel ends normally
    volatile unsigned int* flag = &acc->test_flag;
    int polls = 0;
    while (*flag == 0) {
      if (++polls > test_wait_polls) { atomicOr(&acc->err, (unsigned)ERR_SPIN); break; }
      __nanosleep(256);
    }
  }
  rv_result r;
  memset(&r, 0, sizeof r);
  for (int m = 0; m < 2; ++m) {
    for (int v = 0; v < 6; ++v) r.level_counts[m][v] = acc->level_counts[m][v];
    r.n_nodes[m] = acc->n_nodes[m];
  }
  r.events = n;
  uint64_t v6[6];
  for (int v = 0; v < 6; ++v) v6[v] = acc->level_counts[0][v];
  if (p.nq == 0) {
    r.root = RV_BOT;
    for (int v = 0; v < 6; ++v) if (v6[v]) r.root = v;
  } else {
    for (int v = 0; v < 6; ++v) r.root_counts[v] = v6[v];
    r.root = rvv::valuate(p.tab.q[0].kind, p.tab.q[0].op, p.tab.q[0].num, p.tab.q[0].den, v6);
  }
  const unsigned int e = acc->err;
  r.status = RV_OK;
  if (e & (ERR_LETTER | ERR_TS)) r.status = RV_EINVAL;
  else if (e & ERR_OUTER_FULL) r.status = RV_EAGAIN;   // host retries with a finer split
  else if (e & ERR_SPIN) r.status = RV_ETIMEOUT;       // a bounded device wait gave up
  else if (e) r.status = RV_EINTERNAL;
  *out = r;
}

// ------------------------------------------------------------------ host side
struct Plan {
  int F, B1, B2, P1, P, G_w, nchunk;
  int B2e, hmax;       // heavy routing: B2e = B2 + 1 sub-bucket bits, up to hmax heavy keys per first-level bucket
  int htbits;          // heavy routing: log2 of the sample table
  uint64_t hstride;    // heavy routing: one sample every hstride events
  bool tiled, heavy;
  int test_wait;       // polls of the test wait in k_root (0: none)
  uint64_t n, per_warp, unit, tile2;
  uint64_t max_tiles2, max_units;
  int levels;
  size_t rec_bytes;
  // workspace offsets
  size_t o_acc, o_hist, o_part, o_tot1, o_bstart1, o_recA, o_recB, o_tiles2, o_tf2, o_tk2, o_hist2, o_ssum2,
      o_bstart2, o_units, o_uf, o_uk, o_items0, o_items1, o_groups, o_gf0, o_gk0, o_gf1, o_gk1, o_pool0,
      o_pool1, o_res, o_hkey, o_hpred, o_hts, o_uend, o_htk, o_htc, o_hcnt, o_hlist, o_mids, o_mk, o_mf, o_letters,
      o_hval, total;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int num_sms() { return rv_num_sms(); }

static Plan make_plan(const rv_formula* f, uint64_t n, int host_input, const rv_verify_opts* o, int extra_b2,
                      bool stream = false) {
  Plan pl{};
  pl.n = n;
  pl.test_wait = o && o->test_wait_polls > 0 ? o->test_wait_polls : 0;
  pl.F = f->n_quant == 2 ? FMT_K2 : (f->key_bits == 64 && f->n_quant == 1 ? FMT_K64 : FMT_K32);
  // default: 256 first-level buckets (few open write frontiers in the
  // scatter) and a second-level split down to about 8192 records per bucket
  int b1 = o && o->bucket_bits ? o->bucket_bits : 8;
  pl.B1 = std::min(11, std::max(8, b1));
  pl.P1 = 1 << pl.B1;
  // A bucket splits into at most 256 sub-buckets: 2^B2 light ones, and as
  // many again for heavy keys when heavy routing can be on, so B2 <= 7 then
  // and B2 <= 8 otherwise.  Two variables: the finest split by default,
  // because a fold unit counts the outer bindings of its bucket in a table of
  // UCAP entries, and only the finest split keeps the outer values of any
  // natural trace below that (more than UCAP distinct outer values would have
  // to share 16 hash bits); it also keeps most sub-buckets within one unit.
  const bool heavy_ok = pl.F != FMT_K2 && f->n_quant == 1 && !stream && !(o && o->no_heavy);
  const int b2max = heavy_ok ? 7 : 8;
  int b2 = 0;
  if (o && o->sub_bucket_bits) b2 = o->sub_bucket_bits;
  else if (pl.F == FMT_K2) b2 = b2max;
  else while (b2 < 7 && (n >> (pl.B1 + b2)) > 8192) ++b2;
  b2 += extra_b2;
  pl.B2 = std::min(b2max, std::max(0, b2));
  pl.heavy = heavy_ok && pl.B2 > 0;
  pl.B2e = pl.B2 + (pl.heavy ? 1 : 0);
  pl.hmax = pl.heavy ? std::min(HMAXC, 1 << pl.B2) : 0;
  pl.hstride = std::max<uint64_t>(HSTRIDE, (n >> (HTAB_BITS - 1)) + 1);
  pl.htbits = 10;
  while (pl.htbits < HTAB_BITS && ((uint64_t)1 << (pl.htbits - 1)) < (n + pl.hstride - 1) / pl.hstride) ++pl.htbits;
  pl.P = pl.P1 << pl.B2e;
  const uint64_t unit_max = pl.F == FMT_K32 ? FoldCfg<FMT_K32>::UNIT : FoldCfg<FMT_K64>::UNIT;
  pl.unit = o && o->unit_records ? (uint64_t)o->unit_records : unit_max;
  pl.unit = std::min<uint64_t>(unit_max, std::max<uint64_t>(256, pl.unit));
  pl.tiled = pl.B1 == 8;
  const uint64_t max_w = (uint64_t)num_sms() * 3 * SC_WARPS;
  uint64_t gw = (n + 2047) / 2048;
  if (gw > max_w) gw = max_w;
  if (gw < 1) gw = 1;
  pl.per_warp = ((n + gw - 1) / gw + 31) / 32 * 32;
  if (pl.per_warp == 0) pl.per_warp = 32;
  pl.G_w = (int)((n + pl.per_warp - 1) / pl.per_warp);
  if (pl.G_w < 1) pl.G_w = 1;
  if (pl.tiled) {   // one row of the bucket histogram per CTA tile
    pl.per_warp = pl.F == FMT_K32 ? TileSize<FMT_K32>::v : TileSize<FMT_K64>::v;
    pl.G_w = (int)std::max<uint64_t>(1, (n + pl.per_warp - 1) / pl.per_warp);
  }
  pl.nchunk = (pl.G_w + COLCHUNK - 1) / COLCHUNK;
  pl.tile2 = pl.F == FMT_K32 ? Tile2Len<FMT_K32>::v : Tile2Len<FMT_K64>::v;
  pl.max_tiles2 = n / pl.tile2 + pl.P1 + 1;
  pl.max_units = n / pl.unit + pl.P + 1;
  pl.levels = 0;
  for (uint64_t cap = 1; cap < n / pl.unit + 2; cap *= GC) ++pl.levels;
  pl.rec_bytes = pl.F == FMT_K32 ? 4 : 8;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = align256(off + bytes); return r; };
  pl.o_acc = take(sizeof(Acc));
  pl.o_hist = take((size_t)pl.P1 * pl.G_w * 4);
  pl.o_part = take((size_t)pl.P1 * pl.nchunk * 8);
  pl.o_tot1 = take((size_t)pl.P1 * 8);
  pl.o_bstart1 = take((size_t)(pl.P1 + 1) * 8);
  pl.o_recA = take(n * pl.rec_bytes);
  pl.o_recB = pl.B2 ? take(n * pl.rec_bytes) : pl.o_recA;
  pl.o_tiles2 = pl.B2 ? take(pl.max_tiles2 * sizeof(Tile)) : 0;
  pl.o_tf2 = pl.B2 ? take((size_t)pl.P1 * 4) : 0;
  pl.o_tk2 = pl.B2 ? take((size_t)pl.P1 * 4) : 0;
  pl.o_hist2 = pl.B2 ? take(pl.max_tiles2 * ((size_t)1 << pl.B2e) * 4) : 0;
  pl.o_ssum2 = pl.B2 ? take((size_t)pl.P1 * SCAN2_S * ((size_t)1 << pl.B2e) * 4) : 0;
  pl.o_bstart2 = pl.B2 ? take((size_t)(pl.P + 1) * 8) : pl.o_bstart1;
  pl.o_units = take(pl.max_units * sizeof(Tile));
  pl.o_uf = take((size_t)pl.P * 4);
  pl.o_uk = take((size_t)pl.P * 4);
  pl.o_uend = take((size_t)pl.P * 8);
  pl.o_mids = take((size_t)pl.P * 4);
  pl.o_mk = take((size_t)pl.P * 4);
  pl.o_mf = take((size_t)pl.P * 4);
  pl.o_htk = pl.heavy ? take(((size_t)1 << pl.htbits) * 8) : 0;
  pl.o_htc = pl.heavy ? take(((size_t)1 << pl.htbits) * 4) : 0;
  pl.o_hcnt = pl.heavy ? take((size_t)pl.P1 * 4) : 0;
  pl.o_hlist = pl.heavy ? take((size_t)pl.P1 * pl.hmax * 8) : 0;
  pl.o_items0 = take(pl.max_units * sizeof(Item));
  pl.o_items1 = take(pl.max_units * sizeof(Item));
  pl.o_groups = take(pl.max_units * sizeof(Group));
  pl.o_gf0 = take((size_t)pl.P * 4);
  pl.o_gk0 = take((size_t)pl.P * 4);
  pl.o_gf1 = take((size_t)pl.P * 4);
  pl.o_gk1 = take((size_t)pl.P * 4);
  pl.o_pool0 = take(std::max<uint64_t>(n, 1) * sizeof(Pair));
  pl.o_pool1 = take(std::max<uint64_t>(n, 1) * sizeof(Pair));
  pl.o_res = take(sizeof(rv_result));
  pl.o_hkey = host_input ? take(n * (f->key_bits / 8)) : 0;
  pl.o_hpred = host_input ? take(n) : 0;
  pl.o_hts = host_input ? take(n * 4) : 0;
  pl.o_letters = f->n_cmp ? take(std::max<uint64_t>(n, 1)) : 0;
  pl.o_hval = host_input && f->n_cmp ? take(n * 4) : 0;
  pl.total = off;
  return pl;
}

static MonitorTab make_tab(const rv_formula* f) {
  MonitorTab t;
  memset(&t, 0, sizeof t);
  for (int l = 0; l < RV_MAX_LETTERS; ++l) t.maps[l] = l < f->n_letters ? f->maps[l] : IDENTITY_MAP;
  memcpy(t.labels, f->labels, sizeof t.labels);
  t.n_states = f->n_states;
  t.q0 = f->q0;
  t.n_letters = f->n_letters;
  t.nq = f->n_quant;
  t.q[0] = f->q[0];
  t.q[1] = f->q[1];
  return t;
}

#define RV_CU(call)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return rv_fail(RV_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <int F>
static rv_status launch_all(const Plan& pl, const rv_formula* f, const void* key, const uint8_t* pred,
                            const uint32_t* ts, unsigned char* ws, rv_result* dev_out, const rv_bindings* b,
                            cudaStream_t s, const StreamState* ss = nullptr, const uint32_t* value = nullptr) {
  typedef typename RecT<F>::type Rec;
  Acc* acc = (Acc*)(ws + pl.o_acc);
  RV_CU(cudaMemsetAsync(acc, 0, sizeof(Acc), s));
#ifdef RV_CHECKED
  {
    const CheckCaps caps{pl.n, pl.max_tiles2, pl.max_units, std::max<uint64_t>(pl.n, 1)};
    const unsigned int zero = 0;
    RV_CU(cudaMemcpyToSymbolAsync(g_caps, &caps, sizeof caps, 0, cudaMemcpyHostToDevice, s));
    RV_CU(cudaMemcpyToSymbolAsync(g_bounds_err, &zero, 4, 0, cudaMemcpyHostToDevice, s));
    RV_CU(cudaStreamSynchronize(s));   // the sources are on this stack frame
  }
#endif
  if (f->n_cmp && pl.n) {              // comparison atoms: fold each event's value into its letter
    uint8_t* letters = ws + pl.o_letters;
    const unsigned g = (unsigned)std::min<uint64_t>((pl.n + 255) / 256, (uint64_t)num_sms() * 8);
    RV_LAUNCH("k_cmp_letters", k_cmp_letters, g, 256, 0, s, pred, value, pl.n, cmp_tab(f), letters, &acc->err,
              (unsigned)ERR_LETTER);
    pred = letters;
  }
  Params p;
  memset(&p, 0, sizeof p);
  p.tab = make_tab(f);
  p.B1 = pl.B1;
  p.B2 = pl.B2e;                       // sub-bucket bits of a bucket index
  p.light = pl.heavy ? 1 << pl.B2 : 0;
  p.nq = f->n_quant;
  p.acc = acc;
  if (b) p.out = *b;
  if (ss) { p.stream_mode = 1; p.ss = *ss; }
  const uint64_t n = pl.n;
  if (n > 0) {
    uint32_t* hist = (uint32_t*)(ws + pl.o_hist);
    uint64_t* part = (uint64_t*)(ws + pl.o_part);
    uint64_t* tot1 = (uint64_t*)(ws + pl.o_tot1);
    uint64_t* bstart1 = (uint64_t*)(ws + pl.o_bstart1);
    Rec* recA = (Rec*)(ws + pl.o_recA);
    const int sc_blocks = (pl.G_w + SC_WARPS - 1) / SC_WARPS;
    const size_t sc_smem = (size_t)SC_WARPS * pl.P1 * 4;
    if (pl.tiled)
      RV_LAUNCH("k_hist_tile", k_hist_tile<F>, pl.G_w, TB_THREADS, 0, s, key, ts, n, f->n_quant, hist, acc);
    else
      RV_LAUNCH("k_hist", k_hist<F>, sc_blocks, SC_WARPS * 32, sc_smem, s, key, ts, n, pl.per_warp, pl.G_w, pl.B1, f->n_quant, hist, acc);
    const int ct = pl.P1 * pl.nchunk;
    RV_LAUNCH("k_colscan_a", k_colscan_a, (ct + 255) / 256, 256, 0, s, hist, pl.G_w, pl.P1, pl.nchunk, part);
    RV_LAUNCH("k_colscan_b", k_colscan_b, (pl.P1 + 255) / 256, 256, 0, s, part, pl.P1, pl.nchunk, tot1);
    RV_LAUNCH("k_colscan_c", k_colscan_c, (ct + 255) / 256, 256, 0, s, hist, pl.G_w, pl.P1, pl.nchunk, part);
    RV_LAUNCH("k_bucket_scan", k_scan<uint64_t>, 1, 1024, scan_smem<uint64_t>(), s, tot1, pl.P1, bstart1, bstart1 + pl.P1);
    if (pl.tiled)
      RV_LAUNCH("k_scatter_tile", k_scatter_tile<F>, pl.G_w, TB_THREADS, sizeof(TileShared<F>), s, key, pred, n,
                f->n_quant, f->n_letters, hist, bstart1, recA, acc);
    else
      RV_LAUNCH("k_scatter", k_scatter<F>, sc_blocks, SC_WARPS * 32, sc_smem, s, key, pred, n, pl.per_warp, pl.G_w, pl.B1, f->n_quant,
                f->n_letters, hist, bstart1, recA, acc);
    Rec* recs = recA;
    uint64_t* bstart = bstart1;
    if (pl.B2) {
      Tile* tiles2 = (Tile*)(ws + pl.o_tiles2);
      uint32_t* tf2 = (uint32_t*)(ws + pl.o_tf2);
      uint32_t* tk2 = (uint32_t*)(ws + pl.o_tk2);
      uint32_t* hist2 = (uint32_t*)(ws + pl.o_hist2);
      uint32_t* ssum2 = (uint32_t*)(ws + pl.o_ssum2);
      uint64_t* bstart2 = (uint64_t*)(ws + pl.o_bstart2);
      Rec* recB = (Rec*)(ws + pl.o_recB);
      RV_LAUNCH("k_count_tiles", k_count_tiles, (pl.P1 + 255) / 256, 256, 0, s, bstart1, pl.P1, pl.tile2, tk2);
      RV_LAUNCH("k_scan_u32", k_scan<uint32_t>, 1, 1024, scan_smem<uint32_t>(), s, tk2, pl.P1, tf2, &acc->n_tiles2);
      RV_LAUNCH("k_emit_tiles", k_emit_tiles, (int)((pl.max_tiles2 + 255) / 256), 256, 0, s, bstart1, pl.P1, pl.tile2, tf2, tk2, &acc->n_tiles2, tiles2, pl.max_tiles2);
      const int t2_blocks = (int)((pl.max_tiles2 + SC_WARPS - 1) / SC_WARPS);
      HeavyDev hv{nullptr, nullptr, 0};
      if (pl.heavy) {
        uint64_t* htk = (uint64_t*)(ws + pl.o_htk);
        uint32_t* htc = (uint32_t*)(ws + pl.o_htc);
        uint32_t* hcnt = (uint32_t*)(ws + pl.o_hcnt);
        uint64_t* hlist = (uint64_t*)(ws + pl.o_hlist);
        RV_CU(cudaMemsetAsync(htk, 0, ((size_t)1 << pl.htbits) * 8, s));
        RV_CU(cudaMemsetAsync(htc, 0, ((size_t)1 << pl.htbits) * 4, s));
        RV_CU(cudaMemsetAsync(hcnt, 0, (size_t)pl.P1 * 4, s));
        const uint64_t samples = (n + HS_RUN * pl.hstride - 1) / (HS_RUN * pl.hstride) * HS_RUN;
        const uint32_t thresh = (uint32_t)std::max<uint64_t>(8, HRECORDS / pl.hstride);
        RV_LAUNCH("k_hsample", k_hsample<F>, (int)((samples + HS_PER * 256 - 1) / (HS_PER * 256)), 256, 0, s, key, n, pl.hstride,
                  pl.htbits, htk, htc);
        RV_LAUNCH("k_hpick", k_hpick<F>, (1 << pl.htbits) / 256, 256, 0, s, htk, htc, pl.htbits, thresh, pl.B1, pl.hmax, hcnt,
                  hlist);
        hv = HeavyDev{hcnt, hlist, pl.hmax};
      }
      RV_LAUNCH("k_hist2", k_hist2<F>, t2_blocks, SC_WARPS * 32, 0, s, recA, tiles2, &acc->n_tiles2, pl.B1, pl.B2, hist2, hv);
      RV_LAUNCH("k_scan2_sums", k_scan2_sums, pl.P1 * SCAN2_S, 1024, 0, s, hist2, tf2, tk2, pl.B2e, ssum2);
      RV_LAUNCH("k_scan2", k_scan2, pl.P1 * SCAN2_S, 1024, 0, s, hist2, tf2, tk2, pl.P1, pl.B2e, ssum2, bstart1, bstart2);
      if (F == FMT_K32)
        RV_LAUNCH("k_scatter2", k_scatter2<F>, t2_blocks, SC_WARPS * 32, 0, s, recA, tiles2, &acc->n_tiles2, pl.B1, pl.B2, hist2,
                  bstart2, recB, hv);
      else
        RV_LAUNCH("k_scatter2_tile", k_scatter2_tile<F>, (int)pl.max_tiles2, TB_THREADS, sizeof(Tile2Shared<F>), s, recA, tiles2,
                  &acc->n_tiles2, pl.B1, pl.B2, hist2, bstart2, recB, hv);
      recs = recB;
      bstart = bstart2;
    }
    Tile* units = (Tile*)(ws + pl.o_units);
    uint32_t* uf = (uint32_t*)(ws + pl.o_uf);
    uint32_t* uk = (uint32_t*)(ws + pl.o_uk);
    Item* items0 = (Item*)(ws + pl.o_items0);
    Item* items1 = (Item*)(ws + pl.o_items1);
    Group* groups = (Group*)(ws + pl.o_groups);
    Pair* pool0 = (Pair*)(ws + pl.o_pool0);
    Pair* pool1 = (Pair*)(ws + pl.o_pool1);
    uint64_t* uend = (uint64_t*)(ws + pl.o_uend);
    RV_LAUNCH("k_count_units", k_count_units, (pl.P + 255) / 256, 256, 0, s, bstart, pl.P, pl.B2e, pl.unit, F != FMT_K2 ? 1 : 0, uk, uend,
              pl.heavy ? 1 << pl.B2 : 0);
    RV_LAUNCH("k_scan_u32", k_scan<uint32_t>, 1, 1024, scan_smem<uint32_t>(), s, uk, pl.P, uf, &acc->n_units);
    RV_LAUNCH("k_emit_tiles", k_emit_tiles, (int)((pl.max_units + 255) / 256), 256, 0, s, bstart, pl.P, pl.unit, uf, uk, &acc->n_units, units, pl.max_units,
              F != FMT_K2 ? uend : nullptr);
    const int grid = (int)std::min<uint64_t>(pl.max_units, (uint64_t)num_sms() * FoldCfg<F>::MINB);
    RV_LAUNCH("k_fold", k_fold<F>, grid, FOLD_THREADS, sizeof(FoldShared<F>), s, recs, units, &acc->n_units, p, items0, pool0);
    uint32_t* mids = (uint32_t*)(ws + pl.o_mids);
    uint32_t* mk = (uint32_t*)(ws + pl.o_mk);
    uint32_t* mf = (uint32_t*)(ws + pl.o_mf);
    RV_LAUNCH("k_list_multi", k_list_multi, (pl.P + 255) / 256, 256, 0, s, uk, uf, pl.P, &acc->n_multi, mids, mk, mf);
    const uint32_t* fin = mf;
    const uint32_t* kin = mk;
    uint32_t* gf[2] = {(uint32_t*)(ws + pl.o_gf0), (uint32_t*)(ws + pl.o_gf1)};
    uint32_t* gk[2] = {(uint32_t*)(ws + pl.o_gk0), (uint32_t*)(ws + pl.o_gk1)};
    Item* iin = items0;
    Item* iout = items1;
    Pair* pin = pool0;
    Pair* pout = pool1;
    for (int l = 0; l < pl.levels; ++l) {
      const int dst = (l + 1) & 1;
      RV_CU(cudaMemsetAsync(&acc->pair_top[dst], 0, sizeof(unsigned long long), s));
      RV_LAUNCH("k_groups", k_groups, 1, 1024, 0, s, fin, kin, &acc->n_multi, mids, gf[l & 1], gk[l & 1], groups,
                &acc->n_groups[l]);
      const int cgrid = (int)std::min<uint64_t>(pl.max_units / GC + pl.P, (uint64_t)num_sms() * 2);
      RV_LAUNCH("k_combine", k_combine<F>, cgrid, FOLD_THREADS, sizeof(CombineShared), s, iin, pin, groups, &acc->n_groups[l], &acc->next_group[l], p,
                                                                      iout, pout, dst);
      fin = gf[l & 1];
      kin = gk[l & 1];
      std::swap(iin, iout);
      std::swap(pin, pout);
    }
  }
#ifdef RV_CHECKED
  RV_LAUNCH("k_bounds", k_bounds, 1, 1, 0, s, acc);
#endif
  if (!ss) RV_LAUNCH("k_root", k_root, 1, 32, 0, s, acc, p, n, dev_out, pl.test_wait);
  RV_CU(cudaGetLastError());
  return RV_OK;
}

template <int F>
static rv_status set_attrs_now() {
  RV_CU(cudaFuncSetAttribute(k_fold<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FoldShared<F>)));
  RV_CU(cudaFuncSetAttribute(k_combine<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CombineShared)));
  RV_CU(cudaFuncSetAttribute(k_hist<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, SC_WARPS * 2048 * 4));
  RV_CU(cudaFuncSetAttribute(k_scatter<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, SC_WARPS * 2048 * 4));
  RV_CU(cudaFuncSetAttribute(k_scatter_tile<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileShared<F>)));
  RV_CU(cudaFuncSetAttribute(k_scan<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scan_smem<uint32_t>()));
  RV_CU(cudaFuncSetAttribute(k_scan<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scan_smem<uint64_t>()));
  RV_CU(cudaFuncSetAttribute(k_scatter2_tile<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Tile2Shared<F>)));
  return RV_OK;
}

// the attributes apply to the current device: set them once per device
template <int F>
static rv_status set_attrs() {
  return rv_once_per_device(F == FMT_K32 ? RV_ONCE_FOLD32 : F == FMT_K64 ? RV_ONCE_FOLD64 : RV_ONCE_FOLD2,
                            &set_attrs_now<F>);
}

static rv_status dispatch(const Plan& pl, const rv_formula* f, const void* key, const uint8_t* pred, const uint32_t* ts,
                          unsigned char* ws, rv_result* dev_out, const rv_bindings* b, cudaStream_t s,
                          const StreamState* ss = nullptr, const uint32_t* value = nullptr) {
  rv_status st;
  switch (pl.F) {
    case FMT_K32: st = set_attrs<FMT_K32>(); if (st) return st; return launch_all<FMT_K32>(pl, f, key, pred, ts, ws, dev_out, b, s, ss, value);
    case FMT_K64: st = set_attrs<FMT_K64>(); if (st) return st; return launch_all<FMT_K64>(pl, f, key, pred, ts, ws, dev_out, b, s, ss, value);
    default: st = set_attrs<FMT_K2>(); if (st) return st; return launch_all<FMT_K2>(pl, f, key, pred, ts, ws, dev_out, b, s, ss, value);
  }
}

rv_alloc_fn g_alloc = nullptr;
rv_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

}  // namespace

// allocator hooks (also used by the streaming service)
void* rv_dev_alloc(size_t bytes) {
  if (g_alloc) return g_alloc(bytes, g_alloc_ctx);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  return p;
}
void rv_dev_free(void* p) {
  if (!p) return;
  if (g_free) g_free(p, g_alloc_ctx);
  else cudaFree(p);
}

// Streaming: fold one batch whose keys are dense ids (nq == 2: (outer << 32) |
// binding, 64-bit; nq == 1: binding id as a 64-bit key) into the state ss.
rv_status rv_offline_stream_batch(const rv_formula* f, const uint64_t* key, const uint8_t* pred, uint64_t n,
                                  void* ws, size_t ws_bytes, const StreamState* ss, unsigned int* err_out,
                                  cudaStream_t s) {
  rv_formula g = *f;
  g.key_bits = 64;                       // ids are passed as 64-bit keys
  Plan pl = make_plan(&g, n, 0, nullptr, 0, true);
  if (ws_bytes < pl.total) return rv_fail(RV_ENOMEM, "stream workspace of %zu bytes, need %zu", ws_bytes, pl.total);
  rv_status st = dispatch(pl, &g, key, pred, nullptr, (unsigned char*)ws, nullptr, nullptr, s, ss);
  if (st) return st;
  if (err_out && cudaMemcpyAsync(err_out, &((Acc*)((unsigned char*)ws + pl.o_acc))->err, 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return rv_fail(RV_ECUDA, "status copy failed");
  return RV_OK;
}

size_t rv_offline_stream_ws(const rv_formula* f, uint64_t n) {
  rv_formula g = *f;
  g.key_bits = 64;
  return make_plan(&g, n, 0, nullptr, 0, true).total;
}

extern "C" void rv_set_allocator(rv_alloc_fn alloc, rv_free_fn free_fn, void* ctx) {
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = ctx;
}

extern "C" size_t rv_verify_workspace_size(const rv_formula* f, uint64_t n, int host_input, const rv_verify_opts* opts) {
  if (!f) return 0;
  size_t worst = 0;
  for (int extra = 0; extra <= 7; extra += 2) worst = std::max(worst, make_plan(f, n, host_input, opts, extra).total);
  return worst;
}

static rv_status check_args(const rv_formula* f, const rv_trace* t) {
  if (!f || !t) return rv_fail(RV_EINVAL, "null formula or trace");
  if (t->n > 0xFFFFFFFFull) return rv_fail(RV_EINVAL, "traces are limited to 2^32-1 events");
  if (t->n && (!t->key || !t->pred)) return rv_fail(RV_EINVAL, "null key or pred array");
  if (f->n_quant == 0 && t->n == 0) return rv_fail(RV_EINVAL, "an unquantified property needs a non-empty trace");
  if (f->n_cmp && t->n && !t->value)
    return rv_fail(RV_EINVAL, "the formula compares the value column: the trace needs its value array");
  return RV_OK;
}

extern "C" rv_status rv_verify_trace_async(const rv_formula* f, const rv_trace* t, void* ws, size_t ws_bytes,
                                           rv_result* dev_out, const rv_bindings* bindings,
                                           const rv_verify_opts* opts, cudaStream_t s) {
  rv_status st = check_args(f, t);
  if (st) return st;
  if (!ws || !dev_out) return rv_fail(RV_EINVAL, "the asynchronous form needs a workspace and a device result");
  Plan pl = make_plan(f, t->n, 0, opts, 0);
  if (ws_bytes < pl.total) return rv_fail(RV_ENOMEM, "workspace of %zu bytes, need %zu", ws_bytes, pl.total);
  return dispatch(pl, f, t->key, t->pred, t->ts, (unsigned char*)ws, dev_out, bindings, s, nullptr, t->value);
}

extern "C" rv_status rv_verify_trace(const rv_formula* f, const rv_trace* t, int on_device, void* ws, size_t ws_bytes,
                                     rv_result* out, const rv_bindings* bindings, const rv_verify_opts* opts,
                                     cudaStream_t s) {
  rv_status st = check_args(f, t);
  if (st) return st;
  if (!out) return rv_fail(RV_EINVAL, "null result");
  static thread_local rv_result* pinned = nullptr;
  if (!pinned && cudaMallocHost(&pinned, sizeof(rv_result)) != cudaSuccess)
    return rv_fail(RV_ECUDA, "cannot allocate pinned result buffer");
  for (int extra = 0; extra <= 7; extra += 2) {
    Plan pl = make_plan(f, t->n, !on_device, opts, extra);
    unsigned char* w = (unsigned char*)ws;
    bool owned = false;
    if (!w) {
      w = (unsigned char*)rv_dev_alloc(pl.total);
      if (!w) return rv_fail(RV_ENOMEM, "cannot allocate %zu bytes of workspace", pl.total);
      owned = true;
    } else if (ws_bytes < pl.total) {
      return rv_fail(RV_ENOMEM, "workspace of %zu bytes, need %zu", ws_bytes, pl.total);
    }
    const void* key = t->key;
    const uint8_t* pred = t->pred;
    const uint32_t* ts = t->ts;
    const uint32_t* value = t->value;
    st = RV_OK;
    if (!on_device && t->n) {
      const size_t kb = (size_t)t->n * (f->key_bits / 8);
      if (cudaMemcpyAsync(w + pl.o_hkey, t->key, kb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
          cudaMemcpyAsync(w + pl.o_hpred, t->pred, t->n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
          (t->ts && cudaMemcpyAsync(w + pl.o_hts, t->ts, t->n * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) ||
          (f->n_cmp && cudaMemcpyAsync(w + pl.o_hval, t->value, t->n * 4, cudaMemcpyHostToDevice, s) != cudaSuccess))
        st = rv_fail(RV_ECUDA, "host-to-device copy failed");
      key = w + pl.o_hkey;
      pred = w + pl.o_hpred;
      ts = t->ts ? (const uint32_t*)(w + pl.o_hts) : nullptr;
      value = f->n_cmp ? (const uint32_t*)(w + pl.o_hval) : nullptr;
    }
    rv_result* dres = (rv_result*)(w + pl.o_res);
    if (!st) st = dispatch(pl, f, key, pred, ts, w, dres, bindings, s, nullptr, value);
    if (!st && cudaMemcpyAsync(pinned, dres, sizeof(rv_result), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      st = rv_fail(RV_ECUDA, "device-to-host copy failed");
    cudaError_t e = cudaStreamSynchronize(s);
    if (!st && e != cudaSuccess) st = rv_fail(RV_ECUDA, "stream synchronize: %s", cudaGetErrorString(e));
    if (owned) rv_dev_free(w);
    if (st) return st;
    *out = *pinned;
    if (out->status == RV_EAGAIN && f->n_quant == 2 && pl.B2 < 7 && !(opts && opts->sub_bucket_bits)) continue;
    if (out->status == RV_EINVAL) return rv_fail(RV_EINVAL, "trace rejected: predicate code out of range or timestamps decreasing");
    if (out->status == RV_ETIMEOUT) return rv_fail(RV_ETIMEOUT, "a bounded device wait gave up (device status word)");
    if (out->status != RV_OK) return rv_fail((rv_status)out->status, "device status %d", out->status);
    return RV_OK;
  }
  return rv_fail(RV_EINTERNAL, "too many outer bindings per bucket even at the finest split");
}
