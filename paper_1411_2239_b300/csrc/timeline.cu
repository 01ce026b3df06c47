// Per-event verdict timeline and first violation of every binding.
//
// The online mode of Algorithm 1 (Sec. 4.2) yields an evolving verdict; here
// it is given at event granularity: for event j of binding D (the innermost
// value vector of the event, Sec. 2.4.1), the LTL4 verdict of D's projection
// u^D (Sec. 2.4.3) up to and including j, i.e. lambda(delta*(q0, prefix)) of
// the body's Moore monitor (Sec. 2.2.3), and for every binding whose verdict
// becomes F the index of the first event at which it does (F is permanent,
// Def. "LTL4 semantics", so that event is unique).
//
// Steps:
//   sort   the events grouped by key, trace order kept inside a key: a stable
//          LSD radix sort of (key, event index) by 8-bit key digits (digits on
//          which every key agrees are skipped);
//   scan   an inclusive segmented scan over the sorted events whose operator
//          composes the letters' 64-bit transition maps ("M then m"), segment
//          heads where the key changes.  Three phases: per tile of TT * TV
//          events the aggregate (head seen, map since the last head); an
//          exclusive scan of the tile aggregates; per tile again, each thread
//          starting from its carried state and stepping states, so a binding
//          of any length is spread over every tile it covers;
//   emit   each event's verdict written at its trace position; a binding's
//          first F event recorded as (key, index).
#include <algorithm>
#include <cstring>

#include "profile.h"
#include "rv_device.cuh"

using namespace rvd;

namespace {

constexpr int TT = 256;               // threads per CTA of the scan
constexpr int TV = 16;                // events per thread of the scan
constexpr int TTILE = TT * TV;
constexpr unsigned TFULL = 0xFFFFFFFFu;

struct Agg { uint64_t map; uint32_t head, pad; };   // head: a segment starts inside

// ------------------------------------------------------------------ radix passes
// A pass splits the (key, index) pairs stably by one 8-bit digit.  It works on
// CTA tiles of RT pairs: k_t_hist counts each tile's digits, k_t_colscan turns
// the counts into every tile's offset per digit, and k_t_scatter stages its
// tile in shared memory, orders it by digit there (warps own contiguous
// slices, lanes of equal digits ranked by ballots), and writes each digit's
// run contiguously, so the global stores are runs rather than scattered words.
constexpr int RT = 4096;              // pairs per tile
constexpr int RTT = 256;              // threads per tile
constexpr int RTW = RTT / 32;

template <typename K>
__global__ void __launch_bounds__(RTT) k_t_hist(const K* key, uint64_t n, int shift, uint32_t* hist, int ntiles) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t b0 = (uint64_t)blockIdx.x * RT;
  const int len = (int)min((uint64_t)RT, n - b0);
  // a whole, aligned tile: each thread's keys arrive by 16-byte loads issued
  // together (one memory round trip, not one per key); counts do not depend
  // on the order, so thread t takes words t, t + RTT, ...
  constexpr int PER = RT / RTT;                       // keys per thread
  constexpr int KW = 16 / sizeof(K);                  // keys per 16-byte word
  if (len == RT && ((uintptr_t)(key + b0) & 15) == 0) {
    const uint4* w = reinterpret_cast<const uint4*>(key + b0);
    uint4 x[PER / KW];
#pragma unroll
    for (int q = 0; q < PER / KW; ++q) x[q] = w[q * RTT + threadIdx.x];
#pragma unroll
    for (int q = 0; q < PER / KW; ++q) {
      const K* kk = reinterpret_cast<const K*>(&x[q]);
#pragma unroll
      for (int e = 0; e < KW; ++e) atomicAdd(&cnt[(uint32_t)(kk[e] >> shift) & 255u], 1u);
    }
  } else {
    for (int i = threadIdx.x; i < len; i += RTT) atomicAdd(&cnt[(uint32_t)(key[b0 + i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];   // digit-major
}

// one CTA per digit value: exclusive prefix of its row over the tiles
// (rows are contiguous, the histogram being stored digit-major)
__global__ void __launch_bounds__(1024) k_t_colscan(uint32_t* hist, int G_w, uint64_t* tot) {
  __shared__ uint64_t wsum[32];
  const int r = blockIdx.x;
  uint32_t* row = hist + (uint64_t)r * G_w;
  const int per = (G_w + blockDim.x - 1) / blockDim.x;
  const int j0 = threadIdx.x * per, j1 = min(G_w, j0 + per);
  uint64_t mine = 0;
  for (int j = j0; j < j1; j += 8) {            // eight loads in flight before their sums
    uint32_t x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = j + e < j1 ? row[j + e] : 0u;
#pragma unroll
    for (int e = 0; e < 8; ++e) mine += x[e];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t incl = mine;
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t y = __shfl_up_sync(TFULL, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    uint64_t x = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t y = __shfl_up_sync(TFULL, x, d);
      if (lane >= d) x += y;
    }
    wsum[lane] = x;
  }
  __syncthreads();
  uint64_t run = (w ? wsum[w - 1] : 0) + incl - mine;
  for (int j = j0; j < j1; j += 8) {
    uint32_t x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = j + e < j1 ? row[j + e] : 0u;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (j + e < j1) {
        row[j + e] = (uint32_t)run;
        run += x[e];
      }
  }
  if (threadIdx.x == blockDim.x - 1) tot[r] = run;
}

// the digits' segment starts: exclusive scan of their 256 totals (one CTA)
__global__ void __launch_bounds__(256) k_t_segs(const uint64_t* tot, uint64_t* seg) {
  __shared__ uint64_t ws[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t mine = tot[threadIdx.x];
  uint64_t incl = mine;
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t y = __shfl_up_sync(TFULL, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) ws[w] = incl;
  __syncthreads();
  uint64_t before = 0;
  for (int q = 0; q < w; ++q) before += ws[q];
  seg[threadIdx.x] = before + incl - mine;
}

// lanes whose 8-bit values equal this lane's (invalid lanes form their own group)
__device__ __forceinline__ uint32_t match8(uint32_t v, bool valid) {
  const uint32_t vb = __ballot_sync(TFULL, valid);
  uint32_t m = valid ? vb : ~vb;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t bk = __ballot_sync(TFULL, (v >> k) & 1u);
    m &= ((v >> k) & 1u) ? bk : ~bk;
  }
  return m;
}

template <typename K>
struct RadixShared {
  K key[RT];
  uint32_t idx[RT];
  uint8_t let[RT];
  uint8_t dig[RT];
  uint16_t perm[RT];                  // perm[j]: the pair at position j of the digit order
  uint32_t wcur[RTW][256];
  uint32_t loc[256];
  uint64_t gbase[256];
  uint32_t tsum[RTW];
};

template <typename K>
__global__ void __launch_bounds__(RTT)
k_t_scatter(const K* key, const uint32_t* idx, const uint8_t* let, uint64_t n, int shift, const uint32_t* pre,
            int ntiles, const uint64_t* seg, K* key_out, uint32_t* idx_out, uint8_t* let_out) {
  extern __shared__ __align__(16) unsigned char radix_smem[];
  RadixShared<K>& S = *reinterpret_cast<RadixShared<K>*>(radix_smem);
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const uint64_t b0 = (uint64_t)blockIdx.x * RT;
  const int len = (int)min((uint64_t)RT, n - b0);
  for (int i = threadIdx.x; i < RTW * 256; i += RTT) S.wcur[i / 256][i % 256] = 0;
  // 1. the tile, staged (letters travel with their events).  A whole tile
  // whose arrays are 16-byte aligned (the radix buffers always are) arrives
  // by 16-byte loads all issued before any of them is stored; otherwise one
  // event at a time.
  constexpr int KW = 16 / sizeof(K);
  const bool vec = len == RT && ((((uintptr_t)(key + b0)) | ((uintptr_t)(let + b0)) |
                                  (idx ? (uintptr_t)(idx + b0) : (uintptr_t)0)) & 15) == 0;
  if (vec) {
    const uint4* kw = reinterpret_cast<const uint4*>(key + b0);
    const uint4* iw = reinterpret_cast<const uint4*>(idx + b0);
    const uint4* lw = reinterpret_cast<const uint4*>(let + b0);
    uint4 xk[RT / KW / RTT], xi[RT / 4 / RTT];
#pragma unroll
    for (int q = 0; q < RT / KW / RTT; ++q) xk[q] = kw[q * RTT + threadIdx.x];
    if (idx) {
#pragma unroll
      for (int q = 0; q < RT / 4 / RTT; ++q) xi[q] = iw[q * RTT + threadIdx.x];
    }
    static_assert(RT / 16 == RTT, "one 16-byte word of letters per thread");
    const uint4 xl = lw[threadIdx.x];
    uint4* sk = reinterpret_cast<uint4*>(S.key);
#pragma unroll
    for (int q = 0; q < RT / KW / RTT; ++q) {
      const int wi = q * RTT + threadIdx.x;
      sk[wi] = xk[q];
      const K* kk = reinterpret_cast<const K*>(&xk[q]);
#pragma unroll
      for (int e = 0; e < KW; ++e) S.dig[wi * KW + e] = (uint8_t)((uint32_t)(kk[e] >> shift) & 255u);
    }
    uint4* si = reinterpret_cast<uint4*>(S.idx);
#pragma unroll
    for (int q = 0; q < RT / 4 / RTT; ++q) {
      const int wi = q * RTT + threadIdx.x;
      if (idx) {
        si[wi] = xi[q];
      } else {
        const uint32_t i0 = (uint32_t)(b0 + 4 * wi);
        si[wi] = make_uint4(i0, i0 + 1, i0 + 2, i0 + 3);
      }
    }
    reinterpret_cast<uint4*>(S.let)[threadIdx.x] = xl;
  } else {
    for (int i = threadIdx.x; i < len; i += RTT) {
      const K k = key[b0 + i];
      S.key[i] = k;
      S.idx[i] = idx ? idx[b0 + i] : (uint32_t)(b0 + i);
      S.let[i] = let[b0 + i];
      S.dig[i] = (uint8_t)((uint32_t)(k >> shift) & 255u);
    }
  }
  __syncthreads();
  // 2. per-warp counts over contiguous slices
  const int per = (len + RTW - 1) / RTW;
  const int w0 = min(len, wl * per), w1 = min(len, w0 + per);
  for (int i = w0 + lane; i < w1; i += 32) atomicAdd(&S.wcur[wl][S.dig[i]], 1u);
  __syncthreads();
  // 3. thread d: offsets of digit d inside the tile and in the output
  {
    const int d = threadIdx.x;
    uint32_t tsum_d = 0;
    for (int w = 0; w < RTW; ++w) tsum_d += S.wcur[w][d];
    uint32_t x = tsum_d;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(TFULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) S.tsum[wl] = x;
    __syncthreads();
    uint32_t run = x - tsum_d;
    for (int w = 0; w < wl; ++w) run += S.tsum[w];
    S.loc[d] = run;
    S.gbase[d] = seg[d] + pre[(uint64_t)d * ntiles + blockIdx.x];
    for (int w = 0; w < RTW; ++w) { const uint32_t c = S.wcur[w][d]; S.wcur[w][d] = run; run += c; }
  }
  __syncthreads();
  // 4. stable placement by digit
  for (int base = w0; base < w1; base += 32) {
    const int i = base + lane;
    const bool v = i < w1;
    const uint32_t d = v ? S.dig[i] : 0u;
    const uint32_t peers = match8(d, v);
    uint32_t pos = 0;
    if (v) pos = S.wcur[wl][d] + __popc(peers & lt);
    __syncwarp();
    if (v && lane == __ffs(peers) - 1) S.wcur[wl][d] += __popc(peers);
    __syncwarp();
    if (v) S.perm[pos] = (uint16_t)i;
  }
  __syncthreads();
  // 5. each digit's run goes out contiguously
  for (int j = threadIdx.x; j < len; j += RTT) {
    const uint32_t i = S.perm[j], d = S.dig[i];
    const uint64_t o = S.gbase[d] + (j - S.loc[d]);
    key_out[o] = S.key[i];
    idx_out[o] = S.idx[i];
    let_out[o] = S.let[i];
  }
}

// bitwise OR and AND of all keys: a digit on which they agree needs no pass
template <typename K>
__global__ void k_t_bits(const K* key, uint64_t n, unsigned long long* orand) {
  unsigned long long o = 0, a = ~0ull;
  const uint64_t gt = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, gs = (uint64_t)gridDim.x * blockDim.x;
  // the 16-byte words of the aligned middle, four in flight per thread; the
  // ragged ends one key at a time
  constexpr int KW = 16 / sizeof(K);
  const uint64_t head = min(n, (uint64_t)(((16u - ((uint32_t)(uintptr_t)key & 15u)) & 15u) / sizeof(K)));
  const uint64_t nw = (n - head) / KW;
  const uint4* w = reinterpret_cast<const uint4*>(key + head);
  for (uint64_t q0 = gt; q0 < nw; q0 += 4 * gs) {
    uint4 x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = q0 + j * gs < nw ? w[q0 + j * gs] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (q0 + j * gs >= nw) continue;
      const K* kk = reinterpret_cast<const K*>(&x[j]);
#pragma unroll
      for (int e = 0; e < KW; ++e) { o |= (unsigned long long)kk[e]; a &= (unsigned long long)kk[e]; }
    }
  }
  for (uint64_t i = gt; i < head; i += gs) { o |= (unsigned long long)key[i]; a &= (unsigned long long)key[i]; }
  for (uint64_t i = head + nw * KW + gt; i < n; i += gs) { o |= (unsigned long long)key[i]; a &= (unsigned long long)key[i]; }
  for (int d = 16; d > 0; d >>= 1) {
    o |= __shfl_xor_sync(TFULL, o, d);
    a &= __shfl_xor_sync(TFULL, a, d);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicOr(&orand[0], o);
    atomicAnd(&orand[1], a);
  }
}

// ------------------------------------------------------------------ segmented scan of maps
struct TimelineTab {
  uint64_t maps[RV_MAX_LETTERS];
  uint8_t labels[RV_MAX_STATES];
  int n_states, q0, n_letters;
};

// (a then b) for segment aggregates: b restarts at a head
__device__ __forceinline__ Agg agg_then(Agg a, Agg b, int ns) {
  Agg r;
  r.head = a.head | b.head;
  r.map = b.head ? b.map : apply_map(a.map, b.map, ns);
  r.pad = 0;
  return r;
}

// inclusive scan of one aggregate per thread over the CTA; returns the
// exclusive prefix of this thread, and the CTA total in *total
__device__ Agg cta_exscan(Agg mine, int ns, Agg* total) {
  __shared__ Agg wtot[TT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  Agg incl = mine;
  for (int d = 1; d < 32; d <<= 1) {
    Agg y;
    y.map = __shfl_up_sync(TFULL, incl.map, d);
    y.head = __shfl_up_sync(TFULL, incl.head, d);
    if (lane >= d) incl = agg_then(y, incl, ns);
  }
  if (lane == 31) wtot[w] = incl;
  __syncthreads();
  Agg before{IDENTITY_MAP, 0, 0};
  for (int v = 0; v < w; ++v) before = agg_then(before, wtot[v], ns);
  Agg all = before;
  for (int v = w; v < TT / 32; ++v) all = agg_then(all, wtot[v], ns);
  Agg ex;
  ex.map = __shfl_up_sync(TFULL, incl.map, 1);
  ex.head = __shfl_up_sync(TFULL, incl.head, 1);
  if (lane == 0) { ex.map = IDENTITY_MAP; ex.head = 0; }
  *total = all;
  __syncthreads();
  return agg_then(before, ex, ns);
}

// A thread's TV consecutive events in registers: keys, letters (four to a
// word) and, for the emit, trace indices; 16-byte loads when the thread's
// events are whole and aligned (the radix buffers always are), else one by one.
template <typename K>
struct Events {
  K k[TV];
  uint32_t lw[TV / 4];
  int cnt;
  __device__ __forceinline__ uint32_t letter(int v) const { return (lw[v >> 2] >> (8 * (v & 3))) & 0xFFu; }
};

template <typename K>
__device__ __forceinline__ void load_events(const K* key, const uint8_t* let, uint64_t n, uint64_t i0, Events<K>& e) {
  e.cnt = i0 < n ? (int)min((uint64_t)TV, n - i0) : 0;
  const bool vec = e.cnt == TV && ((((uintptr_t)(key + i0)) | ((uintptr_t)(let + i0))) & 15) == 0;
  if (vec) {
    const uint4* kp = reinterpret_cast<const uint4*>(key + i0);
#pragma unroll
    for (int q = 0; q < (int)(TV * sizeof(K) / 16); ++q) {
      const uint4 x = kp[q];
      if constexpr (sizeof(K) == 4) {
        e.k[4 * q] = x.x; e.k[4 * q + 1] = x.y; e.k[4 * q + 2] = x.z; e.k[4 * q + 3] = x.w;
      } else {
        e.k[2 * q] = (K)x.y << 32 | x.x;
        e.k[2 * q + 1] = (K)x.w << 32 | x.z;
      }
    }
    const uint4 lx = *reinterpret_cast<const uint4*>(let + i0);
    e.lw[0] = lx.x; e.lw[1] = lx.y; e.lw[2] = lx.z; e.lw[3] = lx.w;
  } else {
#pragma unroll
    for (int w = 0; w < TV / 4; ++w) e.lw[w] = 0;
#pragma unroll
    for (int v = 0; v < TV; ++v) {
      e.k[v] = v < e.cnt ? key[i0 + v] : (K)0;
      if (v < e.cnt) e.lw[v >> 2] |= (uint32_t)let[i0 + v] << (8 * (v & 3));
    }
  }
}

// the key before the thread's first event; for event 0 of the trace one
// that differs from it (so event 0 starts a segment)
template <typename K>
__device__ __forceinline__ K key_before(const K* key, uint64_t i0, const Events<K>& e) {
  return i0 > 0 ? key[i0 - 1] : (K)~e.k[0];
}

// the letters' maps and the states' labels, staged in shared memory
struct TabShared {
  uint64_t maps[RV_MAX_LETTERS];
  uint8_t labels[RV_MAX_STATES];
};
__device__ __forceinline__ void stage_tab(const TimelineTab& tab, TabShared& T) {
  for (int l = threadIdx.x; l < RV_MAX_LETTERS; l += blockDim.x) T.maps[l] = l < tab.n_letters ? tab.maps[l] : tab.maps[0];
  if (threadIdx.x < RV_MAX_STATES) T.labels[threadIdx.x] = tab.labels[threadIdx.x];
}

template <typename K>
__device__ __forceinline__ Agg thread_agg(const Events<K>& e, K prev, const TabShared& T, int ns) {
  Agg a{IDENTITY_MAP, 0, 0};
#pragma unroll
  for (int v = 0; v < TV; ++v) {
    if (v < e.cnt) {
      const uint64_t m = T.maps[e.letter(v)];
      if (e.k[v] != (v ? e.k[v - 1] : prev)) { a.head = 1; a.map = m; }
      else a.map = apply_map(a.map, m, ns);
    }
  }
  return a;
}

template <typename K>
__global__ void __launch_bounds__(TT)
k_t_tiles(const K* key, const uint8_t* let, uint64_t n, TimelineTab tab, Agg* tiles, unsigned int* err) {
  __shared__ TabShared T;
  stage_tab(tab, T);
  const uint64_t i0 = (uint64_t)blockIdx.x * TTILE + (uint64_t)threadIdx.x * TV;
  Events<K> e;
  load_events(key, let, n, i0, e);
  const K prev = e.cnt ? key_before(key, i0, e) : (K)0;
  bool bad = false;
#pragma unroll
  for (int v = 0; v < TV; ++v)
    if (v < e.cnt && e.letter(v) >= (uint32_t)tab.n_letters) bad = true;
  __syncthreads();
  Agg total;
  const Agg mine = thread_agg(e, prev, T, tab.n_states);
  cta_exscan(mine, tab.n_states, &total);
  if (threadIdx.x == 0) tiles[blockIdx.x] = total;
  if (__any_sync(TFULL, bad) && (threadIdx.x & 31) == 0) atomicOr(err, (unsigned)ERR_LETTER);
}

// exclusive scan of the tile aggregates (one CTA, TT per round)
__global__ void __launch_bounds__(TT) k_t_tilescan(Agg* tiles, uint64_t ntiles, int ns) {
  __shared__ Agg carry;
  if (threadIdx.x == 0) carry = Agg{IDENTITY_MAP, 0, 0};
  __syncthreads();
  for (uint64_t b = 0; b < ntiles; b += TT) {
    const uint64_t i = b + threadIdx.x;
    const Agg mine = i < ntiles ? tiles[i] : Agg{IDENTITY_MAP, 0, 0};
    Agg total;
    const Agg ex = cta_exscan(mine, ns, &total);
    const Agg c = carry;
    if (i < ntiles) tiles[i] = agg_then(c, ex, ns);
    __syncthreads();
    if (threadIdx.x == 0) carry = agg_then(c, total, ns);
    __syncthreads();
  }
}

template <typename K>
__global__ void __launch_bounds__(TT)
k_t_emit(const K* key, const uint32_t* idx, const uint8_t* let, uint64_t n, TimelineTab tab, const Agg* tiles,
         uint8_t* verdict, uint64_t* vkey, uint32_t* vidx, unsigned long long* nviol) {
  __shared__ TabShared T;
  stage_tab(tab, T);
  const uint64_t i0 = (uint64_t)blockIdx.x * TTILE + (uint64_t)threadIdx.x * TV;
  Events<K> e;
  load_events(key, let, n, i0, e);
  const K prev = e.cnt ? key_before(key, i0, e) : (K)0;
  uint32_t jj[TV];
  if (e.cnt == TV && ((uintptr_t)(idx + i0) & 15) == 0) {
    const uint4* ip = reinterpret_cast<const uint4*>(idx + i0);
#pragma unroll
    for (int q = 0; q < TV / 4; ++q) {
      const uint4 x = ip[q];
      jj[4 * q] = x.x; jj[4 * q + 1] = x.y; jj[4 * q + 2] = x.z; jj[4 * q + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int v = 0; v < TV; ++v) jj[v] = v < e.cnt ? idx[i0 + v] : 0u;
  }
  __syncthreads();
  Agg total;
  const Agg mine = thread_agg(e, prev, T, tab.n_states);
  const Agg ex = agg_then(tiles[blockIdx.x], cta_exscan(mine, tab.n_states, &total), tab.n_states);
  // the state before this thread's first event (meaningless if that event is a head)
  uint32_t q = step_state((uint32_t)tab.q0, ex.map);
  uint32_t vprev = T.labels[q];
#pragma unroll
  for (int v = 0; v < TV; ++v) {
    if (v < e.cnt) {
      const uint64_t m = T.maps[e.letter(v)];
      if (e.k[v] != (v ? e.k[v - 1] : prev)) { q = (uint32_t)tab.q0; vprev = 0xFFu; }
      q = step_state(q, m);
      const uint32_t vd = T.labels[q];
      verdict[jj[v]] = (uint8_t)vd;
      if (vd == RV_BOT && vprev != RV_BOT) {       // F is permanent: the binding's first F event
        const unsigned long long slot = atomicAdd(nviol, 1ull);
        vkey[slot] = (uint64_t)e.k[v];
        vidx[slot] = jj[v];
      }
      vprev = vd;
    }
  }
}

// ------------------------------------------------------------------ host side
struct TPlan {
  uint64_t per_warp, ntiles;
  int G_w;
  size_t o_k0, o_k1, o_i0, o_i1, o_l0, o_l1, o_hist, o_tot, o_tiles, o_orand, o_err, o_letters, total;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

TPlan tplan(uint64_t n, int kbytes) {
  TPlan p{};
  p.per_warp = RT;
  p.G_w = (int)std::max<uint64_t>(1, (n + RT - 1) / RT);       // radix tiles
  p.ntiles = std::max<uint64_t>(1, (n + TTILE - 1) / TTILE);
  size_t off = 0;
  auto take = [&](size_t b) { size_t r = off; off = a256(off + b); return r; };
  const uint64_t m = std::max<uint64_t>(n, 1);
  p.o_k0 = take(m * kbytes);
  p.o_k1 = take(m * kbytes);
  p.o_i0 = take(m * 4);
  p.o_i1 = take(m * 4);
  p.o_l0 = take(m);
  p.o_l1 = take(m);
  p.o_hist = take((size_t)p.G_w * 256 * 4);
  p.o_tot = take(512 * 8);                  // digit totals, then segment starts
  p.o_tiles = take(p.ntiles * sizeof(Agg));
  p.o_orand = take(16);
  p.o_err = take(16);
  p.o_letters = take(m);
  p.total = off;
  return p;
}

#define TCU(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return rv_fail(RV_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));  \
  } while (0)

__global__ void k_t_iota(uint32_t* idx, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    idx[i] = (uint32_t)i;
}

template <typename K>
__global__ void k_t_const(K* key, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    key[i] = 0;
}

// innermost binding key of every event: the key (one or two variables), or
// one constant key for an unquantified property
template <typename K>
rv_status run_timeline(const rv_formula* f, const rv_trace* t, unsigned char* ws, const TPlan& p, uint8_t* verdict,
                       uint64_t* vkey, uint32_t* vidx, unsigned long long* nviol, cudaStream_t s) {
  const uint64_t n = t->n;
  K* kbuf[2] = {(K*)(ws + p.o_k0), (K*)(ws + p.o_k1)};
  uint32_t* ibuf[2] = {(uint32_t*)(ws + p.o_i0), (uint32_t*)(ws + p.o_i1)};
  uint8_t* lbuf[2] = {ws + p.o_l0, ws + p.o_l1};
  uint32_t* hist = (uint32_t*)(ws + p.o_hist);
  uint64_t* tot = (uint64_t*)(ws + p.o_tot);
  Agg* tiles = (Agg*)(ws + p.o_tiles);
  unsigned long long* orand = (unsigned long long*)(ws + p.o_orand);
  unsigned int* err = (unsigned int*)(ws + p.o_err);
  TCU(cudaMemsetAsync(nviol, 0, 8, s));
  TCU(cudaMemsetAsync(err, 0, 4, s));
  const uint8_t* pred = t->pred;
  if (f->n_cmp) {                     // comparison atoms: fold each event's value into its letter
    uint8_t* letters = ws + p.o_letters;
    RV_LAUNCH("k_cmp_letters", k_cmp_letters, 1024, 256, 0, s, pred, t->value, n, cmp_tab(f), letters, err,
              (unsigned)ERR_LETTER);
    pred = letters;
  }
  const K* key = (const K*)t->key;
  if (f->n_quant == 0) {              // one binding: the whole trace
    RV_LAUNCH("k_t_const", k_t_const<K>, 1024, 256, 0, s, kbuf[1], n);
    key = kbuf[1];
  }
  // digits on which every key agrees need no pass
  const unsigned long long init[2] = {0ull, ~0ull};
  TCU(cudaMemcpyAsync(orand, init, 16, cudaMemcpyHostToDevice, s));
  RV_LAUNCH("k_t_bits", k_t_bits<K>, 1024, 256, 0, s, key, n, orand);
  unsigned long long h_orand[2];
  TCU(cudaMemcpyAsync(h_orand, orand, 16, cudaMemcpyDeviceToHost, s));
  TCU(cudaStreamSynchronize(s));
  const unsigned long long differ = h_orand[0] ^ h_orand[1];
  const int grid = p.G_w;
  const K* cur_k = key;
  const uint32_t* cur_i = nullptr;      // identity permutation before the first pass
  const uint8_t* cur_l = pred;
  int out = 0;
  for (int shift = 0; shift < (int)sizeof(K) * 8; shift += 8) {
    if (((differ >> shift) & 255ull) == 0) continue;
    RV_LAUNCH("k_t_hist", k_t_hist<K>, grid, RTT, 0, s, cur_k, n, shift, hist, p.G_w);
    RV_LAUNCH("k_t_colscan", k_t_colscan, 256, 1024, 0, s, hist, p.G_w, tot);
    RV_LAUNCH("k_t_segs", k_t_segs, 1, 256, 0, s, tot, tot + 256);
    RV_LAUNCH("k_t_scatter", k_t_scatter<K>, grid, RTT, sizeof(RadixShared<K>), s, cur_k, cur_i, cur_l, n, shift,
              hist, p.G_w, tot + 256, kbuf[out], ibuf[out], lbuf[out]);
    cur_k = kbuf[out];
    cur_i = ibuf[out];
    cur_l = lbuf[out];
    out ^= 1;
  }
  if (!cur_i) {                          // every key equal: the trace order is already grouped
    RV_LAUNCH("k_t_iota", k_t_iota, 1024, 256, 0, s, ibuf[out], n);
    cur_i = ibuf[out];
  }
  TimelineTab tab;
  memset(&tab, 0, sizeof tab);
  for (int l = 0; l < RV_MAX_LETTERS; ++l) tab.maps[l] = l < f->n_letters ? f->maps[l] : IDENTITY_MAP;
  memcpy(tab.labels, f->labels, sizeof tab.labels);
  tab.n_states = f->n_states;
  tab.q0 = f->q0;
  tab.n_letters = f->n_letters;
  RV_LAUNCH("k_t_tiles", k_t_tiles<K>, (unsigned)p.ntiles, TT, 0, s, cur_k, cur_l, n, tab, tiles, err);
  RV_LAUNCH("k_t_tilescan", k_t_tilescan, 1, TT, 0, s, tiles, p.ntiles, tab.n_states);
  RV_LAUNCH("k_t_emit", k_t_emit<K>, (unsigned)p.ntiles, TT, 0, s, cur_k, cur_i, cur_l, n, tab, tiles, verdict,
            vkey, vidx, nviol);
  TCU(cudaGetLastError());
  unsigned int h_err = 0;
  TCU(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s));
  TCU(cudaStreamSynchronize(s));
  if (h_err & ERR_LETTER) return rv_fail(RV_EINVAL, "predicate code out of range");
  return RV_OK;
}

}  // namespace

rv_status radix_attrs() {
  if (cudaFuncSetAttribute(k_t_scatter<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(RadixShared<uint32_t>)) != cudaSuccess ||
      cudaFuncSetAttribute(k_t_scatter<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(RadixShared<uint64_t>)) != cudaSuccess)
    return rv_fail(RV_ECUDA, "cannot set the radix tile's shared memory");
  return RV_OK;
}

extern "C" size_t rv_timeline_workspace_size(const rv_formula* f, uint64_t n) {
  if (!f) return 0;
  return tplan(n, f->key_bits / 8).total;
}

extern "C" rv_status rv_verify_timeline(const rv_formula* f, const rv_trace* t, void* ws, size_t ws_bytes,
                                        uint8_t* event_verdicts, uint64_t* viol_keys, uint32_t* viol_index,
                                        uint64_t* n_viol, cudaStream_t s) {
  if (!f || !t || !n_viol) return rv_fail(RV_EINVAL, "null argument");
  if (t->n > 0xFFFFFFFFull) return rv_fail(RV_EINVAL, "traces are limited to 2^32-1 events");
  if (t->n && (!t->pred || (f->n_quant && !t->key) || !event_verdicts || !viol_keys || !viol_index || !ws))
    return rv_fail(RV_EINVAL, "null array");
  if (t->n && f->n_cmp && !t->value)
    return rv_fail(RV_EINVAL, "the formula compares the value column: the trace needs its value array");
  if (t->n == 0) {
    TCU(cudaMemsetAsync(n_viol, 0, 8, s));
    TCU(cudaStreamSynchronize(s));
    return RV_OK;
  }
  const TPlan p = tplan(t->n, f->key_bits / 8);
  if (ws_bytes < p.total) return rv_fail(RV_ENOMEM, "timeline workspace of %zu bytes, need %zu", ws_bytes, p.total);
  if (rv_status st = rv_once_per_device(RV_ONCE_EXTRA, &radix_attrs)) return st;
  unsigned long long* nv = (unsigned long long*)n_viol;
  if (f->key_bits == 64)
    return run_timeline<uint64_t>(f, t, (unsigned char*)ws, p, event_verdicts, viol_keys, viol_index, nv, s);
  return run_timeline<uint32_t>(f, t, (unsigned char*)ws, p, event_verdicts, viol_keys, viol_index, nv, s);
}
