// Batched verification: many traces of uneven length, each checked against
// its own list of up to 32 single-quantifier formulas, in one fixed sequence
// of launches that is captured once in a CUDA graph and replayed.
//
// Layout: the traces are concatenated (key uint32[n], pred uint8[n]) with CSR
// offsets; trace t owns events offsets[t]..offsets[t+1].  The formulas of a
// trace all quantify the same key, so the trace is grouped once and every
// binding's events are read once for all its formulas (Algorithm 1 with the
// SortTrace/SpawnMonitors work shared by the formulas of a trace).
//
// map      k_bhist / k_bscan_a,b,c / k_scan64 / k_bscatter: each trace gets
//          2^bits_t buckets by the top bits of mix32(key) (bits_t from its
//          length and the autotuned target bucket size, 4 <= bits_t <= 11),
//          so buckets never mix traces.  A record is 4 bytes: the mixed key's
//          bits below the bucket's (at most 28, which identify the binding
//          inside its bucket, mix32 being a bijection) above a 4-bit letter.
//          Warp tiles never cross a trace boundary and keep private cursors,
//          so records keep trace order inside each bucket.
// monitor  k_bfold: per bucket, chunks of records are stably counting-sorted
//          by binding slot in shared memory; then warps walk the bindings'
//          letter runs with lane f stepping formula f's monitor (states in
//          shared memory between chunks, in registers along a run).
// reduce   per (trace, formula) verdict counts; k_broot applies each
//          formula's quantifier constraint (exact integers).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "profile.h"
#include "rv_device.cuh"

using namespace rvd;

void* rv_dev_alloc(size_t bytes);
void rv_dev_free(void* p);

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int BW = 4;                 // warps per CTA in the split kernels (32 KB of cursors)
constexpr int BATCHR = 16;            // load batching
constexpr int MAXF = 32;              // formulas per trace (one per lane)
constexpr int MAXL = 16;              // letters per formula in batched mode
constexpr int MAXBITS = 11;           // at most 2048 buckets per trace
constexpr int MINBITS = 4;            // at least 16: a record keeps the 28 mixed-key bits below the bucket's
// CTAs of the split resident per SM.  Each warp writes its tile's records to
// up to 2048 bucket positions at once; with more tiles in flight the open,
// partly written sectors outgrow L2 and cost DRAM read-modify-writes, so the
// split is launched with enough (unused) dynamic shared memory that no more
// than this many CTAs fit an SM's 228 KB.
constexpr int SCATTER_CPS = 4;
constexpr int SCATTER_STATIC = BW * (1 << MAXBITS) * 4;            // the cursors
constexpr int SCATTER_PAD = (228 * 1024 / SCATTER_CPS - 1024 - SCATTER_STATIC) / 1024 * 1024;
constexpr int FW = 8;                 // warps per CTA in k_bfold (three CTAs per SM)
constexpr int CHUNK = 4096;           // records sorted at once in k_bfold
constexpr int BSLOTS = 512;           // bindings per pass over a bucket held in shared memory
constexpr int SSLOTS = 32;            // bindings of a long bucket's segment kept as composed maps
constexpr int MAXPASSBITS = 16;       // a bucket's bindings split into at most 2^16 passes
constexpr int BHT_BITS = 10;
constexpr int BHT = 1 << BHT_BITS;
constexpr uint16_t NO_SLOT = 0xFFFF, FULL_SLOT = 0xFFFE;
constexpr uint32_t EMPTY32 = 0xFFFFFFFFu;

struct WTile { uint32_t trace, nb; uint64_t begin, end, hist_off; };

struct BatchDev {
  const WTile* tiles;
  const uint32_t* bucket_base;   // [nt+1] first global bucket of trace t
  const uint32_t* bucket_trace;  // [NB] trace of global bucket
  const uint32_t* trace_bits;    // [nt]
  const uint32_t* tile_first;    // [nt+1] first warp tile of trace t
  const uint64_t* maps;          // [nt][MAXL][MAXF]
  const uint8_t* labels;         // [nt][MAXF][16]
  const rv_quant* quants;        // [nt][MAXF]
  const uint32_t* nletters;      // [nt]
  const uint64_t* offsets;       // [nt+1]
  int nt, nf, NB, ntiles;
};


__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

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

__device__ __forceinline__ uint32_t bucket_of(uint32_t key, uint32_t bits) {
  return bits ? mix32(key) >> (32 - bits) : 0u;
}

__global__ void __launch_bounds__(BW * 32)
k_bhist(BatchDev d, const uint32_t* key, const uint8_t* pred, uint32_t* hist, unsigned int* err) {
  __shared__ uint32_t cnt_all[BW][1 << MAXBITS];
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x * BW + wl;
  if (tile >= d.ntiles) return;
  const WTile T = d.tiles[tile];
  const uint32_t bits = d.trace_bits[T.trace], nl = d.nletters[T.trace];
  uint32_t* cnt = cnt_all[wl];
  for (uint32_t b = lane; b < T.nb; b += 32) cnt[b] = 0;
  __syncwarp();
  bool bad = false;
  for (uint64_t base = T.begin; base < T.end; base += 32 * BATCHR) {
    // all BATCHR rounds' keys and predicates are loaded before any is used,
    // so a lane waits for one memory round trip per batch, not per round
    uint32_t k[BATCHR], l[BATCHR];
#pragma unroll
    for (int j = 0; j < BATCHR; ++j) {
      const uint64_t i = base + j * 32 + lane;
      k[j] = i < T.end ? key[i] : 0u;
      l[j] = i < T.end ? (uint32_t)pred[i] : 0u;
    }
#pragma unroll
    for (int j = 0; j < BATCHR; ++j) {
      if (base + j * 32 + lane < T.end) {
        atomicAdd(&cnt[bucket_of(k[j], bits)], 1u);
        if (l[j] >= nl) bad = true;
      }
    }
  }
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(err, (unsigned)ERR_LETTER);
  __syncwarp();
  for (uint32_t b = lane; b < T.nb; b += 32) hist[T.hist_off + b] = cnt[b];
}

// one thread per global bucket: exclusive prefix over the tiles of its trace
// Exclusive prefix of every bucket's counts over the tiles of its trace, in
// chunks of SCAN_CH tiles so that a long trace's columns are scanned by many
// threads: per (bucket, chunk) sums, then each bucket's chunk sums scanned,
// then each chunk's prefixes on top of the earlier chunks'.  Grid y = chunk.
constexpr int SCAN_CH = 64;
constexpr int SCAN_R = 16;            // loads of a column issued before their sums

__device__ __forceinline__ bool chunk_of(const BatchDev& d, int g, int c, uint32_t* b, uint32_t* t0, uint32_t* t1) {
  const uint32_t t = d.bucket_trace[g];
  *b = g - d.bucket_base[t];
  const uint32_t first = d.tile_first[t], last = d.tile_first[t + 1];
  *t0 = first + (uint32_t)c * SCAN_CH;
  *t1 = min(last, *t0 + SCAN_CH);
  return *t0 < last;
}

__global__ void k_bscan_a(BatchDev d, const uint32_t* hist, uint64_t* part) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
  uint32_t b, t0, t1;
  if (g >= d.NB || !chunk_of(d, g, c, &b, &t0, &t1)) return;
  uint64_t sum = 0;
  for (uint32_t j0 = t0; j0 < t1; j0 += SCAN_R) {
    uint32_t x[SCAN_R];
#pragma unroll
    for (int j = 0; j < SCAN_R; ++j) x[j] = j0 + j < t1 ? hist[d.tiles[j0 + j].hist_off + b] : 0u;
#pragma unroll
    for (int j = 0; j < SCAN_R; ++j) sum += x[j];
  }
  part[(uint64_t)c * d.NB + g] = sum;
}

// per bucket: its chunk sums replaced by their exclusive prefix; tot = the bucket's size
__global__ void k_bscan_b(BatchDev d, uint64_t* part, uint64_t* tot) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= d.NB) return;
  const uint32_t t = d.bucket_trace[g];
  const uint32_t nch = (d.tile_first[t + 1] - d.tile_first[t] + SCAN_CH - 1) / SCAN_CH;
  uint64_t run = 0;
  for (uint32_t c = 0; c < nch; ++c) {
    const uint64_t x = part[(uint64_t)c * d.NB + g];
    part[(uint64_t)c * d.NB + g] = run;
    run += x;
  }
  tot[g] = run;
}

__global__ void k_bscan_c(BatchDev d, uint32_t* hist, const uint64_t* part) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
  uint32_t b, t0, t1;
  if (g >= d.NB || !chunk_of(d, g, c, &b, &t0, &t1)) return;
  uint64_t run = part[(uint64_t)c * d.NB + g];
  for (uint32_t j0 = t0; j0 < t1; j0 += SCAN_R) {
    uint32_t x[SCAN_R];
#pragma unroll
    for (int j = 0; j < SCAN_R; ++j) x[j] = j0 + j < t1 ? hist[d.tiles[j0 + j].hist_off + b] : 0u;
#pragma unroll
    for (int j = 0; j < SCAN_R; ++j) {
      if (j0 + j < t1) hist[d.tiles[j0 + j].hist_off + b] = (uint32_t)run;
      run += x[j];
    }
  }
}

__global__ void __launch_bounds__(1024) k_scan64(const uint64_t* tot, int P, uint64_t* out) {
  __shared__ uint64_t wsum[32];
  __shared__ uint64_t carry;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (t == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < P; base += 4096) {
    uint64_t v[4], s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = base + t * 4 + j;
      v[j] = i < P ? tot[i] : 0ull;
      s += v[j];
    }
    uint64_t x = s;
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      uint64_t z = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(FULL, z, o);
        if (lane >= o) z += y;
      }
      wsum[lane] = z;
    }
    __syncthreads();
    uint64_t run = carry + x - s + (w ? wsum[w - 1] : 0ull);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = base + t * 4 + j;
      if (i < P) out[i] = run;
      run += v[j];
    }
    __syncthreads();
    if (t == 1023) carry = run;
    __syncthreads();
  }
  if (t == 0) out[P] = carry;
}

__global__ void __launch_bounds__(BW * 32)
k_bscatter(BatchDev d, const uint32_t* key, const uint8_t* pred, const uint32_t* pre, const uint64_t* bstart,
           uint32_t* recs) {
  __shared__ uint32_t cur_all[BW][1 << MAXBITS];
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x * BW + wl;
  if (tile >= d.ntiles) return;
  const WTile T = d.tiles[tile];
  const uint32_t bits = d.trace_bits[T.trace], nl = d.nletters[T.trace];
  const uint32_t gb = d.bucket_base[T.trace];
  uint32_t* cur = cur_all[wl];
  // the tile's cursors: eight bucket starts and offsets per lane in flight
  // before any cursor is stored
  constexpr int CB = 8;
  for (uint32_t c0 = 0; c0 < T.nb; c0 += 32 * CB) {
    uint64_t bs[CB];
    uint32_t po[CB];
#pragma unroll
    for (int j = 0; j < CB; ++j) {
      const uint32_t b = c0 + j * 32 + lane;
      bs[j] = b < T.nb ? bstart[gb + b] : 0ull;
      po[j] = b < T.nb ? pre[T.hist_off + b] : 0u;
    }
#pragma unroll
    for (int j = 0; j < CB; ++j) {
      const uint32_t b = c0 + j * 32 + lane;
      if (b < T.nb) cur[b] = (uint32_t)(bs[j] + po[j]);
    }
  }
  __syncwarp();
  const uint32_t lt = lanemask_lt();
  for (uint64_t base = T.begin; base < T.end; base += 32 * BATCHR) {
    uint32_t b[BATCHR];
    uint32_t r[BATCHR];
    // all BATCHR rounds' keys and predicates are loaded before any is used
#pragma unroll
    for (int j = 0; j < BATCHR; ++j) {
      const uint64_t i = base + j * 32 + lane;
      r[j] = i < T.end ? key[i] : 0u;
      b[j] = i < T.end ? (uint32_t)pred[i] : 0u;
    }
#pragma unroll
    for (int j = 0; j < BATCHR; ++j) {
      const uint64_t i = base + j * 32 + lane;
      if (i < T.end) {
        uint32_t l = b[j];
        if (l >= nl) l = 0;
        const uint32_t h = mix32(r[j]);
        b[j] = h >> (32 - bits);
        r[j] = ((h & (0xFFFFFFFFu >> bits)) << 4) | l;   // the bucket holds the top bits
      } else {
        b[j] = EMPTY32;
        r[j] = 0;
      }
    }
#pragma unroll
    for (int j = 0; j < BATCHR; ++j) {
      const bool v = b[j] != EMPTY32;
      const uint32_t peers = __match_any_sync(FULL, v ? b[j] : EMPTY32);   // lanes of equal buckets
      uint32_t pos = 0;
      if (v) pos = cur[b[j]] + __popc(peers & lt);
      __syncwarp();
      if (v && lane == __ffs(peers) - 1) cur[b[j]] += __popc(peers);
      __syncwarp();
      if (v) recs[pos] = r[j];
    }
  }
}

// ------------------------------------------------------------------ fold of one bucket
// A long bucket's segment s >= 1 folded into composed maps: one per binding
// and formula (map of the segment's letters, starting from the identity).
struct Slab {
  uint32_t n, valid;             // valid = 0: more than SSLOTS bindings, fold the records instead
  uint32_t keys[SSLOTS];
  uint64_t maps[SSLOTS][MAXF];
};

struct BFoldShared {
  uint64_t lmap[MAXL][MAXF];
  union {                        // k_bseg composes maps, k_bfold steps states: never both
    uint64_t smap[SSLOTS][MAXF]; // segment maps (long-bucket segments)
    uint8_t state[BSLOTS][MAXF];
  };
  uint8_t labels[MAXF][16];
  uint64_t tkey[BHT];            // key | 1 << 32 once claimed, 0 when empty
  uint16_t tslot[BHT];
  uint16_t slot_of[CHUNK];
  uint8_t letter[CHUNK];
  uint8_t sorted[CHUNK];
  uint32_t wcnt[FW][BSLOTS];     // per-warp counts, then per-warp cursors
  uint32_t seg[BSLOTS + 1];
  uint32_t fcount[MAXF][6];
  uint32_t tsum[FW * 32];
  uint32_t pass_bits[MAXPASSBITS + 2], pass_val[MAXPASSBITS + 2];
  unsigned int nslots, ovf, next, npass;
};

// three fold CTAs of FW warps per SM (228 KB of shared memory, 1 KB reserved per CTA)
static_assert(3 * (sizeof(BFoldShared) + 1024) <= 228 * 1024, "three batched fold CTAs per SM");

// the bindings a pass over a bucket folds: low `bits` bits of the binding's
// record key (the mixed key below the bucket's bits) equal to `val`
__device__ __forceinline__ bool in_pass(uint32_t rkey, uint32_t bits, uint32_t val) {
  return bits == 0 || (rkey & ((1u << bits) - 1u)) == val;
}

// slot of `key` in the bucket's table, inserting it when absent (at most cap
// slots); a new slot starts at q0 = 0 (states) or at the identity (maps)
template <bool MAPS>
__device__ int bfind_or_insert(BFoldShared& S, uint32_t key, int cap, unsigned int* err) {
  const uint64_t tag = (uint64_t)key | (1ull << 32);
  uint32_t h = (key * 0x9E3779B9u) >> (32 - BHT_BITS);
  volatile uint64_t* vk = S.tkey;
  volatile uint16_t* vs = S.tslot;
  for (int probe = 0; probe < BHT; ++probe) {
    uint64_t k = vk[h];
    if (k == 0) {
      const unsigned long long prev = atomicCAS((unsigned long long*)&S.tkey[h], 0ull, (unsigned long long)tag);
      if (prev == 0) {
        const unsigned int s = atomicAdd(&S.nslots, 1u);
        if (s >= (unsigned)cap) { S.ovf = 1; __threadfence_block(); vs[h] = FULL_SLOT; return -1; }
        if (MAPS) for (int f = 0; f < MAXF; ++f) S.smap[s][f] = IDENTITY_MAP;
        else for (int f = 0; f < MAXF; ++f) S.state[s][f] = 0;   // q0 = 0 for every compiled monitor
        __threadfence_block();
        vs[h] = (uint16_t)s;
        return (int)s;
      }
      k = prev;
    }
    if (k == tag) {
      uint16_t s;
      int spins = 0;
      while ((s = vs[h]) == NO_SLOT) {
        if (++spins > (1 << 22)) { atomicOr(err, (unsigned)ERR_SPIN); return -1; }
      }
      return s == FULL_SLOT ? -1 : (int)s;
    }
    h = (h + 1) & (BHT - 1);
  }
  S.ovf = 1;
  return -1;
}

constexpr unsigned ERR_BUCKET = 32;   // bindings of one bucket collide in every hash bit of the passes

// Fold records [r0, r1) of a bucket into the table: the bindings of pass
// (pbits, pval) only, at most cap of them.  Chunks of CHUNK records are
// stably counting-sorted by binding slot in shared memory; then warps walk
// the bindings' letter runs with lane f stepping formula f: its state
// (MAPS = false) or its composed map (MAPS = true).  Returns false when the
// pass has more than cap bindings (nothing of the table is then valid).
template <bool MAPS>
__device__ bool fold_records(BFoldShared& S, const uint32_t* recs, uint64_t r0, uint64_t r1, uint32_t pbits,
                             uint32_t pval, int cap, unsigned int* err) {
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31, nthr = FW * 32;
  const uint32_t lt = lanemask_lt();
  for (uint64_t c0 = r0; c0 < r1; c0 += CHUNK) {
    const int cn = (int)min((uint64_t)CHUNK, r1 - c0);
    // 1. binding slot of every record of the chunk (NO_SLOT: not in this
    // pass); a thread's records are all loaded before the first is looked up
    constexpr int RPT = CHUNK / (FW * 32);
    static_assert(CHUNK % (FW * 32) == 0, "whole rounds of records per chunk");
    uint32_t rr[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int i = q * nthr + threadIdx.x;
      rr[q] = i < cn ? recs[c0 + i] : 0u;
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int i = q * nthr + threadIdx.x;
      if (i >= cn) continue;
      const uint32_t r = rr[q];
      const uint32_t key = r >> 4;
      int sl = NO_SLOT;
      if (in_pass(key, pbits, pval)) {
        sl = bfind_or_insert<MAPS>(S, key, cap, err);
        if (sl < 0) sl = 0;
      }
      S.slot_of[i] = (uint16_t)sl;
      S.letter[i] = (uint8_t)(r & 0xFu);
    }
    for (int i = threadIdx.x; i < FW * BSLOTS; i += nthr) S.wcnt[i / BSLOTS][i % BSLOTS] = 0;
    __syncthreads();
    if (S.ovf) return false;
    const int nsl = (int)S.nslots;
    // 2. stable counting sort by slot; warp w owns records [w0, w1) of the chunk
    const int per = (cn + FW - 1) / FW;
    const int w0 = min(cn, wl * per), w1 = min(cn, w0 + per);
    for (int i = w0 + lane; i < w1; i += 32)
      if (S.slot_of[i] != NO_SLOT) atomicAdd(&S.wcnt[wl][S.slot_of[i]], 1u);
    __syncthreads();
    // exclusive scan over (slot, warp): each thread owns 4 consecutive slots
    {
      const int s0 = threadIdx.x * 4;
      uint32_t tot[4], sum = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int sl = s0 + j;
        uint32_t x = 0;
        if (sl < BSLOTS)
          for (int w = 0; w < FW; ++w) x += S.wcnt[w][sl];
        tot[j] = x;
        sum += x;
      }
      uint32_t x = sum;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) S.tsum[wl] = x;
      __syncthreads();
      uint32_t wbase = 0, all = 0;
      for (int w = 0; w < FW; ++w) { if (w < wl) wbase += S.tsum[w]; all += S.tsum[w]; }
      uint32_t run = wbase + x - sum;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int sl = s0 + j;
        if (sl < BSLOTS) {
          S.seg[sl] = run;
          uint32_t r2 = run;
          for (int w = 0; w < FW; ++w) { const uint32_t c = S.wcnt[w][sl]; S.wcnt[w][sl] = r2; r2 += c; }
        }
        run += tot[j];
      }
      if (threadIdx.x == 0) S.seg[BSLOTS] = all;   // records of this pass in the chunk
    }
    __syncthreads();
    for (int base = w0; base < w1; base += 32) {
      const int i = base + lane;
      const uint32_t sl = i < w1 ? S.slot_of[i] : (uint32_t)NO_SLOT;
      const bool v = sl != NO_SLOT;
      const uint32_t peers = __match_any_sync(FULL, v ? sl : 0xFFFFFFFFu);   // lanes of equal slots
      uint32_t pos = 0;
      if (v) pos = S.wcnt[wl][sl] + __popc(peers & lt);
      __syncwarp();
      if (v && lane == __ffs(peers) - 1) S.wcnt[wl][sl] += __popc(peers);
      __syncwarp();
      if (v) S.sorted[pos] = S.letter[i];
    }
    __syncthreads();
    // 3. walk every binding's letters: lane f steps formula f
    for (int sl = wl; sl < nsl; sl += FW) {
      const uint32_t lo = S.seg[sl], hi = S.seg[sl + 1];
      if (MAPS) {
        uint64_t M = S.smap[sl][lane];
        for (uint32_t base = lo; base < hi; base += 32) {
          const uint32_t n = min(32u, hi - base);
          const uint32_t mine = lane < n ? S.sorted[base + lane] : 0u;
          for (uint32_t j = 0; j < n; ++j) M = compose16(M, S.lmap[__shfl_sync(FULL, mine, j)][lane]);
        }
        S.smap[sl][lane] = M;
      } else {
        uint32_t st = S.state[sl][lane];
        for (uint32_t base = lo; base < hi; base += 32) {
          const uint32_t n = min(32u, hi - base);
          const uint32_t mine = lane < n ? S.sorted[base + lane] : 0u;
          if (n == 32) {
            // a full round: the maps do not depend on the state, so all 32
            // are fetched ahead and only the shift-and-mask chain is serial
#pragma unroll
            for (int j0 = 0; j0 < 32; j0 += 8) {
              uint64_t m[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) m[j] = S.lmap[__shfl_sync(FULL, mine, j0 + j)][lane];
#pragma unroll
              for (int j = 0; j < 8; ++j) st = step_state(st, m[j]);
            }
          } else {
            for (uint32_t j = 0; j < n; ++j) st = step_state(st, S.lmap[__shfl_sync(FULL, mine, j)][lane]);
          }
        }
        S.state[sl][lane] = (uint8_t)st;
      }
    }
    __syncthreads();
  }
  return true;
}

__device__ void load_tables(BFoldShared& S, const BatchDev& d, uint32_t t) {
  for (int i = threadIdx.x; i < MAXL * MAXF; i += FW * 32)
    S.lmap[i / MAXF][i % MAXF] = d.maps[(uint64_t)t * MAXL * MAXF + i];
  for (int i = threadIdx.x; i < MAXF * 16; i += FW * 32)
    S.labels[i / 16][i % 16] = d.labels[(uint64_t)t * MAXF * 16 + i];
}

__device__ void reset_table(BFoldShared& S) {
  for (int i = threadIdx.x; i < BHT; i += FW * 32) { S.tkey[i] = 0; S.tslot[i] = NO_SLOT; }
  if (threadIdx.x == 0) { S.nslots = 0; S.ovf = 0; }
}

// Long buckets (more than long_records records) are cut into segments of
// long_records records; segment s >= 1 of such a bucket is work item
// item_base[g] + s - 1.  This is the cluster-size threshold above which a
// bucket's runs are split across CTAs: each later segment is folded into
// composed maps by a CTA of its own (k_bseg), and the bucket's fold applies
// them in order after folding segment 0 from q0.
__global__ void k_bextra(const uint64_t* bstart, int NB, uint64_t long_records, uint64_t* extra) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= NB) return;
  const uint64_t len = bstart[g + 1] - bstart[g];
  extra[g] = len > long_records ? (len + long_records - 1) / long_records - 1 : 0;
}

__global__ void __launch_bounds__(FW * 32)
k_bseg(BatchDev d, const uint32_t* recs, const uint64_t* bstart, const uint64_t* item_base, uint64_t long_records,
       Slab* slabs, unsigned int* err, unsigned int* next) {
  extern __shared__ __align__(16) unsigned char bsm[];
  BFoldShared& S = *reinterpret_cast<BFoldShared*>(bsm);
  const uint64_t total = item_base[d.NB];
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) S.next = atomicAdd(next, 1u);
    __syncthreads();
    const uint64_t u = S.next;
    if (u >= total) break;
    int lo = 0, hi = d.NB - 1;               // the bucket g with item_base[g] <= u < item_base[g + 1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (item_base[mid] <= u) lo = mid; else hi = mid - 1;
    }
    const int g = lo;
    const uint64_t sidx = u - item_base[g] + 1;
    const uint64_t r0 = bstart[g] + sidx * long_records, r1 = min(bstart[g + 1], r0 + long_records);
    load_tables(S, d, d.bucket_trace[g]);
    reset_table(S);
    __syncthreads();
    const bool ok = fold_records<true>(S, recs, r0, r1, 0, 0, SSLOTS, err);
    Slab& out = slabs[u];
    if (!ok) {
      if (threadIdx.x == 0) { out.valid = 0; out.n = 0; }
      continue;
    }
    const int nsl = (int)S.nslots;
    for (int i = threadIdx.x; i < BHT; i += FW * 32) {
      const uint16_t sl = S.tslot[i];
      if (sl != NO_SLOT && sl != FULL_SLOT) out.keys[sl] = (uint32_t)S.tkey[i];
    }
    for (int i = threadIdx.x; i < nsl * MAXF; i += FW * 32) out.maps[i / MAXF][i % MAXF] = S.smap[i / MAXF][i % MAXF];
    if (threadIdx.x == 0) { out.n = (uint32_t)nsl; out.valid = 1; }
  }
}

// Apply segment u's slab to the pass's bindings (new ones start at q0);
// false when the pass's table overflows.
__device__ bool apply_slab(BFoldShared& S, const Slab& sb, uint32_t pbits, uint32_t pval, unsigned int* err) {
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = (int)sb.n;
  for (int e = wl; e < n; e += FW) {
    const uint32_t key = sb.keys[e];
    if (!in_pass(key, pbits, pval)) continue;
    int sl = 0;
    if (lane == 0) sl = bfind_or_insert<false>(S, key, BSLOTS, err);
    sl = __shfl_sync(FULL, sl, 0);
    if (sl < 0) continue;
    S.state[sl][lane] = (uint8_t)step_state(S.state[sl][lane], sb.maps[e][lane]);
  }
  __syncthreads();
  return !S.ovf;
}

__global__ void __launch_bounds__(FW * 32)
k_bfold(BatchDev d, const uint32_t* recs, const uint64_t* bstart, const uint64_t* item_base, uint64_t long_records,
        const Slab* slabs, unsigned long long* counts, unsigned long long* nbind, unsigned int* err,
        unsigned int* next) {
  extern __shared__ __align__(16) unsigned char bsm[];
  BFoldShared& S = *reinterpret_cast<BFoldShared*>(bsm);
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31, nthr = FW * 32;
  const int nf = d.nf;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) S.next = atomicAdd(next, 1u);
    __syncthreads();
    const unsigned int g = S.next;
    if (g >= (unsigned)d.NB) break;
    const uint64_t b0 = bstart[g], b1 = bstart[g + 1];
    if (b0 == b1) continue;
    const uint32_t t = d.bucket_trace[g];
    const uint64_t first_item = item_base[g], n_extra = item_base[g + 1] - first_item;
    const uint64_t seg0_end = n_extra ? b0 + long_records : b1;
    load_tables(S, d, t);
    for (int i = threadIdx.x; i < MAXF * 6; i += nthr) S.fcount[i / 6][i % 6] = 0;
    if (threadIdx.x == 0) { S.npass = 1; S.pass_bits[0] = 0; S.pass_val[0] = 0; }
    __syncthreads();
    unsigned long long bound = 0;
    // passes over subsets of the bucket's bindings, split further whenever
    // one holds more than BSLOTS of them
    while (S.npass > 0) {
      const uint32_t pbits = S.pass_bits[S.npass - 1], pval = S.pass_val[S.npass - 1];
      reset_table(S);
      __syncthreads();
      bool ok = fold_records<false>(S, recs, b0, seg0_end, pbits, pval, BSLOTS, err);
      for (uint64_t k = 0; ok && k < n_extra; ++k) {
        const Slab& sb = slabs[first_item + k];
        if (sb.valid) {
          ok = apply_slab(S, sb, pbits, pval, err);
        } else {
          const uint64_t r0 = b0 + (k + 1) * long_records;
          ok = fold_records<false>(S, recs, r0, min(b1, r0 + long_records), pbits, pval, BSLOTS, err);
        }
      }
      __syncthreads();
      if (!ok) {
        if (threadIdx.x == 0) {
          S.npass -= 1;
          if (pbits >= MAXPASSBITS) {
            atomicOr(err, ERR_BUCKET);
          } else {
            S.pass_bits[S.npass] = pbits + 1; S.pass_val[S.npass] = pval;
            S.pass_bits[S.npass + 1] = pbits + 1; S.pass_val[S.npass + 1] = pval | (1u << pbits);
            S.npass += 2;
          }
        }
        __syncthreads();
        continue;
      }
      // 4. verdict counts per formula of this pass's bindings
      uint32_t c[6] = {0, 0, 0, 0, 0, 0};
      const int nsl = (int)S.nslots;
      for (int sl = wl; sl < nsl; sl += FW) {
        const uint32_t v = S.labels[lane][S.state[sl][lane] & 15];
#pragma unroll
        for (int k = 0; k < 6; ++k) c[k] += v == (uint32_t)k;
      }
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (c[k]) atomicAdd(&S.fcount[lane][k], c[k]);
      bound += (unsigned long long)nsl;
      __syncthreads();
      if (threadIdx.x == 0) S.npass -= 1;
      __syncthreads();
    }
    for (int i = threadIdx.x; i < nf * 6; i += nthr) {
      const uint32_t x = S.fcount[i / 6][i % 6];
      if (x) atomicAdd(&counts[((uint64_t)t * nf + i / 6) * 6 + i % 6], (unsigned long long)x);
    }
    if (threadIdx.x == 0) atomicAdd(&nbind[t], bound);
  }
}

__global__ void k_broot(BatchDev d, const unsigned long long* counts, const unsigned long long* nbind,
                        const unsigned int* err, rv_result* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.nt * d.nf) return;
  const int t = i / d.nf;
  rv_result r;
  memset(&r, 0, sizeof r);
  uint64_t v[6];
  for (int k = 0; k < 6; ++k) v[k] = counts[(uint64_t)i * 6 + k];
  const rv_quant q = d.quants[(uint64_t)t * MAXF + i % d.nf];
  r.root = rvv::valuate(q.kind, q.op, q.num, q.den, v);
  for (int k = 0; k < 6; ++k) { r.root_counts[k] = v[k]; r.level_counts[0][k] = v[k]; }
  r.n_nodes[0] = nbind[t];
  r.events = d.offsets[t + 1] - d.offsets[t];
  const unsigned e = *err;
  r.status = (e & ERR_LETTER) ? RV_EINVAL : (e & ERR_SPIN) ? RV_ETIMEOUT : e ? RV_EINTERNAL : RV_OK;
  out[i] = r;
}

#define BCU(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return rv_fail(RV_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

// ------------------------------------------------------------------ host side
struct rv_batch {
  int nt = 0, nf = 0;
  std::vector<uint64_t> offsets;
  std::vector<uint64_t> maps;     // [nt][MAXL][MAXF]
  std::vector<uint8_t> labels;    // [nt][MAXF][16]
  std::vector<rv_quant> quants;   // [nt][MAXF]
  std::vector<uint32_t> nletters; // [nt]
  int bucket_records = 4096;
  int tile_events = 16384;
  int long_records = 1 << 16;     // 0: no long-bucket segments
  // device plan (rebuilt when the tuning changes)
  void* plan = nullptr;
  size_t plan_bytes = 0;
  BatchDev dev{};
  size_t hist_entries = 0;
  int scan_chunks = 1;            // chunks of SCAN_CH tiles of the longest trace
  // captured graph and the arguments it was captured with
  cudaGraphExec_t exec = nullptr;
  const void* g_key = nullptr;
  const void* g_pred = nullptr;
  const void* g_ws = nullptr;
  const void* g_res = nullptr;
  cudaStream_t cap = nullptr;
};

namespace {

struct BatchLayout {
  size_t o_hist, o_part, o_tot, o_bstart, o_recs, o_extra, o_item, o_slabs, o_counts, o_nbind, o_err, o_next, o_next2, total;
  uint64_t max_items;
};

// long_records as the kernels see it: 0 turns the segments off
uint64_t long_len(int long_records) { return long_records > 0 ? (uint64_t)long_records : ~0ull >> 1; }

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

void plan_shape(const rv_batch* b, int bucket_records, int tile_events, std::vector<uint32_t>* bits,
                std::vector<WTile>* tiles, int* NB, size_t* hist_entries, int* scan_chunks) {
  int nb_total = 0;
  size_t hist = 0;
  uint64_t most = 1;
  for (int t = 0; t < b->nt; ++t) {
    const uint64_t len = b->offsets[t + 1] - b->offsets[t];
    most = std::max<uint64_t>(most, (len + tile_events - 1) / tile_events);
    uint32_t k = MINBITS;
    while (k < (uint32_t)MAXBITS && (len >> k) > (uint64_t)bucket_records) ++k;
    if (bits) bits->push_back(k);
    const uint32_t nb = 1u << k;
    for (uint64_t s = b->offsets[t]; s < b->offsets[t + 1]; s += (uint64_t)tile_events) {
      if (tiles) tiles->push_back(WTile{(uint32_t)t, nb, s, std::min(b->offsets[t + 1], s + (uint64_t)tile_events), hist});
      hist += nb;
    }
    nb_total += (int)nb;
  }
  *NB = nb_total;
  *hist_entries = hist;
  *scan_chunks = (int)((most + SCAN_CH - 1) / SCAN_CH);   // chunks of the trace with the most tiles
}

BatchLayout layout(const rv_batch* b, int NB, size_t hist_entries, int scan_chunks, int long_records) {
  BatchLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = a256(off + bytes); return r; };
  const uint64_t n = b->offsets.back();
  L.o_hist = take(std::max<size_t>(hist_entries, 1) * 4);
  L.o_part = take((size_t)NB * scan_chunks * 8);
  L.o_tot = take((size_t)NB * 8);
  L.o_bstart = take((size_t)(NB + 1) * 8);
  L.o_recs = take(std::max<uint64_t>(n, 1) * 4);
  L.o_extra = take((size_t)NB * 8);
  L.o_item = take((size_t)(NB + 1) * 8);
  // every extra segment holds long_records records of its bucket before it
  L.max_items = long_records > 0 ? n / (uint64_t)long_records + 1 : 0;
  L.o_slabs = take(std::max<uint64_t>(L.max_items, 1) * sizeof(Slab));
  L.o_counts = take((size_t)b->nt * b->nf * 6 * 8);   // from here on zeroed before every run
  L.o_nbind = take((size_t)b->nt * 8);
  L.o_err = take(4);
  L.o_next = take(4);
  L.o_next2 = take(4);
  L.total = off;
  return L;
}

rv_status build_plan(rv_batch* b) {
  std::vector<uint32_t> bits;
  std::vector<WTile> tiles;
  int NB = 0;
  size_t hist_entries = 0;
  int chunks = 1;
  plan_shape(b, b->bucket_records, b->tile_events, &bits, &tiles, &NB, &hist_entries, &chunks);
  std::vector<uint32_t> base(b->nt + 1), btrace(NB), tfirst(b->nt + 1);
  int g = 0;
  for (int t = 0; t < b->nt; ++t) {
    base[t] = (uint32_t)g;
    for (uint32_t j = 0; j < (1u << bits[t]); ++j) btrace[g++] = (uint32_t)t;
  }
  base[b->nt] = (uint32_t)g;
  size_t ti = 0;
  for (int t = 0; t < b->nt; ++t) {
    tfirst[t] = (uint32_t)ti;
    while (ti < tiles.size() && tiles[ti].trace == (uint32_t)t) ++ti;
  }
  tfirst[b->nt] = (uint32_t)ti;
  b->scan_chunks = chunks;
  // one device block for every plan array
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = a256(off + bytes); return r; };
  const size_t o_tiles = take(std::max<size_t>(tiles.size(), 1) * sizeof(WTile));
  const size_t o_base = take(base.size() * 4), o_btrace = take(btrace.size() * 4), o_bits = take(bits.size() * 4 + 4);
  const size_t o_tfirst = take(tfirst.size() * 4), o_maps = take(b->maps.size() * 8),
               o_labels = take(b->labels.size()), o_quants = take(b->quants.size() * sizeof(rv_quant)),
               o_nl = take(b->nletters.size() * 4), o_offs = take(b->offsets.size() * 8);
  if (b->plan) { rv_dev_free(b->plan); b->plan = nullptr; }
  b->plan = rv_dev_alloc(off);
  if (!b->plan) return rv_fail(RV_ENOMEM, "cannot allocate %zu bytes for the batch plan", off);
  b->plan_bytes = off;
  unsigned char* P = (unsigned char*)b->plan;
  BCU(cudaMemcpy(P + o_tiles, tiles.data(), tiles.size() * sizeof(WTile), cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(P + o_base, base.data(), base.size() * 4, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(P + o_btrace, btrace.data(), btrace.size() * 4, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(P + o_bits, bits.data(), bits.size() * 4, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(P + o_tfirst, tfirst.data(), tfirst.size() * 4, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(P + o_maps, b->maps.data(), b->maps.size() * 8, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(P + o_labels, b->labels.data(), b->labels.size(), cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(P + o_quants, b->quants.data(), b->quants.size() * sizeof(rv_quant), cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(P + o_nl, b->nletters.data(), b->nletters.size() * 4, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(P + o_offs, b->offsets.data(), b->offsets.size() * 8, cudaMemcpyHostToDevice));
  BatchDev& d = b->dev;
  d.tiles = (const WTile*)(P + o_tiles);
  d.bucket_base = (const uint32_t*)(P + o_base);
  d.bucket_trace = (const uint32_t*)(P + o_btrace);
  d.trace_bits = (const uint32_t*)(P + o_bits);
  d.tile_first = (const uint32_t*)(P + o_tfirst);
  d.maps = (const uint64_t*)(P + o_maps);
  d.labels = (const uint8_t*)(P + o_labels);
  d.quants = (const rv_quant*)(P + o_quants);
  d.nletters = (const uint32_t*)(P + o_nl);
  d.offsets = (const uint64_t*)(P + o_offs);
  d.nt = b->nt;
  d.nf = b->nf;
  d.NB = NB;
  d.ntiles = (int)tiles.size();
  b->hist_entries = hist_entries;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  return RV_OK;
}

int num_sms_b() { return rv_num_sms(); }

rv_status enqueue(rv_batch* b, const uint32_t* key, const uint8_t* pred, unsigned char* ws, rv_result* res,
                  cudaStream_t s) {
  const BatchDev& d = b->dev;
  const BatchLayout L = layout(b, d.NB, b->hist_entries, b->scan_chunks, b->long_records);
  uint32_t* hist = (uint32_t*)(ws + L.o_hist);
  uint64_t* tot = (uint64_t*)(ws + L.o_tot);
  uint64_t* part = (uint64_t*)(ws + L.o_part);
  uint64_t* bstart = (uint64_t*)(ws + L.o_bstart);
  uint32_t* recs = (uint32_t*)(ws + L.o_recs);
  unsigned long long* counts = (unsigned long long*)(ws + L.o_counts);
  unsigned long long* nbind = (unsigned long long*)(ws + L.o_nbind);
  unsigned int* err = (unsigned int*)(ws + L.o_err);
  unsigned int* next = (unsigned int*)(ws + L.o_next);
  unsigned int* next2 = (unsigned int*)(ws + L.o_next2);
  uint64_t* extra = (uint64_t*)(ws + L.o_extra);
  uint64_t* item_base = (uint64_t*)(ws + L.o_item);
  Slab* slabs = (Slab*)(ws + L.o_slabs);
  const uint64_t lr = long_len(b->long_records);
  BCU(cudaMemsetAsync(ws + L.o_counts, 0, L.total - L.o_counts, s));   // counts, nbind, err, next
  const int tb = (d.ntiles + BW - 1) / BW;
  if (d.ntiles) {
    RV_LAUNCH("k_bhist", k_bhist, tb, BW * 32, 0, s, d, key, pred, hist, err);
    const dim3 sg((d.NB + 255) / 256, b->scan_chunks);
    RV_LAUNCH("k_bscan_a", k_bscan_a, sg, 256, 0, s, d, hist, part);
    RV_LAUNCH("k_bscan_b", k_bscan_b, (d.NB + 255) / 256, 256, 0, s, d, part, tot);
    RV_LAUNCH("k_bscan_c", k_bscan_c, sg, 256, 0, s, d, hist, part);
    RV_LAUNCH("k_scan64", k_scan64, 1, 1024, 0, s, tot, d.NB, bstart);
    RV_LAUNCH("k_bscatter", k_bscatter, tb, BW * 32, SCATTER_PAD, s, d, key, pred, hist, bstart, recs);
    RV_LAUNCH("k_bextra", k_bextra, (d.NB + 255) / 256, 256, 0, s, bstart, d.NB, lr, extra);
    RV_LAUNCH("k_scan64", k_scan64, 1, 1024, 0, s, extra, d.NB, item_base);
    const int grid = std::min(d.NB, num_sms_b() * 4);
    if (L.max_items)
      RV_LAUNCH("k_bseg", k_bseg, (int)std::min<uint64_t>(L.max_items, (uint64_t)num_sms_b() * 4), FW * 32,
                sizeof(BFoldShared), s, d, recs, bstart, item_base, lr, slabs, err, next2);
    RV_LAUNCH("k_bfold", k_bfold, grid, FW * 32, sizeof(BFoldShared), s, d, recs, bstart, item_base, lr, slabs,
              counts, nbind, err, next);
  }
  RV_LAUNCH("k_broot", k_broot, (d.nt * d.nf + 127) / 128, 128, 0, s, d, counts, nbind, err, res);
  BCU(cudaGetLastError());
  return RV_OK;
}

}  // namespace

extern "C" rv_status rv_batch_create(const rv_formula* const* f, int nf, int nt, const uint64_t* offsets,
                                     const rv_batch_opts* opts, rv_batch** out) {
  if (!f || !offsets || !out || nf < 1 || nf > MAXF || nt < 1)
    return rv_fail(RV_EINVAL, "batch needs 1..32 formulas per trace and at least one trace");
  *out = nullptr;
  for (int t = 0; t < nt; ++t)
    if (offsets[t + 1] < offsets[t]) return rv_fail(RV_EINVAL, "offsets must be non-decreasing");
  if (offsets[0] != 0) return rv_fail(RV_EINVAL, "offsets[0] must be 0");
  if (offsets[nt] > 0xFFFFFFFFull) return rv_fail(RV_EINVAL, "a batch is limited to 2^32-1 events");
  rv_batch* b = new (std::nothrow) rv_batch();
  if (!b) return rv_fail(RV_ENOMEM, "out of host memory");
  b->nt = nt;
  b->nf = nf;
  b->offsets.assign(offsets, offsets + nt + 1);
  b->maps.assign((size_t)nt * MAXL * MAXF, IDENTITY_MAP);
  b->labels.assign((size_t)nt * MAXF * 16, 0);
  b->quants.assign((size_t)nt * MAXF, rv_quant{RV_Q_E, RV_GE, 1, 1});
  b->nletters.assign(nt, 0);
  for (int t = 0; t < nt; ++t) {
    for (int j = 0; j < nf; ++j) {
      const rv_formula* F = f[(size_t)t * nf + j];
      if (!F || F->n_quant != 1 || F->key_bits != 32 || F->n_letters > MAXL || F->n_cmp) {
        delete b;
        return rv_fail(RV_EUNSUPPORTED, "batched formulas need one quantifier, 32-bit keys, at most 16 letters "
                                         "and no comparison atoms");
      }
      if (j == 0) b->nletters[t] = (uint32_t)F->n_letters;
      else if (b->nletters[t] != (uint32_t)F->n_letters) {
        delete b;
        return rv_fail(RV_EINVAL, "the formulas of one trace must share its alphabet");
      }
      for (int l = 0; l < F->n_letters; ++l) b->maps[((size_t)t * MAXL + l) * MAXF + j] = F->maps[l];
      for (int s = 0; s < 16; ++s) b->labels[((size_t)t * MAXF + j) * 16 + s] = F->labels[s];
      b->quants[(size_t)t * MAXF + j] = F->q[0];
    }
  }
  if (opts && opts->bucket_records) b->bucket_records = opts->bucket_records;
  if (opts && opts->tile_events) b->tile_events = std::max(1024, opts->tile_events);
  if (opts && opts->long_records) b->long_records = opts->long_records < 0 ? 0 : std::max(CHUNK, opts->long_records);
  rv_status st = build_plan(b);
  if (st) { rv_batch_free(b); return st; }
  *out = b;
  return RV_OK;
}

extern "C" size_t rv_batch_workspace_size(const rv_batch* b) {
  if (!b) return 0;
  size_t worst = 0;
  for (int br : {256, 512, 1024, 2048, 4096, 8192, b->bucket_records})
    for (int te : {8192, 16384, 32768, b->tile_events}) {
      int NB = 0, ch = 1;
      size_t he = 0;
      plan_shape(b, br, te, nullptr, nullptr, &NB, &he, &ch);
      for (int lr : {b->long_records, 16384})
        worst = std::max(worst, layout(b, NB, he, ch, lr).total);
    }
  return worst;
}

// the attribute applies to the current device: set it once per device
static_assert(SCATTER_PAD >= 0, "the split's cursors fit SCATTER_CPS CTAs per SM");
static rv_status set_bfold_attr() {
  BCU(cudaFuncSetAttribute(k_bfold, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BFoldShared)));
  BCU(cudaFuncSetAttribute(k_bseg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BFoldShared)));
  BCU(cudaFuncSetAttribute(k_bscatter, cudaFuncAttributeMaxDynamicSharedMemorySize, SCATTER_PAD));
  return RV_OK;
}

extern "C" rv_status rv_batch_run(rv_batch* b, const uint32_t* key, const uint8_t* pred, void* ws, size_t ws_bytes,
                                  rv_result* dev_results, cudaStream_t s) {
  if (!b || !ws || !dev_results || (b->offsets.back() && (!key || !pred)))
    return rv_fail(RV_EINVAL, "null argument");
  const BatchLayout L = layout(b, b->dev.NB, b->hist_entries, b->scan_chunks, b->long_records);
  if (ws_bytes < L.total) return rv_fail(RV_ENOMEM, "workspace of %zu bytes, need %zu", ws_bytes, L.total);
  if (rv_status st = rv_once_per_device(RV_ONCE_BATCH, &set_bfold_attr)) return st;
  if (rv_prof_enabled())   // per-kernel events need eager launches, not a graph replay
    return enqueue(b, key, pred, (unsigned char*)ws, dev_results, s);
  if (!b->exec || b->g_key != key || b->g_pred != pred || b->g_ws != ws || b->g_res != dev_results) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (!b->cap) BCU(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    BCU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    rv_status st = enqueue(b, key, pred, (unsigned char*)ws, dev_results, b->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (st) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) return rv_fail(RV_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { b->exec = nullptr; return rv_fail(RV_ECUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
    b->g_key = key; b->g_pred = pred; b->g_ws = ws; b->g_res = dev_results;
  }
  BCU(cudaGraphLaunch(b->exec, s));
  rv_count_launch();
  return RV_OK;
}

// Times the launch sequence on the caller's inputs for each candidate and
// keeps the fastest: first the bucket size (t1: a bucket's bindings are
// folded by one CTA, lane = formula) and the warp tile of the split, then,
// with those, the long-bucket threshold (t2: longer buckets are cut into
// segments folded by separate CTAs through composed maps; 0 = never).
extern "C" rv_status rv_batch_autotune(rv_batch* b, const uint32_t* key, const uint8_t* pred, void* ws,
                                       size_t ws_bytes, rv_result* dev_results, cudaStream_t s,
                                       rv_batch_opts* chosen) {
  if (!b || !dev_results) return rv_fail(RV_EINVAL, "null argument");
  const int cand_br[] = {1024, 2048, 4096, 8192};
  const int cand_te[] = {8192, 32768};
  const int cand_lr[] = {16384, 65536, 262144, 0};
  float best = 1e30f;
  int best_br = b->bucket_records, best_te = b->tile_events, best_lr = b->long_records;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rv_status st = RV_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    st = rv_fail(RV_ECUDA, "event creation failed");
  auto trial = [&](int br, int te, int lr) -> bool {
    b->bucket_records = br;
    b->tile_events = te;
    b->long_records = lr;
    if ((st = build_plan(b))) return false;
    if ((st = rv_batch_run(b, key, pred, ws, ws_bytes, dev_results, s))) return false;   // capture + warm-up
    float ms = 0.f;
    if (cudaEventRecord(e0, s) != cudaSuccess) { st = rv_fail(RV_ECUDA, "event record"); return false; }
    for (int r = 0; r < 3 && !st; ++r) st = rv_batch_run(b, key, pred, ws, ws_bytes, dev_results, s);
    if (st || cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      if (!st) st = rv_fail(RV_ECUDA, "timing failed");
      return false;
    }
    if (ms < best) { best = ms; best_br = br; best_te = te; best_lr = lr; }
    return true;
  };
  const int lr0 = b->long_records;
  for (int br : cand_br)
    for (int te : cand_te)
      if (!st && !trial(br, te, lr0)) break;
  const int br1 = best_br, te1 = best_te;
  for (int lr : cand_lr)
    if (!st && lr != lr0 && !trial(br1, te1, lr)) break;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  b->bucket_records = best_br;
  b->tile_events = best_te;
  b->long_records = best_lr;
  const rv_status st2 = build_plan(b);
  if (chosen) {
    chosen->bucket_records = best_br;
    chosen->tile_events = best_te;
    chosen->long_records = best_lr > 0 ? best_lr : -1;
  }
  return st ? st : st2;
}

extern "C" void rv_batch_free(rv_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->plan) rv_dev_free(b->plan);
  delete b;
}
