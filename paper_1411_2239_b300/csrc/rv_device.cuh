// Device building blocks shared by the offline, batched and streaming paths.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "rv_internal.h"
#include "valuate.h"

namespace rvd {

// ------------------------------------------------------------------ bijective key mixing
// MurmurHash3 finalisers (public domain).  Both are bijections, so the bits of
// a mixed key that are not spent on the bucket index identify the key inside
// its bucket, and the original key can be recovered for per-binding outputs.
constexpr uint32_t inv32(uint32_t c) {
  uint32_t x = c;
  for (int i = 0; i < 5; ++i) x *= 2u - c * x;
  return x;
}
constexpr uint64_t inv64(uint64_t c) {
  uint64_t x = c;
  for (int i = 0; i < 6; ++i) x *= 2ull - c * x;
  return x;
}
constexpr uint32_t M32A = 0x85ebca6bu, M32B = 0xc2b2ae35u;
constexpr uint64_t M64A = 0xff51afd7ed558ccdull, M64B = 0xc4ceb9fe1a85ec53ull;
constexpr uint32_t I32A = inv32(M32A), I32B = inv32(M32B);
constexpr uint64_t I64A = inv64(M64A), I64B = inv64(M64B);
static_assert(M32A * I32A == 1u && M32B * I32B == 1u, "32-bit inverses");
static_assert(M64A * I64A == 1ull && M64B * I64B == 1ull, "64-bit inverses");

__host__ __device__ __forceinline__ uint32_t mix32(uint32_t h) {
  h ^= h >> 16; h *= M32A; h ^= h >> 13; h *= M32B; h ^= h >> 16;
  return h;
}
__host__ __device__ __forceinline__ uint32_t unmix32(uint32_t h) {
  h ^= h >> 16; h *= I32B; h ^= (h >> 13) ^ (h >> 26); h *= I32A; h ^= h >> 16;
  return h;
}
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t h) {
  h ^= h >> 33; h *= M64A; h ^= h >> 33; h *= M64B; h ^= h >> 33;
  return h;
}
__host__ __device__ __forceinline__ uint64_t unmix64(uint64_t h) {
  h ^= h >> 33; h *= I64B; h ^= h >> 33; h *= I64A; h ^= h >> 33;
  return h;
}

// ------------------------------------------------------------------ record formats
// A record is a key-grouped event: the letter (predicate byte) in the low 8
// bits and, above it, the part of the mixed key not implied by the bucket.
enum Fmt {
  FMT_K32 = 0,   // one variable, 32-bit key: u32 record = low (32-B1) mixed bits << 8 | letter
  FMT_K64 = 1,   // one variable, 64-bit key: u64 record = low (64-B1) mixed bits << 8 | letter
  FMT_K2 = 2     // two variables, key (d0 << 32) | d1: u64 record = low (32-B1) bits of mix32(d0) << 40 | d1 << 8 | letter
};

template <int F> struct RecT { typedef uint64_t type; };
template <> struct RecT<FMT_K32> { typedef uint32_t type; };

struct Bucketed {
  uint32_t bucket;   // first-level bucket
  uint64_t rec;
};

template <int F>
__device__ __forceinline__ Bucketed make_record(uint64_t key, uint32_t letter, int B1, int nq) {
  Bucketed r;
  if (F == FMT_K32) {
    uint32_t h = nq == 0 ? 0u : mix32((uint32_t)key);
    r.bucket = h >> (32 - B1);
    r.rec = ((uint64_t)(h & (0xFFFFFFFFu >> B1)) << 8) | letter;
  } else if (F == FMT_K64) {
    uint64_t h = mix64(key);
    r.bucket = (uint32_t)(h >> (64 - B1));
    r.rec = ((h & (~0ull >> B1)) << 8) | letter;
  } else {
    uint32_t h = mix32((uint32_t)(key >> 32));
    r.bucket = h >> (32 - B1);
    r.rec = ((uint64_t)(h & (0xFFFFFFFFu >> B1)) << 40) | ((key & 0xFFFFFFFFull) << 8) | letter;
  }
  return r;
}

// bit position of the second-level split inside a record (top B2 bits of the
// local part of the mixed outer key)
template <int F>
__host__ __device__ __forceinline__ int sub_shift(int B1, int B2) {
  if (F == FMT_K32) return 8 + (32 - B1 - B2);
  if (F == FMT_K64) return 8 + (64 - B1 - B2);
  return 40 + (32 - B1 - B2);
}

// original binding key of a slot key (record >> 8) in first-level bucket b1
template <int F>
__device__ __forceinline__ uint64_t original_key(uint64_t slot_key, uint32_t b1, int B1, int nq) {
  if (F == FMT_K32) {
    if (nq == 0) return 0;
    return unmix32((b1 << (32 - B1)) | (uint32_t)slot_key);
  }
  if (F == FMT_K64) return unmix64(((uint64_t)b1 << (64 - B1)) | slot_key);
  uint32_t u = unmix32((b1 << (32 - B1)) | (uint32_t)(slot_key >> 32));
  return ((uint64_t)u << 32) | (slot_key & 0xFFFFFFFFull);
}
template <int F>
__device__ __forceinline__ uint32_t original_outer(uint32_t u_local, uint32_t b1, int B1) {
  return unmix32((b1 << (32 - B1)) | u_local);
}

// ------------------------------------------------------------------ transition maps
// A map is 16 nibbles: nibble s = target state of s.  apply(M, m) is "M then m":
// result nibble s = m[M[s]].
constexpr uint64_t IDENTITY_MAP = 0xFEDCBA9876543210ull;

// Monitors of at most 8 states keep every target in the low word, so a map
// is 8 nibbles there and composition is a handful of byte permutes:
// expand the second map to bytes, select bytes by the first map's nibbles,
// and pack the selected bytes back into nibbles.
__device__ __forceinline__ uint32_t nibbles_to_bytes_lo(uint32_t c, uint32_t& hi4) {
  const uint32_t l = c & 0x0F0F0F0Fu, h = (c >> 4) & 0x0F0F0F0Fu;   // [c0,c2,c4,c6] [c1,c3,c5,c7]
  hi4 = __byte_perm(l, h, 0x7362);                                   // bytes c4 c5 c6 c7
  return __byte_perm(l, h, 0x5140);                                  // bytes c0 c1 c2 c3
}
__device__ __forceinline__ uint32_t bytes_to_nibbles(uint32_t r03, uint32_t r47) {
  const uint32_t p03 = r03 | (r03 >> 4), p47 = r47 | (r47 >> 4);
  return __byte_perm(p03, p47, 0x6420);
}
__device__ __forceinline__ uint32_t compose8(uint32_t M, uint32_t C) {
  uint32_t c47;
  const uint32_t c03 = nibbles_to_bytes_lo(C, c47);
  return bytes_to_nibbles(__byte_perm(c03, c47, M & 0xFFFFu), __byte_perm(c03, c47, M >> 16));
}
// up to 16 states: two 8-byte tables, chosen per byte by bit 3 of the index
__device__ __forceinline__ uint32_t look4(uint32_t sel16, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
  const uint32_t s7 = sel16 & 0x7777u;
  const uint32_t a = __byte_perm(c0, c1, s7), b = __byte_perm(c2, c3, s7);
  const uint32_t e = __byte_perm(sel16 & 0x0F0Fu, (sel16 >> 4) & 0x0F0Fu, 0x5140);   // selector bytes
  const uint32_t mask = ((e >> 3) & 0x01010101u) * 0xFFu;
  return (a & ~mask) | (b & mask);
}
__device__ __forceinline__ uint64_t compose16(uint64_t M, uint64_t C) {
  uint32_t c1, c3;
  const uint32_t c0 = nibbles_to_bytes_lo((uint32_t)C, c1);
  const uint32_t c2 = nibbles_to_bytes_lo((uint32_t)(C >> 32), c3);
  const uint32_t Ml = (uint32_t)M, Mh = (uint32_t)(M >> 32);
  const uint32_t lo = bytes_to_nibbles(look4(Ml & 0xFFFFu, c0, c1, c2, c3), look4(Ml >> 16, c0, c1, c2, c3));
  const uint32_t hi = bytes_to_nibbles(look4(Mh & 0xFFFFu, c0, c1, c2, c3), look4(Mh >> 16, c0, c1, c2, c3));
  return ((uint64_t)hi << 32) | lo;
}

// "M then m": nibble s of the result is m[M[s]]
__device__ __forceinline__ uint64_t apply_map(uint64_t M, uint64_t m, int n_states) {
  if (n_states <= 8) return (M & 0xFFFFFFFF00000000ull) | compose8((uint32_t)M, (uint32_t)m);
  return compose16(M, m);
}

__device__ __forceinline__ uint32_t step_state(uint32_t q, uint64_t m) {
  return (uint32_t)((m >> (4 * q)) & 15ull);
}

// ------------------------------------------------------------------ monitor and formula tables
struct MonitorTab {
  uint64_t maps[RV_MAX_LETTERS];
  uint8_t labels[RV_MAX_STATES];
  int n_states;
  int q0;
  int n_letters;
  int nq;
  rv_quant q[2];
};

// ------------------------------------------------------------------ interpreted comparison atoms
// Body atoms "value ~ c" are folded into the letter at ingest: letter =
// code + n_base * (bit j set iff atom j holds for the event's value).
struct CmpTab {
  int n_base, n_cmp;
  int op[RV_MAX_CMP];
  uint32_t c[RV_MAX_CMP];
};

inline CmpTab cmp_tab(const rv_formula* f) {
  CmpTab t;
  t.n_base = f->n_base;
  t.n_cmp = f->n_cmp;
  for (int j = 0; j < RV_MAX_CMP; ++j) { t.op[j] = f->cmp_op[j]; t.c[j] = f->cmp_c[j]; }
  return t;
}

__device__ __forceinline__ uint32_t cmp_bits(const CmpTab& t, uint32_t v) {
  uint32_t bits = 0;
#pragma unroll
  for (int j = 0; j < RV_MAX_CMP; ++j) {
    if (j >= t.n_cmp) break;
    const uint32_t c = t.c[j];
    const int op = t.op[j];
    const bool on = op == RV_LT ? v < c : op == RV_LE ? v <= c : op == RV_GT ? v > c : op == RV_GE ? v >= c : v == c;
    bits |= (uint32_t)on << j;
  }
  return bits;
}

// letters of n events from their predicate codes and values; a code outside
// the schema sets `bad_bit` in *err (the letter is then 0)
static __global__ void k_cmp_letters(const uint8_t* pred, const uint32_t* value, uint64_t n, CmpTab t,
                                     uint8_t* out, unsigned int* err, unsigned int bad_bit) {
  bool bad = false;
  const uint64_t gt = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, gs = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i0 = gt; i0 < n; i0 += 4 * gs) {
    uint32_t code[4], val[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {              // four events' loads in flight before any store
      const uint64_t i = i0 + j * gs;
      code[j] = i < n ? pred[i] : 0u;
      val[j] = i < n ? value[i] : 0u;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t i = i0 + j * gs;
      if (i >= n) continue;
      if (code[j] >= (uint32_t)t.n_base) { bad = true; out[i] = 0; continue; }
      out[i] = (uint8_t)(code[j] + (uint32_t)t.n_base * cmp_bits(t, val[j]));
    }
  }
  if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, bad_bit);
}

// ------------------------------------------------------------------ accumulators of one verification
enum {
  ERR_LETTER = 1,       // predicate byte out of range
  ERR_TS = 2,           // timestamps decrease
  ERR_OUTER_FULL = 4,   // too many outer bindings in one bucket
  ERR_SPIN = 8,         // a bounded wait gave up
  ERR_POOL = 16,        // pair pool exhausted
  ERR_BOUNDS = 128      // bounds-checked builds: a write fell outside its array (skipped)
};

struct Acc {
  unsigned long long level_counts[2][6];
  unsigned long long n_nodes[2];
  unsigned long long n_out, n_out_outer;
  unsigned int err;
  unsigned int n_units;
  unsigned int n_tiles2;
  unsigned int n_groups[8];
  unsigned long long pair_top[2];
  unsigned int next_unit;       // dynamic work distribution of k_fold
  unsigned int next_group[8];   // and of each k_combine level
  unsigned int n_multi;         // buckets folded by more than one unit
  unsigned int test_flag;       // set by nothing: the bounded wait of rv_verify_opts.test_wait_polls
};

// ------------------------------------------------------------------ streaming state
// Device-resident monitor state of the online mode (Sec. 4.2: repeated
// invocations update the submonitor tree incrementally).  Bindings and outer
// nodes have dense ids assigned by the streaming pre-pass.
struct StreamState {
  uint8_t* bstate;              // [binding] 0x80 | monitor state once seen, 0 before
  uint8_t* bverdict;            // [binding] last LTL4 verdict
  uint16_t* bstream;            // [binding] stream (one-quantifier formulas)
  uint32_t* ocounts;            // [outer][6] child-verdict counts
  uint8_t* overdict;            // [outer] last verdict, 0xFF before the first
  uint16_t* ostream;            // [outer] stream
  unsigned long long* root;     // [stream][6] root child-verdict counts
};

}  // namespace rvd
