// Front end: strace text -> event table.
//
// The paper monitors programs through strace (Sec. 5: its parsing module
// "translates strace strings" into a numerical table).  rv_parse_strace does
// that translation on the GPU: a log of strace lines
//     [pid] TIME NAME(ARGS...) = RET [ERRNO (text)]
// (pid optional, "[pid N] " or "N "; TIME seconds.microseconds (-ttt) or
// HH:MM:SS.microseconds (-tt)) becomes the arrays key / pred / ts of a trace.
// A caller-given rule per system call name gives the event's predicate code
// and where its key comes from: the first argument (a descriptor passed in)
// or the return value (a descriptor made by the call).  Calls split by
// strace -f into "NAME(ARGS <unfinished ...>" and "<... NAME resumed> ...) =
// RET" give one event, from the line that carries their key.  Lines of other
// calls, signals, exits and failed calls (RET < 0, when the rule asks for
// success) are dropped.
//
// One kernel, one CTA per 8 KiB tile of text taken in order by a ticket: the
// tile (with 16 bytes before it and 1 KiB after it) is staged in shared memory
// with 16-byte loads; its newlines are listed by a block scan; one thread
// parses each line that starts in the tile; the tile's count of kept lines is
// chained to the earlier tiles' by a decoupled look-back (bounded waits), and
// the kept events are written at their place in line order.  The text is read
// from DRAM once; only a line longer than the staged window is parsed from
// global memory.
#include <algorithm>
#include <cstring>

#include "profile.h"
#include "rv_internal.h"

namespace {

constexpr int PT = 128;               // threads per CTA
constexpr int TB = 8192;              // text bytes owned by one tile
constexpr int OV = 1024;              // bytes staged after the tile: the end of its last line
constexpr int WB = 16 + TB + OV;      // staged window: 16 bytes before the tile, the tile, the overhang
constexpr int CB = TB / PT;           // tile bytes per thread in the newline scan (64)
constexpr int RREG = 2;               // rounds of lines whose events stay in registers until written
constexpr int MAX_RULES = RV_PARSE_MAX_RULES;
constexpr unsigned PFULL = 0xFFFFFFFFu;
constexpr uint64_t ST_AGG = 1ull << 62;      // tile status: own count published
constexpr uint64_t ST_INC = 2ull << 62;      // tile status: count of every tile up to this one
constexpr uint64_t ST_VAL = (1ull << 62) - 1;
constexpr uint32_t MAX_POLLS = 1u << 22;     // look-back polls of one window before giving up
constexpr uint32_t PERR_SPIN = 1;

struct Rules {
  char name[MAX_RULES][RV_PARSE_NAME_LEN];
  int len[MAX_RULES];
  int code[MAX_RULES];
  int key_from[MAX_RULES];
  int ok_only[MAX_RULES];
  int n;
};

// workspace words after the tile status array
struct PMisc {
  uint32_t ticket;     // next tile to take
  uint32_t err;        // PERR_* bits
  uint64_t total;      // kept lines of the whole text (written by the last tile)
};

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// newline flags of four text bytes: 0x01 in each byte that is '\n'
__device__ __forceinline__ uint32_t nl4(uint32_t w) { return __vcmpeq4(w, 0x0A0A0A0Au) & 0x01010101u; }

// ------------------------------------------------------------------ one line
struct Cursor {
  const unsigned char* p;
  const unsigned char* end;
  __device__ bool more() const { return p < end; }
  __device__ unsigned char c() const { return p < end ? *p : 0; }
  __device__ void skip_spaces() { while (p < end && (*p == ' ' || *p == '\t')) ++p; }
  __device__ bool eat(const char* s) {
    const unsigned char* q = p;
    for (; *s; ++s, ++q)
      if (q >= end || *q != (unsigned char)*s) return false;
    p = q;
    return true;
  }
  // unsigned decimal; false if none
  __device__ bool num(uint64_t* v, int* digits = nullptr) {
    uint64_t x = 0;
    int d = 0;
    while (p < end && *p >= '0' && *p <= '9' && d < 19) { x = x * 10 + (*p - '0'); ++p; ++d; }
    if (digits) *digits = d;
    *v = x;
    return d > 0;
  }
  // signed decimal (or hex with 0x)
  __device__ bool snum(int64_t* v) {
    bool neg = false;
    if (p < end && *p == '-') { neg = true; ++p; }
    uint64_t x = 0;
    if (p + 1 < end && p[0] == '0' && (p[1] == 'x' || p[1] == 'X')) {
      p += 2;
      int d = 0;
      while (p < end && d < 16) {
        const unsigned char ch = *p;
        int h = ch >= '0' && ch <= '9' ? ch - '0' : ch >= 'a' && ch <= 'f' ? ch - 'a' + 10
              : ch >= 'A' && ch <= 'F' ? ch - 'A' + 10 : -1;
        if (h < 0) break;
        x = x * 16 + (uint64_t)h;
        ++p;
        ++d;
      }
      if (!d) return false;
    } else if (!num(&x)) {
      return false;
    }
    *v = neg ? -(int64_t)x : (int64_t)x;
    return true;
  }
};

__device__ __forceinline__ bool name_char(unsigned char ch) {
  return (ch >= 'a' && ch <= 'z') || (ch >= '0' && ch <= '9') || ch == '_' || (ch >= 'A' && ch <= 'Z');
}

// the rule of the name [a, a + n), or -1
__device__ int find_rule(const Rules& R, const unsigned char* a, int n) {
  for (int r = 0; r < R.n; ++r) {
    if (R.len[r] != n) continue;
    bool eq = true;
    for (int k = 0; k < n && eq; ++k) eq = a[k] == (unsigned char)R.name[r][k];
    if (eq) return r;
  }
  return -1;
}

// the return value after the last ") = " of the line; false if none
__device__ bool return_value(const unsigned char* b, const unsigned char* e, int64_t* ret) {
  for (const unsigned char* q = e - 1; q >= b + 3; --q) {
    if (q[0] == ' ' && q[-1] == '=' && q[-2] == ' ' && q[-3] == ')') {
      Cursor c{q + 1, e};
      c.skip_spaces();
      return c.snum(ret);
    }
  }
  return false;
}

struct Parsed { uint32_t key; uint8_t code; uint8_t keep; uint64_t ts_us; };

__device__ Parsed parse_line(const Rules& R, const unsigned char* b, const unsigned char* e) {
  Parsed out{0, 0, 0, 0};
  Cursor c{b, e};
  c.skip_spaces();
  // optional pid: "[pid N] " or "N " before the timestamp
  if (c.eat("[pid")) {
    uint64_t pid;
    c.skip_spaces();
    if (!c.num(&pid) || !c.eat("]")) return out;
    c.skip_spaces();
  } else {
    const unsigned char* save = c.p;
    uint64_t pid;
    int d;
    if (c.num(&pid, &d) && c.c() == ' ') c.skip_spaces();
    else c.p = save;                             // the number was the timestamp
  }
  // timestamp: seconds.micro (-ttt) or HH:MM:SS.micro (-tt)
  uint64_t a, m = 0, s = 0, us = 0;
  int du = 0;
  if (!c.num(&a)) return out;
  uint64_t secs = a;
  if (c.eat(":")) {
    if (!c.num(&m) || !c.eat(":") || !c.num(&s)) return out;
    secs = a * 3600 + m * 60 + s;
  }
  if (c.eat(".")) {
    if (!c.num(&us, &du)) return out;
    for (; du < 6; ++du) us *= 10;
    for (; du > 6; --du) us /= 10;
  }
  out.ts_us = secs * 1000000ull + us;
  c.skip_spaces();
  // NAME(  or  <... NAME resumed>
  bool resumed = false;
  if (c.eat("<... ")) resumed = true;
  const unsigned char* n0 = c.p;
  while (c.more() && name_char(c.c())) ++c.p;
  const int nlen = (int)(c.p - n0);
  if (nlen == 0 || nlen >= RV_PARSE_NAME_LEN) return out;
  const int r = find_rule(R, n0, nlen);
  if (r < 0) return out;
  if (resumed) {
    if (!c.eat(" resumed>")) return out;
  } else if (!c.eat("(")) {
    return out;
  }
  // strace -f ends a call interrupted by another thread's output with "<unfinished ...>"
  bool unfinished = false;
  {
    const char* tail = "<unfinished ...>";
    const int tl = 16;
    if (e - c.p >= tl) {
      unfinished = true;
      for (int k = 0; k < tl; ++k) unfinished &= e[k - tl] == (unsigned char)tail[k];
    }
  }
  int64_t ret = 0;
  const bool has_ret = !unfinished && return_value(c.p, e, &ret);
  if (R.key_from[r] == RV_KEY_ARG0) {
    if (resumed) return out;                     // the call's first argument was on its unfinished line
    c.skip_spaces();
    int64_t k;
    if (!c.snum(&k) || k < 0) return out;
    if (R.ok_only[r] && has_ret && ret < 0) return out;
    out.key = (uint32_t)k;
  } else {
    if (!has_ret || ret < 0) return out;         // the made descriptor is the return value
    out.key = (uint32_t)ret;
  }
  out.code = (uint8_t)R.code[r];
  out.keep = 1;
  return out;
}

struct PShared {
  uint4 win4[WB / 16];               // text [t0 - 16, t0 + TB + OV), zero past the end of the text
  uint16_t nl[TB];                   // window offsets of the tile's newlines, in order
  uint32_t wsum[2][PT / 32];         // per-warp kept counts of one round (two rounds alternate)
  uint64_t base;                     // kept lines of all earlier tiles
  uint32_t tile, nnl;
  int32_t ovend;                     // window offset of the first newline after the tile, or -1
};

// window offsets [b, e) of line L of the tile; -1 in *e: the line runs past the window
__device__ __forceinline__ void line_bounds(const PShared& S, int h, uint32_t L, int* b, int* e) {
  *b = (L == 0 && h) ? 16 : S.nl[L - h] + 1;
  const uint32_t j = L - h + 1;
  *e = j < S.nnl ? S.nl[j] : S.ovend;
}

// the parse of line L; a line past the window is read from global memory
__device__ Parsed parse_at(const PShared& S, const Rules& R, const unsigned char* text, uint64_t bytes,
                           uint64_t t0, int h, uint32_t L) {
  int b, e;
  line_bounds(S, h, L, &b, &e);
  const unsigned char* win = reinterpret_cast<const unsigned char*>(S.win4);
  const unsigned char *pb, *pe;
  if (e >= 0) {
    pb = win + b;
    pe = win + e;
  } else {
    uint64_t q = t0 + TB + OV;                 // global position of window offset WB
    while (q < bytes && text[q] != '\n') ++q;
    pb = text + (t0 + b - 16);
    pe = text + q;
  }
  if (pe > pb && pe[-1] == '\r') --pe;
  return parse_line(R, pb, pe);
}

// rank of this thread's keep bit among the CTA's threads in round r; *round_total: the round's count
__device__ __forceinline__ uint32_t round_rank(PShared& S, int r, bool keep, uint32_t* round_total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned m = __ballot_sync(PFULL, keep);
  if (lane == 0) S.wsum[r & 1][w] = __popc(m);
  __syncthreads();
  uint32_t before = 0, all = 0;
#pragma unroll
  for (int v = 0; v < PT / 32; ++v) {
    const uint32_t c = S.wsum[r & 1][v];
    before += v < w ? c : 0;
    all += c;
  }
  *round_total = all;
  return before + __popc(m & ((1u << lane) - 1));
}

__global__ void __launch_bounds__(PT) k_p_parse(const unsigned char* text, uint64_t bytes, Rules R, uint64_t* st,
                                                PMisc* misc, uint64_t cap, uint32_t* key_out, uint8_t* pred_out,
                                                uint64_t* ts_out) {
  __shared__ PShared S;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) S.tile = atomicAdd(&misc->ticket, 1u);
  __syncthreads();
  const uint32_t tile = S.tile;
  const uint64_t t0 = (uint64_t)tile * TB;
  const uint64_t tb = min((uint64_t)TB, bytes - t0);           // bytes of the tile inside the text
  unsigned char* win = reinterpret_cast<unsigned char*>(S.win4);

  // 1. stage [t0 - 16, t0 + TB + OV); before the text's first byte a virtual newline
  // the window's 16-byte words are all loaded before any is stored (one memory
  // round trip, not one per word); words outside the text, or of unaligned
  // text, are filled byte by byte
  const bool aligned = ((uintptr_t)text & 15) == 0;
  constexpr int NW = WB / 16, WPT = (NW + PT - 1) / PT;
  uint4 wv[WPT];
#pragma unroll
  for (int q = 0; q < WPT; ++q) {
    const int u = q * PT + tid;
    const int64_t g = (int64_t)t0 - 16 + 16 * (int64_t)u;
    wv[q] = u < NW && g >= 0 && aligned && (uint64_t)g + 16 <= bytes ? *reinterpret_cast<const uint4*>(text + g)
                                                                     : make_uint4(0u, 0u, 0u, 0u);
  }
#pragma unroll
  for (int q = 0; q < WPT; ++q) {
    const int u = q * PT + tid;
    if (u >= NW) continue;
    const int64_t g = (int64_t)t0 - 16 + 16 * (int64_t)u;
    if (g < 0) {
      S.win4[u] = make_uint4(0x0A0A0A0Au, 0x0A0A0A0Au, 0x0A0A0A0Au, 0x0A0A0A0Au);
    } else if (aligned && (uint64_t)g + 16 <= bytes) {
      S.win4[u] = wv[q];
    } else {
      for (int k = 0; k < 16; ++k) win[16 * u + k] = (uint64_t)g + k < bytes ? text[g + k] : 0;
    }
  }
  __syncthreads();

  // 2. newlines of the tile, listed in order; the first newline of the overhang
  uint32_t c = 0;
  const uint32_t* w32 = reinterpret_cast<const uint32_t*>(win + 16 + tid * CB);
#pragma unroll
  for (int k = 0; k < CB / 4; ++k) c += __popc(nl4(w32[k]));
  // block exclusive scan of c
  uint32_t incl = c;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(PFULL, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) S.wsum[0][tid >> 5] = incl;
  __syncthreads();
  uint32_t at = incl - c, nnl = 0;
#pragma unroll
  for (int v = 0; v < PT / 32; ++v) {
    at += v < (tid >> 5) ? S.wsum[0][v] : 0;
    nnl += S.wsum[0][v];
  }
#pragma unroll
  for (int k = 0; k < CB / 4; ++k) {
    uint32_t m = nl4(w32[k]);
    while (m) {
      const int bit = __ffs(m) - 1;
      S.nl[at++] = (uint16_t)(16 + tid * CB + 4 * k + (bit >> 3));
      m &= m - 1;
    }
  }
  if (tid < 32) {
    int32_t found = -1;
    if (t0 + TB >= bytes) {
      found = (int32_t)(16 + tb);                              // the text ends in this tile
    } else {
      const uint32_t* ov = reinterpret_cast<const uint32_t*>(win + 16 + TB);
      for (int k = 0; k < OV / 128 && found < 0; ++k) {
        const uint32_t m = nl4(ov[32 * k + lane]);
        const unsigned any = __ballot_sync(PFULL, m != 0);
        if (any) {
          const int l = __ffs(any) - 1;
          const uint32_t ml = __shfl_sync(PFULL, m, l);
          found = 16 + TB + 4 * (32 * k + l) + ((__ffs(ml) - 1) >> 3);
        }
      }
      if (found < 0 && t0 + TB + OV >= bytes) found = (int32_t)(16 + (bytes - t0));   // the text ends in the overhang
    }
    if (tid == 0) {
      S.ovend = found;
      S.nnl = nnl;
    }
  }
  __syncthreads();
  // a line starts after each newline at [t0 - 1, t0 + tb - 1)
  const int h = win[15] == '\n';
  const uint32_t n_lines = h + nnl - (tb && win[16 + tb - 1] == '\n' ? 1u : 0u);
  const int rounds = (int)((n_lines + PT - 1) / PT);

  // 3. parse; the first RREG rounds keep their events in registers
  Parsed keep_p[RREG];
  uint32_t keep_at[RREG];
  uint32_t kept = 0, kept_reg = 0;
  for (int r = 0; r < rounds; ++r) {
    if (r == RREG) kept_reg = kept;
    const uint32_t L = (uint32_t)r * PT + tid;
    Parsed p{0, 0, 0, 0};
    if (L < n_lines) p = parse_at(S, R, text, bytes, t0, h, L);
    uint32_t rt;
    const uint32_t rk = kept + round_rank(S, r, p.keep, &rt);
#pragma unroll
    for (int q = 0; q < RREG; ++q)
      if (q == r) { keep_p[q] = p; keep_at[q] = rk; }
    kept += rt;
  }

  // 4. decoupled look-back: kept lines of every earlier tile
  if (tid < 32) {
    uint64_t excl = 0;
    if (tile == 0) {
      if (lane == 0) st_relaxed(&st[0], ST_INC | kept);
    } else {
      if (lane == 0) st_relaxed(&st[tile], ST_AGG | kept);
      int64_t j = (int64_t)tile - 1;
      bool gave_up = false;
      for (;;) {
        const int64_t idx = j - lane;
        uint64_t v = idx >= 0 ? ld_relaxed(&st[idx]) : ST_INC;
        uint32_t polls = 0;
        while (__any_sync(PFULL, (v >> 62) == 0)) {
          if (++polls > MAX_POLLS) { gave_up = true; break; }
          if ((v >> 62) == 0) v = ld_relaxed(&st[idx]);
        }
        if (gave_up) break;
        const unsigned inc = __ballot_sync(PFULL, (v >> 62) == 2);
        const int stop = inc ? __ffs(inc) - 1 : 31;
        uint64_t x = lane <= stop ? (v & ST_VAL) : 0;
#pragma unroll
        for (int d = 16; d; d >>= 1) x += __shfl_xor_sync(PFULL, x, d);
        excl += x;
        if (inc) break;
        j -= 32;
      }
      if (lane == 0) {
        if (gave_up) atomicOr(&misc->err, PERR_SPIN);
        st_relaxed(&st[tile], ST_INC | ((excl + kept) & ST_VAL));
      }
    }
    if (lane == 0) {
      S.base = excl;
      if (t0 + TB >= bytes) misc->total = excl + kept;
    }
  }
  __syncthreads();
  const uint64_t base = S.base;
  uint32_t run = kept_reg;

  // 5. events written in line order
  for (int r = 0; r < rounds; ++r) {
    Parsed p{0, 0, 0, 0};
    uint32_t rk = 0;
    if (r < RREG) {
#pragma unroll
      for (int q = 0; q < RREG; ++q)
        if (q == r) { p = keep_p[q]; rk = keep_at[q]; }
    } else {                                   // lines past the registers' rounds are parsed again
      const uint32_t L = (uint32_t)r * PT + tid;
      if (L < n_lines) p = parse_at(S, R, text, bytes, t0, h, L);
      uint32_t rt;
      rk = run + round_rank(S, r, p.keep, &rt);
      run += rt;
    }
    if (p.keep) {
      const uint64_t o = base + rk;
      if (o < cap) {
        key_out[o] = p.key;
        pred_out[o] = p.code;
        if (ts_out) ts_out[o] = p.ts_us;
      }
    }
  }
}

struct PPlan {
  uint64_t ntiles;
  size_t o_st, o_misc, total;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

PPlan pplan(uint64_t bytes) {
  PPlan p{};
  p.ntiles = std::max<uint64_t>(1, (bytes + TB - 1) / TB);
  p.o_st = 0;
  p.o_misc = a256(p.ntiles * 8);
  p.total = p.o_misc + a256(sizeof(PMisc));
  return p;
}

#define PCU(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return rv_fail(RV_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));  \
  } while (0)

}  // namespace

extern "C" size_t rv_parse_workspace_size(uint64_t bytes) { return pplan(bytes).total; }

extern "C" rv_status rv_parse_strace(const char* text, uint64_t bytes, const rv_syscall_rule* rules, int n_rules,
                                     void* ws, size_t ws_bytes, uint32_t* key_out, uint8_t* pred_out,
                                     uint64_t* ts_out, uint64_t capacity, uint64_t* n_events, cudaStream_t s) {
  if (!n_events || (bytes && (!text || !ws || !key_out || !pred_out)) || (n_rules && !rules))
    return rv_fail(RV_EINVAL, "null argument");
  if (n_rules < 1 || n_rules > MAX_RULES) return rv_fail(RV_EINVAL, "1..%d rules", MAX_RULES);
  Rules R;
  memset(&R, 0, sizeof R);
  R.n = n_rules;
  for (int r = 0; r < n_rules; ++r) {
    const size_t L = rules[r].name ? strlen(rules[r].name) : 0;
    if (L == 0 || L >= RV_PARSE_NAME_LEN) return rv_fail(RV_EINVAL, "rule %d: name of 1..%d characters", r,
                                                         RV_PARSE_NAME_LEN - 1);
    if (rules[r].code < 0 || rules[r].code > 255) return rv_fail(RV_EINVAL, "rule %d: code outside 0..255", r);
    if (rules[r].key_from != RV_KEY_ARG0 && rules[r].key_from != RV_KEY_RET)
      return rv_fail(RV_EINVAL, "rule %d: key_from must be RV_KEY_ARG0 or RV_KEY_RET", r);
    memcpy(R.name[r], rules[r].name, L);
    R.len[r] = (int)L;
    R.code[r] = rules[r].code;
    R.key_from[r] = rules[r].key_from;
    R.ok_only[r] = rules[r].ok_only;
  }
  *n_events = 0;
  if (bytes == 0) return RV_OK;
  const PPlan p = pplan(bytes);
  if (p.ntiles > 0x7FFFFFFFull) return rv_fail(RV_EINVAL, "text of %llu bytes: at most 2^31 - 1 tiles of %d bytes",
                                               (unsigned long long)bytes, TB);
  if (ws_bytes < p.total) return rv_fail(RV_ENOMEM, "parse workspace of %zu bytes, need %zu", ws_bytes, p.total);
  unsigned char* W = (unsigned char*)ws;
  uint64_t* st = (uint64_t*)(W + p.o_st);
  PMisc* misc = (PMisc*)(W + p.o_misc);
  PCU(cudaMemsetAsync(W, 0, p.total, s));
  RV_LAUNCH("k_p_parse", k_p_parse, (unsigned)p.ntiles, PT, 0, s, (const unsigned char*)text, bytes, R, st, misc,
            capacity, key_out, pred_out, ts_out);
  PCU(cudaGetLastError());
  PMisc h{};
  PCU(cudaMemcpyAsync(&h, misc, sizeof h, cudaMemcpyDeviceToHost, s));
  PCU(cudaStreamSynchronize(s));
  if (h.err & PERR_SPIN) return rv_fail(RV_ETIMEOUT, "parse: look-back wait gave up");
  *n_events = h.total;
  if (h.total > capacity) return rv_fail(RV_ENOMEM, "%llu events parsed, capacity %llu: only the first were written",
                                         (unsigned long long)h.total, (unsigned long long)capacity);
  return RV_OK;
}
