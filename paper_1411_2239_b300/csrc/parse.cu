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
// Steps: newlines counted per tile and scanned, line ends emitted in order;
// one thread parses each line; kept lines compacted in order by a second
// count/scan/emit.
#include <algorithm>
#include <cstring>

#include "profile.h"
#include "rv_internal.h"

namespace {

constexpr int PT = 256;               // threads per CTA
constexpr int PB = 64;                // text bytes per thread in the newline pass
constexpr int PTILE = PT * PB;        // 16 KiB of text per CTA
constexpr int LT = PT * 8;            // lines per CTA in the compaction
constexpr int MAX_RULES = RV_PARSE_MAX_RULES;
constexpr unsigned PFULL = 0xFFFFFFFFu;

struct Rules {
  char name[MAX_RULES][RV_PARSE_NAME_LEN];
  int len[MAX_RULES];
  int code[MAX_RULES];
  int key_from[MAX_RULES];
  int ok_only[MAX_RULES];
  int n;
};

// newlines in this thread's PB bytes (16-byte loads, byte compares)
__device__ __forceinline__ uint32_t count_nl(const unsigned char* text, uint64_t bytes, uint64_t b0) {
  uint32_t c = 0;
  if (b0 + PB <= bytes && ((uintptr_t)(text + b0) & 15) == 0) {
    const uint4* p = reinterpret_cast<const uint4*>(text + b0);
#pragma unroll
    for (int k = 0; k < PB / 16; ++k) {
      const uint4 v = p[k];
      c += __popc(__vcmpeq4(v.x, 0x0A0A0A0Au) & 0x01010101u) + __popc(__vcmpeq4(v.y, 0x0A0A0A0Au) & 0x01010101u) +
           __popc(__vcmpeq4(v.z, 0x0A0A0A0Au) & 0x01010101u) + __popc(__vcmpeq4(v.w, 0x0A0A0A0Au) & 0x01010101u);
    }
  } else {
    for (uint64_t i = b0; i < min(bytes, b0 + PB); ++i) c += text[i] == '\n';
  }
  return c;
}

// block-wide exclusive scan of one value per thread; *total = the CTA's sum
__device__ uint64_t block_exscan(uint64_t x, uint64_t* total) {
  __shared__ uint64_t ws[PT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t incl = x;
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t y = __shfl_up_sync(PFULL, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) ws[w] = incl;
  __syncthreads();
  uint64_t before = 0, all = 0;
  for (int v = 0; v < PT / 32; ++v) { if (v < w) before += ws[v]; all += ws[v]; }
  *total = all;
  __syncthreads();
  return before + incl - x;
}

__global__ void __launch_bounds__(PT) k_p_count(const unsigned char* text, uint64_t bytes, uint64_t* tile_nl) {
  const uint64_t b0 = (uint64_t)blockIdx.x * PTILE + (uint64_t)threadIdx.x * PB;
  uint64_t total;
  block_exscan(count_nl(text, bytes, b0), &total);
  if (threadIdx.x == 0) tile_nl[blockIdx.x] = total;
}

// exclusive scan of per-tile counts in place (one CTA, PT per round); total at [n]
__global__ void __launch_bounds__(PT) k_p_scan(uint64_t* v, uint64_t n) {
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t b = 0; b < n; b += PT) {
    const uint64_t i = b + threadIdx.x;
    const uint64_t x = i < n ? v[i] : 0;
    uint64_t total;
    const uint64_t ex = block_exscan(x, &total);
    const uint64_t c = carry;
    if (i < n) v[i] = c + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry = c + total;
    __syncthreads();
  }
  if (threadIdx.x == 0) v[n] = carry;
}

// position of every newline, in order
__global__ void __launch_bounds__(PT) k_p_lines(const unsigned char* text, uint64_t bytes, const uint64_t* tile_base,
                                                uint64_t* nl_pos) {
  const uint64_t b0 = (uint64_t)blockIdx.x * PTILE + (uint64_t)threadIdx.x * PB;
  uint64_t total;
  uint64_t at = tile_base[blockIdx.x] + block_exscan(count_nl(text, bytes, b0), &total);
  for (uint64_t i = b0; i < min(bytes, b0 + PB); ++i)
    if (text[i] == '\n') nl_pos[at++] = i;
}

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

__device__ __forceinline__ void line_span(const unsigned char* text, uint64_t bytes, const uint64_t* nl_pos,
                                          uint64_t n_nl, uint64_t i, const unsigned char** b, const unsigned char** e) {
  const uint64_t start = i == 0 ? 0 : nl_pos[i - 1] + 1;
  const uint64_t stop = i < n_nl ? nl_pos[i] : bytes;
  *b = text + start;
  *e = text + stop;
  if (*e > *b && (*e)[-1] == '\r') --*e;
}

__global__ void __launch_bounds__(PT) k_p_keep(const unsigned char* text, uint64_t bytes, const uint64_t* nl_pos,
                                               uint64_t n_nl, uint64_t n_lines, Rules R, uint64_t* tile_keep) {
  uint64_t kept = 0;
  const uint64_t l0 = (uint64_t)blockIdx.x * LT + (uint64_t)threadIdx.x * (LT / PT);
  for (uint64_t i = l0; i < min(n_lines, l0 + LT / PT); ++i) {
    const unsigned char *b, *e;
    line_span(text, bytes, nl_pos, n_nl, i, &b, &e);
    kept += parse_line(R, b, e).keep;
  }
  uint64_t total;
  block_exscan(kept, &total);
  if (threadIdx.x == 0) tile_keep[blockIdx.x] = total;
}

__global__ void __launch_bounds__(PT) k_p_emit(const unsigned char* text, uint64_t bytes, const uint64_t* nl_pos,
                                               uint64_t n_nl, uint64_t n_lines, Rules R, const uint64_t* tile_base,
                                               uint64_t cap, uint32_t* key_out, uint8_t* pred_out, uint64_t* ts_out) {
  const uint64_t l0 = (uint64_t)blockIdx.x * LT + (uint64_t)threadIdx.x * (LT / PT);
  uint64_t kept = 0;
  for (uint64_t i = l0; i < min(n_lines, l0 + LT / PT); ++i) {
    const unsigned char *b, *e;
    line_span(text, bytes, nl_pos, n_nl, i, &b, &e);
    kept += parse_line(R, b, e).keep;
  }
  uint64_t total;
  uint64_t at = tile_base[blockIdx.x] + block_exscan(kept, &total);
  for (uint64_t i = l0; i < min(n_lines, l0 + LT / PT); ++i) {
    const unsigned char *b, *e;
    line_span(text, bytes, nl_pos, n_nl, i, &b, &e);
    const Parsed p = parse_line(R, b, e);
    if (!p.keep) continue;
    if (at < cap) {
      key_out[at] = p.key;
      pred_out[at] = p.code;
      if (ts_out) ts_out[at] = p.ts_us;
    }
    ++at;
  }
}

struct PPlan {
  uint64_t ntiles, max_lines, ltiles;
  size_t o_tnl, o_nl, o_tkeep, total;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

PPlan pplan(uint64_t bytes) {
  PPlan p{};
  p.ntiles = std::max<uint64_t>(1, (bytes + PTILE - 1) / PTILE);
  p.max_lines = bytes + 1;                      // at most one line per byte, plus a last unterminated one
  p.ltiles = std::max<uint64_t>(1, (p.max_lines + LT - 1) / LT);
  size_t off = 0;
  auto take = [&](size_t b) { size_t r = off; off = a256(off + b); return r; };
  p.o_tnl = take((p.ntiles + 1) * 8);
  p.o_nl = take(std::max<uint64_t>(bytes, 1) * 8);
  p.o_tkeep = take((p.ltiles + 1) * 8);
  p.total = off;
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
  if (ws_bytes < p.total) return rv_fail(RV_ENOMEM, "parse workspace of %zu bytes, need %zu", ws_bytes, p.total);
  unsigned char* W = (unsigned char*)ws;
  uint64_t* tnl = (uint64_t*)(W + p.o_tnl);
  uint64_t* nl = (uint64_t*)(W + p.o_nl);
  uint64_t* tkeep = (uint64_t*)(W + p.o_tkeep);
  const unsigned char* T = (const unsigned char*)text;
  RV_LAUNCH("k_p_count", k_p_count, (unsigned)p.ntiles, PT, 0, s, T, bytes, tnl);
  RV_LAUNCH("k_p_scan", k_p_scan, 1, PT, 0, s, tnl, p.ntiles);
  RV_LAUNCH("k_p_lines", k_p_lines, (unsigned)p.ntiles, PT, 0, s, T, bytes, tnl, nl);
  uint64_t n_nl = 0, last_nl = 0;
  PCU(cudaMemcpyAsync(&n_nl, tnl + p.ntiles, 8, cudaMemcpyDeviceToHost, s));
  PCU(cudaStreamSynchronize(s));
  if (n_nl) {
    PCU(cudaMemcpyAsync(&last_nl, nl + n_nl - 1, 8, cudaMemcpyDeviceToHost, s));
    PCU(cudaStreamSynchronize(s));
  }
  // a last line without a newline counts too
  const uint64_t n_lines = n_nl + (n_nl == 0 || last_nl + 1 < bytes ? 1 : 0);
  const uint64_t ltiles = (n_lines + LT - 1) / LT;
  RV_LAUNCH("k_p_keep", k_p_keep, (unsigned)ltiles, PT, 0, s, T, bytes, nl, n_nl, n_lines, R, tkeep);
  RV_LAUNCH("k_p_scan", k_p_scan, 1, PT, 0, s, tkeep, ltiles);
  RV_LAUNCH("k_p_emit", k_p_emit, (unsigned)ltiles, PT, 0, s, T, bytes, nl, n_nl, n_lines, R, tkeep, capacity,
            key_out, pred_out, ts_out);
  PCU(cudaGetLastError());
  uint64_t kept = 0;
  PCU(cudaMemcpyAsync(&kept, tkeep + ltiles, 8, cudaMemcpyDeviceToHost, s));
  PCU(cudaStreamSynchronize(s));
  *n_events = kept;
  if (kept > capacity) return rv_fail(RV_ENOMEM, "%llu events parsed, capacity %llu: only the first were written",
                                      (unsigned long long)kept, (unsigned long long)capacity);
  return RV_OK;
}
