// Host formula front-end: LTL4-C parser (Def. 1, Sec. 2.1) and synthesis of
// the minimal LTL4 Moore monitor of the body (Def. "LTL4 Monitor", Sec. 2.2.3).
//
// Monitor construction.  Let the *type* of a position of a word be the set of
// subformulas of psi true there.  The type at position i is a function of the
// letter at i and the type at i+1 (prep): X g holds iff g holds at i+1, and
// f U g holds iff g holds now or (f holds now and f U g holds at i+1).  For a
// finite prefix u, the map f_u : tau -> type of (u . suffix of type tau) is the
// composition of the letters' prep maps, and it decides [u |=_4 psi]:
//   T  iff psi is in f_u(tau) for every type tau of an infinite word,
//   F  iff psi is in f_u(tau) for no such type,
//   Tp / Fp otherwise by psi in f_u(end), "end" being the type of the empty
//          suffix (every X and U false: strong next and bounded until of
//          Def. "FLTL semantics").
// The types of infinite words (realisable types) come from an elimination
// tableau: candidates are (letter, truth of every X/U subformula); a candidate
// survives while it has a surviving successor consistent with the X and U
// expansion laws and, for every until it claims, a surviving path to a
// candidate where the until's right operand holds.  The reachable maps f_u
// form a Moore machine labelled as above; Moore partition refinement gives the
// unique minimal monitor, which must have at most 16 states so that a state
// fits a nibble and a letter's transition map fits a 64-bit word.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>
#include <algorithm>

#include "rv_internal.h"
#include "valuate.h"

static thread_local std::string g_err = "no error";

rv_status rv_fail(rv_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

extern "C" const char* rv_last_error(void) { return g_err.c_str(); }

namespace {

struct ParseFail { rv_status st; std::string msg; };

enum { N_TRUE, N_AP, N_NOT, N_AND, N_X, N_U };
struct CNode { int op, a, b; };

struct Builder {
  std::vector<CNode> nodes;
  std::map<std::tuple<int, int, int>, int> ids;
  int mk(int op, int a, int b) {
    auto key = std::make_tuple(op, a, b);
    auto it = ids.find(key);
    if (it != ids.end()) return it->second;
    nodes.push_back({op, a, b});
    int id = (int)nodes.size() - 1;
    ids[key] = id;
    return id;
  }
  int top() { return mk(N_TRUE, -1, -1); }
  int bot() { return neg(top()); }
  int ap(int i) { return mk(N_AP, i, -1); }
  int neg(int a) { return nodes[a].op == N_NOT ? nodes[a].a : mk(N_NOT, a, -1); }
  int conj(int a, int b) { return mk(N_AND, std::min(a, b), std::max(a, b)); }
  int disj(int a, int b) { return neg(conj(neg(a), neg(b))); }
  int next(int a) { return mk(N_X, a, -1); }
  int until(int a, int b) { return mk(N_U, a, b); }
  int eventually(int a) { return until(top(), a); }
  int always(int a) { return neg(eventually(neg(a))); }
};

// ------------------------------------------------------------------ tokenizer
static std::string ascii_ops(const std::string& s) {
  static const std::pair<const char*, const char*> rep[] = {
      {"\xC2\xAC", " ! "},  {"\xE2\x88\xA7", " && "}, {"\xE2\x88\xA8", " || "},
      {"\xE2\x86\x92", " -> "}, {"\xE2\x86\x94", " <-> "}, {"\xE2\x87\x92", " => "},
      {"\xE2\x89\xA5", " >= "}, {"\xE2\x89\xA4", " <= "}, {"\xE2\x8A\xA4", " true "},
      {"\xE2\x8A\xA5", " false "}};
  std::string out = s;
  for (auto& r : rep) {
    size_t pos = 0;
    while ((pos = out.find(r.first, pos)) != std::string::npos) {
      out.replace(pos, strlen(r.first), r.second);
      pos += strlen(r.second);
    }
  }
  return out;
}

static bool is_alpha(char c) { return (c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z'); }
static bool is_digit(char c) { return c >= '0' && c <= '9'; }
static bool is_alnum(char c) { return is_alpha(c) || is_digit(c); }

static std::vector<std::string> tokenize(const std::string& text) {
  std::string s = ascii_ops(text);
  std::vector<std::string> t;
  size_t i = 0;
  static const char* multi[] = {"<->", "->", "=>", "&&", "||", "<=", ">="};
  while (i < s.size()) {
    char c = s[i];
    if (c == ' ' || c == '\t' || c == '\n' || c == '\r') { ++i; continue; }
    bool done = false;
    for (const char* m : multi) {
      size_t L = strlen(m);
      if (s.compare(i, L, m) == 0) { t.push_back(m); i += L; done = true; break; }
    }
    if (done) continue;
    if (strchr("()!&|<>=:,_{}%~", c)) { t.push_back(std::string(1, c == '~' ? '!' : c)); ++i; continue; }
    if (is_digit(c) || (c == '.' && i + 1 < s.size() && is_digit(s[i + 1]))) {
      size_t j = i;
      while (j < s.size() && is_digit(s[j])) ++j;
      if (j < s.size() && s[j] == '.') { ++j; while (j < s.size() && is_digit(s[j])) ++j; }
      t.push_back(s.substr(i, j - i));
      i = j;
      continue;
    }
    if (is_alpha(c)) {
      size_t j = i + 1;
      while (j < s.size()) {
        if (is_alnum(s[j])) { ++j; continue; }
        if (s[j] == '_' && j + 1 < s.size() && is_alnum(s[j + 1])) { j += 2; continue; }
        break;
      }
      t.push_back(s.substr(i, j - i));
      i = j;
      continue;
    }
    throw ParseFail{RV_EPARSE, std::string("unexpected character '") + c + "'"};
  }
  return t;
}

static uint64_t gcd64(uint64_t a, uint64_t b) { while (b) { uint64_t t = a % b; a = b; b = t; } return a; }

// ------------------------------------------------------------------ parser
struct Parser {
  std::vector<std::string> t;
  size_t i = 0;
  Builder& B;
  std::vector<std::string> aps;     // distinct body propositions, in order of appearance
  struct Cmp { std::string name; int op; uint64_t c; };
  std::vector<Cmp> cmp;             // per proposition: a comparison atom (op >= 0) or a predicate code (op < 0)
  std::vector<rv_quant> quants;
  explicit Parser(Builder& b) : B(b) {}

  const std::string* peek(size_t k = 0) const { return i + k < t.size() ? &t[i + k] : nullptr; }
  bool at(const char* s, size_t k = 0) const { auto p = peek(k); return p && *p == s; }
  std::string take() {
    if (i >= t.size()) throw ParseFail{RV_EPARSE, "unexpected end of formula"};
    return t[i++];
  }
  void expect(const char* s) {
    if (!at(s)) throw ParseFail{RV_EPARSE, std::string("expected '") + s + "' near '" + (peek() ? *peek() : "end") + "'"};
    ++i;
  }
  static bool ident(const std::string& s) { return !s.empty() && is_alpha(s[0]); }
  bool quant_start(size_t k) const {
    return (at("A", k) || at("E", k)) && (at("_", k + 1) || at(":", k + 2));
  }

  void quantifier() {
    rv_quant q{};
    q.kind = take() == "A" ? RV_Q_A : RV_Q_E;
    bool explicit_c = false;
    if (at("_")) {
      take();
      bool braced = at("{");
      if (braced) take();
      std::string op = take();
      if (op == "<") q.op = RV_LT; else if (op == "<=") q.op = RV_LE; else if (op == ">") q.op = RV_GT;
      else if (op == ">=") q.op = RV_GE; else if (op == "=") q.op = RV_EQ;
      else throw ParseFail{RV_EPARSE, "bad comparison '" + op + "'"};
      std::string num = take();
      if (!is_digit(num[0]) && num[0] != '.') throw ParseFail{RV_EPARSE, "bad constant '" + num + "'"};
      uint64_t n = 0, d = 1;
      bool frac = false;
      int digits = 0;
      for (char c : num) {
        if (c == '.') { frac = true; continue; }
        if (++digits > 15) throw ParseFail{RV_EUNSUPPORTED, "constant has too many digits"};
        n = n * 10 + (uint64_t)(c - '0');
        if (frac) d *= 10;
      }
      if (at("%")) { take(); d *= 100; }
      if (braced) expect("}");
      uint64_t g = gcd64(n, d);
      if (g == 0) g = 1;
      q.num = n / g; q.den = d / g;
      explicit_c = true;
    }
    if (!explicit_c) {  // defaults stated after Def. 1
      if (q.kind == RV_Q_A) { q.op = RV_EQ; q.num = 1; q.den = 1; }
      else { q.op = RV_GE; q.num = 1; q.den = 1; }
    }
    if (q.kind == RV_Q_A && q.num > q.den) throw ParseFail{RV_EPARSE, "A constant must lie in [0,1]"};
    if (q.kind == RV_Q_E && q.den != 1) throw ParseFail{RV_EPARSE, "E constant must be a non-negative integer"};
    std::string var = take();
    if (!ident(var)) throw ParseFail{RV_EPARSE, "bad variable '" + var + "'"};
    expect(":");
    std::string pred = take();
    if (!ident(pred)) throw ParseFail{RV_EPARSE, "bad binding predicate '" + pred + "'"};
    if (at("(")) args();
    expect("=>");
    quants.push_back(q);
  }
  void args() {
    expect("(");
    while (!at(")")) { take(); if (at(",")) take(); }
    expect(")");
  }
  int qformula() {
    if (at("(") && quant_start(1)) { take(); int f = qformula(); expect(")"); return f; }
    if (quant_start(0)) { quantifier(); return qformula(); }
    return iff();
  }
  int iff() {
    int f = imp();
    while (at("<->")) {
      take();
      int g = imp();
      f = B.disj(B.conj(f, g), B.conj(B.neg(f), B.neg(g)));
    }
    return f;
  }
  int imp() {
    int f = disj();
    if (at("->")) { take(); int g = imp(); return B.disj(B.neg(f), g); }
    return f;
  }
  int disj() {
    int f = conj();
    while (at("||") || at("|")) { take(); f = B.disj(f, conj()); }
    return f;
  }
  int conj() {
    int f = until();
    while (at("&&") || at("&")) { take(); f = B.conj(f, until()); }
    return f;
  }
  int until() {
    int f = unary();
    if (at("U") || at("R") || at("W")) {
      std::string op = take();
      int g = until();
      if (op == "U") return B.until(f, g);
      if (op == "R") return B.neg(B.until(B.neg(f), B.neg(g)));
      return B.disj(B.until(f, g), B.always(f));    // W
    }
    return f;
  }
  int unary() {
    if (at("!")) { take(); return B.neg(unary()); }
    if (at("X")) { take(); return B.next(unary()); }
    if (at("F")) { take(); return B.eventually(unary()); }
    if (at("G")) { take(); return B.always(unary()); }
    if (at("(")) { take(); int f = iff(); expect(")"); return f; }
    if (at("true")) { take(); return B.top(); }
    if (at("false")) { take(); return B.bot(); }
    auto p = peek();
    if (p && ident(*p) && *p != "U" && *p != "R" && *p != "W" && *p != "A" && *p != "E") {
      std::string name = take();
      if (at("(")) args();
      int op = -1;
      uint64_t c = 0;
      static const char* cmps[] = {"<", "<=", ">", ">=", "="};
      for (int k = 0; k < 5; ++k)
        if (at(cmps[k])) op = k;             // RV_LT, RV_LE, RV_GT, RV_GE, RV_EQ in that order
      std::string atom = name;
      if (op >= 0) {                         // interpreted predicate: value ~ integer constant
        take();
        const std::string num = take();
        if (num.empty() || !is_digit(num[0]) || num.find('.') != std::string::npos || num.size() > 10)
          throw ParseFail{RV_EPARSE, "a comparison needs an integer constant, got '" + num + "'"};
        c = strtoull(num.c_str(), nullptr, 10);
        if (c > 0xFFFFFFFFull) throw ParseFail{RV_EPARSE, "comparison constant beyond 2^32-1"};
        atom = name + cmps[op] + std::to_string(c);
      }
      size_t k = std::find(aps.begin(), aps.end(), atom) - aps.begin();
      if (k == aps.size()) { aps.push_back(atom); cmp.push_back(Cmp{name, op, c}); }
      return B.ap((int)k);
    }
    throw ParseFail{RV_EPARSE, std::string("unexpected token '") + (p ? *p : "end") + "'"};
  }
};

// ------------------------------------------------------------------ monitor synthesis
struct Synth {
  const std::vector<CNode>& nd;
  int root;
  explicit Synth(const std::vector<CNode>& n, int r) : nd(n), root(r) {}

  uint64_t prep(uint64_t mask, uint64_t next) const {
    uint64_t t = 0;
    for (size_t i = 0; i < nd.size(); ++i) {
      const CNode& c = nd[i];
      bool v = false;
      switch (c.op) {
        case N_TRUE: v = true; break;
        case N_AP: v = (mask >> c.a) & 1; break;
        case N_NOT: v = !((t >> c.a) & 1); break;
        case N_AND: v = ((t >> c.a) & 1) && ((t >> c.b) & 1); break;
        case N_X: v = (next >> c.a) & 1; break;
        case N_U: v = ((t >> c.b) & 1) || (((t >> c.a) & 1) && ((next >> i) & 1)); break;
      }
      if (v) t |= 1ull << i;
    }
    return t;
  }
  // type of a candidate: letter mask plus chosen truth of the X/U nodes
  uint64_t candidate(uint64_t mask, uint64_t temporal_bits) const {
    uint64_t t = temporal_bits;
    for (size_t i = 0; i < nd.size(); ++i) {
      const CNode& c = nd[i];
      bool v;
      switch (c.op) {
        case N_TRUE: v = true; break;
        case N_AP: v = (mask >> c.a) & 1; break;
        case N_NOT: v = !((t >> c.a) & 1); break;
        case N_AND: v = ((t >> c.a) & 1) && ((t >> c.b) & 1); break;
        default: continue;
      }
      if (v) t |= 1ull << i;
    }
    return t;
  }

  // realisable types (types of infinite words over the letters in sigma)
  rv_status realisable(const std::vector<uint64_t>& sigma, std::vector<uint64_t>& out) const {
    std::vector<int> temp;
    for (size_t i = 0; i < nd.size(); ++i)
      if (nd[i].op == N_X || nd[i].op == N_U) temp.push_back((int)i);
    const int k = (int)temp.size();
    if (k > 16 || ((uint64_t)sigma.size() << k) > (1u << 20))
      return rv_fail(RV_EUNSUPPORTED, "formula body too large for monitor synthesis (%d temporal operators)", k);
    std::vector<uint64_t> cand;
    for (uint64_t m : sigma)
      for (uint64_t bits = 0; bits < (1ull << k); ++bits) {
        uint64_t tb = 0;
        for (int j = 0; j < k; ++j) if ((bits >> j) & 1) tb |= 1ull << temp[j];
        cand.push_back(candidate(m, tb));
      }
    const size_t C = cand.size();
    // signature a predecessor constrains: child of each X, and each U itself
    auto sig_of = [&](uint64_t t) {
      uint64_t s = 0;
      for (int j = 0; j < k; ++j) {
        const CNode& c = nd[temp[j]];
        bool b = c.op == N_X ? ((t >> c.a) & 1) : ((t >> temp[j]) & 1);
        if (b) s |= 1ull << j;
      }
      return s;
    };
    std::unordered_map<uint64_t, std::vector<int>> by_sig;
    for (size_t j = 0; j < C; ++j) by_sig[sig_of(cand[j])].push_back((int)j);
    std::vector<std::vector<int>> succ(C), pred(C);
    for (size_t a = 0; a < C; ++a) {
      uint64_t t = cand[a], fixed = 0, freemask = 0;
      bool ok = true;
      for (int j = 0; j < k && ok; ++j) {
        const CNode& c = nd[temp[j]];
        bool self = (t >> temp[j]) & 1;
        if (c.op == N_X) { if (self) fixed |= 1ull << j; continue; }
        bool A = (t >> c.a) & 1, Bv = (t >> c.b) & 1;
        if (Bv) { if (!self) ok = false; else freemask |= 1ull << j; }
        else if (A) { if (self) fixed |= 1ull << j; }
        else { if (self) ok = false; else freemask |= 1ull << j; }
      }
      if (!ok) continue;
      // enumerate subsets of freemask
      uint64_t sub = 0;
      while (true) {
        auto it = by_sig.find(fixed | sub);
        if (it != by_sig.end())
          for (int b : it->second) { succ[a].push_back(b); pred[b].push_back((int)a); }
        if (sub == freemask) break;
        sub = (sub - freemask) & freemask;
      }
    }
    std::vector<char> alive(C, 1);
    std::vector<int> nsucc(C);
    for (size_t a = 0; a < C; ++a) nsucc[a] = (int)succ[a].size();
    bool changed = true;
    std::vector<char> reach(C);
    std::vector<int> stack;
    while (changed) {
      changed = false;
      // candidates with no surviving successor
      for (size_t a = 0; a < C; ++a) {
        if (!alive[a]) continue;
        bool any = false;
        for (int b : succ[a]) if (alive[b]) { any = true; break; }
        if (!any) { alive[a] = 0; changed = true; }
      }
      // unfulfillable untils
      for (int j = 0; j < k; ++j) {
        const CNode& c = nd[temp[j]];
        if (c.op != N_U) continue;
        std::fill(reach.begin(), reach.end(), 0);
        stack.clear();
        for (size_t a = 0; a < C; ++a)
          if (alive[a] && ((cand[a] >> c.b) & 1)) { reach[a] = 1; stack.push_back((int)a); }
        while (!stack.empty()) {
          int b = stack.back(); stack.pop_back();
          for (int a : pred[b]) if (alive[a] && !reach[a]) { reach[a] = 1; stack.push_back(a); }
        }
        for (size_t a = 0; a < C; ++a)
          if (alive[a] && ((cand[a] >> temp[j]) & 1) && !reach[a]) { alive[a] = 0; changed = true; }
      }
    }
    out.clear();
    for (size_t a = 0; a < C; ++a) if (alive[a]) out.push_back(cand[a]);
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
    if (out.empty()) return rv_fail(RV_EINTERNAL, "no realisable type");
    return RV_OK;
  }
};

struct VecHash {
  size_t operator()(const std::vector<uint16_t>& v) const {
    uint64_t h = 1469598103934665603ull;
    for (uint16_t x : v) { h ^= x; h *= 1099511628211ull; }
    return (size_t)h;
  }
};

rv_status synthesise(const Builder& B, int root, const std::vector<uint64_t>& letter_mask, rv_formula* f) {
  if (B.nodes.size() > 64) return rv_fail(RV_EUNSUPPORTED, "formula body has more than 64 subformulas");
  Synth S(B.nodes, root);
  std::vector<uint64_t> sigma(letter_mask);
  std::sort(sigma.begin(), sigma.end());
  sigma.erase(std::unique(sigma.begin(), sigma.end()), sigma.end());
  std::vector<uint64_t> R;
  rv_status st = S.realisable(sigma, R);
  if (st != RV_OK) return st;
  // domain: realisable types followed by the finite-word types reachable from "end"
  std::vector<uint64_t> D(R);
  std::unordered_map<uint64_t, int> idx;
  for (size_t i = 0; i < D.size(); ++i) idx[D[i]] = (int)i;
  const size_t nR = R.size();
  std::vector<uint64_t> work{0};
  if (!idx.count(0)) { idx[0] = (int)D.size(); D.push_back(0); }
  const int end_idx = idx[0];
  while (!work.empty()) {
    uint64_t t = work.back(); work.pop_back();
    for (uint64_t m : sigma) {
      uint64_t u = S.prep(m, t);
      if (!idx.count(u)) { idx[u] = (int)D.size(); D.push_back(u); work.push_back(u); }
    }
    if (D.size() > 60000) return rv_fail(RV_EUNSUPPORTED, "too many finite-trace types");
  }
  const size_t nD = D.size();
  if (nD > 65535) return rv_fail(RV_EUNSUPPORTED, "type domain too large");
  std::vector<std::vector<uint16_t>> P(sigma.size(), std::vector<uint16_t>(nD));
  for (size_t s = 0; s < sigma.size(); ++s)
    for (size_t d = 0; d < nD; ++d) {
      auto it = idx.find(S.prep(sigma[s], D[d]));
      if (it == idx.end()) return rv_fail(RV_EINTERNAL, "type domain not closed under prepend");
      P[s][d] = (uint16_t)it->second;
    }
  // reachable prefix maps f_u, f_{ua}[d] = f_u[P_a[d]]
  std::vector<std::vector<uint16_t>> states;
  std::unordered_map<std::vector<uint16_t>, int, VecHash> sid;
  std::vector<uint16_t> id(nD);
  for (size_t d = 0; d < nD; ++d) id[d] = (uint16_t)d;
  states.push_back(id);
  sid[id] = 0;
  std::vector<std::vector<int>> delta;
  for (size_t q = 0; q < states.size(); ++q) {
    std::vector<int> row(sigma.size());
    for (size_t s = 0; s < sigma.size(); ++s) {
      std::vector<uint16_t> g(nD);
      const std::vector<uint16_t>& fq = states[q];
      for (size_t d = 0; d < nD; ++d) g[d] = fq[P[s][d]];
      auto it = sid.find(g);
      int to;
      if (it == sid.end()) {
        to = (int)states.size();
        if (to > 200000) return rv_fail(RV_EUNSUPPORTED, "monitor construction exceeds 200000 states");
        sid.emplace(g, to);
        states.push_back(std::move(g));
      } else {
        to = it->second;
      }
      row[s] = to;
    }
    delta.push_back(row);
  }
  const size_t Q = states.size();
  std::vector<int> label(Q);
  for (size_t q = 0; q < Q; ++q) {
    size_t yes = 0;
    for (size_t d = 0; d < nR; ++d) yes += (D[states[q][d]] >> root) & 1;
    if (yes == nR) label[q] = RV_TOP;
    else if (yes == 0) label[q] = RV_BOT;
    else label[q] = ((D[states[q][end_idx]] >> root) & 1) ? RV_TOP_P : RV_BOT_P;
  }
  // Moore partition refinement
  std::vector<int> cls(label);
  size_t ncls = 0;
  while (true) {
    std::map<std::vector<int>, int> key;
    std::vector<int> nc(Q);
    for (size_t q = 0; q < Q; ++q) {
      std::vector<int> sig{cls[q]};
      for (size_t s = 0; s < sigma.size(); ++s) sig.push_back(cls[delta[q][s]]);
      auto it = key.find(sig);
      if (it == key.end()) { int c = (int)key.size(); key.emplace(sig, c); nc[q] = c; }
      else nc[q] = it->second;
    }
    size_t n = key.size();
    cls.swap(nc);
    if (n == ncls) break;
    ncls = n;
  }
  // renumber classes breadth-first from the initial state
  std::vector<int> order(ncls, -1), rep(ncls, -1);
  for (size_t q = 0; q < Q; ++q) if (rep[cls[q]] < 0) rep[cls[q]] = (int)q;
  std::vector<int> queue{cls[0]};
  order[cls[0]] = 0;
  int next_id = 1;
  for (size_t h = 0; h < queue.size(); ++h) {
    int c = queue[h];
    for (size_t s = 0; s < sigma.size(); ++s) {
      int c2 = cls[delta[rep[c]][s]];
      if (order[c2] < 0) { order[c2] = next_id++; queue.push_back(c2); }
    }
  }
  if (next_id > RV_MAX_STATES)
    return rv_fail(RV_EUNSUPPORTED, "minimal LTL4 monitor has %d states (more than 16)", next_id);
  f->n_states = next_id;
  f->q0 = 0;
  for (int s = 0; s < RV_MAX_STATES; ++s) f->labels[s] = RV_BOT;
  for (size_t c = 0; c < ncls; ++c) if (order[c] >= 0) f->labels[order[c]] = (uint8_t)label[rep[c]];
  for (int l = 0; l < f->n_letters; ++l) {
    size_t s = std::lower_bound(sigma.begin(), sigma.end(), letter_mask[l]) - sigma.begin();
    uint64_t m = 0;
    for (int st = 0; st < RV_MAX_STATES; ++st) {
      uint64_t to = (uint64_t)st;
      if (st < next_id) {
        int c = -1;
        for (size_t cc = 0; cc < ncls; ++cc) if (order[cc] == st) { c = (int)cc; break; }
        to = (uint64_t)order[cls[delta[rep[c]][s]]];
      }
      m |= to << (4 * st);
    }
    f->maps[l] = m;
  }
  return RV_OK;
}

}  // namespace

extern "C" rv_status rv_compile_formula(const char* text, const rv_schema* schema, rv_formula** out,
                                        char* err, size_t errlen) {
  auto report = [&](rv_status st) {
    if (err && errlen) { snprintf(err, errlen, "%s", rv_last_error()); }
    return st;
  };
  if (!text || !schema || !out) return report(rv_fail(RV_EINVAL, "null argument"));
  *out = nullptr;
  if (schema->alphabet != RV_ONEHOT && schema->alphabet != RV_BITMASK)
    return report(rv_fail(RV_EINVAL, "unknown alphabet mode"));
  if (schema->n_codes < 1 || (schema->alphabet == RV_ONEHOT && schema->n_codes > 256) ||
      (schema->alphabet == RV_BITMASK && schema->n_codes > 8))
    return report(rv_fail(RV_EINVAL, "n_codes out of range"));
  if (schema->key_bits != 32 && schema->key_bits != 64) return report(rv_fail(RV_EINVAL, "key_bits must be 32 or 64"));
  if (!schema->code_names) return report(rv_fail(RV_EINVAL, "code_names is NULL"));
  Builder B;
  Parser p(B);
  int root;
  try {
    p.t = tokenize(text);
    root = p.qformula();
    if (p.peek()) throw ParseFail{RV_EPARSE, "trailing input at '" + *p.peek() + "'"};
  } catch (const ParseFail& e) {
    return report(rv_fail(e.st, "%s", e.msg.c_str()));
  } catch (...) {
    return report(rv_fail(RV_EINTERNAL, "parser failure"));
  }
  if (p.quants.size() > 2) return report(rv_fail(RV_EUNSUPPORTED, "at most two counting quantifiers"));
  if (p.quants.size() == 2 && schema->key_bits != 64)
    return report(rv_fail(RV_EINVAL, "two quantified variables need 64-bit keys (d0 << 32 | d1)"));
  if (p.aps.size() > 64) return report(rv_fail(RV_EUNSUPPORTED, "too many propositions"));
  std::vector<int> ap_code(p.aps.size(), -1), ap_cmp(p.aps.size(), -1);
  int n_cmp = 0;
  for (size_t a = 0; a < p.aps.size(); ++a) {
    if (p.cmp[a].op >= 0) {
      if (!schema->value_name || p.cmp[a].name != schema->value_name)
        return report(rv_fail(RV_EPARSE, "comparison on '%s', which is not the schema's value column",
                              p.cmp[a].name.c_str()));
      if (n_cmp >= RV_MAX_CMP) return report(rv_fail(RV_EUNSUPPORTED, "more than %d comparison atoms", RV_MAX_CMP));
      ap_cmp[a] = n_cmp++;
      continue;
    }
    for (int c = 0; c < schema->n_codes; ++c)
      if (schema->code_names[c] && p.aps[a] == schema->code_names[c]) { ap_code[a] = c; break; }
    if (ap_code[a] < 0) return report(rv_fail(RV_EPARSE, "body proposition '%s' is not a predicate code", p.aps[a].c_str()));
  }
  const int n_base = schema->alphabet == RV_ONEHOT ? schema->n_codes : (1 << schema->n_codes);
  if (n_base << n_cmp > RV_MAX_LETTERS)
    return report(rv_fail(RV_EUNSUPPORTED, "%d predicate letters times %d comparison outcomes exceed %d letters",
                          n_base, 1 << n_cmp, RV_MAX_LETTERS));
  rv_formula* f = new (std::nothrow) rv_formula();
  if (!f) return report(rv_fail(RV_ENOMEM, "out of host memory"));
  f->n_quant = (int)p.quants.size();
  for (int i = 0; i < f->n_quant; ++i) f->q[i] = p.quants[i];
  f->key_bits = schema->key_bits;
  f->alphabet = schema->alphabet;
  f->n_codes = schema->n_codes;
  f->n_base = n_base;
  f->n_cmp = n_cmp;
  for (size_t a = 0; a < p.aps.size(); ++a)
    if (ap_cmp[a] >= 0) { f->cmp_op[ap_cmp[a]] = p.cmp[a].op; f->cmp_c[ap_cmp[a]] = (uint32_t)p.cmp[a].c; }
  f->n_letters = n_base << n_cmp;
  f->text = text;
  // comparison outcomes some value can produce: the atoms are thresholds on one
  // variable, so the values 0, 2^32-1 and c-1, c, c+1 of every constant meet
  // every outcome there is
  std::vector<char> realisable((size_t)1 << n_cmp, 0);
  {
    std::vector<uint64_t> cand{0ull, 0xFFFFFFFFull};
    for (int j = 0; j < n_cmp; ++j)
      for (int d = -1; d <= 1; ++d) {
        const int64_t v = (int64_t)f->cmp_c[j] + d;
        if (v >= 0 && v <= 0xFFFFFFFFll) cand.push_back((uint64_t)v);
      }
    for (uint64_t v : cand) {
      unsigned bits = 0;
      for (int j = 0; j < n_cmp; ++j) {
        const uint64_t c = f->cmp_c[j];
        const int op = f->cmp_op[j];
        const bool on = op == RV_LT ? v < c : op == RV_LE ? v <= c : op == RV_GT ? v > c : op == RV_GE ? v >= c : v == c;
        if (on) bits |= 1u << j;
      }
      realisable[bits] = 1;
    }
  }
  unsigned first_real = 0;
  while (!realisable[first_real]) ++first_real;
  std::vector<uint64_t> mask(f->n_letters, 0);
  for (int l = 0; l < f->n_letters; ++l) {
    const int base = l % n_base;
    unsigned bits = (unsigned)(l / n_base);
    if (!realisable[bits]) bits = first_real;   // never produced; kept out of the effective alphabet
    for (size_t a = 0; a < p.aps.size(); ++a) {
      bool on;
      if (ap_cmp[a] >= 0) on = (bits >> ap_cmp[a]) & 1u;
      else on = schema->alphabet == RV_ONEHOT ? (ap_code[a] == base) : ((base >> ap_code[a]) & 1);
      if (on) mask[l] |= 1ull << a;
    }
  }
  rv_status st;
  try {
    st = synthesise(B, root, mask, f);
  } catch (...) {
    st = rv_fail(RV_ENOMEM, "monitor synthesis ran out of memory");
  }
  if (st != RV_OK) { delete f; return report(st); }
  *out = f;
  return RV_OK;
}

extern "C" rv_status rv_formula_get_info(const rv_formula* f, rv_formula_info* info) {
  if (!f || !info) return rv_fail(RV_EINVAL, "null argument");
  info->n_quant = f->n_quant;
  info->n_states = f->n_states;
  info->n_letters = f->n_letters;
  info->q0 = f->q0;
  info->key_bits = f->key_bits;
  info->alphabet = f->alphabet;
  info->n_base = f->n_base;
  info->n_cmp = f->n_cmp;
  return RV_OK;
}

extern "C" rv_status rv_formula_tables(const rv_formula* f, uint64_t* maps, int n_maps, uint8_t labels[16]) {
  if (!f) return rv_fail(RV_EINVAL, "null formula");
  if (maps) {
    if (n_maps < f->n_letters) return rv_fail(RV_EINVAL, "maps array shorter than n_letters");
    memcpy(maps, f->maps, sizeof(uint64_t) * f->n_letters);
  }
  if (labels) memcpy(labels, f->labels, 16);
  return RV_OK;
}

extern "C" rv_status rv_formula_quantifier(const rv_formula* f, int level, int* kind, int* op,
                                           uint64_t* num, uint64_t* den) {
  if (!f || level < 0 || level >= f->n_quant) return rv_fail(RV_EINVAL, "no quantifier at that level");
  if (kind) *kind = f->q[level].kind;
  if (op) *op = f->q[level].op;
  if (num) *num = f->q[level].num;
  if (den) *den = f->q[level].den;
  return RV_OK;
}

extern "C" void rv_formula_free(rv_formula* f) { delete f; }

extern "C" rv_status rv_valuate(int kind, int op, uint64_t num, uint64_t den, const uint64_t v[6], int* verdict) {
  if (!v || !verdict || (kind != RV_Q_A && kind != RV_Q_E) || op < RV_LT || op > RV_EQ || den == 0)
    return rv_fail(RV_EINVAL, "bad valuation arguments");
  *verdict = rvv::valuate(kind, op, num, den, v);
  return RV_OK;
}
