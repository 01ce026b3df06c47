// Six-valued valuation of a counting-quantifier node (Eq. S, Def. "LTL4-C
// Semantics", Table 1), shared by the host entry rv_valuate and the reduce
// kernels.  All arithmetic is in integers: an A constraint n ~ c*N with
// c = num/den is decided as n*den ~ num*N in 128-bit.
//
// Readings of the garbled definition (the six cases tried top-down in
// lattice order, first match wins):
//   ~ in {>=, >}:  T  if C(v_T) and permanently satisfied
//                  Tc if C(v_T + v_Tc)
//                  Tp if C(v_T + v_Tc + v_Tp)
//                  Fp if C(v_T + v_Tc + v_Tp + v_Fp)     (printed "= 0" read as "= 1")
//                  F  if permanently violated, else Fc
//   ~ in {<=, <}:  the same cascade on the mirrored counts
//                  N - v_F, N - v_F - v_Fc, v_T + v_Tc + v_Tp, v_T + v_Tc
//   ~ is '=':      the same rungs with the constraint an exact equality:
//                  Tc if C(v_T + v_Tc) and C(v_T + v_Tc + v_Tp + v_Fp),
//                  Tp if C(v_T + v_Tc + v_Tp), Fp if some count between the
//                  first two meets it, F if permanently violated, else Fc
//                  (never T: a continuation can always break an equality).
// Permanence: E follows Table 1 (>, >=: satisfied for good once C(v_T);
// =, <=, <: violated for good once !C(v_T)).  A with c = num/den:
//   >=: sat iff c = 0, viol iff c = 1 and v_F >= 1
//   > : sat iff c = 0 and v_T >= 1, viol iff c = 1
//   <=: sat iff c = 1, viol iff c = 0 and v_T >= 1
//   < : sat iff c = 1 and v_F >= 1, viol iff c = 0
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define RV_HD __host__ __device__ __forceinline__
#else
#define RV_HD inline
#endif

namespace rvv {

enum { VF = 0, VFC = 1, VFP = 2, VTP = 3, VTC = 4, VT = 5 };
enum { LT = 0, LE = 1, GT = 2, GE = 3, EQ = 4 };
enum { QA = 0, QE = 1 };

typedef unsigned __int128 u128;

RV_HD bool cmp(int op, u128 a, u128 b) {
  switch (op) {
    case LT: return a < b;
    case LE: return a <= b;
    case GT: return a > b;
    case GE: return a >= b;
    default: return a == b;
  }
}

RV_HD bool constraint(int kind, int op, uint64_t num, uint64_t den, uint64_t n, uint64_t N) {
  if (kind == QA) return cmp(op, (u128)n * den, (u128)num * N);
  return cmp(op, (u128)n, (u128)num);
}

RV_HD bool perm_sat(int kind, int op, uint64_t num, uint64_t den, const uint64_t* v) {
  if (kind == QE) return (op == GT || op == GE) ? constraint(kind, op, num, den, v[VT], 0) : false;
  const bool c0 = num == 0, c1 = num == den;
  switch (op) {
    case GE: return c0;
    case GT: return c0 && v[VT] >= 1;
    case LE: return c1;
    default: return c1 && v[VF] >= 1;   // LT
  }
}

RV_HD bool perm_viol(int kind, int op, uint64_t num, uint64_t den, const uint64_t* v) {
  if (kind == QE) return (op == LT || op == LE) ? !constraint(kind, op, num, den, v[VT], 0) : false;
  const bool c0 = num == 0, c1 = num == den;
  switch (op) {
    case GE: return c1 && v[VF] >= 1;
    case GT: return c1;
    case LE: return c0 && v[VT] >= 1;
    default: return c0;                 // LT
  }
}

RV_HD int ladder(int kind, int op, uint64_t num, uint64_t den, const uint64_t* v) {
  const uint64_t N = v[0] + v[1] + v[2] + v[3] + v[4] + v[5];
  uint64_t n1, n2, n3, n4;
  if (op == GE || op == GT) {
    n1 = v[VT];
    n2 = n1 + v[VTC];
    n3 = n2 + v[VTP];
    n4 = n3 + v[VFP];
  } else {
    n1 = N - v[VF];
    n2 = n1 - v[VFC];
    n3 = v[VT] + v[VTC] + v[VTP];
    n4 = v[VT] + v[VTC];
  }
  if (constraint(kind, op, num, den, n1, N) && perm_sat(kind, op, num, den, v)) return VT;
  if (constraint(kind, op, num, den, n2, N)) return VTC;
  if (constraint(kind, op, num, den, n3, N)) return VTP;
  if (constraint(kind, op, num, den, n4, N)) return VFP;
  if (perm_viol(kind, op, num, den, v)) return VF;
  return VFC;
}

RV_HD int equality(int kind, uint64_t num, uint64_t den, const uint64_t* v) {
  const uint64_t N = v[0] + v[1] + v[2] + v[3] + v[4] + v[5];
  const uint64_t lo = v[VT] + v[VTC], hi = lo + v[VTP] + v[VFP];
  if (constraint(kind, EQ, num, den, lo, N) && constraint(kind, EQ, num, den, hi, N)) return VTC;
  if (constraint(kind, EQ, num, den, lo + v[VTP], N)) return VTP;
  // is there an integer count n in [lo, hi] with n == l (E) or n * den == num * N (A)?
  if (kind == QE) {
    if (num >= lo && num <= hi) return VFP;
  } else {
    const u128 t = (u128)num * N;
    if (t % den == 0 && t / den >= lo && t / den <= hi) return VFP;
  }
  const bool viol = kind == QE ? v[VT] > num
                               : ((num == den && v[VF] >= 1) || (num == 0 && v[VT] >= 1));
  return viol ? VF : VFC;
}

RV_HD int valuate(int kind, int op, uint64_t num, uint64_t den, const uint64_t* v) {
  if (op == EQ) return equality(kind, num, den, v);
  return ladder(kind, op, num, den, v);
}

}  // namespace rvv
