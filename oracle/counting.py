"""Counting quantifiers and six-valued semantics (Sec. 2.4).  Test infrastructure only.

Truth values B6 are coded in their lattice order (Sec. 2.3):
    F = 0 < Fc = 1 < Fp = 2 < Tp = 3 < Tc = 4 < T = 5.

Eq. S: for the quantifier tuple <Q, ~, c, x, p> of a node with child vector
counts v (v[b] = |B(phi, u, D|^m, b)|, Sec. 3.4) and N = |P(phi, u, D|^m)|
children, and a set B of truth values with n = sum of v[b] over b in B,
    A:  n ~ c * N      (decided exactly as n * q ~ p * N, c = p / q)
    E:  n ~ c
Def. "LTL4-C Semantics" assigns one of the six values from such constraints
plus permanence conditions.  The definition as printed is garbled in places,
so this module fixes one reading and every other part of the project follows
it:

 * cases are tried top-down in lattice order and the first one that applies
   wins (Sec. 2.3: Tp only when Tc fails, Fp only when Tp and Tc fail);
 * the Fp case's second conjunct is read S(B6 - {F, Fc}) = 1 (printed = 0,
   which contradicts the Fc case and the prose about phi_2);
 * for ~ in {>=, >} the ladder is the one printed:  T if S({T}) and the
   constraint is permanently satisfied, Tc if S({T,Tc}), Tp if
   S({T,Tc,Tp}), Fp if S(B6 - {F,Fc}), F if permanently violated, else Fc;
 * for ~ in {<=, <} the ladder runs the mirrored counts -- the children that
   could still be true are the ones that push the count up -- so:
   T if (N - v[F]) ~ and permanently satisfied, Tc if (N - v[F] - v[Fc]) ~,
   Tp if (v[T]+v[Tc]+v[Tp]) ~, Fp if (v[T]+v[Tc]) ~, F if permanently violated,
   else Fc (this makes Table 1's direction hold: E_{<=c} is violated for good
   once more than c children are definitely true);
 * ~ is '=' : the same rungs with Eq. S an exact equality n*q = p*N:
   Tc if both v[T]+v[Tc] and v[T]+v[Tc]+v[Tp]+v[Fp] meet it (so does every
   count between), Tp if v[T]+v[Tc]+v[Tp] meets it, Fp if some count of true
   children between those two meets it, F if permanently violated (E: v[T] > l,
   Table 1; A: c = 1 and v[F] >= 1, or c = 0 and v[T] >= 1), else Fc; never T,
   since a continuation can always add a child that breaks the equality.  This
   gives E_{=0} = E_{<=0} (case study 3) and A_{=1} = A_{>=1} (Sec. 2.4.5);
 * permanence: the E rules of Table 1 (>, >=: permanently satisfied once the
   constraint holds on v[T]; =, <, <=: permanently violated once it fails on
   v[T]) and, for A with c = p/q, the rules obtained by letting a
   continuation add any number of children of any verdict while T and F
   children stay as they are: '>=': sat iff c = 0, viol iff c = 1 and
   v[F] >= 1;  '>': sat iff c = 0 and v[T] >= 1, viol iff c = 1;  '<=': sat
   iff c = 1, viol iff c = 0 and v[T] >= 1;  '<': sat iff c = 1 and
   v[F] >= 1, viol iff c = 0.  The paper states the A rule only for A_{=1}
   (one F child makes it F), which this reproduces.
 * N = 0 (a root with no bindings) is decided by the same integer comparisons.

Pins: beyond the worked example, Table 1, the A_{=1} rule and the
case-study thresholds, every rung and permanence rule here is checked against
an enumeration of how a node's children can still turn out (a T or F child
keeps its value, any other child may end either way, a continuation may add
children of any verdict; tests/test_oracle_permanence.py), for every count
vector with at most six children, every comparison and several constants, and
held to the order of B6 and to negation by the invariant tests.
"""
from __future__ import annotations

from fractions import Fraction

F, FC, FP, TP, TC, T = 0, 1, 2, 3, 4, 5
NAMES = {F: "F", FC: "Fc", FP: "Fp", TP: "Tp", TC: "Tc", T: "T"}

_CMP = {
    "<": lambda a, b: a < b,
    "<=": lambda a, b: a <= b,
    ">": lambda a, b: a > b,
    ">=": lambda a, b: a >= b,
    "=": lambda a, b: a == b,
}


def constraint(kind: str, op: str, const: Fraction, n: int, N: int) -> bool:
    """S of Eq. S for a count n out of N children."""
    if kind == "A":
        return _CMP[op](n * const.denominator, const.numerator * N)
    return _CMP[op](n, int(const))


def permanently_satisfied(kind, op, const, v) -> bool:
    if kind == "E":
        if op in (">", ">="):
            return constraint(kind, op, const, v[T], None)
        return False
    if op == ">=":
        return const == 0
    if op == ">":
        return const == 0 and v[T] >= 1
    if op == "<=":
        return const == 1
    if op == "<":
        return const == 1 and v[F] >= 1
    raise ValueError(op)


def permanently_violated(kind, op, const, v) -> bool:
    if kind == "E":
        if op in ("<", "<="):
            return not constraint(kind, op, const, v[T], None)
        return False
    if op == ">=":
        return const == 1 and v[F] >= 1
    if op == ">":
        return const == 1
    if op == "<=":
        return const == 0 and v[T] >= 1
    if op == "<":
        return const == 0
    raise ValueError(op)


def _ladder(kind, op, const, v):
    N = sum(v)
    if op in (">=", ">"):
        n1 = v[T]
        n2 = v[T] + v[TC]
        n3 = v[T] + v[TC] + v[TP]
        n4 = v[T] + v[TC] + v[TP] + v[FP]
    else:
        n1 = N - v[F]
        n2 = N - v[F] - v[FC]
        n3 = v[T] + v[TC] + v[TP]
        n4 = v[T] + v[TC]
    C = lambda n: constraint(kind, op, const, n, N)  # noqa: E731
    if C(n1) and permanently_satisfied(kind, op, const, v):
        return T
    if C(n2):
        return TC
    if C(n3):
        return TP
    if C(n4):
        return FP
    if permanently_violated(kind, op, const, v):
        return F
    return FC


def _equality(kind, const, v):
    N = sum(v)
    lo = v[T] + v[TC]                 # presumptive children all false
    hi = lo + v[TP] + v[FP]           # presumptive children all true
    C = lambda n: constraint(kind, "=", const, n, N)  # noqa: E731
    if C(lo) and C(hi):
        return TC
    if C(lo + v[TP]):
        return TP
    if any(C(n) for n in range(lo, hi + 1)):
        return FP
    if kind == "E":
        viol = v[T] > int(const)
    else:
        viol = (const == 1 and v[F] >= 1) or (const == 0 and v[T] >= 1)
    return F if viol else FC


def valuate(q, v) -> int:
    """Six-valued verdict of a quantifier node with child-verdict counts v[0..5]."""
    if len(v) != 6:
        raise ValueError("v must have six entries")
    if q.op == "=":
        return _equality(q.kind, q.const, v)
    return _ladder(q.kind, q.op, q.const, v)
