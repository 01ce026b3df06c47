"""Brute-force pin of the six-valued valuation of one quantifier node (no GPU).

Def. "LTL4-C Semantics" (Sec. 2.4.5) gives the six verdicts of a node by its
constraint S (Eq. S) and, for T and F, by a condition on every continuation of
the trace ("for all v in Sigma^omega, [uv |=_6 phi] = T", resp. F).  Sec. 2.3
describes the middle values informally: Tc/Fc are what the node's children
currently establish, Tp/Fp what holds if the program stops now.  The oracle
(oracle/counting.py) turns this into a ladder of closed-form count sums and
permanence rules, most of which the paper never prints (the A rules beyond
A_{=1}, the <=/< ladder, '=').  This module decides the same verdicts with no
closed form, by enumerating how the node's children can still turn out:

  * a child whose verdict is T or F keeps it in every continuation (LTL4 T/F
    and six-valued T/F are permanent by their definitions); a child with any
    of the four other verdicts may still end up true or false;
  * a continuation of the trace may move every undecided child to any verdict
    and add new children of any verdict (here: up to K more fixed-true, K more
    fixed-false and K more undecided children, with K raised until the
    answers stop changing);
  * a "resolution" assigns a truth value to every undecided child; the
    constraint of Eq. S is then evaluated on the number of true children out
    of all children, in exact integers (A: n*q ~ p*N; E: n ~ l).

With these, the six rungs, tried top-down in lattice order (Sec. 2.3), are:

  T   every continuation, under every resolution, satisfies the constraint
  Tc  every resolution of the presumptive (Tp, Fp) children satisfies it, the
      Tc children counted true and the Fc children false (what is currently
      established cannot be undone by how the presumptive ones end)
  Tp  the presumed resolution (Tp, Tc true; Fp, Fc false) satisfies it
  Fp  some resolution of the presumptive children satisfies it (Tc true, Fc
      false)
  F   no continuation has a resolution that satisfies it
  Fc  otherwise

and the oracle must agree with them on every child-count vector with at most
six children, for every comparison and the constants below.  The
permanence predicates are compared on their own as well (T rung: "every
continuation satisfies"; F rung: "no continuation can").
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import counting
from oracle.counting import F, FC, FP, T, TC, TP
from oracle.formula import Quantifier

OPS = ("<", "<=", ">", ">=", "=")
CONSTS = {"A": [Fraction(0), Fraction(1, 4), Fraction(1, 2), Fraction(1)],
          "E": [Fraction(k) for k in range(4)]}
MAX_N = 6
K_STABLE = 30          # enough to push A_{>=1/4} below 1/4 from six true children


def _holds(kind, op, c, n, N):
    """Eq. S on n true children out of N, as exact integers (arrays allowed)."""
    lhs, rhs = (n * c.denominator, c.numerator * N) if kind == "A" else (n, int(c) + 0 * n)
    return {"<": lhs < rhs, "<=": lhs <= rhs, ">": lhs > rhs, ">=": lhs >= rhs, "=": lhs == rhs}[op]


def _vectors(max_n):
    """Every vector of six child-verdict counts with 0 <= N <= max_n."""
    out = []

    def rec(prefix, left):
        if len(prefix) == 5:
            out.append(tuple(prefix) + (left,))
            return
        for k in range(left + 1):
            rec(prefix + [k], left - k)
    for N in range(max_n + 1):
        rec([], N)
    return out


def _reach(t_fixed, f_fixed, free, K, KU=2):
    """Boolean table R[t, N]: a continuation has a resolution with t true
    children out of N.  Existing undecided children: i move to T, j to F, the
    rest stay undecided; new children: aT <= K fixed true, aF <= K fixed
    false, aU <= KU undecided; then x of all undecided children resolve true."""
    tmax = t_fixed + free + K + KU
    nmax = t_fixed + f_fixed + free + 2 * K + KU
    R = np.zeros((tmax + 1, nmax + 1), dtype=bool)
    aT = np.arange(K + 1)[:, None, None]
    aF = np.arange(K + 1)[None, :, None]
    N0 = t_fixed + f_fixed + free
    for i in range(free + 1):
        for j in range(free - i + 1):
            for aU in range(KU + 1):
                x = np.arange(free - i - j + aU + 1)[None, None, :]
                t = t_fixed + i + aT + x + 0 * aF
                n = N0 + aT + aF + aU + 0 * x
                R[t, n] = True
    return R


def _brute(kinds_consts, K):
    """Verdict, 'every continuation satisfies' and 'no continuation can' by
    enumeration, keyed by (kind, op, const, v)."""
    reach_cache = {}
    out = {}
    vectors = _vectors(MAX_N)
    for v in vectors:
        N = sum(v)
        und = N - v[T] - v[F]
        key = (v[T], v[F], und)
        if key not in reach_cache:
            reach_cache[key] = _reach(v[T], v[F], und, K)
        R = reach_cache[key]
        tt, nn = np.nonzero(R)
        pres = v[TP] + v[FP]
        xs = np.arange(pres + 1)
        cur = v[T] + v[TC] + xs                     # Tc true, Fc false, x presumptive true
        for kind, c in kinds_consts:
            for op in OPS:
                sat = _holds(kind, op, c, tt, nn)
                all_sat, none_sat = bool(sat.all()), not bool(sat.any())
                cs = _holds(kind, op, c, cur, N)
                if all_sat:
                    b = T
                elif cs.all():
                    b = TC
                elif _holds(kind, op, c, v[T] + v[TC] + v[TP], N):
                    b = TP
                elif cs.any():
                    b = FP
                elif none_sat:
                    b = F
                else:
                    b = FC
                out[(kind, op, c, v)] = (b, all_sat, none_sat)
    return out


_KC = [(k, c) for k in ("A", "E") for c in CONSTS[k]]


@pytest.fixture(scope="module")
def brute():
    a = _brute(_KC, K_STABLE)
    b = _brute(_KC, K_STABLE + 1)
    assert a == b, "enumeration bound too small: answers change from K to K+1"
    return a


def _mismatches(brute):
    bad = []
    for (kind, op, c, v), (b, all_sat, none_sat) in brute.items():
        q = Quantifier(kind, op, c, "x", "p")
        got = counting.valuate(q, list(v))
        if got != b:
            bad.append(("valuate", kind, op, c, v, got, b))
        if op != "=":
            ps = counting.permanently_satisfied(kind, op, c, list(v))
            pv = counting.permanently_violated(kind, op, c, list(v))
            if ps != all_sat:
                bad.append(("perm-sat", kind, op, c, v, ps, all_sat))
            if pv != none_sat:
                bad.append(("perm-viol", kind, op, c, v, pv, none_sat))
    return bad


def test_enumeration_covers_every_verdict(brute):
    seen = {}
    for (kind, op, c, v), (b, _, _) in brute.items():
        seen.setdefault((kind, op), set()).add(b)
    # every comparison reaches at least four of the six values somewhere
    assert all(len(s) >= 4 for s in seen.values()), seen
    assert len(brute) == len(_vectors(MAX_N)) * len(_KC) * len(OPS)


def test_oracle_valuation_matches_enumeration(brute):
    bad = _mismatches(brute)
    assert not bad, bad[:10]


def test_table1_is_what_the_enumeration_gives(brute):
    # Table 1 as printed (E quantifiers): '>' and '>=' become permanently
    # satisfied once the definite count satisfies them; '=', '<' and '<=' are
    # permanently violated once it exceeds what they allow
    for (kind, op, c, v), (_, all_sat, none_sat) in brute.items():
        if kind != "E":
            continue
        l, t = int(c), v[T]
        if op == ">":
            assert all_sat == (t > l)
        elif op == ">=":
            assert all_sat == (t >= l)
        elif op == "=":
            assert none_sat == (t > l) and not all_sat
        elif op == "<":
            assert none_sat == (t >= l) and not all_sat
        elif op == "<=":
            assert none_sat == (t > l) and not all_sat


def test_A_eq_1_rule_is_what_the_enumeration_gives(brute):
    # Sec. 2.4.5: under A (= A_{=1}) one violated child violates the node for good
    for (kind, op, c, v), (b, _, none_sat) in brute.items():
        if kind == "A" and op == "=" and c == 1:
            assert none_sat == (v[F] >= 1)
            if v[F] >= 1:
                assert b == F


def _strict_gt_without_witness(kind, op, const, v):
    # planted: A_{>0} counted permanently satisfied without any true child
    if kind == "A" and op == ">" and const == 0:
        return True
    return _orig_ps(kind, op, const, v)


_orig_ps = counting.permanently_satisfied


def _A_ge_one_without_false_child(kind, op, const, v):
    # planted: A_{>=1} counted permanently violated before any child is false
    if kind == "A" and op == ">=" and const == 1:
        return True
    return _orig_pv(kind, op, const, v)


_orig_pv = counting.permanently_violated


def _mirrored_fp_without_tc(kind, op, const, v):
    # planted: the <= ladder's Fp rung leaves out the Tc children
    b = _orig_ladder(kind, op, const, v)
    if op in ("<=", "<") and b in (FC, F) and counting.constraint(kind, op, const, v[T], sum(v)):
        return FP
    return b


_orig_ladder = counting._ladder


@pytest.mark.parametrize("attr,fake", [
    ("permanently_satisfied", _strict_gt_without_witness),
    ("permanently_violated", _A_ge_one_without_false_child),
    ("_ladder", _mirrored_fp_without_tc),
])
def test_enumeration_catches_planted_mistakes(monkeypatch, brute, attr, fake):
    monkeypatch.setattr(counting, attr, fake)
    assert _mismatches(brute)
