"""Invariants of the six-valued semantics, checked on the oracle (no GPU),
and planted mistakes that the pins must catch."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import counting, fltl, ltl4
from oracle.counting import F, T
from oracle.verify import Schema, verify
from tests import test_oracle_pins as pins

SCH = Schema(["a", "b", "c", "d"])
BODIES = ["G(a -> F b)", "F c", "a U b", "G !d", "X a || c", "(a -> X b) W c"]
QUANTS = ["A_{>=0.5}", "A_{>0}", "A_{<=0.25}", "A_{<1}", "A", "A_{=0.5}",
          "E_{>=2}", "E_{>1}", "E_{<=1}", "E_{<2}", "E", "E_{=1}"]


def _formula(rng, nest):
    body = BODIES[rng.integers(len(BODIES))]
    q0 = QUANTS[rng.integers(len(QUANTS))]
    if nest:
        q1 = QUANTS[rng.integers(len(QUANTS))]
        return f"{q0} x: p(x) => {q1} y: q(x,y) => {body}", 2
    return f"{q0} x: p(x) => {body}", 1


def _trace(rng, n, nvars, nkeys=5):
    if nvars == 1:
        keys = rng.integers(0, nkeys, size=n).astype(np.uint64)
    else:
        keys = (rng.integers(0, 3, size=n).astype(np.uint64) << np.uint64(32)) | \
            rng.integers(0, nkeys, size=n).astype(np.uint64)
    return keys, rng.integers(0, 4, size=n)


def test_counts_sum_to_bindings():
    rng = np.random.default_rng(11)
    for _ in range(60):
        text, nv = _formula(rng, rng.integers(2))
        keys, preds = _trace(rng, int(rng.integers(1, 40)), nv)
        r = verify(text, SCH, keys, preds)
        assert sum(r.root_counts) == r.n_nodes[0]
        for m in range(nv):
            assert sum(r.level_counts[m]) == r.n_nodes[m] == len(r.verdicts[m])


def test_definite_verdicts_are_monotone():
    # T and F are permanent: every extension of the trace, including events of
    # new bindings, keeps them (Def. LTL4-C Semantics, first two cases)
    rng = np.random.default_rng(12)
    seen = {T: 0, F: 0}
    for _ in range(300):
        text, nv = _formula(rng, rng.integers(2))
        keys, preds = _trace(rng, int(rng.integers(1, 30)), nv)
        r0 = verify(text, SCH, keys, preds)
        if r0.root not in (T, F):
            continue
        seen[r0.root] += 1
        for _ in range(4):
            k2, p2 = _trace(rng, int(rng.integers(1, 30)), nv, nkeys=8)
            r1 = verify(text, SCH, np.concatenate([keys, k2]), np.concatenate([preds, p2]))
            assert r1.root == r0.root, (text, r0.root, r1.root)
            for m in range(nv):
                for D, b in r0.verdicts[m].items():
                    if b in (T, F):
                        assert r1.verdicts[m][D] == b
    assert seen[T] > 5 and seen[F] > 5


def test_equality_readings():
    # E_{=0} is E_{<=0} (case study 3); A_{=1} is A_{>=1} (Sec. 2.4.5)
    rng = np.random.default_rng(13)
    for _ in range(80):
        keys, preds = _trace(rng, int(rng.integers(1, 40)), 2)
        for a, b in [("E_{=0}", "E_{<=0}"), ("A_{=1}", "A_{>=1}"), ("A", "A_{>=1}")]:
            body = BODIES[rng.integers(len(BODIES))]
            fa = f"A_{{>=0.5}} x: p(x) => {a} y: q(y) => {body}"
            fb = f"A_{{>=0.5}} x: p(x) => {b} y: q(y) => {body}"
            ra, rb = verify(fa, SCH, keys, preds), verify(fb, SCH, keys, preds)
            assert ra.root == rb.root and ra.verdicts == rb.verdicts


def _count_vectors(max_n):
    """Every vector of six child-verdict counts with 1 <= N <= max_n."""
    def rec(i, left):
        if i == 5:
            yield (left,)
            return
        for k in range(left + 1):
            for rest in rec(i + 1, left - k):
                yield (k,) + rest
    for N in range(1, max_n + 1):
        yield from rec(0, N)


def _check_ladder_monotone():
    # B6 is a chain (F < Fc < Fp < Tp < Tc < T, Sec. 2.4.4): moving one child
    # up the chain, with the number of children fixed, makes more of them count
    # as true at every level of certainty, so it can never lower the verdict of
    # a '>=' or '>' node nor raise that of a '<=' or '<' node
    consts = {"E": [Fraction(k) for k in range(4)],
              "A": [Fraction(0), Fraction(1, 4), Fraction(1, 3), Fraction(1, 2), Fraction(2, 3), Fraction(1)]}
    moves = 0
    for kind in ("E", "A"):
        for op in (">=", ">", "<=", "<"):
            for c in consts[kind]:
                q = counting_quant(kind, op, c)
                for v in _count_vectors(4):
                    b0 = counting.valuate(q, list(v))
                    for i in range(6):
                        if not v[i]:
                            continue
                        for j in range(i + 1, 6):
                            w = list(v)
                            w[i] -= 1
                            w[j] += 1
                            b1 = counting.valuate(q, w)
                            moves += 1
                            if op in (">=", ">"):
                                assert b1 >= b0, (kind, op, c, v, i, j, b0, b1)
                            else:
                                assert b1 <= b0, (kind, op, c, v, i, j, b0, b1)
    assert moves > 10000


def counting_quant(kind, op, const):
    from oracle.formula import Quantifier
    return Quantifier(kind, op, const, "x", "p")


def test_ladder_monotone_in_child_verdicts():
    _check_ladder_monotone()


def _check_negation_duality():
    # a node whose constraint is negated (>= and <, > and <=) decides the
    # negated proposition, so its verdict is the dual one in B6 (T <-> F,
    # Tc <-> Fc, Tp <-> Fp; index b <-> 5 - b), as LTL4 is for negated formulas
    consts = {"E": [Fraction(k) for k in range(5)],
              "A": [Fraction(0), Fraction(1, 4), Fraction(1, 3), Fraction(1, 2), Fraction(2, 3), Fraction(1)]}
    n = 0
    for kind in ("E", "A"):
        for op, neg in ((">=", "<"), (">", "<=")):
            for c in consts[kind]:
                for v in _count_vectors(5):
                    b = counting.valuate(counting_quant(kind, op, c), list(v))
                    d = counting.valuate(counting_quant(kind, neg, c), list(v))
                    assert d == 5 - b, (kind, op, c, v, b, d)
                    n += 1
    assert n > 5000


def test_negated_constraint_gives_dual_verdict():
    _check_negation_duality()


def test_negated_outer_constraint_on_traces():
    # the same through the whole trace -> verdict function: negating the
    # outermost constraint gives the dual root verdict and changes nothing below
    rng = np.random.default_rng(14)
    neg = {">=": "<", "<": ">=", ">": "<=", "<=": ">"}
    outer = [("A", "0.5"), ("A", "0.25"), ("A", "1"), ("A", "0"), ("E", "2"), ("E", "0"), ("E", "1")]
    for _ in range(80):
        kind, c = outer[rng.integers(len(outer))]
        op = list(neg)[rng.integers(4)]
        body = BODIES[rng.integers(len(BODIES))]
        nested = bool(rng.integers(2))
        inner = f"{QUANTS[rng.integers(len(QUANTS))]} y: q(x,y) => " if nested else ""
        keys, preds = _trace(rng, int(rng.integers(1, 40)), 2 if nested else 1)
        fa = f"{kind}_{{{op}{c}}} x: p(x) => {inner}{body}"
        fb = f"{kind}_{{{neg[op]}{c}}} x: p(x) => {inner}{body}"
        ra, rb = verify(fa, SCH, keys, preds), verify(fb, SCH, keys, preds)
        assert rb.root == 5 - ra.root, (fa, ra.root, rb.root)
        assert ra.root_counts == rb.root_counts and ra.verdicts == rb.verdicts


# ------------------------------------------------------------------ planted mistakes
def _weak_next(f, letters, ap_truth, memo=None):
    if f[0] == "X":
        g = _orig_eval(f[1], letters, ap_truth, memo)
        r = np.ones(len(letters), dtype=bool)
        r[:-1] = g[1:]
        return r
    return _orig_eval(f, letters, ap_truth, memo)


_orig_eval = fltl.evaluate


def _swap_sign(kind, op, const, n, N):
    flip = {"<": ">", ">": "<", "<=": ">=", ">=": "<=", "=": "="}[op]
    return _orig_constraint(kind, flip, const, n, N)


_orig_constraint = counting.constraint


def _progress_drops_until_now(f, letter):
    # forgets that f U g can be fulfilled by the current letter
    if f[0] == "U":
        return ltl4.mk_and([_orig_progress(f[1], letter), f])
    return _orig_progress(f, letter)


_orig_progress = ltl4.progress


@pytest.mark.parametrize("target,attr,fake,checks", [
    (fltl, "evaluate", _weak_next, [pins.test_fltl_closed_forms]),
    (counting, "constraint", _swap_sign, [pins.test_table1_exhaustive, pins.test_case_study1_threshold]),
    (counting, "permanently_violated", lambda *a: False, [pins.test_worked_example]),
    (counting, "_equality", lambda kind, const, v: counting.FC if v[F] else counting.TC,
     [pins.test_A_eq_1_single_violation]),
    (ltl4, "progress", _progress_drops_until_now, [pins.test_ltl4_fig1_monitor_shape]),
])
def test_pins_catch_planted_mistakes(monkeypatch, target, attr, fake, checks):
    monkeypatch.setattr(target, attr, fake)
    for check in checks:
        with pytest.raises(AssertionError):
            check()


def test_ladder_mutation_caught_by_threshold_pin(monkeypatch):
    # dropping the Tp rung must break the case-study-1 threshold pin
    orig = counting._ladder

    def no_tp(kind, op, const, v):
        b = orig(kind, op, const, v)
        return counting.FP if b == counting.TP else b
    monkeypatch.setattr(counting, "_ladder", no_tp)
    with pytest.raises(AssertionError):
        pins.test_case_study1_threshold()
    assert Fraction(1) == 1


def test_ladder_wrong_index_caught_by_monotonicity(monkeypatch):
    # a '>=' ladder whose Tc rung sums the Fc children instead of the Tc ones
    # must break the monotonicity invariant
    orig = counting._ladder

    def wrong_index(kind, op, const, v):
        b = orig(kind, op, const, v)
        if op not in (">=", ">") or b == T:
            return b
        N = sum(v)
        if counting.constraint(kind, op, const, v[T] + v[counting.FC], N):
            return counting.TC
        if b == counting.TC:          # the rung the right sum satisfied, now missed
            return counting.TP
        return b
    monkeypatch.setattr(counting, "_ladder", wrong_index)
    with pytest.raises(AssertionError):
        _check_ladder_monotone()


def test_ladder_wrong_sum_caught_by_duality(monkeypatch):
    # a '<=' ladder whose Tc rung also leaves out the Fp children must break
    # the duality with '>'
    orig = counting._ladder

    def wrong_sum(kind, op, const, v):
        b = orig(kind, op, const, v)
        if op not in ("<=", "<") or b in (T, counting.TC):
            return b
        N = sum(v)
        if counting.constraint(kind, op, const, N - v[F] - v[counting.FC] - v[counting.FP], N):
            return counting.TC
        return b
    monkeypatch.setattr(counting, "_ladder", wrong_sum)
    with pytest.raises(AssertionError):
        _check_negation_duality()
