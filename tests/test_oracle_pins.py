"""Pins of the CPU oracle to the paper and to the mathematics (no GPU).

Each test ties one part of the oracle to something other than the oracle: a
value the paper prints, a closed form, an independent brute force, or an
invariant of the semantics.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import counting, fltl
from oracle.counting import F, FC, FP, T, TC, TP
from oracle.formula import ParseError, Quantifier, parse
from oracle.ltl4 import LTL4
from oracle.verify import Checker, Schema, letter_sets, verify
from tests.bruteforce import all_verdicts

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NAME = {"F": F, "Fc": FC, "Fp": FP, "Tp": TP, "Tc": TC, "T": T}
PROPS3 = ["a", "b", "c"]
SETS3 = [frozenset(p for i, p in enumerate(PROPS3) if (m >> i) & 1) for m in range(8)]


# ------------------------------------------------------------------ syntax
def test_default_constraints():
    # Sec. 2.1: bare A means A_{=1}, bare E means E_{>=1}
    q = parse("A x: p(x) => a").quants[0]
    assert (q.kind, q.op, q.const) == ("A", "=", 1)
    q = parse("E x: p(x) => a").quants[0]
    assert (q.kind, q.op, q.const) == ("E", ">=", 1)


def test_constants_exact():
    assert parse("A_{>=0.95} s: socket(s) => a").quants[0].const == Fraction(19, 20)
    assert parse("A_{>= 50%} f: intrace(f) => a").quants[0].const == Fraction(1, 2)
    assert parse("E_{=0} r: req(r) => a").quants[0].const == 0
    with pytest.raises(ParseError):
        parse("A_{>=1.5} x: p(x) => a")
    with pytest.raises(ParseError):
        parse("E_{<=2.5} x: p(x) => a")


@pytest.mark.parametrize("text", [
    # introduction and Eq. prop (Sec. 4.1), with the binder => made explicit
    "A_{>=0.95} s: socket(s) => G(receive(s) -> F respond(s))",
    "A x: user(x) => (E_{<=3} r: rid(r) => (login && unauthorized))",
    # Eq. 1 and Eq. 2 (Sec. 2.3)
    "A_{>=50%} f: intrace(f) => (opened(f) U close(f))",
    "A_{>=50%} f: intrace(f) => G(opened(f) U close(f))",
    # case studies 2 and 3 (Sec. 5.1)
    "A u: user(u) => F chunk_ok(u)",
    "A v: vid(v) => E_{=0} r: req(r) => (cached(v) && external(r))",
    # Fig. 1
    "G a || (b U c)",
])
def test_paper_formulas_parse(text):
    f = parse(text)
    assert f.body[0] in ("not", "or", "and", "U", "X", "ap")


def test_precedence():
    # the binder => binds loosest; U binds tighter than &&; -> is right assoc.
    f = parse("A x: p(x) => a && b U c -> d")
    assert f.body == parse("(a && (b U c)) -> d").body
    assert parse("a -> b -> c").body == parse("a -> (b -> c)").body


# ------------------------------------------------------------------ FLTL closed forms
def _word(rng, n, p=0.5):
    return rng.integers(0, 8, size=n)


def test_fltl_closed_forms():
    rng = np.random.default_rng(1)
    truth = {nm: np.array([nm in s for s in SETS3]) for nm in PROPS3}
    F_a, G_a, X_a, nX_a = (parse(t).body for t in ("F a", "G a", "X a", "!X a"))
    for _ in range(300):
        n = int(rng.integers(1, 12))
        w = _word(rng, n)
        has = truth["a"][w]
        assert fltl.holds(F_a, w, truth) == bool(has.any())
        assert fltl.holds(G_a, w, truth) == bool(has.all())
        # strong next: X a is false on a one-letter trace, !X a is true
        assert fltl.holds(X_a, w, truth) == (n > 1 and bool(has[1]))
        assert fltl.holds(nX_a, w, truth) == (n == 1 or not bool(has[1]))
        # X^n a needs n+1 letters (Def. FLTL: u_1 must be non-empty)
        xs = parse("X " * n + "true").body
        assert fltl.holds(xs, w, truth) is False


# ------------------------------------------------------------------ LTL4 pins
def test_ltl4_against_lasso_bruteforce_len6():
    # all 299,592 traces of length <= 6 over 3 propositions (bitmask letters)
    for text in ["G a || (b U c)", "G(a -> F b)", "X(a U !b) && F c"]:
        f = parse(text)
        bf, stable = all_verdicts(f.body, SETS3, 6)
        assert stable
        m = LTL4(f.body, SETS3)
        bad = [w for w, v in bf.items() if m.verdict(np.array(w)) != v]
        assert not bad, (text, bad[:5])


RANDOM_BODIES = [
    "a U (X b R c)", "(a U b) U (X c)", "!X a", "X X a", "F G a", "G F a", "a W b",
    "G(a -> X b)", "F(a && X !a)", "(a -> F c) U b", "X(a <-> b) || G c",
    "!(a U b) && F(b && c)", "G(a U b)", "a R (b || X c)",
]


@pytest.mark.parametrize("text", RANDOM_BODIES)
def test_ltl4_against_lasso_bruteforce_len4(text):
    f = parse(text)
    bf, stable = all_verdicts(f.body, SETS3, 4)
    assert stable
    m = LTL4(f.body, SETS3)
    bad = [w for w, v in bf.items() if m.verdict(np.array(w)) != v]
    assert not bad, bad[:5]


def test_ltl4_fig1_monitor_shape():
    # Fig. 1: the monitor of G a || (b U c) has traps T and F; a-runs are Tp,
    # b-runs are Fp.  Letters over {a, b, c}.
    f = parse("G a || (b U c)")
    m = LTL4(f.body, SETS3)
    A, B, C, N = 1, 2, 4, 0
    assert m.verdict([A, A, A]) == TP
    assert m.verdict([B, B]) == FP
    assert m.verdict([B, C]) == T and m.verdict([B, C, N, N]) == T
    assert m.verdict([N]) == F and m.verdict([N, A, B, C]) == F
    assert m.verdict([A | B, A]) == TP         # both disjuncts alive
    assert m.verdict([A | B, B]) == FP         # G a died, b U c pending


def test_response_property_is_never_definite():
    # G(receive -> F respond) over one-hot letters {socket, receive, respond}:
    # no finite trace decides it permanently (Def. LTL4).
    f = parse("G(receive -> F respond)")
    sets = letter_sets(Schema(["socket", "receive", "respond"]), f.aps())
    m = LTL4(f.body, sets)
    for n in range(1, 7):
        for w in itertools.product(range(3), repeat=n):
            v = m.verdict(np.array(w))
            assert v in (TP, FP)
            pending = [x for x in w if x in (1, 2)]
            assert (v == FP) == (bool(pending) and pending[-1] == 1)


# ------------------------------------------------------------------ projection (Sec. 2.4.3)
def test_projection_example():
    g = json.load(open(os.path.join(GOLDEN, "projection_example.json")))
    keys = np.array([(x << 32) | y for x, y in g["values"]], dtype=np.uint64)
    ch = Checker("A x: px(x) => A y: py(y) => G q", Schema(["q", "r"]))
    assert list(ch.projection(keys, (1, 2))) == g["expect"]["u^<1,2>"]
    assert list(ch.projection(keys, (1, 3))) == g["expect"]["u^<1,3>"]
    res = ch.run(keys, np.zeros(3, dtype=np.int64))
    children = sorted(D for D in res.verdicts[1] if D[:1] == (1,))
    assert [list(D) for D in children] == g["expect"]["P(<1>)"]
    assert res.n_nodes == [1, 2]


# ------------------------------------------------------------------ worked example
def test_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "worked_example.json")))
    codes = g["codes"]
    keys = np.array([(g["users"][e["user"]] << 32) | e["rid"] for e in g["events"]], dtype=np.uint64)
    preds = np.array([sum(1 << codes.index(p) for p in e["preds"]) for e in g["events"]])
    res = verify(g["formula"], Schema(codes, "bitmask"), keys, preds)
    ex = g["expect"]
    assert res.n_nodes == [ex["children_of_root"], ex["distinct_value_vectors"]]
    adam = g["users"]["Adam"]
    adam_children = [v for D, v in res.verdicts[1].items() if D[0] == adam]
    assert adam_children.count(T) == ex["adam_children_true"]
    assert res.verdicts[0][(adam,)] == NAME[ex["adam"]]
    assert res.root == NAME[ex["root"]]


# ------------------------------------------------------------------ Table 1 and the A_{=1} rule
def _counts(rng):
    return [int(x) for x in rng.integers(0, 4, size=6)]


def test_table1_exhaustive():
    # Table 1: E_{>c}/E_{>=c} permanently satisfied once v[T] >c / >=c;
    # E_{=c}/E_{<=c} permanently violated once v[T] > c, E_{<c} once v[T] >= c.
    rule = {">": (T, lambda t, c: t > c), ">=": (T, lambda t, c: t >= c),
            "=": (F, lambda t, c: t > c), "<=": (F, lambda t, c: t > c),
            "<": (F, lambda t, c: t >= c)}
    for op, (perm, fires) in rule.items():
        for c in range(0, 5):
            q = Quantifier("E", op, Fraction(c), "x", "p")
            for v in itertools.product(range(3), repeat=6):
                if sum(v) > 8:
                    continue
                b = counting.valuate(q, list(v))
                assert (b == perm) == fires(v[T], c), (op, c, v, b)


def test_A_eq_1_single_violation():
    # Sec. 2.4.5: under A_{=1} one F child makes the property F for good
    q = parse("A x: p(x) => a").quants[0]
    for v in itertools.product(range(3), repeat=6):
        b = counting.valuate(q, list(v))
        assert (b == F) == (v[F] >= 1)


def test_case_study1_threshold():
    # A_{>=0.95}: children are Tp (served) or Fp (pending receive); exactly 95%
    # served is still Tp, one socket fewer is Fp.
    q = parse("A_{>=0.95} s: socket(s) => a").quants[0]
    assert counting.valuate(q, [0, 0, 50, 950, 0, 0]) == TP
    assert counting.valuate(q, [0, 0, 51, 949, 0, 0]) == FP
    assert counting.valuate(q, [0, 0, 0, 1, 0, 0]) == TP


def test_phi2_never_currently_true():
    # Sec. 2.3: phi_2 = A_{>=50%} f: intrace(f) => G(opened U close) can never be Tc
    rng = np.random.default_rng(7)
    sch = Schema(["opened", "close", "other"])
    for _ in range(40):
        n = int(rng.integers(1, 60))
        keys = rng.integers(0, 6, size=n).astype(np.uint32)
        preds = rng.integers(0, 3, size=n)
        r = verify("A_{>=50%} f: intrace(f) => G(opened U close)", sch, keys, preds)
        assert r.root != TC
        assert r.root_counts[T] == 0


def test_empty_root():
    sch = Schema(["a", "b"])
    e = np.zeros(0, dtype=np.uint32)
    assert verify("A_{>=0.5} x: p(x) => a", sch, e, e).root == TC   # 0 >= 0
    assert verify("A_{>0.5} x: p(x) => a", sch, e, e).root == FC    # 0 > 0 fails
    assert verify("E x: p(x) => a", sch, e, e).root == FC
