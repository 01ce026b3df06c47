"""Host-side checks of librv (no GPU work): the C ABI, the monitor compiler and
the exact-integer valuation, each against the CPU oracle."""
import itertools
import re
from fractions import Fraction
import os

import numpy as np
import pytest

from oracle import counting
from oracle.formula import Quantifier, parse
from oracle.ltl4 import LTL4
from oracle.verify import Schema, letter_sets
from paper_1411_2239_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol(rv):
    header = open(os.path.join(ROOT, "include", "rv.h")).read()
    header = re.sub(r"/\*.*?\*/", "", header, flags=re.S)
    names = set(re.findall(r"\b(rv_[a-z0-9_]+)\s*\(", header))
    assert "rv_verify_trace" in names and "rv_compile_formula" in names
    L = rv.lib()
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_parse_errors(rv):
    with pytest.raises(rv.RVError) as e:
        rv.Formula("A x: p(x) => G(", ["a"])
    assert e.value.status == rv.RV_EPARSE
    with pytest.raises(rv.RVError) as e:
        rv.Formula("A x: p(x) => G nope", ["a"])
    assert e.value.status == rv.RV_EPARSE
    with pytest.raises(rv.RVError) as e:
        rv.Formula("A x: p(x) => E y: q(y) => a", ["a"], key_bits=32)
    assert e.value.status == rv.RV_EINVAL
    with pytest.raises(rv.RVError) as e:
        rv.Formula("A_{>=1.5} x: p(x) => a", ["a"])
    assert e.value.status == rv.RV_EPARSE


def test_quantifier_constants_match_oracle(rv):
    for text in ["A_{>=0.95} s: socket(s) => a", "A_{<50%} s: p(s) => a", "E_{=0} r: q(r) => a",
                 "A x: p(x) => a", "E x: p(x) => a", "A_{>0.125} x: p(x) => a"]:
        f = rv.Formula(text, ["a"])
        oq = parse(text).quants[0]
        q = f.quantifier(0)
        assert q.kind == (rv.Q_A if oq.kind == "A" else rv.Q_E)
        assert q.op == rv.OPS[oq.op]
        assert Fraction(q.num, q.den) == oq.const


def _simulate(maps, labels, word, q0=0):
    q = q0
    for l in word:
        q = (maps[l] >> (4 * q)) & 15
    return labels[q]


BODIES = ["G a || (b U c)", "G(a -> F b)", "X(a U !b) && F c", "a U (X b R c)", "F G a", "G F a",
          "!X a", "X X a", "(a U b) U (X c)", "G(a U b)", "a W b", "G(a -> X b)", "(a -> F c) U b",
          "X(a <-> b) || G c", "!(a U b) && F(b && c)", "a R (b || X c)", "true", "false", "a"]


@pytest.mark.parametrize("body", BODIES)
def test_monitor_matches_oracle_on_all_short_words(rv, body):
    props = ["a", "b", "c"]
    f = rv.Formula(body, props, alphabet="bitmask")
    maps, labels = f.tables()
    assert 1 <= f.n_states <= 16
    sets = [frozenset(p for i, p in enumerate(props) if (m >> i) & 1) for m in range(8)]
    m = LTL4(parse(body).body, sets)
    for n in range(1, 5):
        for w in itertools.product(range(8), repeat=n):
            assert _simulate(maps, labels, w, f.q0) == m.verdict(np.array(w)), (body, w)


def test_monitor_onehot_random_bodies(rv):
    rng = np.random.default_rng(5)
    codes = ["p0", "p1", "p2", "p3", "p4"]
    done = 0
    while done < 25:
        body = synth.random_body(rng, codes[:3], depth=int(rng.integers(1, 4)))
        try:
            f = rv.Formula(body, codes)
        except rv.RVError as e:
            assert e.status == rv.RV_EUNSUPPORTED
            continue
        maps, labels = f.tables()
        m = LTL4(parse(body).body, letter_sets(Schema(codes), parse(body).aps()))
        for _ in range(300):
            w = rng.integers(0, 5, size=int(rng.integers(1, 25)))
            assert _simulate(maps, labels, w, f.q0) == m.verdict(w), (body, w)
        done += 1


def test_case_study_monitors(rv):
    f = rv.Formula("A_{>=0.95} s: socket(s) => G(receive -> F respond)", synth.SOCKET_CODES)
    assert f.n_quant == 1 and f.n_states <= 3
    f = rv.Formula("A_{>=0.90} u: user(u) => E_{<=3} f: file(u,f) => open && !F close", synth.FILE_CODES,
                   key_bits=64)
    assert f.n_quant == 2 and f.n_states <= 3
    # Fig. 1: G a || (b U c) -- five reachable verdict states after the initial one
    f = rv.Formula("G a || (b U c)", ["a", "b", "c"], alphabet="bitmask")
    assert f.n_states == 6


def test_valuation_matches_oracle_exhaustively(rv):
    consts_A = [Fraction(0), Fraction(1, 4), Fraction(1, 2), Fraction(19, 20), Fraction(1)]
    consts_E = [Fraction(0), Fraction(1), Fraction(2), Fraction(3)]
    vecs = [v for v in itertools.product(range(3), repeat=6)]
    for kind, consts in (("A", consts_A), ("E", consts_E)):
        for op in ["<", "<=", ">", ">=", "="]:
            for c in consts:
                q = Quantifier(kind, op, c, "x", "p")
                for v in vecs:
                    want = counting.valuate(q, list(v))
                    got = rv.valuate(rv.Q_A if kind == "A" else rv.Q_E, rv.OPS[op], c.numerator, c.denominator, v)
                    assert got == want, (kind, op, c, v)


def test_valuation_large_counts_exact(rv):
    # 128-bit cross-multiplication: counts near 2^40 with a 15-digit constant
    num, den = 999999999999999, 10**15
    N = 1 << 40
    for tp in [N - 1, N - 2, N // 2]:
        v = [0, 0, N - tp, tp, 0, 0]
        q = Quantifier("A", ">=", Fraction(num, den), "x", "p")
        assert rv.valuate(rv.Q_A, rv.OPS[">="], num, den, v) == counting.valuate(q, v)


def _header_structs():
    """Field names, in order, of every `typedef struct { ... } name;` in rv.h."""
    import re
    text = open(os.path.join(os.path.dirname(__file__), "..", "include", "rv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            first, *rest = decl.split(",")          # `uint64_t a, b, c;` declares three fields
            for d in [first] + rest:
                fields.append(re.findall(r"(\w+)\s*(?:\[[^\]]*\])*\s*$", d.strip())[0])
        out[name] = fields
    return out


def test_binding_structs_mirror_the_header():
    # the ctypes mirrors of the C structs keep the header's fields and order
    from paper_1411_2239_b300 import rv
    hs = _header_structs()
    pairs = {"rv_schema": rv._Schema, "rv_formula_info": rv._Info, "rv_trace": rv._Trace, "rv_result": rv._Result,
             "rv_bindings": rv._Bindings, "rv_verify_opts": rv._Opts, "rv_batch_opts": rv._BatchOpts,
             "rv_service_cfg": rv._SvcCfg, "rv_stream_verdict": rv._Verdict, "rv_service_counters": rv._SvcCounters}
    for cname, cls in pairs.items():
        assert cname in hs, cname
        assert [f[0] for f in cls._fields_] == hs[cname], (cname, hs[cname])


def test_noalloc_scratch_covers_a_million_events_in_every_key_format(rv):
    # the no-allocation entry point's fixed scratch array is 64 MiB and it
    # accepts traces of up to 1,000,000 events: the workspace of such a trace
    # must fit for one 32-bit key, one 64-bit key and two variables
    cases = [("A_{>=0.95} s: socket(s) => G(receive -> F respond)", synth.SOCKET_CODES, 32),
             ("A_{>=0.95} s: socket(s) => G(receive -> F respond)", synth.SOCKET_CODES, 64),
             ("A_{>=0.90} u: user(u) => E_{<=3} f: file(u,f) => open && !F close", synth.FILE_CODES, 64)]
    for text, codes, bits in cases:
        f = rv.Formula(text, codes, key_bits=bits)
        assert rv.workspace_size(f, 1_000_000) <= 64 << 20, (text, bits)


def test_batch_arguments_are_checked_before_any_device_work(rv):
    # rv_batch_create validates its formulas and offsets on the host and
    # returns an error before it allocates or copies anything
    import numpy as np
    c2, c3 = ["p0", "p1"], ["p0", "p1", "p2"]
    f2 = rv.Formula("A x: p(x) => G p0", c2)
    f3 = rv.Formula("A x: p(x) => G p0", c3)
    nested = rv.Formula("A_{>=0.90} u: user(u) => E_{<=3} f: file(u,f) => open && !F close",
                        ["user", "file", "open", "close"], key_bits=64)
    off = np.array([0, 10, 20], dtype=np.uint64)
    cases = [([[f2, f3], [f2, f2]], off, rv.RV_EINVAL),                              # alphabets differ in a trace
             ([[nested], [nested]], off, rv.RV_EUNSUPPORTED),                        # two quantifiers
             ([[f2], [f2]], np.array([0, 20, 10], dtype=np.uint64), rv.RV_EINVAL),   # decreasing offsets
             ([[f2], [f2]], np.array([5, 10, 20], dtype=np.uint64), rv.RV_EINVAL),   # offsets[0] != 0
             ([[f2] * 33, [f2] * 33], off, rv.RV_EINVAL)]                            # more than 32 formulas
    for forms, o, want in cases:
        with pytest.raises(rv.RVError) as e:
            rv.Batch(forms, o)
        assert e.value.status == want, (e.value, want)
