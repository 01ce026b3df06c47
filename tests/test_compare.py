"""Interpreted comparison predicates (case study 2, Sec. 5.1: an atom such as
avg_chunksize(u) <= maximum compares a program variable carried by the event
with a constant), host side: oracle pins and the monitor compiler against the
oracle.  No GPU."""
import itertools

import numpy as np
import pytest

from oracle import verify as ov
from oracle.verify import Checker, Schema, verify
from paper_1411_2239_b300 import synth

SCH = Schema(["user", "upload"], value_name="avg")


def _trace(rng, n, nk=5):
    return (rng.integers(0, nk, size=n).astype(np.uint32), rng.integers(0, 2, size=n),
            rng.integers(0, 40, size=n).astype(np.uint32))


def test_closed_forms_per_binding():
    # F(avg <= 10): T once some event's value is <= 10 (permanent), else Fp;
    # G(avg < 30): F once some value is >= 30, else Tp
    rng = np.random.default_rng(101)
    for _ in range(20):
        keys, preds, vals = _trace(rng, int(rng.integers(1, 50)))
        rf = verify("A u: user(u) => F(avg <= 10)", SCH, keys, preds, vals)
        rg = verify("A u: user(u) => G(avg(u) < 30)", SCH, keys, preds, vals)
        for k in np.unique(keys):
            v = vals[keys == k]
            assert rf.verdicts[0][(int(k),)] == (5 if v.min() <= 10 else 2)
            assert rg.verdicts[0][(int(k),)] == (0 if v.max() >= 30 else 3)


def test_unrealisable_outcomes_are_not_letters():
    # no value is both <= 10 and >= 20: F(avg <= 10 && avg >= 20) can never hold,
    # so every binding is violated for good at its first event (LTL4's F
    # quantifies continuations over the letters the trace can produce)
    rng = np.random.default_rng(102)
    keys, preds, vals = _trace(rng, 30)
    r = verify("A u: user(u) => F(avg <= 10 && avg >= 20)", SCH, keys, preds, vals)
    assert set(r.verdicts[0].values()) == {0}
    # with the outcome allowed (a planted mistake) the verdict is only presumptive
    ck = Checker("A u: user(u) => F(avg <= 10 && avg >= 20)", SCH)
    assert (True, True) not in {o for (_, o) in ck.ext}


def test_equality_and_mixed_atoms():
    rng = np.random.default_rng(103)
    for _ in range(20):
        keys, preds, vals = _trace(rng, int(rng.integers(1, 40)))
        r = verify("A u: user(u) => G(upload -> avg = 7)", SCH, keys, preds, vals)
        for k in np.unique(keys):
            sel = keys == k
            bad = ((preds[sel] == 1) & (vals[sel] != 7)).any()
            assert r.verdicts[0][(int(k),)] == (0 if bad else 3)


def test_values_required():
    with pytest.raises(ValueError):
        verify("A u: user(u) => F(avg <= 10)", SCH, np.zeros(3, np.uint32), np.zeros(3, int))
    with pytest.raises(ValueError):
        verify("A u: user(u) => F(size <= 10)", SCH, np.zeros(3, np.uint32), np.zeros(3, int), np.zeros(3))


def _simulate(maps, labels, word, q0):
    q = q0
    for l in word:
        q = (maps[l] >> (4 * q)) & 15
    return labels[q]


@pytest.mark.parametrize("body", ["F(avg <= 10)", "G(upload -> avg > 20)", "(avg < 5) U (upload && avg >= 30)",
                                  "G(avg <= 10 -> X avg = 11)", "F(avg <= 10 && avg >= 20)"])
def test_monitor_with_comparisons_matches_oracle(rv, body):
    f = rv.Formula(f"A u: user(u) => {body}", SCH.code_names, value_name="avg")
    maps, labels = f.tables()
    ck = Checker(f"A u: user(u) => {body}", SCH)
    assert f.n_base == 2 and f.n_letters == 2 << f.n_cmp
    # a value from every region the constants cut out of [0, 2^32)
    values = [0, 4, 5, 6, 10, 11, 12, 19, 20, 21, 29, 30, 31, 2**32 - 1]
    for n in range(1, 4):
        for codes in itertools.product(range(2), repeat=n):
            for vals in itertools.product(values, repeat=n):
                gl = [c + f.n_base * _bits(f, body, v) for c, v in zip(codes, vals)]
                ol = ck.letters(np.array(codes), np.array(vals))
                assert _simulate(maps, labels, gl, f.q0) == ck.ltl4.verdict(ol), (body, codes, vals)


def _bits(f, body, v):
    # the library numbers comparison atoms in order of first appearance
    import re
    atoms = []
    for m in re.finditer(r"avg\s*(<=|>=|<|>|=)\s*(\d+)", body):
        a = (m.group(1), int(m.group(2)))
        if a not in atoms:
            atoms.append(a)
    fn = {"<": v.__lt__, "<=": v.__le__, ">": v.__gt__, ">=": v.__ge__, "=": v.__eq__}
    return sum(1 << j for j, (op, c) in enumerate(atoms) if fn[op](c))


def test_comparison_parse_errors(rv):
    with pytest.raises(rv.RVError) as e:
        rv.Formula("A u: user(u) => F(size <= 10)", SCH.code_names, value_name="avg")
    assert e.value.status == rv.RV_EPARSE
    with pytest.raises(rv.RVError) as e:
        rv.Formula("A u: user(u) => F(avg <= 1.5)", SCH.code_names, value_name="avg")
    assert e.value.status == rv.RV_EPARSE
    with pytest.raises(rv.RVError) as e:
        rv.Formula("A u: user(u) => F(avg <= 1 && avg <= 2 && avg <= 3 && avg <= 4 && avg <= 5)",
                   SCH.code_names, value_name="avg")
    assert e.value.status == rv.RV_EUNSUPPORTED
