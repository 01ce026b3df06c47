"""Pins of the oracle's per-event timeline (no GPU): every event's verdict is
the whole-trace verdict of its binding on the trace cut after that event
(computed by oracle.verify, itself pinned), the last event of a binding
carries the binding's verdict, and T and F never change once reached."""
import numpy as np
import pytest

from oracle import timeline as tl
from oracle.verify import Schema, verify

SCH = Schema(["a", "b", "c"])
CASES = [("A x: p(x) => G(a -> F b)", 1), ("E_{<=2} x: p(x) => F c", 1), ("A x: p(x) => a U b", 1),
         ("A_{>=0.5} x: p(x) => E y: q(x,y) => G !c", 2), ("G(a -> X b)", 0)]


def _trace(rng, n, nq):
    if nq == 2:
        keys = (rng.integers(0, 3, size=n).astype(np.uint64) << np.uint64(32)) | \
            rng.integers(0, 4, size=n).astype(np.uint64)
    else:
        keys = rng.integers(0, 6, size=n).astype(np.uint64)
    return keys, rng.integers(0, 3, size=n)


def _check(text, nq, keys, preds, timeline=tl.timeline):
    v, first = timeline(text, SCH, keys, preds)
    for j in range(len(preds)):
        r = verify(text, SCH, keys[:j + 1], preds[:j + 1])
        if nq == 0:
            want = r.root
        else:
            D = tuple(int(x) for x in ((int(keys[j]) >> 32, int(keys[j]) & 0xFFFFFFFF) if nq == 2 else (int(keys[j]),)))
            want = r.verdicts[nq - 1][D]
        assert v[j] == want, (text, j)
    return v, first


@pytest.mark.parametrize("text,nq", CASES)
def test_each_event_is_the_verdict_of_the_cut_trace(text, nq):
    rng = np.random.default_rng(81)
    for _ in range(4):
        keys, preds = _trace(rng, int(rng.integers(1, 60)), nq)
        v, first = _check(text, nq, keys, preds)
        # first violations: the earliest F event of each binding, and F stays F
        seen = {}
        for j in range(len(preds)):
            D = () if nq == 0 else ((int(keys[j]) >> 32, int(keys[j]) & 0xFFFFFFFF) if nq == 2 else (int(keys[j]),))
            if v[j] == 0:
                seen.setdefault(D, j)
            if D in seen:
                assert v[j] == 0
        assert first == seen


def test_last_event_carries_the_binding_verdict():
    rng = np.random.default_rng(82)
    text = "A x: p(x) => G(a -> F b)"
    keys, preds = _trace(rng, 400, 1)
    v, _ = tl.timeline(text, SCH, keys, preds)
    r = verify(text, SCH, keys, preds)
    for D, b in r.verdicts[0].items():
        last = np.flatnonzero(keys == D[0])[-1]
        assert v[last] == b


def _off_by_one(text, schema, keys, preds):
    # planted: each event gets the verdict of the prefix before it
    v, first = tl.timeline(text, schema, keys, preds)
    out = v.copy()
    nq = text.count(":")
    last = {}
    for j in range(len(preds)):
        D = int(keys[j]) if nq else 0
        if D in last:
            out[j] = v[last[D]]
        last[D] = j
    return out, first


def test_planted_off_by_one_is_caught():
    rng = np.random.default_rng(83)
    keys, preds = _trace(rng, 40, 1)
    with pytest.raises(AssertionError):
        _check("A x: p(x) => a U b", 1, keys, preds, timeline=_off_by_one)
