"""GPU parity of the per-event timeline (rv_verify_timeline) with the oracle:
every event's verdict and every binding's first violation, on reduced
socket-shaped (one variable) and file-shaped (two variables) traces, a
binding long enough to span many scan tiles, and edge cases."""
import numpy as np
import pytest

from oracle.timeline import timeline as oracle_timeline
from oracle.verify import Schema
from paper_1411_2239_b300 import synth

pytestmark = pytest.mark.gpu

C1 = "A_{>=0.95} s: socket(s) => G(receive -> F respond)"
C3 = "A_{>=0.90} u: user(u) => E_{<=3} f: file(u,f) => open && !F close"


def _dev(torch, a):
    a = np.ascontiguousarray(a)
    view = {8: np.int64, 4: np.int32, 1: np.uint8}[a.dtype.itemsize]
    return torch.from_numpy(a.view(view)).cuda()


def _check(rv, text, codes, key, pred, key_bits=32, nq=1):
    import torch
    f = rv.Formula(text, codes, key_bits=key_bits)
    v, first = rv.timeline(f, _dev(torch, key), _dev(torch, pred))
    ov, ofirst = oracle_timeline(text, Schema(codes), key, pred)
    assert (v == ov).all(), int(np.flatnonzero(v != ov)[0])
    if nq == 2:
        want = {(D[0] << 32) | D[1]: j for D, j in ofirst.items()}
    elif nq == 1:
        want = {D[0]: j for D, j in ofirst.items()}
    else:
        want = {0: j for D, j in ofirst.items()}
    assert first == want
    return v


def test_socket_trace_uniform(rv):
    tr = synth.socket_trace(100_000, 1_000, n_pending=50, seed=91)
    v = _check(rv, C1, tr.codes, tr.key, tr.pred)
    assert set(np.unique(v).tolist()) <= {2, 3}


def test_socket_trace_zipf_with_violations(rv):
    # a safety body: bindings that see two receives in a row are violated for good
    tr = synth.socket_trace(60_000, 3_000, pending_frac=0.05, zipf_s=1.1, seed=92)
    v = _check(rv, "A s: socket(s) => G(receive -> X !receive)", tr.codes, tr.key, tr.pred)
    assert (v == 0).any()


def test_file_trace_two_variables(rv):
    tr = synth.file_trace(80_000, 100, 2_000, seed=93)
    _check(rv, C3, tr.codes, tr.key, tr.pred, key_bits=64, nq=2)


def test_one_binding_over_many_tiles(rv):
    # 11,000 events of one key: its segment crosses three scan tiles of 4096
    # events, so every state after the first tile comes from a carried map
    rng = np.random.default_rng(94)
    n = 12_000
    key = np.full(n, 12345, dtype=np.uint32)
    key[rng.random(n) < 0.08] = 777
    pred = rng.choice(np.array([0, 1, 2], dtype=np.uint8), size=n, p=[0.5, 0.05, 0.45])
    _check(rv, C1, synth.SOCKET_CODES, key, pred)
    _check(rv, "A s: socket(s) => G(receive -> X !receive)", synth.SOCKET_CODES, key, pred)


def test_unquantified_and_tiny_traces(rv):
    rng = np.random.default_rng(95)
    for n in (1, 2, 31, 4097):
        pred = rng.integers(0, 3, size=n).astype(np.uint8)
        key = rng.integers(0, 3, size=n).astype(np.uint32)
        _check(rv, "G(receive -> X !receive)", synth.SOCKET_CODES, key, pred, nq=0)
        _check(rv, C1, synth.SOCKET_CODES, key, pred)
