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


def test_full_size_trace_sampled_and_against_offline(rv):
    """The 1e8-event Zipf socket trace the bench times, in the bench's
    launch configuration.  Sampled bindings (their whole projections, and the
    first 400 events of the heaviest sampled binding) against the oracle: one
    binding's per-event verdicts and first violation depend only on its own
    events.  Every binding's verdict after its last event against the
    offline path's verdict of that binding (itself checked against the
    oracle), for all bindings."""
    import torch
    import bench
    w = dict(bench.WORKLOADS["c2"])
    tr = bench.make_trace(w, 1000 * w["cfg"])
    f = rv.Formula(w["formula"], tr.codes)
    key = _dev(torch, tr.key)
    pred = _dev(torch, tr.pred)
    v, first = rv.timeline(f, key, pred)
    n = tr.n
    assert len(v) == n

    rng = np.random.default_rng(96)
    cand = np.unique(tr.key[rng.integers(0, n, size=3000)])
    mask = np.isin(tr.key, cand)
    pos = np.flatnonzero(mask)
    kk = tr.key[pos]
    order = np.argsort(kk, kind="stable")
    kk, pos = kk[order], pos[order]
    starts = np.flatnonzero(np.r_[True, kk[1:] != kk[:-1]])
    ends = np.r_[starts[1:], len(kk)]
    sizes = ends - starts
    short = [i for i in range(len(starts)) if sizes[i] <= 400]
    picked = [short[i] for i in rng.choice(len(short), size=min(60, len(short)), replace=False)]
    heavy = int(np.argmax(sizes))
    checks = [(int(kk[starts[i]]), pos[starts[i]:ends[i]], True) for i in picked]
    checks.append((int(kk[starts[heavy]]), pos[starts[heavy]:starts[heavy] + 400], False))
    for k, idx, whole in checks:
        ov, ofirst = oracle_timeline(w["formula"], Schema(tr.codes), np.full(len(idx), k, dtype=np.uint32),
                                     tr.pred[idx])
        assert (v[idx] == ov).all(), (k, int(np.flatnonzero(v[idx] != ov)[0]))
        if whole:
            want = int(idx[ofirst[(k,)]]) if (k,) in ofirst else None
            assert first.get(k) == want, k
        elif (k,) in ofirst:
            assert first.get(k) == int(idx[ofirst[(k,)]]), k

    # every binding's last verdict equals its offline verdict
    kt = key.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    uniq, inv = torch.unique(kt, return_inverse=True)
    last = torch.full((uniq.numel(),), -1, dtype=torch.int64, device="cuda")
    last.scatter_reduce_(0, inv, torch.arange(n, device="cuda", dtype=torch.int64), reduce="amax")
    vd = torch.from_numpy(v).cuda()
    last_v = vd[last].cpu().numpy()
    off = rv.verify(f, key, pred, want_bindings=True)
    assert len(off.bindings) == uniq.numel()
    ok = uniq.cpu().numpy()
    got = np.array([off.bindings[int(x)] for x in ok], dtype=np.uint8)
    assert (got == last_v).all(), int(ok[np.flatnonzero(got != last_v)[0]])
    # F is permanent: a binding's first violation is its first F event, and its last verdict is F
    fk = np.fromiter(first.keys(), dtype=np.uint64, count=len(first))
    assert len(first) == int((last_v == 0).sum())
    assert all(v[j] == 0 for j in list(first.values())[:1000])
    assert set(fk.tolist()) == set(ok[last_v == 0].tolist())


def test_unaligned_input_arrays(rv):
    # the radix passes and the scan read 16-byte words where a tile's arrays
    # are aligned, one event at a time otherwise: a key and a predicate array
    # starting one element past a 16-byte boundary take the second way in
    # the first pass
    import torch
    tr = synth.socket_trace(70_000, 2_000, pending_frac=0.05, zipf_s=1.1, seed=97)
    key = torch.from_numpy(np.concatenate([[0], tr.key]).astype(np.uint32).view(np.int32)).cuda()[1:]
    pred = torch.from_numpy(np.concatenate([[0], tr.pred]).astype(np.uint8)).cuda()[1:]
    assert key.data_ptr() % 16 == 4 and pred.data_ptr() % 16 == 1
    for text in (C1, "A s: socket(s) => G(receive -> X !receive)"):
        f = rv.Formula(text, tr.codes)
        v, first = rv.timeline(f, key, pred)
        ov, ofirst = oracle_timeline(text, Schema(tr.codes), tr.key, tr.pred)
        assert (v == ov).all(), (text, int(np.flatnonzero(v != ov)[0]))
        assert first == {D[0]: j for D, j in ofirst.items()}, text
