"""GPU test of rv_verify_trace_noalloc, the entry point that allocates nothing.

It exists for callers that cannot allocate device memory while they verify
(work recorded during CUDA graph capture, hosts whose device memory belongs to
another allocator, loops that must not block on an allocation).  Its workspace
is one fixed array inside the library that every call shares, so this test
calls it several times in a row, on different traces, and checks each result
against the ordinary entry point rv_verify_trace_async.  Results are integers
(verdicts and counts), so they must be identical.  The file sorts last so a
stop-at-first-failure run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1411_2239_b300 import rv, synth

pytestmark = pytest.mark.gpu

C1 = "A_{>=0.95} s: socket(s) => G(receive -> F respond)"
C3 = "A_{>=0.90} u: user(u) => E_{<=3} f: file(u,f) => open && !F close"


def _lib():
    L = rv.lib()
    L.rv_verify_trace_noalloc.argtypes = [ctypes.c_void_p, ctypes.POINTER(rv._Trace), ctypes.c_void_p,
                                          ctypes.c_void_p]
    return L


def _dev(torch, a):
    a = np.ascontiguousarray(a)
    view = {8: np.int64, 4: np.int32, 1: np.uint8}[a.dtype.itemsize]
    return torch.from_numpy(a.view(view)).cuda()


def _noalloc(torch, f, key, pred):
    out = torch.zeros(rv.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    tr = rv._Trace(key.data_ptr(), pred.data_ptr(), None, int(pred.shape[0]))
    st = _lib().rv_verify_trace_noalloc(f.handle, ctypes.byref(tr), ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, rv.parse_result(bytes(out.cpu().numpy()))


def _reference(torch, f, key, pred):
    n = int(pred.shape[0])
    ws = torch.empty(rv.workspace_size(f, n), dtype=torch.uint8, device="cuda")
    out = torch.zeros(rv.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    rv.verify_async(f, key, pred, ws, out)
    torch.cuda.synchronize()
    return rv.parse_result(bytes(out.cpu().numpy()))


def _same(a, b):
    return (a.root, a.status, a.root_counts, a.level_counts, a.n_nodes, a.events) == \
           (b.root, b.status, b.root_counts, b.level_counts, b.n_nodes, b.events)


def test_noalloc_matches_workspace_entry_on_consecutive_calls():
    import torch
    t1 = synth.socket_trace(100_000, 1000, n_pending=50, seed=1)
    t2 = synth.socket_trace(900_000, 20_000, pending_frac=0.03, zipf_s=1.1, seed=2)
    t3 = synth.file_trace(500_000, 300, 10_000, seed=3)
    f1 = rv.Formula(C1, t1.codes)
    f3 = rv.Formula(C3, t3.codes, key_bits=64)
    cases = [(f1, t1), (f1, t2), (f3, t3), (f1, t1), (f3, t3)]   # repeated calls share the scratch array
    for f, t in cases:
        key, pred = _dev(torch, t.key), _dev(torch, t.pred)
        st, got = _noalloc(torch, f, key, pred)
        assert st == rv.RV_OK, rv.last_error()
        want = _reference(torch, f, key, pred)
        assert want.status == 0
        assert _same(got, want), (got, want)


def test_noalloc_two_variables_at_the_event_limit():
    # exactly 1,000,000 events of the nested workload's shape: the largest
    # trace the entry point accepts, in the key format with the largest plan
    import torch
    t = synth.file_trace(1_200_000, 2_000, 50_000, seed=4)
    assert len(t.pred) >= 1_000_000
    t.key, t.pred = t.key[:1_000_000], t.pred[:1_000_000]      # a prefix is a trace too
    f = rv.Formula(C3, t.codes, key_bits=64)
    key, pred = _dev(torch, t.key), _dev(torch, t.pred)
    for _ in range(2):
        st, got = _noalloc(torch, f, key, pred)
        assert st == rv.RV_OK, rv.last_error()
        want = _reference(torch, f, key, pred)
        assert want.status == 0 and _same(got, want), (got, want)


def _fmix32(x):
    """MurmurHash3's 32-bit finaliser (public domain): the library takes a
    two-variable key's bucket from the top bits of this mix of the outer value."""
    x = x.astype(np.uint64)
    x ^= x >> np.uint64(16)
    x = (x * np.uint64(0x85EBCA6B)) & np.uint64(0xFFFFFFFF)
    x ^= x >> np.uint64(13)
    x = (x * np.uint64(0xC2B2AE35)) & np.uint64(0xFFFFFFFF)
    x ^= x >> np.uint64(16)
    return x.astype(np.uint32)


def _users_sharing(top_bits, count, seed):
    rng = np.random.default_rng(seed)
    cand = np.unique(rng.integers(1, 2**32, size=20_000_000, dtype=np.uint64).astype(np.uint32))
    top = _fmix32(cand) >> np.uint32(32 - top_bits)
    vals, counts = np.unique(top, return_counts=True)
    users = cand[top == vals[np.argmax(counts)]][:count]
    assert len(users) == count
    return users


def _nested_trace(users, files_per_user, seed):
    # per (user, file): open, read, then close unless it is the user's last
    # file (one leaked file per user, so the inner E_{<=3} stays satisfied);
    # the pairs are interleaved at random times, each keeping its own order
    rng = np.random.default_rng(seed)
    keys, preds, times = [], [], []
    for u in users:
        for f in range(files_per_user):
            k = (int(u) << 32) | (f + 1)
            seq = [0, 2] + ([1] if f + 1 < files_per_user else [])
            keys += [k] * len(seq)
            preds += seq
            times += sorted(rng.random(len(seq)).tolist())
    order = np.argsort(np.array(times), kind="stable")
    return np.array(keys, dtype=np.uint64)[order], np.array(preds, dtype=np.uint8)[order]


def test_noalloc_many_outer_values_in_one_first_level_bucket():
    # 400 users whose hashes share the 8 bits of the first-level split: more
    # outer values than a fold unit counts (256) unless the second-level split
    # separates them, which the default plan for two variables does
    import torch
    from oracle.verify import Schema, verify
    users = _users_sharing(8, 400, seed=5)
    k, p = _nested_trace(users, 3, seed=6)
    f = rv.Formula(C3, synth.FILE_CODES, key_bits=64)
    key, pred = _dev(torch, k), _dev(torch, p)
    st, got = _noalloc(torch, f, key, pred)
    assert st == rv.RV_OK, rv.last_error()
    o = verify(C3, Schema(synth.FILE_CODES), k, p)
    assert got.status == rv.RV_OK
    assert (got.root, got.root_counts, got.level_counts) == (o.root, o.root_counts, o.level_counts)


def test_noalloc_reports_outer_values_crafted_to_collide():
    # 300 users whose hashes share all 16 bits of the finest split land in one
    # key bucket: the call is accepted and queued, and the device result says
    # RV_EAGAIN (more outer values than a fold unit counts), as documented
    import torch
    users = _users_sharing(16, 300, seed=7)
    k, p = _nested_trace(users, 2, seed=8)
    f = rv.Formula(C3, synth.FILE_CODES, key_bits=64)
    st, got = _noalloc(torch, f, _dev(torch, k), _dev(torch, p))
    assert st == rv.RV_OK, rv.last_error()
    assert got.status == rv.RV_EAGAIN


def test_noalloc_rejects_traces_over_the_limit():
    import torch
    f = rv.Formula(C1, synth.SOCKET_CODES)
    n = 1_000_001
    key = torch.zeros(n, dtype=torch.int32, device="cuda")
    pred = torch.zeros(n, dtype=torch.uint8, device="cuda")
    st, _ = _noalloc(torch, f, key, pred)
    assert st == rv.RV_EINVAL
    assert "1000000" in rv.last_error()
