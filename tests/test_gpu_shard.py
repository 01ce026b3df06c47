"""One trace over several ranks on one GPU: the device split (rv_shard_trace)
against its host form, then every part verified through the real path in
sequence and combined (rv_combine_results), against the unsharded result and
the oracle.  Each part is what one rank would verify after the exchange."""
import numpy as np
import pytest

from oracle.verify import Schema, verify as oracle_verify
from paper_1411_2239_b300 import synth

pytestmark = pytest.mark.gpu

C1 = "A_{>=0.95} s: socket(s) => G(receive -> F respond)"
C3 = "A_{>=0.90} u: user(u) => E_{<=3} f: file(u,f) => open && !F close"


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def _dev(torch, a):
    a = np.ascontiguousarray(a)
    view = {8: np.int64, 4: np.int32, 1: np.uint8}[a.dtype.itemsize]
    return torch.from_numpy(a.view(view)).cuda()


def _split_and_check(rv, torch, f, key_np, pred_np, world, ts_np=None):
    key, pred = _dev(torch, key_np), _dev(torch, pred_np)
    ts = None if ts_np is None else _dev(torch, ts_np)
    ko, po, to, counts = rv.shard_trace(f, key, pred, world, ts=ts)
    torch.cuda.synchronize()
    counts = counts.cpu().numpy().astype(np.int64)
    ranks = rv.shard_of(f, key_np, world)
    assert counts.tolist() == np.bincount(ranks, minlength=world).tolist()
    # segment r holds exactly the events of rank r, in trace order
    order = np.argsort(ranks, kind="stable")
    kview = np.uint64 if f.key_bits == 64 else np.uint32
    assert (ko.cpu().numpy().view(kview) == key_np[order]).all()
    assert (po.cpu().numpy() == pred_np[order]).all()
    if ts_np is not None:
        assert (to.cpu().numpy().view(np.uint32) == ts_np[order]).all()
    parts, start = [], 0
    for r in range(world):
        c = int(counts[r])
        parts.append(rv.verify(f, ko[start:start + c], po[start:start + c]))
        start += c
    return rv.combine_results(f, parts)


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_sharded_zipf_socket_trace_equals_unsharded(rv, torch_cuda, world):
    tr = synth.socket_trace(400_000, 20_000, pending_frac=0.03, zipf_s=1.1, seed=51)
    f = rv.Formula(C1, tr.codes)
    got = _split_and_check(rv, torch_cuda, f, tr.key, tr.pred, world, ts_np=tr.ts)
    whole = rv.verify(f, _dev(torch_cuda, tr.key), _dev(torch_cuda, tr.pred))
    o = oracle_verify(C1, Schema(tr.codes), tr.key, tr.pred)
    assert got.status == 0
    assert (got.root, got.root_counts, got.level_counts, got.n_nodes, got.events) == \
           (whole.root, whole.root_counts, whole.level_counts, whole.n_nodes, whole.events)
    assert (got.root, got.root_counts) == (o.root, o.root_counts)


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_nested_trace_equals_oracle(rv, torch_cuda, world):
    tr = synth.file_trace(300_000, 500, 20_000, seed=52)
    f = rv.Formula(C3, tr.codes, key_bits=64)
    got = _split_and_check(rv, torch_cuda, f, tr.key, tr.pred, world)
    o = oracle_verify(C3, Schema(tr.codes), tr.key, tr.pred)
    assert got.status == 0
    assert (got.root, got.root_counts, got.level_counts, list(got.n_nodes)) == \
           (o.root, o.root_counts, o.level_counts, list(o.n_nodes))


def test_shard_of_an_empty_trace(rv, torch_cuda):
    f = rv.Formula(C1, synth.SOCKET_CODES)
    key = torch_cuda.empty(0, dtype=torch_cuda.int32, device="cuda")
    pred = torch_cuda.empty(0, dtype=torch_cuda.uint8, device="cuda")
    _, _, _, counts = rv.shard_trace(f, key, pred, 4)
    assert counts.cpu().tolist() == [0, 0, 0, 0]


def test_full_size_split_of_the_bench_trace(rv, torch_cuda):
    """The 1e8-event Zipf socket trace split 8 ways, as the bench times it:
    every segment holds exactly its rank's events in trace order (against the
    host form), and the parts verified one after another combine to the
    unsharded result and to the counts the generator's construction fixes."""
    import bench
    w = dict(bench.WORKLOADS["c2"])
    tr = bench.make_trace(w, 1000 * w["cfg"])
    f = rv.Formula(w["formula"], tr.codes)
    got = _split_and_check(rv, torch_cuda, f, tr.key, tr.pred, 8)
    whole = rv.verify(f, _dev(torch_cuda, tr.key), _dev(torch_cuda, tr.pred))
    assert got.status == 0
    assert (got.root, got.root_counts, got.level_counts, got.n_nodes, got.events) == \
           (whole.root, whole.root_counts, whole.level_counts, whole.n_nodes, whole.events)
    assert bench.matches(got, bench.expected_counts(dict(w, kind="socket"), tr))
