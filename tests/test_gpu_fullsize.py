"""Parity at full size, in the launch configuration bench.py times.

The oracle cannot verify 1e8-2e8 events in a test, so it checks sampled
outputs one by one -- the per-binding verdicts of sampled bindings (including
the longest cluster) and the per-user subtrees of sampled users -- and the
rest is checked through properties that hold at any size: the verdict counts
sum to the number of bindings, the bindings are the distinct keys, and the
root verdict is the valuation of the root counts.
"""
import numpy as np
import pytest

from oracle import counting
from oracle.formula import parse
from oracle.verify import Checker, Schema
from paper_1411_2239_b300 import synth

pytestmark = pytest.mark.gpu

C2 = "A_{>=0.95} s: socket(s) => G(receive -> F respond)"
C3 = "A_{>=0.90} u: user(u) => E_{<=3} f: file(u,f) => open && !F close"


def _dev(torch, a):
    view = {8: np.int64, 4: np.int32, 1: np.uint8}[a.dtype.itemsize]
    return torch.from_numpy(np.ascontiguousarray(a).view(view)).cuda()


def test_c2_full_size(rv):
    import torch
    tr = synth.socket_trace(100_000_000, 1_000_000, pending_frac=0.03, zipf_s=1.1, seed=2000)
    f = rv.Formula(C2, tr.codes)
    g = rv.verify(f, _dev(torch, tr.key), _dev(torch, tr.pred), want_bindings=True)
    assert g.status == 0
    # properties at full size
    assert g.n_nodes[0] == tr.meta["appearing"] == len(g.bindings)
    assert sum(g.root_counts) == g.n_nodes[0]
    q = parse(C2).quants[0]
    assert g.root == counting.valuate(q, g.root_counts)
    pend = set(int(x) for x in tr.meta["pending_ids"])
    assert g.root_counts == [0, 0, len(pend), g.n_nodes[0] - len(pend), 0, 0]
    # sampled bindings: the head cluster, heavy ones and random ones, each by the oracle
    ch = Checker(C2, Schema(tr.codes))
    uniq, counts = np.unique(tr.key, return_counts=True)
    order = np.argsort(-counts)
    rng = np.random.default_rng(0)
    sample = list(uniq[order[:3]]) + list(uniq[order[rng.integers(3, 2000, size=4)]]) + \
        list(rng.choice(uniq, size=12, replace=False)) + list(rng.choice(np.array(sorted(pend), dtype=np.uint32), 3))
    assert counts[order[0]] > 10_000_000
    for k in sample:
        idx = np.flatnonzero(tr.key == k)
        want = ch.instance_verdict(tr.pred[idx])
        assert g.bindings[int(k)] == want, (int(k), len(idx))


def test_c3_full_size(rv):
    import torch
    tr = synth.file_trace(200_000_000, 100_000, 1_000_000, seed=3000)
    f = rv.Formula(C3, tr.codes, key_bits=64)
    g = rv.verify(f, _dev(torch, tr.key), _dev(torch, tr.pred), want_bindings=True)
    assert g.status == 0
    assert g.n_nodes[0] == 100_000 == len(g.outer)
    assert g.n_nodes[1] == tr.meta["n_pairs"] == len(g.bindings)
    assert sum(g.root_counts) == g.n_nodes[0] and sum(g.level_counts[1]) == g.n_nodes[1]
    q0 = parse(C3).quants[0]
    assert g.root == counting.valuate(q0, g.root_counts)
    # every inner verdict histogram entry matches the per-binding outputs
    hist = [0] * 6
    for v in g.bindings.values():
        hist[v] += 1
    assert hist == g.level_counts[1]
    # sampled users: the oracle verifies each user's whole subtree
    ch = Checker(C3, Schema(tr.codes))
    users = tr.key >> np.uint64(32)
    rng = np.random.default_rng(1)
    sample = list(rng.choice(np.unique(users[:2_000_000]), size=10, replace=False))
    sample += [int(u) for u in tr.meta["violating_users"][:4]]
    for u in sample:
        idx = np.flatnonzero(users == np.uint64(u))
        sub = ch.run(tr.key[idx], tr.pred[idx])
        assert g.outer[int(u)] == sub.verdicts[0][(int(u),)], int(u)
        for D, v in sub.verdicts[1].items():
            assert g.bindings[(int(D[0]) << 32) | int(D[1])] == v
