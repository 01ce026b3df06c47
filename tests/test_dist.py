"""Multi-rank host logic of bench.py on CPU (gloo, two ranks).

Whole-job numbers take the slowest rank's step time, AND the ranks'
verification and sum their events.  The sharded N > 1 step (each rank holds
a slice of one trace, splits it by the outer-value hash, exchanges the parts
with an all-to-all, verifies its part and all-reduces the counts) is run
here with host tensors: the device split is stood in for by its host form
(rv_shard_of plus a stable sort) and the per-part verification by the
oracle; the combined result must equal the oracle on the whole trace."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, ok, value = bench.combine_ranks(ms=10.0 * (rank + 1), verified=(rank == 0), n_local=1000 * (rank + 1),
                                        world=world)
    w = dict(bench.WORKLOADS["c1"], n=5000, n_ids=50, n_pending=5)
    tr = bench.make_trace(w, 1000 * w["cfg"] + rank)
    out[rank] = (ms, ok, value, int(tr.key[:100].astype(np.uint64).sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_over_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, ok, value, _ = res[r]
        assert ms == 20.0                      # slowest rank
        assert ok is False                     # rank 1 reported a failed check
        assert abs(value - 3000 / 0.020) < 1e-6
    assert res[0][3] != res[1][3]              # ranks verify different traces


def test_single_rank_is_identity():
    import bench
    assert bench.combine_ranks(5.0, True, 100, 1) == (5.0, True, 100 / 0.005)


def _slices(world):
    """The slices of one trace (socket ids disjoint between slices), as bench's sharded run draws them."""
    import bench
    w = dict(bench.WORKLOADS["c2"], n=6_000, n_ids=300)
    ids = np.random.default_rng(7).choice(np.iinfo(np.uint32).max, size=world * w["n_ids"],
                                          replace=False).astype(np.uint32)
    return w, [bench.make_trace(w, 100 + r, ids=ids[r * w["n_ids"]:(r + 1) * w["n_ids"]]) for r in range(world)]


def _shard_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench
    from oracle.verify import Schema, verify
    from paper_1411_2239_b300 import rv
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, slices = _slices(world)
    tr = slices[rank]
    f = rv.Formula(w["formula"], tr.codes)
    ranks = rv.shard_of(f, tr.key, world)
    order = np.argsort(ranks, kind="stable")                 # the device split, on the host
    counts = torch.tensor(np.bincount(ranks, minlength=world), dtype=torch.int64)
    ks = torch.from_numpy(tr.key[order].view(np.int32).copy())
    ps = torch.from_numpy(tr.pred[order].copy())
    kr, pr = bench.exchange(ks, ps, counts)
    key = kr.numpy().view(np.uint32)
    assert (rv.shard_of(f, key, world) == rank).all()       # only this rank's socket ids arrive
    o = verify(w["formula"], Schema(tr.codes), key, pr.numpy())
    part = rv.Result(o.root, 0, list(o.root_counts), [list(o.level_counts[0]), [0] * 6], [o.n_nodes[0], 0],
                     len(key))
    res = bench.reduce_result(rv, f, part)
    exp = torch.tensor(bench.expected_counts(w, tr)["root_counts"], dtype=torch.int64)
    dist.all_reduce(exp)
    out[rank] = (res.root, res.root_counts, res.events, exp.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_step_over_two_gloo_ranks():
    from oracle.verify import Schema, verify
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    w, slices = _slices(world)
    key = np.concatenate([s.key for s in slices])            # slice r follows slice r - 1 in time
    pred = np.concatenate([s.pred for s in slices])
    o = verify(w["formula"], Schema(slices[0].codes), key, pred)
    for r in range(world):
        root, counts, events, exp = res[r]
        assert (root, counts, events) == (o.root, o.root_counts, len(pred))
        assert counts == exp                                # the construction of the slices adds up
