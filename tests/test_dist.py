"""Multi-rank host logic of bench.py on CPU (gloo, two ranks): whole-job
numbers take the slowest rank's step time, AND the ranks' verification and
sum their events; every rank draws its own seeded trace."""
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
