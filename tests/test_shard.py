"""One trace over several ranks, host side (no GPU): the partition by outer
value is exact and the parts' counts add up to the whole trace's result.

Algorithm 1 (Sec. 4.2) evaluates each binding on its own projection; the
bindings of one outer value form one subtree (Sec. 3.3), and ApplyQuantifiers
only counts verdicts per level (Sec. 3.4).  Two gloo ranks on CPU each take
their part of the same seeded trace (rv_shard_of, the library's host form of
the device split), verify it with the oracle (the test's checker), and
combine the counts through the library (rv_combine_results) after an
all-reduce and after an all-gather of the parts: both must equal the oracle
on the whole trace, and no outer value may appear on two ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1411_2239_b300 import synth

C1 = "A_{>=0.95} s: socket(s) => G(receive -> F respond)"
C3 = "A_{>=0.90} u: user(u) => E_{<=3} f: file(u,f) => open && !F close"
E2 = "E_{<=40} s: socket(s) => G(receive -> F respond)"


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _cases():
    t1 = synth.socket_trace(20_000, 400, n_pending=20, seed=41)
    t2 = synth.socket_trace(30_000, 2_000, pending_frac=0.03, zipf_s=1.1, seed=42)
    t3 = synth.file_trace(30_000, 60, 2_000, seed=43)
    return [(C1, t1, 32), (C1, t2, 32), (E2, t2, 32), (C1, t2, 64), (C3, t3, 64)]


def _as_rv(o, nq, n):
    from paper_1411_2239_b300 import rv
    lc = [list(o.level_counts[m]) if m < nq else [0] * 6 for m in range(2)]
    nn = [o.n_nodes[m] if m < nq else 0 for m in range(2)]
    return rv.Result(o.root, 0, list(o.root_counts), lc, nn, n)


def _outer_values(key, nq):
    k = np.asarray(key).astype(np.uint64)
    return set((k >> np.uint64(32)).tolist() if nq == 2 else k.tolist())


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    from oracle.verify import Schema, verify
    from paper_1411_2239_b300 import rv
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = []
    for text, tr, bits in _cases():
        f = rv.Formula(text, tr.codes, key_bits=bits)
        key = tr.key.astype(np.uint64 if bits == 64 else np.uint32)
        mine = rv.shard_of(f, key, world) == rank
        k, p = key[mine], tr.pred[mine]                      # trace order kept
        o = verify(text, Schema(tr.codes), k, p)
        part = _as_rv(o, f.n_quant, int(mine.sum()))
        # all-reduce of the counts, then one re-valuation of the root
        v = torch.tensor(part.root_counts + part.level_counts[0] + part.level_counts[1] + part.n_nodes +
                         [part.events, part.status], dtype=torch.int64)
        dist.all_reduce(v)
        v = v.tolist()
        summed = rv.Result(0, 0, v[0:6], [v[6:12], v[12:18]], v[18:20], v[20])
        by_reduce = rv.combine_results(f, [summed])
        # all-gather of the parts, combined by the library
        parts = [None] * world
        dist.all_gather_object(parts, part)
        by_gather = rv.combine_results(f, parts)
        vals = [None] * world
        dist.all_gather_object(vals, sorted(_outer_values(k, f.n_quant)))
        res.append((by_reduce, by_gather, vals))
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_exactly_and_combine_to_the_oracle():
    from oracle.verify import Schema, verify
    from paper_1411_2239_b300 import rv
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for i, (text, tr, bits) in enumerate(_cases()):
        f = rv.Formula(text, tr.codes, key_bits=bits)
        o = verify(text, Schema(tr.codes), tr.key, tr.pred)
        whole = _as_rv(o, f.n_quant, len(tr.pred))
        for rank in range(world):
            by_reduce, by_gather, vals = res[rank][i]
            for got in (by_reduce, by_gather):
                assert (got.root, got.root_counts, got.level_counts, got.n_nodes, got.events) == \
                       (whole.root, whole.root_counts, whole.level_counts, whole.n_nodes, whole.events), text
            # exact partition: no outer value on two ranks, every value somewhere
            a, b = set(vals[0]), set(vals[1])
            assert not (a & b)
            assert a | b == _outer_values(tr.key, f.n_quant)
            assert a and b                                      # both ranks got work


def test_rank_depends_on_the_outer_value_only(rv):
    rng = np.random.default_rng(44)
    f = rv.Formula(C3, synth.FILE_CODES, key_bits=64)
    users = rng.integers(0, 2**32, size=500, dtype=np.uint64)
    files = rng.integers(0, 2**32, size=(500, 4), dtype=np.uint64)
    key = ((users[:, None] << np.uint64(32)) | files).reshape(-1)
    for world in (2, 3, 7, 256):
        r = rv.shard_of(f, key, world).reshape(500, 4)
        assert (r == r[:, :1]).all() and r.max() < world
        counts = np.bincount(r[:, 0], minlength=world)
        if world <= 7:
            assert counts.min() > 0.5 * 500 / world       # spread over every rank
    assert (rv.shard_of(f, key, 1) == 0).all()


def test_shard_arguments_are_checked(rv):
    f = rv.Formula(C1, synth.SOCKET_CODES)
    key = np.arange(10, dtype=np.uint32)
    for world in (0, 257):
        with pytest.raises(rv.RVError) as e:
            rv.shard_of(f, key, world)
        assert e.value.status == rv.RV_EINVAL
    g = rv.Formula("G(receive -> F respond)", synth.SOCKET_CODES)
    with pytest.raises(rv.RVError) as e:
        rv.shard_of(g, key, 2)
    assert e.value.status == rv.RV_EINVAL
    with pytest.raises(rv.RVError):
        rv.combine_results(g, [rv.Result(3, 0, [0] * 6, [[0] * 6] * 2, [0, 0], 5)] * 2)
