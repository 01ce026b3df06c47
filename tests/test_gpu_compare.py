"""GPU parity of interpreted comparison predicates (case study 2, Sec. 5.1:
A u: user(u) => F(avg_chunksize(u) <= maximum)) with the oracle: the value
column is folded into the letters on the device; results, per-binding
verdicts and the per-event timeline must equal the oracle's."""
import numpy as np
import pytest

from oracle.timeline import timeline as oracle_timeline
from oracle.verify import Schema, verify as oracle_verify
from paper_1411_2239_b300 import synth

pytestmark = pytest.mark.gpu

CS2 = "A u: user(u) => F(avg_chunksize(u) <= 2097152)"


def _dev(torch, a):
    a = np.ascontiguousarray(a)
    view = {8: np.int64, 4: np.int32, 1: np.uint8}[a.dtype.itemsize]
    return torch.from_numpy(a.view(view)).cuda()


@pytest.mark.parametrize("text", [CS2, "A_{>=0.9} u: user(u) => G(upload -> avg_chunksize < 3000000)",
                                  "E_{<=5} u: user(u) => F(avg_chunksize <= 100000 && X avg_chunksize > 200000)"])
def test_chunk_trace_matches_oracle(rv, text):
    import torch
    tr = synth.chunk_trace(300_000, 2_000, seed=111)
    sch = Schema(tr.codes, value_name="avg_chunksize")
    f = rv.Formula(text, tr.codes, value_name="avg_chunksize")
    assert f.n_cmp >= 1
    o = oracle_verify(text, sch, tr.key, tr.pred, tr.value)
    g = rv.verify(f, _dev(torch, tr.key), _dev(torch, tr.pred), value=_dev(torch, tr.value), want_bindings=True)
    assert g.status == 0 and (g.root, g.root_counts) == (o.root, o.root_counts)
    assert g.bindings == {int(D[0]): v for D, v in o.verdicts[0].items()}
    h = rv.verify(f, tr.key, tr.pred, value=tr.value)             # host input path
    assert (h.root, h.root_counts) == (o.root, o.root_counts)


def test_case_study_shape(rv):
    # heavy users keep a session average of the maximum chunk: presumably violated
    import torch
    tr = synth.chunk_trace(200_000, 1_000, seed=112)
    f = rv.Formula(CS2, tr.codes, value_name="avg_chunksize")
    g = rv.verify(f, _dev(torch, tr.key), _dev(torch, tr.pred), value=_dev(torch, tr.value))
    heavy = len(tr.meta["heavy_users"])
    assert g.root_counts == [0, 0, heavy, 0, 0, tr.meta["appearing"] - heavy]


def test_two_variables_with_comparison(rv):
    import torch
    rng = np.random.default_rng(113)
    n = 100_000
    key = (rng.integers(0, 50, size=n).astype(np.uint64) << np.uint64(32)) | rng.integers(0, 40, size=n).astype(np.uint64)
    pred = rng.integers(0, 2, size=n).astype(np.uint8)
    value = rng.integers(0, 1000, size=n).astype(np.uint32)
    text = "A_{>=0.5} u: user(u) => E_{<=2} f: file(u,f) => F(upload && avg > 995)"
    sch = Schema(["user", "upload"], value_name="avg")
    f = rv.Formula(text, sch.code_names, key_bits=64, value_name="avg")
    o = oracle_verify(text, sch, key, pred, value)
    g = rv.verify(f, _dev(torch, key), _dev(torch, pred), value=_dev(torch, value))
    assert (g.root, g.root_counts, g.level_counts) == (o.root, o.root_counts, o.level_counts)


def test_timeline_with_comparison(rv):
    import torch
    tr = synth.chunk_trace(60_000, 500, seed=114)
    text = "A u: user(u) => G(upload -> avg_chunksize < 3500000)"
    f = rv.Formula(text, tr.codes, value_name="avg_chunksize")
    v, first = rv.timeline(f, _dev(torch, tr.key), _dev(torch, tr.pred), value=_dev(torch, tr.value))
    ov, ofirst = oracle_timeline(text, Schema(tr.codes, value_name="avg_chunksize"), tr.key, tr.pred, tr.value)
    assert (v == ov).all()
    assert first == {D[0]: j for D, j in ofirst.items()}


def test_missing_values_rejected(rv):
    import torch
    f = rv.Formula(CS2, synth.CHUNK_CODES, value_name="avg_chunksize")
    key = torch.zeros(10, dtype=torch.int32, device="cuda")
    pred = torch.zeros(10, dtype=torch.uint8, device="cuda")
    with pytest.raises(rv.RVError) as e:
        rv.verify(f, key, pred)
    assert e.value.status == rv.RV_EINVAL


def test_sharded_with_values(rv):
    # the split moves the value column with the events; the parts' counts add up
    import torch
    tr = synth.chunk_trace(200_000, 1_500, seed=115)
    f = rv.Formula(CS2, tr.codes, value_name="avg_chunksize")
    key, pred, value = _dev(torch, tr.key), _dev(torch, tr.pred), _dev(torch, tr.value)
    ko, po, _, counts = rv.shard_trace(f, key, pred, 3, value=value)
    vo = rv.shard_trace.last_value
    counts = counts.cpu().tolist()
    parts, a = [], 0
    for c in counts:
        parts.append(rv.verify(f, ko[a:a + c], po[a:a + c], value=vo[a:a + c]))
        a += c
    got = rv.combine_results(f, parts)
    o = oracle_verify(CS2, Schema(tr.codes, value_name="avg_chunksize"), tr.key, tr.pred, tr.value)
    assert (got.root, got.root_counts) == (o.root, o.root_counts)
