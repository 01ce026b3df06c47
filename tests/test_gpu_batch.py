"""GPU parity of the batched path (rv_batch_*): every (trace, formula) result
equals the CPU oracle and the single-trace launch."""
import numpy as np
import pytest

from oracle.verify import Schema, verify as oracle_verify
from paper_1411_2239_b300 import synth

pytestmark = pytest.mark.gpu


def _formulas(rv, rng, codes, nf):
    out, texts = [], []
    while len(out) < nf:
        body = synth.random_body(rng, codes, depth=int(rng.integers(1, 4)))
        text = f"{synth.random_quantifier(rng)} x: p(x) => {body}"
        try:
            out.append(rv.Formula(text, codes))
            texts.append(text)
        except rv.RVError:
            continue
    return out, texts


def _make(rv, seed, lens, nf):
    rng = np.random.default_rng(seed)
    keys, preds, forms, texts, codes_all = [], [], [], [], []
    for n in lens:
        nc = int(rng.integers(2, 7))
        codes = [f"p{j}" for j in range(nc)]
        nk = max(1, n // 16)
        keys.append(rng.integers(0, nk, size=n).astype(np.uint32) * np.uint32(2654435761))
        preds.append(rng.integers(0, nc, size=n).astype(np.uint8))
        f, t = _formulas(rv, rng, codes, nf)
        forms.append(f)
        texts.append(t)
        codes_all.append(codes)
    off = np.zeros(len(lens) + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens)
    return keys, preds, forms, texts, codes_all, off


def _run(rv, torch, forms, keys, preds, off, **kw):
    b = rv.Batch(forms, off, **kw)
    k = torch.from_numpy(np.concatenate(keys).view(np.int32)).cuda()
    p = torch.from_numpy(np.concatenate(preds)).cuda()
    ws = torch.empty(b.workspace_size(), dtype=torch.uint8, device="cuda")
    res = torch.empty(b.nt * b.nf * rv.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    b.run(k, p, ws, res)
    torch.cuda.synchronize()
    return b, k, p, ws, res, b.results(res)


def test_batch_matches_oracle(rv):
    import torch
    lens = [0, 1, 7, 100, 999, 5000, 20000, 64, 3000, 12345]
    keys, preds, forms, texts, codes, off = _make(rv, 1, lens, 8)
    _, _, _, _, _, out = _run(rv, torch, forms, keys, preds, off, bucket_records=512)
    for t in range(len(lens)):
        for j in range(8):
            r = out[t * 8 + j]
            o = oracle_verify(texts[t][j], Schema(codes[t]), keys[t], preds[t])
            assert r.status == 0
            assert r.root == o.root and r.root_counts == o.root_counts, (t, j, texts[t][j])
            assert r.n_nodes[0] == o.n_nodes[0] and r.events == lens[t]


def test_batch_matches_single_launch_and_autotune(rv):
    import torch
    lens = [int(x) for x in np.exp(np.random.default_rng(2).uniform(np.log(1e3), np.log(3e5), size=12))]
    keys, preds, forms, texts, codes, off = _make(rv, 2, lens, 32)
    b, k, p, ws, res, out = _run(rv, torch, forms, keys, preds, off)
    for t in range(len(lens)):
        kt = torch.from_numpy(keys[t].view(np.int32)).cuda()
        pt = torch.from_numpy(preds[t]).cuda()
        for j in range(0, 32, 5):
            s = rv.verify(forms[t][j], kt, pt)
            r = out[t * 32 + j]
            assert (r.root, r.root_counts, r.n_nodes[0]) == (s.root, s.root_counts, s.n_nodes[0])
    chosen = b.autotune(k, p, ws, res)
    assert chosen["bucket_records"] in (1024, 2048, 4096, 8192)
    b.run(k, p, ws, res)
    torch.cuda.synchronize()
    out2 = b.results(res)
    assert [(r.root, r.root_counts) for r in out2] == [(r.root, r.root_counts) for r in out]


def test_batch_bad_predicate(rv):
    import torch
    keys, preds, forms, texts, codes, off = _make(rv, 3, [100, 200], 2)
    preds[1][17] = len(codes[1])          # out of this trace's alphabet
    _, _, _, _, _, out = _run(rv, torch, forms, keys, preds, off)
    assert all(r.status == rv.RV_EINVAL for r in out)


def test_buckets_of_many_bindings_fold_in_passes(rv):
    # every event its own binding: buckets of thousands of bindings, folded in
    # passes of at most 512 bindings each (hash-selected subsets)
    import torch
    rng = np.random.default_rng(4)
    n = 60_000
    keys = [np.arange(n, dtype=np.uint32) * np.uint32(2654435761), rng.integers(0, 7_000, size=n).astype(np.uint32)]
    preds = [rng.integers(0, 2, size=n).astype(np.uint8) for _ in range(2)]
    texts = ["E x: p(x) => F a", "A_{>=0.4} x: p(x) => G(a -> X b)"]
    forms = [[rv.Formula(t, ["a", "b"]) for t in texts] for _ in range(2)]
    off = np.array([0, n, 2 * n], dtype=np.uint64)
    for br in (8192, 256):
        _, _, _, _, _, out = _run(rv, torch, forms, keys, preds, off, bucket_records=br)
        for t in range(2):
            for j, text in enumerate(texts):
                o = oracle_verify(text, Schema(["a", "b"]), keys[t], preds[t])
                r = out[t * 2 + j]
                assert r.status == 0 and r.root == o.root and r.root_counts == o.root_counts, (br, t, j)
                assert r.n_nodes[0] == o.n_nodes[0]


def _zipf_head_batch(rv, seed, head_events, nf):
    # trace 0: one binding with head_events events among 4000 light ones;
    # traces 1..3: ordinary uniform traces
    rng = np.random.default_rng(seed)
    codes = ["p0", "p1", "p2"]
    n0 = head_events + 200_000
    k0 = rng.integers(1, 4_000, size=n0).astype(np.uint32) * np.uint32(2654435761)
    k0[rng.random(n0) < head_events / n0] = np.uint32(77)
    keys = [k0] + [rng.integers(0, 3_000, size=50_000).astype(np.uint32) for _ in range(3)]
    preds = [rng.integers(0, 3, size=len(k)).astype(np.uint8) for k in keys]
    forms, texts = [], []
    for _ in keys:
        f, t = _formulas(rv, rng, codes, nf)
        forms.append(f)
        texts.append(t)
    off = np.zeros(len(keys) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(k) for k in keys])
    return keys, preds, forms, texts, codes, off


def test_long_cluster_segments_match_single_launch_and_oracle(rv):
    # a binding of more than a million events: its bucket is cut into
    # segments folded by separate CTAs into composed maps (long_records), or
    # folded whole (long_records < 0); both equal the single-trace launch and,
    # for some formulas, the oracle
    import torch
    keys, preds, forms, texts, codes, off = _zipf_head_batch(rv, 6, 1_100_000, 16)
    assert (keys[0] == 77).sum() > 1_000_000
    outs = []
    for br, lr in ((4096, 16384), (4096, 65536), (4096, -1), (8192, 65536)):
        _, _, _, _, _, out = _run(rv, torch, forms, keys, preds, off, bucket_records=br, long_records=lr)
        outs.append([(r.status, r.root, r.root_counts, r.n_nodes[0]) for r in out])
    assert outs[0] == outs[1] == outs[2] == outs[3]
    out = outs[0]
    for t in range(len(keys)):
        kt = torch.from_numpy(keys[t].view(np.int32)).cuda()
        pt = torch.from_numpy(preds[t]).cuda()
        for j in range(16):
            s = rv.verify(forms[t][j], kt, pt)
            assert out[t * 16 + j] == (0, s.root, s.root_counts, s.n_nodes[0]), (t, j)
    for j in range(0, 16, 5):
        o = oracle_verify(texts[0][j], Schema(codes), keys[0], preds[0])
        assert out[j][1:3] == (o.root, o.root_counts), texts[0][j]


def test_autotune_reports_thresholds(rv):
    import torch
    keys, preds, forms, texts, codes, off = _zipf_head_batch(rv, 7, 300_000, 8)
    b, k, p, ws, res, out = _run(rv, torch, forms, keys, preds, off)
    chosen = b.autotune(k, p, ws, res)
    assert chosen["bucket_records"] in (1024, 2048, 4096, 8192)
    assert chosen["long_records"] in (16384, 65536, 262144, -1)
    b.run(k, p, ws, res)
    torch.cuda.synchronize()
    assert [(r.root, r.root_counts) for r in b.results(res)] == [(r.root, r.root_counts) for r in out]


SMALL = ["E_{>=6} x: p(x) => (((!p3) U (p3)) U (X(p3))) -> ((G(p3)) -> ((p2) U (!p3)))",
         "E_{<7} x: p(x) => (F(p2)) -> (F(p0))",
         "A_{>=85%} x: p(x) => ((X(p0)) -> (X(p3))) U (X(G(p2)))",
         "A_{=100%} x: p(x) => X(X(G(p1)))",
         "E_{>6} x: p(x) => ((F(X(p2))) -> (G((p0) U (!p0)))) -> (X(F((p0) U (p1))))",
         "A_{<75%} x: p(x) => X((((p1) && (p3)) U ((p2) -> (p3))) && ((G(p1)) U (F(!p0))))"]
LARGE = ["A_{>75%} x: p(x) => ((((p1) -> (p3)) U ((!p3) && (p0))) && (X((!p3) -> (!p2)))) U (X(X((p1) && (p1))))",
         "A_{<15%} x: p(x) => (X(G(F(p2)))) -> (X(X(X(p2))))"]


def test_small_and_large_monitor_traces(rv):
    # traces whose monitors all have at most 8 states (every map target in
    # the low word of the nibble map) and traces that mix in monitors of 9
    # and 12 states, with runs of full and partial rounds of 32 letters and
    # two bucket sizes: every (trace, formula) against the oracle
    import torch
    codes = ["p0", "p1", "p2", "p3"]
    sets = [SMALL + SMALL[:2], SMALL[:6] + LARGE, LARGE + SMALL[2:] + SMALL[:2], SMALL[::-1] + SMALL[:2]]
    assert all(len(s) == 8 for s in sets)
    forms = [[rv.Formula(t, codes) for t in s] for s in sets]
    assert all(f.n_states <= 8 for f in forms[0]) and all(f.n_states <= 8 for f in forms[3])
    assert any(f.n_states > 8 for f in forms[1]) and any(f.n_states > 8 for f in forms[2])
    rng = np.random.default_rng(11)
    shape = [(40_000, 300), (40_000, 300), (30_000, 3_000), (30_000, 3_000)]   # ~130 and ~10 events a key
    keys = [rng.integers(0, nk, size=n).astype(np.uint32) * np.uint32(2654435761) for n, nk in shape]
    preds = [rng.integers(0, 4, size=n).astype(np.uint8) for n, _ in shape]
    off = np.zeros(len(keys) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(k) for k in keys])
    for br in (4096, 512):
        _, _, _, _, _, out = _run(rv, torch, forms, keys, preds, off, bucket_records=br)
        for t in range(len(keys)):
            for j, text in enumerate(sets[t]):
                o = oracle_verify(text, Schema(codes), keys[t], preds[t])
                r = out[t * 8 + j]
                assert r.status == 0 and r.root == o.root and r.root_counts == o.root_counts, (br, t, j, text)
                assert r.n_nodes[0] == o.n_nodes[0]
