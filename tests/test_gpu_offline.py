"""GPU parity of the offline path (rv_verify_trace) against the CPU oracle.

Every verdict, count and per-binding verdict must be identical (all
arithmetic is integer).  Sizes are small enough for the oracle to finish in
seconds while still spanning many buckets, multi-unit buckets (tree combine)
and ragged tails."""
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
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda()
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda()
    return torch.from_numpy(a).cuda()


def _check(rv, torch, text, codes, key, pred, alphabet="onehot", key_bits=32, opts=None, ts=None, host=False):
    f = rv.Formula(text, codes, alphabet=alphabet, key_bits=key_bits)
    if host:
        g = rv.verify(f, key, pred, ts=ts, opts=opts)
    else:
        g = rv.verify(f, _dev(torch, key), _dev(torch, pred), ts=None if ts is None else _dev(torch, ts),
                      want_bindings=True, opts=opts)
    o = oracle_verify(text, Schema(codes, alphabet), key, pred)
    assert g.status == 0
    assert g.root == o.root, (g.root, o.root)
    nq = f.n_quant
    if nq:
        assert g.root_counts == o.root_counts
        for m in range(nq):
            assert g.level_counts[m] == o.level_counts[m]
            assert g.n_nodes[m] == o.n_nodes[m]
    if not host and nq:
        inner = o.verdicts[nq - 1]
        if nq == 1:
            want = {int(D[0]): v for D, v in inner.items()}
        else:
            want = {(int(D[0]) << 32) | int(D[1]): v for D, v in inner.items()}
        assert g.bindings == want
        if nq == 2:
            assert g.outer == {int(D[0]): v for D, v in o.verdicts[0].items()}
    return g, o


def test_c1_full(rv, torch_cuda):
    tr = synth.socket_trace(100_000, 1000, n_pending=50, seed=1)
    g, _ = _check(rv, torch_cuda, C1, tr.codes, tr.key, tr.pred)
    assert g.root == 3 and g.root_counts == [0, 0, 50, 950, 0, 0]


@pytest.mark.parametrize("pending,root", [(51, 2), (49, 3), (0, 3)])
def test_c1_threshold(rv, torch_cuda, pending, root):
    tr = synth.socket_trace(100_000, 1000, n_pending=pending, seed=2)
    g, _ = _check(rv, torch_cuda, C1, tr.codes, tr.key, tr.pred)
    assert g.root == root


@pytest.mark.parametrize("opts", [None, {"unit_records": 256}, {"bucket_bits": 8, "unit_records": 1024},
                                  {"bucket_bits": 11}])
def test_c2_shape_reduced(rv, torch_cuda, opts):
    tr = synth.socket_trace(2_000_000, 20_000, pending_frac=0.03, zipf_s=1.1, seed=3)
    assert tr.meta["max_cluster"] > 100_000          # long clusters span many units
    _check(rv, torch_cuda, C1, tr.codes, tr.key, tr.pred, opts=opts)


@pytest.mark.parametrize("opts", [None, {"sub_bucket_bits": 3, "unit_records": 512}, {"bucket_bits": 8}])
def test_c3_shape_reduced(rv, torch_cuda, opts):
    tr = synth.file_trace(1_000_000, 500, 1_000_000, seed=4)
    _check(rv, torch_cuda, C3, tr.codes, tr.key, tr.pred, key_bits=64, opts=opts)


def test_random_formulas_one_quantifier(rv, torch_cuda):
    rng = np.random.default_rng(6)
    codes = ["a", "b", "c", "d"]
    n_done = 0
    while n_done < 40:
        body = synth.random_body(rng, codes[:3], depth=int(rng.integers(1, 4)))
        text = f"{synth.random_quantifier(rng)} x: p(x) => {body}"
        n = int(rng.integers(1, 3000))
        key = rng.integers(0, int(rng.integers(1, 200)), size=n).astype(np.uint32)
        pred = rng.integers(0, 4, size=n).astype(np.uint8)
        try:
            _check(rv, torch_cuda, text, codes, key, pred, opts={"unit_records": 256})
        except rv.RVError as e:
            assert e.status == rv.RV_EUNSUPPORTED
            continue
        n_done += 1


def test_random_formulas_two_quantifiers(rv, torch_cuda):
    rng = np.random.default_rng(7)
    codes = ["a", "b", "c", "d"]
    n_done = 0
    while n_done < 30:
        body = synth.random_body(rng, codes[:3], depth=int(rng.integers(1, 3)))
        text = f"{synth.random_quantifier(rng)} x: p(x) => {synth.random_quantifier(rng)} y: q(x,y) => {body}"
        n = int(rng.integers(1, 4000))
        u = rng.integers(0, int(rng.integers(1, 40)), size=n).astype(np.uint64)
        fi = rng.integers(0, int(rng.integers(1, 50)), size=n).astype(np.uint64)
        key = (u << np.uint64(32)) | fi
        pred = rng.integers(0, 4, size=n).astype(np.uint8)
        try:
            _check(rv, torch_cuda, text, codes, key, pred, key_bits=64,
                   opts={"unit_records": 256, "sub_bucket_bits": int(rng.integers(0, 4))})
        except rv.RVError as e:
            assert e.status == rv.RV_EUNSUPPORTED
            continue
        n_done += 1


def test_one_long_cluster_many_levels(rv, torch_cuda):
    # a single binding of 300k events folded by 1172 units -> three combine levels
    rng = np.random.default_rng(8)
    n = 300_000
    key = np.full(n, 77, dtype=np.uint32)
    pred = rng.integers(0, 3, size=n).astype(np.uint8)
    for body in ["G(receive -> F respond)", "F(receive && X respond)", "G !socket", "(receive U respond) || F socket"]:
        _check(rv, torch_cuda, f"E x: p(x) => {body}", synth.SOCKET_CODES, key, pred, opts={"unit_records": 256})


def test_unquantified_property(rv, torch_cuda):
    rng = np.random.default_rng(9)
    pred = rng.integers(0, 3, size=50_000).astype(np.uint8)
    key = rng.integers(0, 5, size=50_000).astype(np.uint32)
    for body in ["G(receive -> F respond)", "F socket", "X X receive", "G(socket -> X receive)"]:
        _check(rv, torch_cuda, body, synth.SOCKET_CODES, key, pred, opts={"unit_records": 1024})


def test_empty_and_tiny_traces(rv, torch_cuda):
    e32 = np.zeros(0, dtype=np.uint32)
    e8 = np.zeros(0, dtype=np.uint8)
    for text in ["A_{>=0.5} x: p(x) => socket", "A_{>0.5} x: p(x) => socket", "E x: p(x) => socket",
                 "E_{<=0} x: p(x) => socket"]:
        f = rv.Formula(text, synth.SOCKET_CODES)
        g = rv.verify(f, e32, e8)
        o = oracle_verify(text, Schema(synth.SOCKET_CODES), e32, e8)
        assert g.root == o.root and g.n_nodes[0] == 0
    for n in [1, 2, 31, 32, 33]:
        key = np.arange(n, dtype=np.uint32) % 3
        pred = (np.arange(n) % 3).astype(np.uint8)
        _check(rv, torch_cuda, C1, synth.SOCKET_CODES, key, pred)


def test_worked_example_bitmask(rv, torch_cuda):
    codes = ["login", "unauthorized", "authorized"]
    key = np.array([(1 << 32) | 12, (1 << 32) | 13, (2 << 32) | 14, (1 << 32) | 15, (1 << 32) | 16], dtype=np.uint64)
    pred = np.array([3, 3, 5, 3, 3], dtype=np.uint8)
    g, _ = _check(rv, torch_cuda, "A x: user(x) => E_{<=3} r: rid(r) => (login && unauthorized)", codes, key, pred,
                  alphabet="bitmask", key_bits=64)
    assert g.root == 0


def test_invalid_inputs_rejected(rv, torch_cuda):
    f = rv.Formula(C1, synth.SOCKET_CODES)
    key = np.arange(100, dtype=np.uint32)
    pred = np.zeros(100, dtype=np.uint8)
    pred[57] = 3                                     # only codes 0..2 exist
    with pytest.raises(rv.RVError) as e:
        rv.verify(f, _dev(torch_cuda, key), _dev(torch_cuda, pred))
    assert e.value.status == rv.RV_EINVAL
    pred[57] = 0
    ts = np.arange(100, dtype=np.uint32)
    ts[40] = 5                                        # time goes backwards
    with pytest.raises(rv.RVError) as e:
        rv.verify(f, key, pred, ts=ts)
    assert e.value.status == rv.RV_EINVAL
    ts[40] = 40
    assert rv.verify(f, key, pred, ts=ts).status == 0


def test_host_and_device_inputs_agree(rv, torch_cuda):
    tr = synth.socket_trace(300_000, 5_000, pending_frac=0.05, zipf_s=1.1, seed=10)
    f = rv.Formula(C1, tr.codes)
    a = rv.verify(f, tr.key, tr.pred, ts=tr.ts)
    b = rv.verify(f, _dev(torch_cuda, tr.key), _dev(torch_cuda, tr.pred), ts=_dev(torch_cuda, tr.ts))
    assert (a.root, a.root_counts, a.n_nodes) == (b.root, b.root_counts, b.n_nodes)


def test_repeatable(rv, torch_cuda):
    tr = synth.file_trace(500_000, 300, 10_000, seed=11)
    f = rv.Formula(C3, tr.codes, key_bits=64)
    k, p = _dev(torch_cuda, tr.key), _dev(torch_cuda, tr.pred)
    r = [rv.verify(f, k, p, want_bindings=True) for _ in range(3)]
    assert r[0].bindings == r[1].bindings == r[2].bindings
    assert r[0].outer == r[1].outer == r[2].outer


def _fmix32(x):
    """MurmurHash3's 32-bit finaliser (public domain), the published mix the
    library applies to a 32-bit key before taking bucket bits from its top."""
    x = x.astype(np.uint64)
    x ^= x >> np.uint64(16)
    x = (x * np.uint64(0x85EBCA6B)) & np.uint64(0xFFFFFFFF)
    x ^= x >> np.uint64(13)
    x = (x * np.uint64(0xC2B2AE35)) & np.uint64(0xFFFFFFFF)
    x ^= x >> np.uint64(16)
    return x.astype(np.uint32)


def test_units_that_open_with_one_binding(rv, torch_cuda):
    # 20 keys chosen to share one bucket (equal top 15 bits of the mixed key),
    # cut into 256-record units that each open with a burst of one key: units
    # whose first round is mostly one binding, whatever the rest holds
    rng = np.random.default_rng(21)
    cand = rng.integers(0, 2**32, size=4_000_000, dtype=np.uint64).astype(np.uint32)
    top = _fmix32(cand) >> np.uint32(17)
    vals, counts = np.unique(top, return_counts=True)
    same = np.unique(cand[top == vals[np.argmax(counts)]])[:20]
    assert len(same) == 20
    heavy, light = same[0], same[1:]
    blocks = []
    for u in range(60):
        share = [0.9, 0.5, 0.2][u % 3]            # dominated, balanced and light units
        body = np.where(rng.random(228) < share, heavy, rng.choice(light, size=228))
        blocks.append(np.concatenate([np.full(28, heavy, dtype=np.uint32), body.astype(np.uint32)]))
    key = np.concatenate(blocks)
    noise = rng.integers(0, 2**32, size=5000, dtype=np.uint64).astype(np.uint32)
    key = np.insert(key, rng.integers(0, len(key), size=len(noise)), noise)
    pred = rng.integers(0, 3, size=len(key)).astype(np.uint8)
    opts = {"bucket_bits": 8, "sub_bucket_bits": 7, "unit_records": 256}
    for body in ["G(receive -> F respond)", "F(receive && X respond)", "(receive U respond) || F socket"]:
        _check(rv, torch_cuda, f"A_{{>=0.5}} x: p(x) => {body}", synth.SOCKET_CODES, key, pred, opts=opts)


@pytest.mark.parametrize("opts", [{"sub_bucket_bits": 3}, {"sub_bucket_bits": 3, "no_heavy": 1},
                                  {"sub_bucket_bits": 2, "unit_records": 1024}])
def test_zipf_heads_in_own_sub_buckets(rv, torch_cuda, opts):
    # Zipf(1.1) over 2e4 ids: the head keys are found by sampling and folded
    # in sub-buckets of their own (or not, with no_heavy); both must match
    tr = synth.socket_trace(3_000_000, 20_000, pending_frac=0.03, zipf_s=1.1, seed=31)
    _check(rv, torch_cuda, C1, tr.codes, tr.key, tr.pred, opts=opts)


@pytest.mark.parametrize("opts", [{"sub_bucket_bits": 7}, {"sub_bucket_bits": 3}])
def test_heavy_keys_with_few_records(rv, torch_cuda, opts):
    # The heavy-key sample reads 8 consecutive events out of every 2048 (every
    # 256th event on average, for traces under 2^27 events).  Four keys
    # planted exactly in six of those runs each are counted 48 times, as often
    # as a key of about 12k events, so each gets a sub-bucket of its own that
    # holds only its 48 records: at most half a unit, so the unit's end is
    # taken from the per-bucket unit ends, which must hold it.
    rng = np.random.default_rng(61)
    n = 300_000
    key = rng.choice(rng.integers(0, 2**32, size=30_000, dtype=np.uint64), size=n).astype(np.uint32)
    planted = rng.integers(0, 2**32, size=4, dtype=np.uint64).astype(np.uint32)
    for a, k in enumerate(planted):
        for m in range(6 * a + 3, 6 * a + 9):
            key[2048 * m: 2048 * m + 8] = k
    pred = rng.integers(0, 3, size=n).astype(np.uint8)
    for k in planted:
        assert (key == k).sum() == 48
    _check(rv, torch_cuda, C1, synth.SOCKET_CODES, key, pred, opts=opts)


def test_many_multi_unit_buckets(rv, torch_cuda):
    # 2^14 light sub-buckets of about 300 records cut into 256-record units:
    # over 8192 buckets are folded by two units or more, so the bucket list of
    # every combine level spans more than one staged chunk; one planted
    # binding of 40k events is folded by over 150 units (two combine levels)
    tr = synth.socket_trace(5_000_000, 1_000_000, pending_frac=0.03, seed=41)
    key = tr.key.copy()
    rng = np.random.default_rng(42)
    key[rng.choice(len(key), size=40_000, replace=False)] = key[0]
    top = _fmix32(key) >> np.uint32(32 - 14)
    assert (np.bincount(top, minlength=1 << 14) > 256).sum() > 8192
    opts = {"bucket_bits": 8, "sub_bucket_bits": 6, "unit_records": 256}
    _check(rv, torch_cuda, C1, tr.codes, key, tr.pred, opts=opts)


def test_level2_scan_in_slices(rv, torch_cuda):
    # 40 keys that share one first-level bucket (equal top 8 bits of the mixed
    # key) hold 1.2e6 events: that bucket's 147 level-2 tiles are scanned by
    # two CTAs, the slice sums of the first carried into the second; the keys
    # are heavy, so both light and heavy sub-bucket columns are non-empty
    rng = np.random.default_rng(51)
    cand = rng.integers(0, 2**32, size=200_000, dtype=np.uint64).astype(np.uint32)
    top = _fmix32(cand) >> np.uint32(24)
    vals, counts = np.unique(top, return_counts=True)
    same = np.unique(cand[top == vals[np.argmax(counts)]])[:40]
    assert len(same) == 40
    key = rng.choice(same, size=1_200_000)
    noise = rng.integers(0, 2**32, size=100_000, dtype=np.uint64).astype(np.uint32)
    key = np.insert(key, rng.integers(0, len(key), size=len(noise)), noise)
    assert (_fmix32(key) >> np.uint32(24) == vals[np.argmax(counts)]).sum() > 129 * 8192
    pred = rng.integers(0, 3, size=len(key)).astype(np.uint8)
    for opts in [{"sub_bucket_bits": 3}, {"sub_bucket_bits": 3, "no_heavy": 1}]:
        _check(rv, torch_cuda, C1, synth.SOCKET_CODES, key, pred, opts=opts)


def test_two_devices_in_one_process(rv, torch_cuda):
    # kernel attributes (dynamic shared-memory limits) belong to the device
    # that is current when they are set: the offline path must configure each
    # device it runs on, not only the first
    if torch_cuda.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    tr = synth.socket_trace(200_000, 5_000, pending_frac=0.03, zipf_s=1.1, seed=31)
    for d in (0, 1, 0):
        with torch_cuda.cuda.device(d):
            _check(rv, torch_cuda, C1, tr.codes, tr.key, tr.pred)


def test_bounded_device_wait_gives_up_with_timeout_status(rv, torch_cuda):
    # a wait on a device flag that nothing sets (rv_verify_opts.test_wait_polls)
    # gives up after its polls: the result's status word says RV_ETIMEOUT, the
    # verdict is still computed, and the context stays usable
    tr = synth.socket_trace(50_000, 500, n_pending=20, seed=33)
    f = rv.Formula(C1, tr.codes)
    k, p = _dev(torch_cuda, tr.key), _dev(torch_cuda, tr.pred)
    with pytest.raises(rv.RVError) as e:
        rv.verify(f, k, p, opts={"test_wait_polls": 2000})
    assert e.value.status == rv.RV_ETIMEOUT
    ws = torch_cuda.empty(rv.workspace_size(f, tr.n), dtype=torch_cuda.uint8, device="cuda")
    out = torch_cuda.zeros(rv.RESULT_BYTES, dtype=torch_cuda.uint8, device="cuda")
    rv.verify_async(f, k, p, ws, out, opts={"test_wait_polls": 2000})
    torch_cuda.cuda.synchronize()
    r = rv.parse_result(bytes(out.cpu().numpy()))
    good = rv.verify(f, k, p)
    o = oracle_verify(C1, Schema(tr.codes), tr.key, tr.pred)
    assert r.status == rv.RV_ETIMEOUT
    assert good.status == 0 and (good.root, good.root_counts) == (o.root, o.root_counts)
    assert (r.root, r.root_counts) == (o.root, o.root_counts)
