"""GPU tests of the online service (rv_service / rv_stream): every chunk's
verdict equals the CPU oracle on the stream prefix it closes, whether the
stream runs alone or mixed with others; admission, timeouts and closing."""
import time

import numpy as np
import pytest

from oracle.verify import Schema, verify as oracle_verify
from paper_1411_2239_b300 import synth

pytestmark = pytest.mark.gpu

C1 = "A_{>=0.95} s: socket(s) => G(receive -> F respond)"
C3 = "A_{>=0.90} u: user(u) => E_{<=3} f: file(u,f) => open && !F close"


def _chunks(rng, n):
    cuts = np.sort(rng.choice(np.arange(1, n), size=min(n - 1, int(rng.integers(3, 9))), replace=False))
    return np.split(np.arange(n), cuts)


def _push(rv, st, key, pred, timeout_s=60):
    """Push, retrying while the service refuses admission (as a producer would)."""
    t0 = time.time()
    while True:
        try:
            return st.push(key, pred)
        except rv.RVError as e:
            if e.status != rv.RV_EAGAIN or time.time() - t0 > timeout_s:
                raise
            time.sleep(0.002)


def _drain(streams, want, timeout_s=60):
    got = {i: [] for i in range(len(streams))}
    t0 = time.time()
    while any(len(got[i]) < want[i] for i in got) and time.time() - t0 < timeout_s:
        for i, st in enumerate(streams):
            got[i] += st.poll(64, timeout_us=2000)
    return got


def _run(rv, formula_text, codes, key_bits, traces, seed, **cfg):
    rng = np.random.default_rng(seed)
    f = rv.Formula(formula_text, codes, key_bits=key_bits)
    svc = rv.Service(f, **cfg)
    streams = [svc.open_stream() for _ in traces]
    plans = [_chunks(rng, tr.n) for tr in traces]
    order = [(i, j) for i in range(len(traces)) for j in range(len(plans[i]))]
    # interleave streams, keep each stream's chunks in order
    pos = [0] * len(traces)
    while order:
        i = int(rng.integers(len(traces)))
        if pos[i] >= len(plans[i]):
            order = [o for o in order if pos[o[0]] < len(plans[o[0]])]
            continue
        idx = plans[i][pos[i]]
        _push(rv, streams[i], traces[i].key[idx], traces[i].pred[idx])
        pos[i] += 1
        order = [o for o in order if pos[o[0]] < len(plans[o[0]])]
    got = _drain(streams, [len(p) for p in plans])
    svc.close()
    return plans, got


def _check_prefixes(formula_text, codes, traces, plans, got):
    for i, tr in enumerate(traces):
        assert [v.ticket for v in got[i]] == list(range(1, len(plans[i]) + 1))
        end = 0
        for k, v in enumerate(got[i]):
            end += len(plans[i][k])
            o = oracle_verify(formula_text, Schema(codes), tr.key[:end], tr.pred[:end])
            assert v.status == 0 and v.events == end
            assert v.root == o.root and v.root_counts == o.root_counts, (i, k)
            assert v.latency_us > 0


def test_two_quantifier_streams_match_oracle_prefixes(rv):
    traces = [synth.file_trace(30_000, 40, 500, seed=20 + i) for i in range(3)]
    plans, got = _run(rv, C3, synth.FILE_CODES, 64, traces, 1, max_bindings=1 << 20, max_outer=1 << 17)
    _check_prefixes(C3, synth.FILE_CODES, traces, plans, got)


def test_one_quantifier_streams_match_oracle_prefixes(rv):
    traces = [synth.socket_trace(40_000, 300, pending_frac=0.1, seed=30 + i) for i in range(4)]
    plans, got = _run(rv, C1, synth.SOCKET_CODES, 32, traces, 2, max_bindings=1 << 20)
    _check_prefixes(C1, synth.SOCKET_CODES, traces, plans, got)


def test_alone_equals_mixed(rv):
    a = synth.file_trace(40_000, 50, 300, seed=40)
    others = [synth.file_trace(30_000, 30, 300, seed=41 + i) for i in range(5)]
    plans1, got1 = _run(rv, C3, synth.FILE_CODES, 64, [a], 3)
    # the same chunking of stream a, now interleaved with five other streams
    rng = np.random.default_rng(3)
    f = rv.Formula(C3, synth.FILE_CODES, key_bits=64)
    svc = rv.Service(f)
    sa = svc.open_stream()
    so = [svc.open_stream() for _ in others]
    oplans = [_chunks(np.random.default_rng(100 + i), tr.n) for i, tr in enumerate(others)]
    for k, idx in enumerate(plans1[0]):
        sa.push(a.key[idx], a.pred[idx])
        for i, tr in enumerate(others):
            if k < len(oplans[i]):
                so[i].push(tr.key[oplans[i][k]], tr.pred[oplans[i][k]])
    got = _drain([sa], [len(plans1[0])])[0]
    svc.close()
    assert [(v.ticket, v.root, v.root_counts, v.events) for v in got] == \
           [(v.ticket, v.root, v.root_counts, v.events) for v in got1[0]]


def test_admission_refuses_over_budget(rv):
    f = rv.Formula(C1, synth.SOCKET_CODES)
    svc = rv.Service(f, max_bindings=1000, max_batch_events=4096)
    st = svc.open_stream()
    key = np.arange(5000, dtype=np.uint32)
    pred = np.zeros(5000, dtype=np.uint8)
    with pytest.raises(rv.RVError) as e:        # larger than a batch
        st.push(key, pred)
    assert e.value.status == rv.RV_EINVAL
    with pytest.raises(rv.RVError) as e:        # could need 2000 > 1000 bindings
        st.push(key[:2000], pred[:2000])
    assert e.value.status == rv.RV_EAGAIN
    assert svc.stats()["refused"] >= 1
    st.push(key[:500], pred[:500])
    v = _drain([st], [1])[0]
    assert len(v) == 1 and v[0].status == 0
    svc.close()


def test_malformed_chunks_and_timeouts(rv):
    f = rv.Formula(C1, synth.SOCKET_CODES)
    svc = rv.Service(f)
    st = svc.open_stream()
    assert st.poll(4, timeout_us=1000) == []
    with pytest.raises(rv.RVError) as e:
        st.push(np.arange(10, dtype=np.uint32), np.full(10, 3, dtype=np.uint8))   # code 3 does not exist
    assert e.value.status == rv.RV_EINVAL
    with pytest.raises(rv.RVError) as e:
        st.push(np.arange(10, dtype=np.uint32), np.zeros(10, dtype=np.uint8), ts=np.arange(10, 0, -1, dtype=np.uint32))
    assert e.value.status == rv.RV_EINVAL
    svc.close()


def test_close_mid_flight_keeps_other_streams(rv):
    traces = [synth.socket_trace(20_000, 200, pending_frac=0.1, seed=50 + i) for i in range(2)]
    f = rv.Formula(C1, synth.SOCKET_CODES)
    svc = rv.Service(f)
    a, b = svc.open_stream(), svc.open_stream()
    for idx in np.array_split(np.arange(traces[0].n), 6):
        a.push(traces[0].key[idx], traces[0].pred[idx])
    a.close()
    with pytest.raises(rv.RVError):
        a.push(traces[0].key[:5], traces[0].pred[:5])
    b.push(traces[1].key, traces[1].pred)
    got = _drain([b], [1])[0]
    o = oracle_verify(C1, Schema(synth.SOCKET_CODES), traces[1].key, traces[1].pred)
    assert got[0].root == o.root and got[0].root_counts == o.root_counts
    svc.close()


def _open(rv, svc, timeout_s=30):
    """Open a stream, waiting while every slot is still being retired."""
    t0 = time.time()
    while True:
        try:
            return svc.open_stream()
        except rv.RVError as e:
            if e.status != rv.RV_EAGAIN or time.time() - t0 > timeout_s:
                raise
            time.sleep(0.002)


def test_slots_reused_over_open_close_cycles(rv):
    # 200 streams opened and closed on a 64-slot service, every one with the
    # same socket ids: a reused slot must start from an empty submonitor tree.
    # A long-lived stream runs beside them the whole time.
    f = rv.Formula(C1, synth.SOCKET_CODES)
    svc = rv.Service(f, max_streams=64, max_bindings=1 << 16)
    sch = Schema(synth.SOCKET_CODES)
    keeper = synth.socket_trace(60_000, 500, pending_frac=0.1, seed=60)
    kst = svc.open_stream()
    kparts = np.array_split(np.arange(keeper.n), 50)
    short = [synth.socket_trace(600, 40, n_pending=k % 7, seed=61 + k % 5) for k in range(200)]
    live = []
    for k in range(200):
        st = _open(rv, svc)
        _push(rv, st, short[k].key, short[k].pred)
        live.append((st, short[k]))
        if k % 4 == 0 and k // 4 < len(kparts):
            _push(rv, kst, keeper.key[kparts[k // 4]], keeper.pred[kparts[k // 4]])
        if len(live) > 40:                      # keep 40 short streams open at a time
            st0, tr0 = live.pop(0)
            v = _drain([st0], [1])[0]
            o = oracle_verify(C1, sch, tr0.key, tr0.pred)
            assert v[0].root == o.root and v[0].root_counts == o.root_counts
            st0.close()
    for st0, tr0 in live:
        v = _drain([st0], [1])[0]
        o = oracle_verify(C1, sch, tr0.key, tr0.pred)
        assert v[0].root == o.root and v[0].root_counts == o.root_counts
        st0.close()
    n_k = min(50, 200 // 4)
    got = _drain([kst], [n_k])[0]
    end = sum(len(kparts[i]) for i in range(n_k))
    o = oracle_verify(C1, sch, keeper.key[:end], keeper.pred[:end])
    assert got[-1].root == o.root and got[-1].root_counts == o.root_counts
    kst.close()
    t0 = time.time()
    while svc.stats()["bindings"] > 0 and time.time() - t0 < 30:   # every binding retired
        time.sleep(0.01)
    assert svc.stats()["bindings"] == 0
    svc.close()


def test_memory_readmitted_after_close(rv):
    f = rv.Formula(C1, synth.SOCKET_CODES)
    svc = rv.Service(f, max_bindings=2_000, max_batch_events=4_096)
    a, b = svc.open_stream(), svc.open_stream()
    ka = np.arange(1, 1_501, dtype=np.uint32)
    a.push(ka, np.zeros(1_500, dtype=np.uint8))
    assert _drain([a], [1])[0][0].status == 0
    kb = np.arange(10_001, 11_001, dtype=np.uint32)
    pb = np.zeros(1_000, dtype=np.uint8)
    with pytest.raises(rv.RVError) as e:        # 1500 live + up to 1000 new > 2000
        b.push(kb, pb)
    assert e.value.status == rv.RV_EAGAIN
    a.close()
    _push(rv, b, kb, pb)                        # admitted once a's bindings are retired
    v = _drain([b], [1])[0]
    assert v[0].status == 0 and sum(v[0].root_counts) == 1_000
    assert svc.stats()["bindings"] == 1_000
    svc.close()


def test_bad_chunk_fails_only_its_push(rv):
    traces = [synth.socket_trace(20_000, 200, pending_frac=0.1, seed=70 + i) for i in range(3)]
    f = rv.Formula(C1, synth.SOCKET_CODES)
    svc = rv.Service(f)
    sts = [svc.open_stream() for _ in traces]
    parts = [np.array_split(np.arange(tr.n), 4) for tr in traces]
    for k in range(4):
        for i, (st, tr) in enumerate(zip(sts, traces)):
            if i == 0 and k == 2:
                with pytest.raises(rv.RVError) as e:
                    st.push(tr.key[:10], np.full(10, 7, dtype=np.uint8))
                assert e.value.status == rv.RV_EINVAL
            _push(rv, st, tr.key[parts[i][k]], tr.pred[parts[i][k]])
    got = _drain(sts, [4, 4, 4])
    for i, tr in enumerate(traces):
        o = oracle_verify(C1, Schema(synth.SOCKET_CODES), tr.key, tr.pred)
        assert [v.ticket for v in got[i]] == [1, 2, 3, 4]
        assert got[i][-1].root == o.root and got[i][-1].root_counts == o.root_counts
    svc.close()
