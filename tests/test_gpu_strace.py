"""GPU parity of the strace front end (rv_parse_strace) with the oracle's
parser, element by element, and the whole path: log -> events -> verdict."""
import numpy as np
import pytest

from oracle import strace
from oracle.verify import Schema, verify as oracle_verify
from paper_1411_2239_b300 import synth
from tests.test_strace_oracle import RULES

pytestmark = pytest.mark.gpu

C1 = "A_{>=0.95} s: socket(s) => G(receive -> F respond)"
GPU_RULES = [(r.name, r.code, r.key_from, int(r.ok_only)) for r in RULES]


def _check(rv, text, rules=RULES):
    key, pred, ts = rv.parse_strace(text, [(r.name, r.code, r.key_from, int(r.ok_only)) for r in rules])
    k, c, t = strace.parse(text, rules)
    assert key.cpu().numpy().view(np.uint32).tolist() == [x & 0xFFFFFFFF for x in k]
    assert pred.cpu().numpy().tolist() == c
    assert ts.cpu().numpy().tolist() == t
    return key, pred


@pytest.mark.parametrize("fmt,noise,split", [("ttt", 0.3, 0.1), ("tt", 0.7, 0.3), ("ttt", 0.0, 0.0)])
def test_generated_logs_match_oracle(rv, fmt, noise, split):
    tr = synth.socket_trace(100_000, 1_000, n_pending=50, seed=121)
    text = synth.strace_log(tr, seed=122, noise=noise, split=split, fmt=fmt)
    key, pred = _check(rv, text)
    assert (key.cpu().numpy().view(np.uint32) == tr.key).all() and (pred.cpu().numpy() == tr.pred).all()


def test_log_to_verdict(rv):
    tr = synth.socket_trace(200_000, 3_000, pending_frac=0.05, zipf_s=1.1, seed=123)
    key, pred = _check(rv, synth.strace_log(tr, seed=124))
    f = rv.Formula(C1, tr.codes)
    g = rv.verify(f, key, pred)
    o = oracle_verify(C1, Schema(tr.codes), tr.key, tr.pred)
    assert (g.root, g.root_counts) == (o.root, o.root_counts)


def test_hand_written_and_edge_lines(rv):
    lines = ["1700000000.000021 socket(AF_INET, SOCK_STREAM, IPPROTO_TCP) = 7",
             "12345 1700000000.5 recvfrom(7, \"GET\", 8192, 0, NULL, NULL) = 78",
             "[pid  4242] 10:00:01.000002 sendto(0x1f, \"HTTP\", 12, 0, NULL, 0) = 12",
             "[pid 4242] 1.1234567 accept4(3, {sa_family=AF_INET}, [16], SOCK_CLOEXEC) = 9",
             "1.0 recvfrom(7,  <unfinished ...>", "1.0 <... recvfrom resumed>\"x\", 8192, 0, NULL, NULL) = 1",
             "1.0 socket(AF_INET, SOCK_STREAM, 0 <unfinished ...>", "1.0 <... socket resumed>) = 12",
             "1.0 recvfrom(7, 0x7f, 8192, 0, NULL, NULL) = -1 EAGAIN (Resource temporarily unavailable)",
             "1.0 close(7) = 0\r", "1.0 --- SIGCHLD {si_signo=SIGCHLD} ---", "garbage", "", "   ",
             "1.0 " + "x" * 300 + "(1) = 2", "2.0 sendto(5, \"a\", 1, 0, NULL, 0) = 1"]
    _check(rv, "\n".join(lines))                    # last line without a newline
    _check(rv, "\n".join(lines) + "\n")
    _check(rv, "1.0 socket(AF_INET, 1, 0) = 5")     # one line, no newline
    key, _, _ = rv.parse_strace("", GPU_RULES)
    assert key.numel() == 0


def _pad_line(n):
    """A dropped line of exactly n bytes before its newline (n >= 4)."""
    return "1.0 " + "z" * (n - 4)


def test_lines_on_tile_edges(rv):
    """The front end stages text in tiles of 8 KiB: lines that end on the last
    byte of a tile, start on its first byte, or cross its edge."""
    ev = ["1.0 socket(AF_INET, SOCK_STREAM, IPPROTO_TCP) = 7", "1.5 recvfrom(7, \"a\", 1, 0, NULL, NULL) = 1"]
    for shift in list(range(-3, 4)) + [-len(ev[0]) - 1, -len(ev[0])]:
        pad = 8192 - 1 + shift                       # newline of the pad line at byte 8191 + shift
        text = "\n".join([_pad_line(pad)] + ev * 300) + "\n"
        _check(rv, text)
        _check(rv, text[:-1])
    # an event line exactly filling one tile, then one exactly filling the next
    fill = "1.0 sendto(5, \"" + "q" * (8191 - 36) + "\", 1, 0, NULL, 0) = 1"
    assert len(fill) == 8191
    _check(rv, "\n".join([fill, fill, ev[1]]))


def test_lines_longer_than_the_window(rv):
    """Lines longer than a tile plus its 1 KiB overhang are parsed from global
    memory; they may start anywhere in a tile."""
    long_ev = "2.0 sendto(9, \"" + "L" * 20000 + "\", 20000, 0, NULL, 0) = 20000"
    long_drop = "2.0 write(1, \"" + "D" * 9500 + "\", 9500) = 9500"
    short = "3.0 recvfrom(9, \"x\", 1, 0, NULL, NULL) = 1"
    for lead in (0, 1, 100, 8000, 8191, 8192):
        text = "\n".join([_pad_line(max(4, lead))] * (lead > 0) + [long_ev, short, long_drop, long_ev] + [short] * 50)
        _check(rv, text)
        _check(rv, text + "\n")
    _check(rv, long_ev)                                 # the whole text one long line, no newline


def test_unaligned_text_and_capacity(rv):
    import torch
    tr = synth.socket_trace(20_000, 300, n_pending=10, seed=125)
    text = synth.strace_log(tr, seed=126)
    raw = torch.frombuffer(bytearray(b"#" + text.encode()), dtype=torch.uint8).cuda()
    dev = raw[1:]                                       # the text starts one byte past a 16-byte boundary
    assert dev.data_ptr() % 16 == 1
    key, pred, ts = rv.parse_strace(dev, GPU_RULES)
    k, c, t = strace.parse(text, RULES)
    assert key.cpu().numpy().view(np.uint32).tolist() == [x & 0xFFFFFFFF for x in k]
    assert pred.cpu().numpy().tolist() == c and ts.cpu().numpy().tolist() == t
    with pytest.raises(RuntimeError, match="capacity"):
        rv.parse_strace(text, GPU_RULES, capacity=len(k) - 1)


def test_full_size_log_equals_its_trace(rv):
    """The bench's log (a 1e6-event Zipf socket trace, 152 MB of strace text
    with dropped lines and split calls) parsed on the GPU gives back exactly
    the events of the trace that wrote it, in order."""
    import torch
    import bench
    tr = synth.socket_trace(1_000_000, 10_000, pending_frac=0.03, zipf_s=1.1, seed=6000)
    text = synth.strace_log(tr, seed=6001)
    dev = torch.frombuffer(bytearray(text.encode()), dtype=torch.uint8).cuda()
    key, pred, ts = rv.parse_strace(dev, GPU_RULES, capacity=tr.n + 16)
    assert key.numel() == tr.n
    assert (key.cpu().numpy().view(np.uint32) == tr.key).all()
    assert (pred.cpu().numpy() == tr.pred).all()
    t = ts.cpu().numpy()
    assert (np.diff(t) >= 0).all()
