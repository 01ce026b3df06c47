"""Pins of the oracle's strace front end (no GPU): lines written by hand,
each with the event the format fixes, and the round trip of a generated log."""
import numpy as np

from oracle import strace
from paper_1411_2239_b300 import synth

RULES = [strace.Rule("socket", 0, strace.RET), strace.Rule("recvfrom", 1, strace.ARG0, True),
         strace.Rule("sendto", 2, strace.ARG0, True), strace.Rule("accept4", 0, strace.RET)]
T = {r.name: r for r in RULES}


def test_hand_written_lines():
    cases = [
        ("1700000000.000021 socket(AF_INET, SOCK_STREAM, IPPROTO_TCP) = 7", (7, 0, 1700000000000021)),
        ("12345 1700000000.5 recvfrom(7, \"GET\", 8192, 0, NULL, NULL) = 78", (7, 1, 1700000000500000)),
        ("[pid  4242] 10:00:01.000002 sendto(0x1f, \"HTTP\", 12, 0, NULL, 0) = 12", (31, 2, 36001000002)),
        ("[pid 4242] 1.1234567 accept4(3, {sa_family=AF_INET}, [16], SOCK_CLOEXEC) = 9", (9, 0, 1123456)),
        ("1.0 recvfrom(7,  <unfinished ...>", (7, 1, 1000000)),                    # key in the first half
        ("1.0 <... recvfrom resumed>\"x\", 8192, 0, NULL, NULL) = 1", None),          # ... not in the second
        ("1.0 socket(AF_INET, SOCK_STREAM, 0 <unfinished ...>", None),              # return value still missing
        ("1.0 <... socket resumed>) = 12", (12, 0, 1000000)),
        ("1.0 recvfrom(7, 0x7f, 8192, 0, NULL, NULL) = -1 EAGAIN (Resource temporarily unavailable)", None),
        ("1.0 socket(AF_INET, SOCK_STREAM, 0) = -1 EMFILE (Too many open files)", None),
        ("1.0 close(7) = 0", None),
        ("1.0 --- SIGCHLD {si_signo=SIGCHLD} ---", None),
        ("1.0 +++ exited with 0 +++", None),
        ("garbage", None),
        ("1.0 recvfrom(-1, 0x7f, 1, 0, NULL, NULL) = -1 EBADF (Bad file descriptor)", None),
    ]
    for line, want in cases:
        assert strace.parse_line(line, T) == want, line
        assert strace.parse_line(line + "\r", T) == want, line


def test_unterminated_last_line_and_blank_lines():
    text = "1.0 socket(AF_INET, 1, 0) = 5\n\n2.0 sendto(5, \"a\", 1, 0, NULL, 0) = 1"
    assert strace.parse(text, RULES) == ([5, 5], [0, 2], [1000000, 2000000])


def test_generated_log_round_trips():
    tr = synth.socket_trace(3000, 80, n_pending=4, seed=3)
    for fmt in ("ttt", "tt"):
        k, c, _ = strace.parse(synth.strace_log(tr, seed=4, fmt=fmt), RULES[:3])
        assert (np.array(k, dtype=np.uint32) == tr.key).all() and (np.array(c) == tr.pred).all()
