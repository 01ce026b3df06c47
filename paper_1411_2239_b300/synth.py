"""Seeded synthetic event traces shaped like the paper's case studies.

This module only draws inputs: it holds none of the verification arithmetic
and imports nothing else from the package, so both the CUDA path's tests and
the CPU oracle can use it.  Every trace is a structure of arrays in trace
order (the order the paper's semantics uses, Sec. 2 "Trace"):

    ts   uint32[n]   non-decreasing timestamps
    pred uint8[n]    predicate code (index into ``codes``)
    key  uint32[n]   binding key (one quantified variable), or
         uint64[n]   (d0 << 32) | d1 for two variables

The paper's datasets (Apache/strace, Dropbox, YouTube; Sec. 5.1) are not
available, so these stand in for them:

  socket_trace   -- case study 1 shape: per socket id, a ``socket`` event, then
                    alternating ``receive``/``respond``; an exact number of
                    sockets end with an unanswered receive.  Socket ids are
                    drawn uniformly or from a Zipf law over ranks.
  file_trace     -- nested two-variable shape (users x files): per (user, file)
                    pair an ``open``, then ``read``/``user`` noise, then ``close``
                    unless the pair leaked; log-normal events per pair; an exact
                    share of users leak 4..8 pairs, the others 0..3.
  batch_traces   -- many independent traces of log-uniform length with uniform
                    keys (about 64 events per key) over 2..6 predicate codes.
  random_body    -- random LTL bodies (G/F/U/X nestings) over given names.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SOCKET_CODES = ["socket", "receive", "respond"]
FILE_CODES = ["open", "close", "read", "user"]


@dataclass
class Trace:
    ts: np.ndarray
    pred: np.ndarray
    key: np.ndarray
    codes: list
    meta: dict = field(default_factory=dict)
    value: np.ndarray = None      # optional per-event value column (uint32)

    @property
    def n(self):
        return len(self.pred)


def _timestamps(rng, n):
    return np.cumsum(rng.integers(0, 3, size=n, dtype=np.uint32), dtype=np.uint32)


def _rank_within_key(key_idx, n_keys):
    """Occurrence number of each event within its key (0 for the first)."""
    order = np.argsort(key_idx, kind="stable")
    counts = np.bincount(key_idx, minlength=n_keys)
    starts = np.zeros(n_keys + 1, dtype=np.int64)
    np.cumsum(counts, out=starts[1:])
    rank = np.empty(len(key_idx), dtype=np.int64)
    rank[order] = np.arange(len(key_idx), dtype=np.int64) - np.repeat(starts[:-1], counts)
    return rank, counts, order, starts


def socket_trace(n, n_ids, pending_frac=None, n_pending=None, zipf_s=None, seed=0, ids=None):
    """Case-study-1-shaped trace (see module docstring).

    ``n_pending`` (or ``pending_frac`` of the sockets that appear with at least
    two events) sockets end with a receive that is never answered.  ``ids``
    (n_ids distinct uint32) replaces the random socket ids, e.g. to give
    several slices of one trace disjoint ids."""
    rng = np.random.default_rng(seed)
    drawn = rng.choice(np.iinfo(np.uint32).max, size=n_ids, replace=False).astype(np.uint32)
    ids = drawn if ids is None else np.asarray(ids, dtype=np.uint32)
    assert len(ids) == n_ids
    if zipf_s is None:
        kidx = rng.integers(0, n_ids, size=n, dtype=np.int64)
    else:
        w = np.arange(1, n_ids + 1, dtype=np.float64) ** (-zipf_s)
        cdf = np.cumsum(w)
        cdf /= cdf[-1]
        kidx = np.searchsorted(cdf, rng.random(n)).astype(np.int64)
        np.minimum(kidx, n_ids - 1, out=kidx)
    rank, counts, order, starts = _rank_within_key(kidx, n_ids)
    pred = np.where(rank == 0, 0, np.where(rank % 2 == 1, 1, 2)).astype(np.uint8)
    eligible = np.flatnonzero(counts >= 2)
    if n_pending is None:
        n_pending = int(round((pending_frac or 0.0) * len(eligible)))
    pend = rng.choice(eligible, size=min(n_pending, len(eligible)), replace=False)
    last = order[starts[1:][counts >= 1] - 1]                 # last event of each appearing key
    last_key = kidx[last]
    pending_mask = np.zeros(n_ids, dtype=bool)
    pending_mask[pend] = True
    two = counts[last_key] >= 2
    pred[last[two & pending_mask[last_key]]] = 1               # unanswered receive
    pred[last[two & ~pending_mask[last_key]]] = 2              # answered
    meta = {"n_ids": n_ids, "appearing": int((counts > 0).sum()), "pending_ids": ids[pend],
            "max_cluster": int(counts.max()) if n else 0, "zipf_s": zipf_s}
    return Trace(_timestamps(rng, n), pred, ids[kidx], list(SOCKET_CODES), meta)


def file_trace(n_target, n_users, n_files, pairs_per_user=200, mean_events=10.0, sigma=1.5,
               leak_user_frac=0.02, seed=0):
    """Nested two-variable trace: key = (user << 32) | file.

    Events per (user, file) pair are 2 + floor(exp(mu + sigma Z)) with mu set so
    that their mean is about ``mean_events``; the pair count is chosen so that
    the trace has about ``n_target`` events.  Each pair opens first; ``close``
    ends it unless the pair leaked.  A share ``leak_user_frac`` of the users
    leak 4..8 pairs, every other user 0..3."""
    rng = np.random.default_rng(seed)
    mu = np.log(max(mean_events - 2.0, 0.5)) - sigma * sigma / 2.0
    n_pairs = max(1, int(n_target / mean_events))
    users = rng.choice(np.iinfo(np.uint32).max, size=n_users, replace=False).astype(np.uint64)
    # every user gets at least one pair, the rest are spread uniformly
    p_user = np.concatenate([np.arange(n_users), rng.integers(0, n_users, size=max(0, n_pairs - n_users))])
    p_user.sort()
    p_file = rng.integers(0, n_files, size=len(p_user)).astype(np.uint64)
    key = (p_user.astype(np.uint64) << np.uint64(32)) | p_file
    key, first = np.unique(key, return_index=True)              # distinct (user, file) pairs
    p_user = p_user[first]
    n_pairs = len(key)
    lens = 2 + np.floor(np.exp(mu + sigma * rng.standard_normal(n_pairs))).astype(np.int64)
    # leaks: choose the number of leaked pairs of every user
    per_user = np.bincount(p_user, minlength=n_users)
    violators = rng.random(n_users) < leak_user_frac
    want = np.where(violators, rng.integers(4, 9, size=n_users), rng.integers(0, 4, size=n_users))
    want = np.minimum(want, per_user)
    pstart = np.zeros(n_users + 1, dtype=np.int64)
    np.cumsum(per_user, out=pstart[1:])
    within = np.arange(n_pairs) - pstart[p_user]
    leaked = within < want[p_user]
    # lay events out pair-major, then interleave by random times
    off = np.zeros(n_pairs + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    n = int(off[-1])
    pair_of = np.repeat(np.arange(n_pairs), lens)
    pos = np.arange(n, dtype=np.int64) - off[pair_of]
    pred = rng.choice(np.array([2, 3], dtype=np.uint8), size=n)            # read / user noise
    pred[pos == 0] = 0                                                      # open first
    last = off[1:] - 1
    pred[last[~leaked]] = 1                                                 # close
    # per-pair increasing times inside a random window, then one global sort
    start = rng.random(n_pairs)
    width = rng.random(n_pairs) * (1.0 - start)
    csum = np.cumsum(rng.exponential(size=n))
    base = np.concatenate([[0.0], csum[off[1:-1] - 1]])
    tot = csum[off[1:] - 1] - base + rng.exponential(size=n_pairs)
    t = start[pair_of] + width[pair_of] * (csum - base[pair_of]) / tot[pair_of]
    del csum, pos
    order = np.argsort(t, kind="stable")
    del t
    full_key = (users[p_user] << np.uint64(32)) | (key & np.uint64(0xFFFFFFFF))
    meta = {"n_users": n_users, "n_pairs": n_pairs, "violating_users": users[violators & (want >= 4)],
            "leaked_pairs": int(leaked.sum())}
    return Trace(_timestamps(rng, n), pred[order], full_key[pair_of[order]], list(FILE_CODES), meta)


CHUNK_CODES = ["user", "upload"]


def chunk_trace(n, n_users, max_chunk=4 << 20, heavy_frac=0.05, seed=0):
    """Case-study-2-shaped trace (personal cloud storage uploads): events of
    uniformly chosen users, each carrying a chunk size; a user's first event
    is ``user``, the others ``upload``.  The value column is the average chunk
    size of the user's session so far (integer), the program variable the
    case study's avg_chunksize predicate reads.  A share ``heavy_frac`` of the
    users upload chunks of the maximum size only; the others draw sizes
    log-uniformly in [4 KiB, max_chunk]."""
    rng = np.random.default_rng(seed)
    users = rng.choice(np.iinfo(np.uint32).max, size=n_users, replace=False).astype(np.uint32)
    kidx = rng.integers(0, n_users, size=n, dtype=np.int64)
    heavy = rng.random(n_users) < heavy_frac
    size = np.exp(rng.uniform(np.log(4096), np.log(max_chunk), size=n)).astype(np.uint64)
    size[heavy[kidx]] = max_chunk
    rank, counts, order, starts = _rank_within_key(kidx, n_users)
    csum = np.cumsum(size[order])
    before = np.where(starts[:-1] > 0, csum[np.maximum(starts[:-1] - 1, 0)], 0).astype(np.uint64)
    run = np.empty(n, dtype=np.uint64)
    run[order] = csum - np.repeat(before, counts)
    avg = (run // (rank.astype(np.uint64) + 1)).astype(np.uint32)
    pred = np.where(rank == 0, 0, 1).astype(np.uint8)
    meta = {"heavy_users": users[heavy & (counts > 0)], "appearing": int((counts > 0).sum()), "max_chunk": max_chunk}
    return Trace(_timestamps(rng, n), pred, users[kidx], list(CHUNK_CODES), meta, avg)


def batch_traces(n_traces, min_len=1_000, max_len=10_000_000, per_key=64, seed=0):
    """Independent traces with log-uniform lengths and uniform keys."""
    rng = np.random.default_rng(seed)
    lens = np.exp(rng.uniform(np.log(min_len), np.log(max_len), size=n_traces)).astype(np.int64)
    out = []
    for n in lens:
        n = int(n)
        n_codes = int(rng.integers(2, 7))
        nk = max(1, -(-n // per_key))
        ids = rng.choice(np.iinfo(np.uint32).max, size=nk, replace=False).astype(np.uint32)
        key = ids[rng.integers(0, nk, size=n)]
        pred = rng.integers(0, n_codes, size=n).astype(np.uint8)
        codes = [f"p{j}" for j in range(n_codes)]
        out.append(Trace(_timestamps(rng, n), pred, key, codes, {"n_keys": nk}))
    return out


def random_body(rng, names, depth=3):
    """A random LTL body over the given proposition names (G/F/U/X nestings)."""
    def atom():
        a = names[int(rng.integers(len(names)))]
        return a if rng.random() < 0.7 else f"!{a}"

    def gen(d):
        if d == 0:
            return atom()
        r = rng.random()
        if r < 0.18:
            return f"G({gen(d - 1)})"
        if r < 0.36:
            return f"F({gen(d - 1)})"
        if r < 0.5:
            return f"X({gen(d - 1)})"
        if r < 0.68:
            return f"({gen(d - 1)}) U ({gen(d - 1)})"
        if r < 0.84:
            return f"({gen(d - 1)}) && ({gen(d - 1)})"
        return f"({gen(d - 1)}) -> ({gen(d - 1)})"
    return gen(depth)


def random_quantifier(rng):
    """A random single quantifier prefix text, A with a percentage or E with a count."""
    ops = ["<", "<=", ">", ">=", "="]
    op = ops[int(rng.integers(len(ops)))]
    if rng.random() < 0.5:
        return f"A_{{{op}{int(rng.integers(0, 21)) * 5}%}}"
    return f"E_{{{op}{int(rng.integers(0, 9))}}}"


def strace_log(trace, seed=0, noise=0.3, split=0.1, fmt="ttt"):
    """strace text of a socket trace (codes socket / receive / respond): each
    event becomes a socket(...) = id, recvfrom(id, ...) or sendto(id, ...) line;
    between them come lines the front end must drop (other calls, failed
    receives, signals, exits) and, for a share ``split`` of the events, the
    call is cut into an unfinished and a resumed half with another line in
    between.  Timestamps: strace -ttt or -tt format, microseconds."""
    if not 0.0 <= noise < 1.0:
        raise ValueError("noise is the probability of one more dropped line: it must lie in [0, 1)")
    rng = np.random.default_rng(seed)
    pids = rng.integers(1000, 99999, size=4)
    t0 = 1_700_000_000 * 1_000_000
    out = []

    def stamp(t):
        sec, us = divmod(int(t), 1_000_000)
        if fmt == "ttt":
            return f"{sec}.{us:06d}"
        h, rem = divmod(sec % 86400, 3600)
        return f"{h:02d}:{rem // 60:02d}:{rem % 60:02d}.{us:06d}"

    def pid():
        p = int(pids[int(rng.integers(len(pids)))])
        return f"[pid {p:5d}] " if rng.random() < 0.5 else f"{p} "

    noise_lines = ["epoll_wait(4, [], 512, 0) = 0", "futex(0x7f3a2c0, FUTEX_WAKE_PRIVATE, 1) = 1",
                   "mmap(NULL, 8192, PROT_READ|PROT_WRITE, MAP_PRIVATE|MAP_ANONYMOUS, -1, 0) = 0x7f3a2c000000",
                   "recvfrom(9, 0x7ffd, 8192, 0, NULL, NULL) = -1 EAGAIN (Resource temporarily unavailable)",
                   "--- SIGCHLD {si_signo=SIGCHLD, si_code=CLD_EXITED, si_pid=4242} ---",
                   "+++ exited with 0 +++", "close(11) = 0", "accept4(3, NULL, NULL, SOCK_CLOEXEC) = -1 EAGAIN (x)"]
    t = t0
    for key, code in zip(trace.key.tolist(), trace.pred.tolist()):
        t += int(rng.integers(1, 50))
        while rng.random() < noise:
            out.append(f"{pid()}{stamp(t)} {noise_lines[int(rng.integers(len(noise_lines)))]}")
        n = int(rng.integers(1, 4000))
        if code == 0:
            head, tail = "socket(AF_INET, SOCK_STREAM, IPPROTO_TCP", f") = {key}"
            name = "socket"
        elif code == 1:
            head, tail = f'recvfrom({key}, "GET /index.html HTTP/1.1\r\n"..., 8192, 0, NULL', f", NULL) = {n}"
            name = "recvfrom"
        else:
            head, tail = f'sendto({key}, "HTTP/1.1 200 OK\r\n"..., {n}, MSG_NOSIGNAL, NULL', f", 0) = {n}"
            name = "sendto"
        if rng.random() < split:
            p = pid()
            out.append(f"{p}{stamp(t)} {head} <unfinished ...>")
            out.append(f"{pid()}{stamp(t)} {noise_lines[0]}")
            out.append(f"{p}{stamp(t + 1)} <... {name} resumed>{tail}")
        else:
            out.append(f"{pid()}{stamp(t)} {head}{tail}")
    return "\n".join(out) + "\n"

