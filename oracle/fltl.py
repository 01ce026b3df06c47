"""Finite-trace LTL (Def. "FLTL semantics", Sec. 2.2.1).  Test infrastructure only.

[u |=_F X f] is [u_1 |=_F f] when the suffix u_1 is non-empty and false
otherwise (strong next).  [u |=_F f U g] holds iff some k in [0, n-1] has g at
k and f at every l in [0, k).  Atomic propositions and Boolean connectives are
as in LTL.  F and G are derived (F f = true U f, G f = !F !f), so they arrive
here already rewritten by ``formula.core``.

A word is given as an integer array of letter ids plus ``ap_truth``: for each
atomic proposition name, a boolean array indexed by letter id.  Every
subformula is evaluated at every position of the word, bottom-up:

  * X f at i is f at i+1, and false at the last position;
  * f U g at i: look at the first position j >= i where g holds or f fails.
    The until holds iff such a j exists and g holds there (if g holds at j,
    then j is a witness k; if f fails at j first, no later k can work, because
    f must hold at every position before k).
"""
from __future__ import annotations

import numpy as np


def evaluate(f, letters: np.ndarray, ap_truth: dict, memo=None) -> np.ndarray:
    """Boolean array over positions: entry i is [u^(i) |=_F f], u^(i) the suffix at i."""
    if memo is None:
        memo = {}
    if f in memo:
        return memo[f]
    n = len(letters)
    op = f[0]
    if op == "true":
        r = np.ones(n, dtype=bool)
    elif op == "false":
        r = np.zeros(n, dtype=bool)
    elif op == "ap":
        r = ap_truth[f[1]][letters]
    elif op == "not":
        r = ~evaluate(f[1], letters, ap_truth, memo)
    elif op == "and":
        r = evaluate(f[1], letters, ap_truth, memo) & evaluate(f[2], letters, ap_truth, memo)
    elif op == "or":
        r = evaluate(f[1], letters, ap_truth, memo) | evaluate(f[2], letters, ap_truth, memo)
    elif op == "X":
        g = evaluate(f[1], letters, ap_truth, memo)
        r = np.zeros(n, dtype=bool)
        r[:-1] = g[1:]
    elif op == "U":
        a = evaluate(f[1], letters, ap_truth, memo)
        b = evaluate(f[2], letters, ap_truth, memo)
        stop = b | ~a
        pos = np.where(stop, np.arange(n), n)
        first = np.minimum.accumulate(pos[::-1])[::-1]   # first stop at or after i
        r = (first < n) & b[np.minimum(first, n - 1)]
    else:
        raise ValueError(op)
    memo[f] = r
    return r


def holds(f, letters: np.ndarray, ap_truth: dict) -> bool:
    """[u |=_F f] for a non-empty finite word u."""
    if len(letters) == 0:
        raise ValueError("FLTL is only evaluated on non-empty traces")
    return bool(evaluate(f, np.asarray(letters), ap_truth)[0])
