"""Per-event verdict timeline of a trace.  Test infrastructure only.

Algorithm 1's online mode (Sec. 4.2) gives an evolving verdict as the trace
grows.  At event granularity: for event j whose innermost value vector is D
(Sec. 2.4.1), the verdict is [u^D_{<=j} |=_4 psi], the LTL4 verdict (Def.
"LTL4 semantics", module ltl4) of D's projection (Sec. 2.4.3) cut after
event j.  A binding's first violation is the first event at which that
verdict is F; F is permanent, so afterwards it stays F.

The residual of each prefix is obtained by progressing the previous prefix's
residual through the new letter (the same rewriting ltl4 applies letter by
letter); the FLTL bit of each prefix is evaluated on the whole prefix.
"""
from __future__ import annotations

import numpy as np

from . import fltl
from .ltl4 import B4_BOT, B4_BOT_P, B4_TOP_P, progress
from .verify import Checker, Schema, value_vectors


def timeline(formula, schema: Schema, keys, preds, values=None):
    """(verdicts, first_violation): verdicts[j] is the code (0 F, 2 Fp, 3 Tp,
    5 T) of event j's binding after event j; first_violation maps each
    binding's value vector (a tuple) to the index of its first F event."""
    ck = Checker(formula, schema)
    preds = np.asarray(preds)
    ck.check_preds(preds)
    preds = ck.letters(preds, values)
    n = len(preds)
    nq = len(ck.formula.quants)
    L = ck.ltl4
    vv = value_vectors(nq, keys) if nq else np.zeros((n, 0), dtype=np.uint64)
    groups = {}
    for j in range(n):
        groups.setdefault(tuple(int(x) for x in vv[j]), []).append(j)
    verdicts = np.zeros(n, dtype=np.uint8)
    first = {}
    for D, idx in groups.items():
        letters = preds[idx].astype(np.int64)
        r = L.start
        for k, j in enumerate(idx):
            r = progress(r, L.letter_sets[letters[k]])
            d = L.definite(r)
            if d is None:
                d = B4_TOP_P if fltl.holds(L.body, letters[:k + 1], L.ap_truth) else B4_BOT_P
            verdicts[j] = d
            if d == B4_BOT and D not in first:
                first[D] = j
    return verdicts, first
