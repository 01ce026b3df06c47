"""[u |=_6 phi] for a whole trace: the result the method computes.  Test infrastructure only.

Steps, in the paper's order (Sec. 2.4 and Sec. 3):

1. Variable valuation (Sec. 2.4.1).  Every event j carries a value for each
   quantified variable; D_j is the value vector of event j.  The binding
   predicate p_i(d_i) is read as "event j carries value d_i for x_i" (key
   presence), so the set of value vectors of Eq. D is {D_j}.  A trace has one
   key column: with one variable it is the key itself; with two it is a 64-bit
   word (d_0 << 32) | d_1.
2. Projection (Sec. 2.4.3): u^D is the subsequence of events whose value
   vector is D, in trace (array) order.
3. Property instances of the innermost level are LTL4 properties evaluated on
   their projections (module ltl4).  Letters: with the one-hot alphabet the
   predicate code c of an event is the letter {name(c)} restricted to the
   propositions of the body; with the bitmask alphabet bit i of the code means
   proposition name(i) holds.
4. Canonical valuations (Sec. 2.4.2): the level-m nodes are the distinct
   prefixes D|^m; the children of a node are given by the parent function P.
5. Bottom-up evaluation (Sec. 3.4): each quantifier node counts its children
   by verdict (the vector v) and applies its constraint (module counting).
   The root's verdict is the verdict of the trace.
"""
from __future__ import annotations

import re
from dataclasses import dataclass, field

import numpy as np

from . import counting
from .formula import Formula, parse
from .ltl4 import LTL4


@dataclass
class Schema:
    code_names: list          # name of each predicate code
    alphabet: str = "onehot"  # 'onehot' or 'bitmask'
    value_name: str = None    # name of the events' value column (comparison atoms)

    @property
    def n_letters(self):
        return len(self.code_names) if self.alphabet == "onehot" else 1 << len(self.code_names)


def letter_sets(schema: Schema, aps) -> list:
    """Letter id -> frozenset of body propositions true in that letter."""
    aps = set(aps)
    out = []
    for lid in range(schema.n_letters):
        if schema.alphabet == "onehot":
            s = {schema.code_names[lid]}
        else:
            s = {nm for i, nm in enumerate(schema.code_names) if (lid >> i) & 1}
        out.append(frozenset(s & aps))
    return out


@dataclass
class Result:
    root: int
    root_counts: list
    level_counts: list = field(default_factory=list)   # [m]: verdict histogram of level-(m+1) nodes
    n_nodes: list = field(default_factory=list)        # [m]: number of level-(m+1) nodes
    verdicts: list = field(default_factory=list)       # [m]: {value vector prefix: verdict}


def value_vectors(n_vars: int, keys: np.ndarray):
    """Per-event value vectors as an (n, n_vars) integer array."""
    keys = np.asarray(keys)
    if n_vars == 0:
        return np.zeros((len(keys), 0), dtype=np.uint64)
    if n_vars == 1:
        return keys.astype(np.uint64).reshape(-1, 1)
    if n_vars == 2:
        k = keys.astype(np.uint64)
        return np.stack([k >> np.uint64(32), k & np.uint64(0xFFFFFFFF)], axis=1)
    raise ValueError("at most two quantified variables")


_CMP_ATOM = re.compile(r"([A-Za-z]\w*?)(<=|>=|<|>|=)(\d+)")
_CMP_FN = {"<": lambda v, c: v < c, "<=": lambda v, c: v <= c, ">": lambda v, c: v > c,
           ">=": lambda v, c: v >= c, "=": lambda v, c: v == c}


class Checker:
    """The formula, schema and LTL4 evaluator of one verification problem.

    Comparison atoms "name~c" hold at an event iff its value compares so with
    c.  Each event is then a letter (its predicate code's propositions plus
    the comparison atoms its value makes true); the letters the trace can
    produce, over which LTL4 quantifies continuations, are every code with
    every set of comparison outcomes that some value in [0, 2^32) gives."""

    def __init__(self, formula, schema: Schema):
        self.formula: Formula = parse(formula) if isinstance(formula, str) else formula
        self.schema = schema
        aps = self.formula.aps()
        self.cmps = sorted(a for a in aps if _CMP_ATOM.fullmatch(a))
        for a in self.cmps:
            if _CMP_ATOM.fullmatch(a).group(1) != schema.value_name:
                raise ValueError(f"comparison atom {a} is not on the schema's value column")
        missing = aps - set(self.cmps) - set(schema.code_names)
        if missing:
            raise ValueError(f"body propositions not in the schema: {sorted(missing)}")
        base = letter_sets(schema, aps - set(self.cmps))
        if not self.cmps:
            self.ltl4 = LTL4(self.formula.body, base)
            self.ext = None
            return
        # outcome sets that some value produces: the atoms are thresholds on one
        # number, so the values 0, 2^32 - 1 and c - 1, c, c + 1 of every
        # constant c meet each of them
        parsed = [_CMP_ATOM.fullmatch(a).groups() for a in self.cmps]
        cand = {0, 0xFFFFFFFF}
        for _, _, c in parsed:
            cand |= {v for v in (int(c) - 1, int(c), int(c) + 1) if 0 <= v <= 0xFFFFFFFF}
        outcomes = sorted({self._outcome(parsed, v) for v in cand})
        sets, self.ext = [], {}
        for code in range(schema.n_letters):
            for o in outcomes:
                self.ext[(code, o)] = len(sets)
                sets.append(frozenset(base[code] | {a for a, on in zip(self.cmps, o) if on}))
        self._parsed = parsed
        self.ltl4 = LTL4(self.formula.body, sets)

    @staticmethod
    def _outcome(parsed, v):
        return tuple(bool(_CMP_FN[op](v, int(c))) for _, op, c in parsed)

    def letters(self, preds, values):
        """Letter of every event: its code, with the comparison outcomes of its value."""
        preds = np.asarray(preds)
        if self.ext is None:
            return preds
        if values is None:
            raise ValueError("the formula compares the value column: values are needed")
        values = np.asarray(values)
        return np.array([self.ext[(int(p), self._outcome(self._parsed, int(v)))] for p, v in zip(preds, values)],
                        dtype=np.int64)

    def check_preds(self, preds):
        preds = np.asarray(preds)
        if preds.size and int(preds.max()) >= self.schema.n_letters:
            raise ValueError("predicate code out of range")

    def instance_verdict(self, letters) -> int:
        """LTL4 verdict of one innermost property instance on its projection."""
        return self.ltl4.verdict(np.asarray(letters, dtype=np.int64))

    def projection(self, keys, D):
        """Indices of u^D (events whose value vector is D), in trace order."""
        vv = value_vectors(len(self.formula.quants), keys)
        mask = np.all(vv == np.asarray(D, dtype=np.uint64).reshape(1, -1), axis=1)
        return np.flatnonzero(mask)

    def run(self, keys, preds, values=None) -> Result:
        preds = np.asarray(preds)
        self.check_preds(preds)
        preds = self.letters(preds, values)
        quants = self.formula.quants
        nq = len(quants)
        if nq == 0:
            if len(preds) == 0:
                raise ValueError("an unquantified property needs a non-empty trace")
            return Result(self.instance_verdict(preds), [0] * 6)
        vv = value_vectors(nq, keys)
        # group events by full value vector, keeping trace order inside a group
        uniq, inverse = np.unique(vv, axis=0, return_inverse=True)
        inverse = inverse.reshape(-1)
        order = np.argsort(inverse, kind="stable")
        bounds = np.searchsorted(inverse[order], np.arange(len(uniq) + 1))
        level = {}
        for b in range(len(uniq)):
            idx = order[bounds[b]:bounds[b + 1]]
            level[tuple(int(x) for x in uniq[b])] = self.instance_verdict(preds[idx])
        verdicts = [None] * nq
        verdicts[nq - 1] = level
        # quantifier nodes, innermost first: node D|^m applies Q_m to its children
        for m in range(nq - 1, -1, -1):
            counts = {}
            for D, b in verdicts[m].items():
                counts.setdefault(D[:m], [0] * 6)[b] += 1
            if m == 0:
                v = counts.get((), [0] * 6)
                root = counting.valuate(quants[0], v)
                break
            verdicts[m - 1] = {P: counting.valuate(quants[m], v) for P, v in counts.items()}
        level_counts, n_nodes = [], []
        for m in range(nq):
            h = [0] * 6
            for b in verdicts[m].values():
                h[b] += 1
            level_counts.append(h)
            n_nodes.append(len(verdicts[m]))
        return Result(root, list(v), level_counts, n_nodes, verdicts)


def verify(formula, schema: Schema, keys, preds, values=None) -> Result:
    return Checker(formula, schema).run(keys, preds, values)
