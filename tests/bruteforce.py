"""Brute-force LTL4 verdicts by enumeration of lasso continuations.

An independent route to [u |=_4 psi] (Def. "LTL4 semantics", Sec. 2.2.2), used
only to pin the oracle.  It never progresses formulas and never builds a
tableau.  Instead:

* The *type* of a position of a word is the set of subformulas of psi that
  hold there.  The type at position i is a function of the letter at i and the
  type at i+1 ("prepend"): X g holds iff g holds at i+1; f U g holds iff g holds
  now, or f holds now and f U g holds at i+1.
* For a cycle w, the types along w^omega are computed exactly, subformula by
  subformula: X g reads the next cycle position; f U g holds at i iff, walking
  forward around the cycle from i, a position with g is met before a position
  without f (at most one lap is needed).
* R_L = all types of v.w^omega with |w| <= L, closed under prepending letters.
  Every ultimately periodic word is covered once L reaches its cycle length,
  and the test checks that R_L no longer grows from L to L+1 before it trusts
  it.
* [u |=_4 psi] = T if psi is in the type of u.t for every t in R_L, F if in
  none, otherwise Tp/Fp by the finite-trace type of u (prepend u onto the
  "end" type in which every X and U formula is false: strong next and bounded
  until of Def. "FLTL semantics").
"""
from __future__ import annotations

import itertools

import numpy as np


class Types:
    def __init__(self, body_core, letter_sets):
        nodes = []

        def walk(f):
            for g in f[1:]:
                if isinstance(g, tuple):
                    walk(g)
            if f not in nodes:
                nodes.append(f)
        walk(body_core)
        self.nodes = nodes
        self.idx = {f: i for i, f in enumerate(nodes)}
        self.root = self.idx[body_core]
        self.letters = [frozenset(s) for s in letter_sets]
        self.types = []          # list of frozenset of node indices
        self.type_id = {}
        self.prep_tab = {}

    def tid(self, t):
        t = frozenset(t)
        if t not in self.type_id:
            self.type_id[t] = len(self.types)
            self.types.append(t)
        return self.type_id[t]

    def prepend(self, lid, nxt_id):
        key = (lid, nxt_id)
        if key in self.prep_tab:
            return self.prep_tab[key]
        letter, nxt = self.letters[lid], self.types[nxt_id]
        val = {}
        for i, f in enumerate(self.nodes):
            op = f[0]
            if op == "true":
                val[i] = True
            elif op == "false":
                val[i] = False
            elif op == "ap":
                val[i] = f[1] in letter
            elif op == "not":
                val[i] = not val[self.idx[f[1]]]
            elif op == "and":
                val[i] = val[self.idx[f[1]]] and val[self.idx[f[2]]]
            elif op == "or":
                val[i] = val[self.idx[f[1]]] or val[self.idx[f[2]]]
            elif op == "X":
                val[i] = self.idx[f[1]] in nxt
            elif op == "U":
                val[i] = val[self.idx[f[2]]] or (val[self.idx[f[1]]] and i in nxt)
        r = self.tid(i for i, v in val.items() if v)
        self.prep_tab[key] = r
        return r

    def cycle_type(self, cyc):
        m = len(cyc)
        val = {}
        for i, f in enumerate(self.nodes):
            op = f[0]
            if op == "true":
                v = [True] * m
            elif op == "false":
                v = [False] * m
            elif op == "ap":
                v = [f[1] in self.letters[a] for a in cyc]
            elif op == "not":
                v = [not x for x in val[self.idx[f[1]]]]
            elif op == "and":
                a, b = val[self.idx[f[1]]], val[self.idx[f[2]]]
                v = [x and y for x, y in zip(a, b)]
            elif op == "or":
                a, b = val[self.idx[f[1]]], val[self.idx[f[2]]]
                v = [x or y for x, y in zip(a, b)]
            elif op == "X":
                g = val[self.idx[f[1]]]
                v = [g[(p + 1) % m] for p in range(m)]
            elif op == "U":
                a, b = val[self.idx[f[1]]], val[self.idx[f[2]]]
                v = []
                for p in range(m):
                    res = False
                    for s in range(m):
                        q = (p + s) % m
                        if b[q]:
                            res = True
                            break
                        if not a[q]:
                            break
                    v.append(res)
            val[i] = v
        return self.tid(i for i in val if val[i][0])

    def realizable(self, max_cycle):
        seen = set()
        for m in range(1, max_cycle + 1):
            for cyc in itertools.product(range(len(self.letters)), repeat=m):
                seen.add(self.cycle_type(cyc))
        frontier = list(seen)
        while frontier:
            t = frontier.pop()
            for lid in range(len(self.letters)):
                u = self.prepend(lid, t)
                if u not in seen:
                    seen.add(u)
                    frontier.append(u)
        return sorted(seen)


def all_verdicts(body_core, letter_sets, max_len, max_cycle=3):
    """{word tuple: verdict code} for every non-empty word of length <= max_len.

    Also returns whether R_L was stable from max_cycle to max_cycle+1."""
    ty = Types(body_core, letter_sets)
    R = ty.realizable(max_cycle)
    R2 = ty.realizable(max_cycle + 1)
    stable = set(R) == set(R2)
    end = ty.tid(())
    cols = np.array(list(R) + [end], dtype=np.int64)
    out = {}
    L = len(letter_sets)

    def holds(tids):
        return np.array([ty.root in ty.types[t] for t in tids], dtype=bool)

    frontier = [((), cols)]
    for _ in range(max_len):
        nxt = []
        for suffix, vec in frontier:
            for a in range(L):
                newvec = np.array([ty.prepend(a, int(t)) for t in vec], dtype=np.int64)
                word = (a,) + suffix
                h = holds(newvec)
                inf, fin = h[:-1], h[-1]
                if inf.all():
                    v = 5
                elif not inf.any():
                    v = 0
                else:
                    v = 3 if fin else 2
                out[word] = v
                nxt.append((word, newvec))
        frontier = nxt
    return out, stable
