"""Four-valued LTL (Def. "LTL4 semantics", Sec. 2.2.2).  Test infrastructure only.

[u |=_4 f] is
  T   if every infinite continuation v (v in Sigma^omega) has uv |= f,
  F   if no continuation has uv |= f,
  Tp  otherwise, when [u |=_F f] holds (finite-trace LTL, module fltl),
  Fp  otherwise.

The two quantifications over Sigma^omega are decided here without any
automaton for f:

1. Progression.  For an infinite word, uv |= f iff v |= prog(f, u), where
   prog rewrites a formula through one letter:
     prog(p, a) = true if p in a else false,  prog(X f, a) = f,
     prog(f U g, a) = prog(g, a) || (prog(f, a) && f U g),
   and distributes over !, &&, ||.  Residuals are kept modulo
   associativity, commutativity and idempotence of && and || (n-ary frozensets),
   which keeps the set of residuals of a formula finite.
2. Satisfiability of the residual r over Sigma^omega by the textbook atom
   tableau (Lichtenstein and Pnueli): an atom is a letter plus a truth value for
   every X- and U-subformula of r; atom A may be followed by atom B when every
   X g in A agrees with g in B and every f U g in A obeys the expansion law
   f U g = g || (f && X(f U g)).  r is satisfiable iff an atom containing r
   reaches a non-trivial strongly connected component in which every until that
   occurs is fulfilled (its right operand holds in some atom of the component).

Then every continuation satisfies f iff !r is unsatisfiable, and none does iff
r is unsatisfiable.  Sigma is the set of letters the trace can produce (the
schema's effective alphabet): continuations are drawn from it.
"""
from __future__ import annotations

from itertools import product

from . import fltl

TRUE = ("true",)
FALSE = ("false",)

# T, F, Tp, Fp as their codes in the six-valued lattice F < Fc < Fp < Tp < Tc < T
B4_TOP, B4_BOT, B4_TOP_P, B4_BOT_P = 5, 0, 3, 2


# ---------------------------------------------------------------- normal form
def mk_not(f):
    if f == TRUE:
        return FALSE
    if f == FALSE:
        return TRUE
    if f[0] == "not":
        return f[1]
    return ("not", f)


def _mk_nary(kind, items):
    unit, zero = (TRUE, FALSE) if kind == "AND" else (FALSE, TRUE)
    flat = set()
    for g in items:
        if g == unit:
            continue
        if g == zero:
            return zero
        if g[0] == kind:
            flat |= g[1]
        else:
            flat.add(g)
    for g in flat:
        if mk_not(g) in flat:
            return zero
    if not flat:
        return unit
    if len(flat) == 1:
        return next(iter(flat))
    return (kind, frozenset(flat))


def mk_and(items):
    return _mk_nary("AND", items)


def mk_or(items):
    return _mk_nary("OR", items)


def norm(f):
    """Core AST (binary and/or) -> normal form with n-ary AND/OR."""
    op = f[0]
    if op in ("true", "false", "ap"):
        return f
    if op == "not":
        return mk_not(norm(f[1]))
    if op == "and":
        return mk_and([norm(f[1]), norm(f[2])])
    if op == "or":
        return mk_or([norm(f[1]), norm(f[2])])
    if op == "X":
        return ("X", norm(f[1]))
    if op == "U":
        return ("U", norm(f[1]), norm(f[2]))
    raise ValueError(op)


# ---------------------------------------------------------------- progression
def progress(f, letter: frozenset):
    op = f[0]
    if op in ("true", "false"):
        return f
    if op == "ap":
        return TRUE if f[1] in letter else FALSE
    if op == "not":
        return mk_not(progress(f[1], letter))
    if op == "AND":
        return mk_and([progress(g, letter) for g in f[1]])
    if op == "OR":
        return mk_or([progress(g, letter) for g in f[1]])
    if op == "X":
        return f[1]
    if op == "U":
        return mk_or([progress(f[2], letter), mk_and([progress(f[1], letter), f])])
    raise ValueError(op)


# ---------------------------------------------------------------- tableau
def _closure(f, acc):
    if f in acc:
        return
    op = f[0]
    if op in ("AND", "OR"):
        for g in f[1]:
            _closure(g, acc)
    elif op in ("not", "X"):
        _closure(f[1], acc)
    elif op == "U":
        _closure(f[1], acc)
        _closure(f[2], acc)
    acc[f] = None        # children first


def satisfiable(r, sigma) -> bool:
    """Is there w in sigma^omega with w |= r?  sigma: iterable of frozensets of APs."""
    if r == TRUE:
        return True
    if r == FALSE:
        return False
    order = {}
    _closure(r, order)
    nodes = list(order)
    temporal = [g for g in nodes if g[0] in ("X", "U")]
    xs = [g for g in temporal if g[0] == "X"]
    us = [g for g in temporal if g[0] == "U"]

    def evaluate(letter, choice):
        val = dict(zip(temporal, choice))
        for g in nodes:
            op = g[0]
            if op in ("X", "U"):
                continue
            if op == "true":
                val[g] = True
            elif op == "false":
                val[g] = False
            elif op == "ap":
                val[g] = g[1] in letter
            elif op == "not":
                val[g] = not val[g[1]]
            elif op == "AND":
                val[g] = all(val[h] for h in g[1])
            elif op == "OR":
                val[g] = any(val[h] for h in g[1])
        return val

    atoms = []
    for letter in sigma:
        for choice in product((False, True), repeat=len(temporal)):
            atoms.append(evaluate(letter, choice))

    # successors: B may follow A iff X g in A <-> g in B, and the expansion law
    # f U g in A <-> (g in A or (f in A and f U g in B)).  Atoms are indexed by
    # the part of their valuation that a predecessor constrains.
    by_sig = {}
    for j, b in enumerate(atoms):
        sig = tuple(b[x[1]] for x in xs) + tuple(b[u] for u in us)
        by_sig.setdefault(sig, []).append(j)
    succ = [[] for _ in atoms]
    for i, a in enumerate(atoms):
        xpart = tuple(a[x] for x in xs)
        allowed = []
        for u in us:
            allowed.append([bu for bu in (False, True)
                            if a[u] == (a[u[2]] or (a[u[1]] and bu))])
        for upart in product(*allowed):
            succ[i].extend(by_sig.get(xpart + tuple(upart), ()))

    comp = _scc(len(atoms), succ)
    members = {}
    for i, c in enumerate(comp):
        members.setdefault(c, []).append(i)
    good = set()
    for c, mem in members.items():
        nontrivial = len(mem) > 1 or mem[0] in succ[mem[0]]
        if not nontrivial:
            continue
        fulfilled = all(any(atoms[k][u[2]] for k in mem)
                        for u in us if any(atoms[k][u] for k in mem))
        if fulfilled:
            good.add(c)
    # atoms that reach a good component
    pred = [[] for _ in atoms]
    for i, s in enumerate(succ):
        for j in s:
            pred[j].append(i)
    live = set(i for i, c in enumerate(comp) if c in good)
    stack = list(live)
    while stack:
        j = stack.pop()
        for i in pred[j]:
            if i not in live:
                live.add(i)
                stack.append(i)
    return any(atoms[i][r] for i in live)


def _scc(n, succ):
    """Tarjan's strongly connected components (iterative); returns component ids."""
    index, low, comp = [None] * n, [0] * n, [None] * n
    onstack, stack, counter, ncomp = [False] * n, [], 0, 0
    for root in range(n):
        if index[root] is not None:
            continue
        work = [(root, 0)]
        while work:
            v, k = work.pop()
            if k == 0:
                index[v] = low[v] = counter
                counter += 1
                stack.append(v)
                onstack[v] = True
            if k < len(succ[v]):
                work.append((v, k + 1))
                w = succ[v][k]
                if index[w] is None:
                    work.append((w, 0))
                elif onstack[w]:
                    low[v] = min(low[v], index[w])
                continue
            if low[v] == index[v]:
                while True:
                    w = stack.pop()
                    onstack[w] = False
                    comp[w] = ncomp
                    if w == v:
                        break
                ncomp += 1
            if work:
                parent = work[-1][0]
                low[parent] = min(low[parent], low[v])
    return comp


# ---------------------------------------------------------------- verdicts
class LTL4:
    """Evaluator of [u |=_4 psi] for one body psi over one effective alphabet."""

    def __init__(self, body_core, letter_sets):
        # letter_sets[i]: frozenset of the body's APs true in letter i
        self.body = body_core
        self.letter_sets = [frozenset(s) for s in letter_sets]
        self.sigma = sorted(set(self.letter_sets), key=sorted)
        self.start = norm(body_core)
        aps = set()
        for s in self.letter_sets:
            aps |= s
        from .formula import body_aps
        aps |= body_aps(body_core)
        import numpy as np
        self.ap_truth = {p: np.array([p in s for s in self.letter_sets], dtype=bool) for p in aps}
        self._step = {}
        self._sat = {}

    def residual(self, letters):
        r = self.start
        step = self._step
        for lid in letters:
            key = (r, lid)
            nxt = step.get(key)
            if nxt is None:
                nxt = progress(r, self.letter_sets[lid])
                step[key] = nxt
            r = nxt
        return r

    def sat(self, r):
        v = self._sat.get(r)
        if v is None:
            v = satisfiable(r, self.sigma)
            self._sat[r] = v
        return v

    def definite(self, r):
        """T / F if the residual decides every continuation, else None."""
        if not self.sat(mk_not(r)):
            return B4_TOP
        if not self.sat(r):
            return B4_BOT
        return None

    def verdict(self, letters) -> int:
        """[u |=_4 psi] as a code in {0 (F), 2 (Fp), 3 (Tp), 5 (T)}."""
        d = self.definite(self.residual(letters))
        if d is not None:
            return d
        return B4_TOP_P if fltl.holds(self.body, letters, self.ap_truth) else B4_BOT_P
