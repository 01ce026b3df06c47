"""Syntax of LTL4-C (Def. 1, Sec. 2.1) for the oracle.  Test infrastructure only.

A formula is a string of counting quantifiers followed by a quantifier-free
LTL body (the canonical form of Eq. genprop / Eq. bigq, Sec. 2.4):

    A_{>=0.95} s: socket(s) => G(receive(s) -> F respond(s))
    A u: user(u) => E_{<=3} f: open(u,f) => open && !F close

Quantifier tuple <Q_i, ~_i, c_i, x_i, p_i> (Eq. bigq).  A bare ``A`` means
A_{=1} and a bare ``E`` means E_{>=1} (the defaults stated after Def. 1).  The
constant of an A quantifier is a real in [0,1]; it is kept as an exact
``fractions.Fraction`` parsed from its decimal or percent text, so that the
constraint |B| ~ k*|P| of Eq. S can be decided in integers.  The constant of an
E quantifier is a non-negative integer (the paper writes l in Z+, yet uses
E_{=0} in case study 3, so 0 is admitted).

Body grammar (loosest first): ``<->``, ``->`` (right assoc.), ``||``, ``&&``,
``U``/``R``/``W`` (right assoc.), unary ``!``/``X``/``F``/``G``, atoms
``true``, ``false``, ``name`` or ``name(args)`` (arguments are the bound
variables and are ignored: within a projected trace u^D the predicate instances
of the binding hold by construction, Sec. 2.4.3), and comparisons
``name ~ c`` / ``name(args) ~ c`` of the event's value with an integer
constant (interpreted predicates such as case study 2's
``avg_chunksize(u) <= maximum``, Sec. 5.1), kept as the atom ``name~c``.

The AST is made of plain tuples so that structurally equal formulas are equal:
  ('true',) ('false',) ('ap', name) ('not', f) ('and', f, g) ('or', f, g)
  ('X', f) ('U', f, g)
``core()`` removes the derived operators: F f = true U f, G f = !F !f
(Sec. 2.2.1), f -> g = !f || g, f <-> g = (f && g) || (!f && !g),
f R g = !(!f U !g), f W g = (f U g) || G f.
"""
from __future__ import annotations

import re
from dataclasses import dataclass
from fractions import Fraction

OPS = ("<", "<=", ">", ">=", "=")


class ParseError(ValueError):
    pass


@dataclass(frozen=True)
class Quantifier:
    """One tuple <Q_i, ~_i, c_i, x_i, p_i> of Eq. bigq."""
    kind: str          # 'A' (percentage counting) or 'E' (instance counting)
    op: str            # one of OPS
    const: Fraction    # k in [0,1] for A, integer l >= 0 for E (as Fraction)
    var: str
    pred: str


@dataclass(frozen=True)
class Formula:
    quants: tuple      # tuple[Quantifier]; may be empty (plain LTL4 property)
    body: tuple        # core AST of the quantifier-free body psi

    def aps(self):
        return body_aps(self.body)


_TOKEN = re.compile(r"""
    (?P<ws>\s+)
  | (?P<sym><->|->|=>|&&|\|\||<=|>=|[()!&|<>=:,_{}%~])
  | (?P<num>\d+(?:\.\d*)?|\.\d+)
  | (?P<id>[A-Za-z][A-Za-z0-9]*(?:_[A-Za-z0-9]+)*)
""", re.VERBOSE)

_UNICODE = {"¬": "!", "∧": "&&", "∨": "||", "→": "->", "↔": "<->", "⇒": "=>",
            "≥": ">=", "≤": "<=", "⊤": "true", "⊥": "false"}


def _tokens(text: str):
    for u, a in _UNICODE.items():
        text = text.replace(u, f" {a} ")
    out, i = [], 0
    while i < len(text):
        m = _TOKEN.match(text, i)
        if not m:
            raise ParseError(f"unexpected character {text[i]!r} at {i}")
        i = m.end()
        if m.lastgroup == "ws":
            continue
        tok = m.group(m.lastgroup)
        if tok == "~":
            tok = "!"
        out.append(tok)
    return out


class _P:
    def __init__(self, toks):
        self.t, self.i = toks, 0

    def peek(self, k=0):
        j = self.i + k
        return self.t[j] if j < len(self.t) else None

    def take(self, want=None):
        tok = self.peek()
        if tok is None or (want is not None and tok != want):
            raise ParseError(f"expected {want!r}, found {tok!r}")
        self.i += 1
        return tok

    # quantifier prefix ---------------------------------------------------
    def quantifier(self):
        kind = self.take()
        op, const = None, None
        if self.peek() == "_":
            self.take("_")
            braced = self.peek() == "{"
            if braced:
                self.take("{")
            op = self.take()
            if op not in OPS:
                raise ParseError(f"bad comparison {op!r}")
            num = self.take()
            if not re.fullmatch(r"\d+(?:\.\d*)?|\.\d+", num):
                raise ParseError(f"bad constant {num!r}")
            const = Fraction(num)
            if self.peek() == "%":
                self.take("%")
                const = const / 100
            if braced:
                self.take("}")
        if op is None:  # defaults stated after Def. 1
            op, const = ("=", Fraction(1)) if kind == "A" else (">=", Fraction(1))
        if kind == "A" and not (0 <= const <= 1):
            raise ParseError("A constant must lie in [0,1]")
        if kind == "E" and (const.denominator != 1 or const < 0):
            raise ParseError("E constant must be a non-negative integer")
        var = self.take()
        if not re.fullmatch(r"[A-Za-z]\w*", var):
            raise ParseError(f"bad variable {var!r}")
        self.take(":")
        pred = self.take()
        if self.peek() == "(":
            self.args()
        self.take("=>")
        return Quantifier(kind, op, const, var, pred)

    def args(self):
        self.take("(")
        while self.peek() != ")":
            self.take()
            if self.peek() == ",":
                self.take(",")
        self.take(")")

    # body ------------------------------------------------------------------
    def iff(self):
        f = self.imp()
        while self.peek() == "<->":
            self.take()
            g = self.imp()
            f = ("iff", f, g)
        return f

    def imp(self):
        f = self.disj()
        if self.peek() == "->":
            self.take()
            return ("imp", f, self.imp())
        return f

    def disj(self):
        f = self.conj()
        while self.peek() in ("||", "|"):
            self.take()
            f = ("or", f, self.conj())
        return f

    def conj(self):
        f = self.until()
        while self.peek() in ("&&", "&"):
            self.take()
            f = ("and", f, self.until())
        return f

    def until(self):
        f = self.unary()
        if self.peek() in ("U", "R", "W"):
            op = self.take()
            return (op, f, self.until())
        return f

    def unary(self):
        tok = self.peek()
        if tok == "!":
            self.take()
            return ("not", self.unary())
        if tok in ("X", "F", "G"):
            self.take()
            return (tok, self.unary())
        if tok == "(":
            self.take("(")
            f = self.iff()
            self.take(")")
            return f
        if tok == "true":
            self.take()
            return ("true",)
        if tok == "false":
            self.take()
            return ("false",)
        if tok is not None and re.fullmatch(r"[A-Za-z]\w*", tok) and tok not in ("U", "R", "W", "A", "E"):
            self.take()
            if self.peek() == "(":
                self.args()
            if self.peek() in OPS:
                # interpreted predicate: the event's value compared with an
                # integer constant (case study 2, Sec. 5.1)
                op = self.take()
                num = self.take()
                if not re.fullmatch(r"\d+", num or "") or int(num) > 0xFFFFFFFF:
                    raise ParseError(f"a comparison needs an integer constant in [0, 2^32), got {num!r}")
                return ("ap", f"{tok}{op}{int(num)}")
            return ("ap", tok)
        raise ParseError(f"unexpected token {tok!r}")


def core(f):
    """Rewrite derived operators into true/false/ap/not/and/or/X/U."""
    op = f[0]
    if op in ("true", "false", "ap"):
        return f
    if op == "not":
        return ("not", core(f[1]))
    if op in ("and", "or"):
        return (op, core(f[1]), core(f[2]))
    if op == "X":
        return ("X", core(f[1]))
    if op == "U":
        return ("U", core(f[1]), core(f[2]))
    if op == "F":
        return ("U", ("true",), core(f[1]))
    if op == "G":
        return ("not", ("U", ("true",), ("not", core(f[1]))))
    if op == "imp":
        return ("or", ("not", core(f[1])), core(f[2]))
    if op == "iff":
        a, b = core(f[1]), core(f[2])
        return ("or", ("and", a, b), ("and", ("not", a), ("not", b)))
    if op == "R":
        a, b = core(f[1]), core(f[2])
        return ("not", ("U", ("not", a), ("not", b)))
    if op == "W":
        a, b = core(f[1]), core(f[2])
        return ("or", ("U", a, b), ("not", ("U", ("true",), ("not", a))))
    raise ValueError(op)


def body_aps(f):
    if f[0] == "ap":
        return {f[1]}
    out = set()
    for g in f[1:]:
        if isinstance(g, tuple):
            out |= body_aps(g)
    return out


def parse(text: str) -> Formula:
    """Parse an LTL4-C formula into canonical form Q_0..Q_{n-1} psi."""
    p = _P(_tokens(text))
    quants = []

    def quant_start(k):
        return p.peek(k) in ("A", "E") and (p.peek(k + 1) == "_" or p.peek(k + 2) == ":")

    def qformula():
        # a parenthesised quantified sub-formula, as in Eq. example3
        if p.peek() == "(" and quant_start(1):
            p.take("(")
            body = qformula()
            p.take(")")
            return body
        if quant_start(0):
            quants.append(p.quantifier())
            return qformula()
        return p.iff()

    body = qformula()
    if p.peek() is not None:
        raise ParseError(f"trailing input at {p.peek()!r}")
    return Formula(tuple(quants), core(body))


def subformulas(f, acc=None):
    """All subformulas of a core formula, children before parents."""
    if acc is None:
        acc = []
    for g in f[1:]:
        if isinstance(g, tuple):
            subformulas(g, acc)
    if f not in acc:
        acc.append(f)
    return acc
