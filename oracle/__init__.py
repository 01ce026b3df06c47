"""Plain CPU oracle for LTL4-C runtime verification (test infrastructure only).

This package is the slow, obviously-correct restatement of the semantics of
"Accelerated Runtime Verification of LTL Specifications with Counting
Semantics" (Medhat, Joshi, Bonakdarpour, Fischmeister).  It exists to check the
CUDA path, and only the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it.  The product path never routes
through this package and shares no code with it.

Modules
  formula   -- syntax of Def. 1 (Sec. 2.1) with the default constraints, and
               the exact rational/integer constants of the quantifiers.
  fltl      -- finite-trace LTL, Def. "FLTL semantics" (Sec. 2.2.1).
  ltl4      -- four-valued LTL, Def. "LTL4 semantics" (Sec. 2.2.2): formula
               progression plus an atom tableau for satisfiability.
  counting  -- value vectors, projection u^D, parent function P, the count
               function B, constraint S (Eq. S) and the six-valued inductive
               semantics (Def. "LTL4-C Semantics", Table 1).
  verify    -- the whole trace -> verdict function (the method's result).
  timeline  -- the verdict of every event's binding after that event, and
               each binding's first violation (the online mode, Sec. 4.2).

Parity status: every function is pinned by tests/test_oracle_*.py; the
readings of the six-valued valuation beyond the cases the paper works out
(the ladder for <=/< and =, the percentage-quantifier permanence rules) are
pinned by an enumeration of how a node's children can still turn out
(tests/test_oracle_permanence.py).
"""
