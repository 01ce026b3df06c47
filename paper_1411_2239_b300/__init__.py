"""B300-native runtime verification of LTL4-C formulas (map -> monitor -> reduce).

The compute path lives in the C-ABI library ``librv.so`` built from ``csrc/``;
``paper_1411_2239_b300.rv`` is its thin ctypes binding.  Importing this package
loads nothing; ``rv`` loads the library on first use and raises if it is
missing.
"""
