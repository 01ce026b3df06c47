"""Host logic of bench.py that needs no GPU: the kernel-source hash that keys
the committed DRAM-traffic record."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_only_drops_comments_keeps_strings():
    src = 'int a = 1;  // one\n/* block\n comment */ int b = 2;\n\nconst char* s = "x // y /* z */";\n'
    out = bench.code_only(src)
    assert "one" not in out and "block" not in out
    assert '"x // y /* z */"' in out
    assert "int a = 1;" in out and "int b = 2;" in out


def test_hash_ignores_comment_edits_only():
    files = {p: open(os.path.join(ROOT, p)).read()
             for p in ["include/rv.h"] + ["paper_1411_2239_b300/csrc/" + f for f in bench.OFFLINE_SOURCES]}
    base = bench.kernel_source_hash(files.__getitem__)
    assert base == bench.kernel_source_hash()
    k = "paper_1411_2239_b300/csrc/offline.cu"
    commented = dict(files)
    commented[k] = files[k].replace("namespace {", "// a new comment line\nnamespace {  /* and one here */", 1)
    assert bench.kernel_source_hash(commented.__getitem__) == base
    changed = dict(files)
    changed[k] = files[k].replace("constexpr int SPIN_LIMIT = 1 << 22;", "constexpr int SPIN_LIMIT = 1 << 21;", 1)
    assert changed[k] != files[k]
    assert bench.kernel_source_hash(changed.__getitem__) != base
