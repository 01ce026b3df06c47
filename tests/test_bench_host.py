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


def _run_bench(args, env_extra=None):
    import json
    import subprocess
    env = dict(os.environ, **(env_extra or {}))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(ln) for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_reference_arm_line():
    # the reference arm is the oracle on the host cores: one JSON line with
    # the contract's keys, no GPU needed; ranks other than 0 print nothing
    lines = _run_bench(["--impl", "reference", "--events", "300000", "--steps", "1", "--warmup", "1"])
    assert len(lines) == 1
    d = lines[0]
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert _run_bench(["--impl", "reference", "--events", "300000", "--steps", "1", "--warmup", "1"],
                      {"RANK": "1"}) == []
