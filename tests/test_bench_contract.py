"""The benchmark's reference arm on the CPU: one JSON line with the keys the
benchmark contract asks for (the oracle timed on the host cores)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["metric"] == d["unit"] == "grid-pt-steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("ch2d_periodic_2048sq")


def test_bench_refers_to_no_undefined_name():
    # the GPU arm cannot run here, so a missing module-level name would only show
    # on the GPU machine: every name the script loads must be a builtin, a module
    # global, or bound somewhere in it
    import ast
    import builtins

    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    known = set(dir(builtins)) | {"__file__", "__name__"}
    for n in ast.walk(tree):
        if isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
            known.add(n.id)
        elif isinstance(n, ast.arg):
            known.add(n.arg)
        elif isinstance(n, (ast.FunctionDef, ast.ClassDef)):
            known.add(n.name)
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            known.update((a.asname or a.name).split(".")[0] for a in n.names)
        elif isinstance(n, ast.ExceptHandler) and n.name:
            known.add(n.name)
    used = {n.id for n in ast.walk(tree) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load)}
    assert not used - known, sorted(used - known)


def test_bench_kernel_tables_name_profile_slots():
    # the roofline tables are keyed by the library's profile slot names
    import re
    import sys as _sys

    _sys.path.insert(0, ROOT)
    import bench

    src = open(os.path.join(ROOT, "paper_2101_06550_gb300", "csrc", "ch.cu")).read()
    table = src[src.index("kSlotName[kSlots] = {"):]
    slots = set(re.findall(r'"([a-z0-9_]+)"', table[:table.index("};")]))
    for name in list(bench.KERNEL_FP64_OPS) + list(bench.KERNEL_BYTES) + list(bench.KERNEL_TRAFFIC_BYTES):
        assert name in slots, name
    assert set(bench.KERNEL_FP64_OPS) == set(bench.KERNEL_BYTES)
