"""The Python entry points on the host: every name a function reads resolves
(module globals, builtins or an enclosing scope), so no benchmark mode or
binding call fails with a NameError on the GPU machine; and the benchmark's
argument parser accepts every mode."""
import builtins
import os
import subprocess
import sys
import symtable

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MODULE_DUNDERS = {"__file__", "__name__", "__doc__", "__spec__", "__package__"}


def _unresolved(table, module_names):
    out = []
    for child in table.get_children():
        if child.get_type() == "function":
            for sym in child.get_symbols():
                if sym.is_global() and not sym.is_assigned() and sym.is_referenced():
                    name = sym.get_name()
                    if name not in module_names and not hasattr(builtins, name) and name not in MODULE_DUNDERS:
                        out.append((child.get_name(), name))
        out += _unresolved(child, module_names)
    return out


SOURCES = ["bench.py", "__graft_entry__.py", "paper_1401_4441_gb300/lc.py", "paper_1401_4441_gb300/inputs.py",
           "paper_1401_4441_gb300/autotune.py", "paper_1401_4441_gb300/build.py",
           "paper_1401_4441_gb300/checkpoint.py", "oracle/__init__.py", "oracle/dag.py", "oracle/build.py"]


def test_names_resolve():
    bad = []
    for rel in SOURCES:
        path = os.path.join(ROOT, rel)
        top = symtable.symtable(open(path).read(), path, "exec")
        module_names = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()}
        bad += [(rel,) + u for u in _unresolved(top, module_names)]
    assert bad == []


def test_bench_help():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0
    for opt in ("--schedule", "--skin", "--workload", "--impl", "--dag", "--profile"):
        assert opt in r.stdout


def test_reference_arm_line_on_the_host():
    """The reference arm (the FP64 oracle's Verlet steps on the host cores)
    needs no GPU: its one JSON line carries the keys of the benchmark
    contract, with the arm's own value as cpu_baseline and e2e."""
    import json
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in d
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] >= 3 and d["higher_is_better"] is True
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
