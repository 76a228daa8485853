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
