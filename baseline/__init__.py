"""CPU baselines for bench.py (not the product path, not the oracle).

strategy1: the paper's Strategy 1 (Sec. VI, Fig. 6: loop exchange and
2-strided colouring) for the link-cell force sweep with Newton's third law,
FP64, on all host cores with OpenMP.  Built with gcc on first use into
baseline/_build/.  tests/test_baseline_strategy1.py checks it against the
oracle.
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "strategy1.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libstrategy1.so")
_lib = None


def build(force=False):
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall", SRC, "-o", tmp, "-lm"],
                   check=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.s1_forces.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double, dp, dp, dp,
                                  ctypes.POINTER(ctypes.c_int64)]
        lib.s1_forces.restype = ctypes.c_int
        lib.s1_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads():
    return int(_load().s1_threads())


def forces(pos, box, rc):
    """(forces [n, 3] by ID, U, W, npairs) of positions pos [n, 3]."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    L = np.ascontiguousarray(np.asarray(box, np.float64)[:3])
    n = pos.shape[0]
    f = np.zeros((n, 3), np.float64)
    U, W = ctypes.c_double(), ctypes.c_double()
    npairs = ctypes.c_int64()
    dp = ctypes.POINTER(ctypes.c_double)
    r = lib.s1_forces(n, pos.ctypes.data_as(dp), L.ctypes.data_as(dp), float(rc), f.ctypes.data_as(dp),
                      ctypes.byref(U), ctypes.byref(W), ctypes.byref(npairs))
    if r:
        raise RuntimeError(f"s1_forces failed ({r})")
    return f, U.value, W.value, npairs.value
