"""Plain FP64 CPU oracle for the link-cell Lennard-Jones force sweep.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of bench.py may import this
package.  It shares no code with the CUDA path (``paper_1401_4441_gb300``);
inputs come from the seeded generators in ``paper_1401_4441_gb300.inputs``,
which hold none of the method's arithmetic.

Functions (all FP64, positions indexed by particle ID):
  grid(L, rc)                 -> nc[3]                      (Sec. IV: cells of side >= r_c)
  bin(x, y, z, L, rc)         -> dict(cell_of, count, start, perm, colour, ncolours)
  nsq_forces(x, y, z, L, rc)  -> (f[n,3], U, W, npairs)      O(N^2) minimum image
  lc_forces(x, y, z, L, rc)   -> (f[n,3], U, W, npairs)      serial link-cell, literature order
  forces_sample(..., ids)     -> (f[len(ids),3], nneigh)     per-particle sums
  force_scale(x, y, z, L, rc) -> s[n]                       sum_j |F_ij| per particle
  verlet(xyz, v, L, rc, dt, nsteps) -> (xyz, v, f, energies[nsteps+1, 3])
  half_shell()                -> int[13,3]                   forward half-shell offsets
  offset_groups()             -> int[13]                     parity-pattern groups
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lp = ctypes.POINTER(ctypes.c_int64)
        bp = ctypes.POINTER(ctypes.c_int8)
        lib.orc_grid.argtypes = [dp, ctypes.c_double, ip]
        lib.orc_grid.restype = ctypes.c_int
        lib.orc_wrap.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_wrap.restype = ctypes.c_double
        lib.orc_bin.argtypes = [ctypes.c_int64, dp, dp, dp, dp, ctypes.c_double,
                                ip, ip, ip, ip, bp, ip]
        lib.orc_bin.restype = ctypes.c_int
        lib.orc_nsq_forces.argtypes = [ctypes.c_int64, dp, dp, dp, dp, ctypes.c_double,
                                       dp, dp, dp, lp]
        lib.orc_nsq_forces.restype = None
        lib.orc_lc_forces.argtypes = [ctypes.c_int64, dp, dp, dp, dp, ctypes.c_double,
                                      dp, dp, dp, lp]
        lib.orc_lc_forces.restype = ctypes.c_int
        lib.orc_forces_sample.argtypes = [ctypes.c_int64, dp, dp, dp, dp, ctypes.c_double,
                                          ctypes.c_int64, lp, dp, lp]
        lib.orc_forces_sample.restype = ctypes.c_int
        lib.orc_verlet.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_int, dp,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]
        lib.orc_verlet.restype = ctypes.c_int
        lib.orc_force_scale.argtypes = [ctypes.c_int64, dp, dp, dp, dp, ctypes.c_double, dp]
        lib.orc_force_scale.restype = None
        lib.orc_half_shell.argtypes = [ip]
        lib.orc_half_shell.restype = None
        lib.orc_offset_groups.argtypes = [ip]
        lib.orc_offset_groups.restype = None
        _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _l(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _b(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _box(L):
    L = np.asarray(L, dtype=np.float64)
    if L.ndim == 0:
        L = np.full(3, float(L))
    return np.ascontiguousarray(L)


def grid(L, rc):
    lib = _load()
    nc = np.zeros(3, np.int32)
    bad = lib.orc_grid(_d(_box(L)), float(rc), _i(nc))
    return nc, bool(bad)


def wrap(x, L):
    return _load().orc_wrap(float(x), float(L))


def bin(x, y, z, L, rc):
    lib = _load()
    x, y, z, L = _f64(x), _f64(y), _f64(z), _box(L)
    nc, bad = grid(L, rc)
    if bad:
        raise ValueError("box too small: every L_d must hold at least 3 cells")
    n = x.shape[0]
    ncell = int(nc[0]) * int(nc[1]) * int(nc[2])
    cell_of = np.zeros(n, np.int32)
    count = np.zeros(ncell, np.int32)
    start = np.zeros(ncell, np.int32)
    perm = np.zeros(n, np.int32)
    colour = np.zeros(ncell, np.int8)
    ncol = np.zeros(1, np.int32)
    r = lib.orc_bin(n, _d(x), _d(y), _d(z), _d(L), float(rc), _i(cell_of), _i(count),
                    _i(start), _i(perm), _b(colour), _i(ncol))
    if r:
        raise RuntimeError(f"orc_bin failed ({r})")
    return dict(nc=nc, cell_of=cell_of, count=count, start=start, perm=perm,
                colour=colour, ncolours=int(ncol[0]))


def nsq_forces(x, y, z, L, rc):
    lib = _load()
    x, y, z, L = _f64(x), _f64(y), _f64(z), _box(L)
    n = x.shape[0]
    f = np.zeros((n, 3), np.float64)
    U = np.zeros(1); W = np.zeros(1); npairs = np.zeros(1, np.int64)
    lib.orc_nsq_forces(n, _d(x), _d(y), _d(z), _d(L), float(rc), _d(f), _d(U), _d(W), _l(npairs))
    return f, float(U[0]), float(W[0]), int(npairs[0])


def lc_forces(x, y, z, L, rc):
    lib = _load()
    x, y, z, L = _f64(x), _f64(y), _f64(z), _box(L)
    n = x.shape[0]
    f = np.zeros((n, 3), np.float64)
    U = np.zeros(1); W = np.zeros(1); npairs = np.zeros(1, np.int64)
    r = lib.orc_lc_forces(n, _d(x), _d(y), _d(z), _d(L), float(rc), _d(f), _d(U), _d(W), _l(npairs))
    if r:
        raise RuntimeError(f"orc_lc_forces failed ({r})")
    return f, float(U[0]), float(W[0]), int(npairs[0])


def forces_sample(x, y, z, L, rc, ids):
    lib = _load()
    x, y, z, L = _f64(x), _f64(y), _f64(z), _box(L)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    f = np.zeros((ids.shape[0], 3), np.float64)
    nn = np.zeros(ids.shape[0], np.int64)
    r = lib.orc_forces_sample(x.shape[0], _d(x), _d(y), _d(z), _d(L), float(rc),
                              ids.shape[0], _l(ids), _d(f), _l(nn))
    if r:
        raise RuntimeError(f"orc_forces_sample failed ({r})")
    return f, nn


def force_scale(x, y, z, L, rc):
    """Per-particle sum of pair-force magnitudes, S_i = sum_j |F_ij|."""
    lib = _load()
    x, y, z, L = _f64(x), _f64(y), _f64(z), _box(L)
    out = np.zeros(x.shape[0])
    lib.orc_force_scale(x.shape[0], _d(x), _d(y), _d(z), _d(L), float(rc), _d(out))
    return out


def verlet(xyz, v, L, rc, dt, nsteps, f=None):
    """Velocity Verlet in FP64; returns (xyz, v, f, energies[nsteps+1, (U, K, W)]).
    If f (forces of xyz) is given the initial force evaluation is skipped."""
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).copy()
    v = np.ascontiguousarray(v, dtype=np.float64).copy()
    n = xyz.shape[0]
    have_f = f is not None
    f = np.zeros((n, 3), np.float64) if f is None else np.ascontiguousarray(f, dtype=np.float64).copy()
    e = np.zeros((nsteps + 1, 3), np.float64)
    r = lib.orc_verlet(n, _d(xyz), _d(v), _d(f), int(have_f), _d(_box(L)), float(rc), float(dt),
                       int(nsteps), _d(e))
    if r:
        raise RuntimeError(f"orc_verlet failed ({r})")
    return xyz, v, f, e


def half_shell():
    out = np.zeros(39, np.int32)
    _load().orc_half_shell(_i(out))
    return out.reshape(13, 3)


def offset_groups():
    out = np.zeros(13, np.int32)
    _load().orc_offset_groups(_i(out))
    return out
