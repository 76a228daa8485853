"""Thin ctypes binding of liblc.so (include/lc.h).

Argument marshalling only: every step of the force sweep, binning and
integration runs in the library's CUDA kernels.  There is no CPU fallback:
if the compiled library is missing, loading raises.  PyTorch is used for
device buffers and streams only (``torch.cuda.current_stream()``).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblc.so")

SCHED = {"colour": 0, "atomic": 1, "fullshell": 2, "buffer": 3, "list": 4}
PREC = {"fp64": 0, "mixed": 1}
ORDER = {"cell": 0, "loopex": 1}
DAG_WITHHOLD = 1
QUEUE_WITHHOLD = 1
GET = {"cell_count": 0, "cell_start": 1, "perm": 2, "colour": 3, "forces": 4, "pos": 5, "vel": 6}
STATUS = {0: "LC_OK", 1: "LC_ERR_INVALID_ARG", 2: "LC_ERR_BOX_TOO_SMALL", 3: "LC_ERR_CUDA",
          4: "LC_ERR_OOM", 5: "LC_ERR_NONFINITE", 6: "LC_ERR_TIMEOUT", 7: "LC_ERR_STATE",
          8: "LC_ERR_RACE", 9: "LC_ERR_TOO_LARGE"}

_lib = None


class LCError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        name = STATUS.get(code, str(code))
        msg = _load().lc_status_str(code).decode() if _lib is not None else name
        super().__init__(f"{where}: {name} ({msg})")


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"liblc.so not built ({LIB_PATH}); run paper_1401_4441_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, ip, lp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), \
        ctypes.POINTER(ctypes.c_int64)
    ctx_pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "lc_create": ([dp, ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctx_pp], ctypes.c_int),
        "lc_set_state": ([vp, vp, vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "lc_bin": ([vp, vp], ctypes.c_int),
        "lc_forces": ([vp, ctypes.c_int, vp], ctypes.c_int),
        "lc_verlet_step": ([vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, vp], ctypes.c_int),
        "lc_energy_virial": ([vp, dp, dp, dp, lp, vp], ctypes.c_int),
        "lc_get": ([vp, ctypes.c_int, vp, ctypes.c_int, vp], ctypes.c_int),
        "lc_grid": ([vp, ip, ip, ip], ctypes.c_int),
        "lc_schedule_check": ([vp, ctypes.c_int, lp, lp, vp], ctypes.c_int),
        "lc_set_tile": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "lc_launch_counts": ([vp, ip, ip], ctypes.c_int),
        "lc_launch_counts_graphs": ([vp, ip, ip], ctypes.c_int),
        "lc_batch_create": ([ctypes.c_int32, dp, dp, lp, ctypes.c_int, ctx_pp], ctypes.c_int),
        "lc_batch_energies": ([vp, dp, dp, dp, lp, vp], ctypes.c_int),
        "lc_batch_info": ([vp, ip, lp, lp], ctypes.c_int),
        "lc_dag_build": ([vp, ctypes.c_int, lp, lp, lp], ctypes.c_int),
        "lc_dag_forces": ([vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, vp, vp], ctypes.c_int),
        "lc_dag_plan": ([ip, ctypes.c_int, ip, ctypes.c_int32, lp, lp, lp], ctypes.c_int),
        "lc_dag_stencil_order": ([vp, ip, ctypes.c_int32], ctypes.c_int),
        "lc_create_2d": ([dp, ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctx_pp], ctypes.c_int),
        "lc_stage_state": ([vp, vp, vp, ctypes.c_int32, vp], ctypes.c_int),
        "lc_set_state_staged": ([vp, ctypes.c_int32, vp], ctypes.c_int),
        "lc_energy_virial_async": ([vp, vp, vp], ctypes.c_int),
        "lc_result_decode": ([vp, dp, dp, dp, lp], ctypes.c_int),
        "lc_set_skin": ([vp, ctypes.c_double, ctypes.c_int32], ctypes.c_int),
        "lc_list_info": ([vp, lp, lp, lp, lp, lp, ip, vp], ctypes.c_int),
        "lc_batch_step": ([vp, ctypes.c_double, ctypes.c_int32, vp], ctypes.c_int),
        "lc_set_queue_wait": ([vp, ctypes.c_double, ctypes.c_int32], ctypes.c_int),
        "lc_probe_fp32": ([ctypes.c_int32, dp, dp, vp], ctypes.c_int),
        "lc_destroy": ([vp], None),
        "lc_status_str": ([ctypes.c_int], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def lib():
    return _load()


def _check(code, where):
    if code != 0:
        raise LCError(code, where)


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def _ptr(a):
    """(pointer, on_device) of a host numpy array or a CUDA torch tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        return ctypes.c_void_p(a.ctypes.data), 0
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported array type {type(a)}")


def _perm(perm):
    if perm is None:
        return None, 0
    perm = [int(x) for x in perm]
    return (ctypes.c_int32 * len(perm))(*perm), len(perm)


def decode(out):
    """(U, K, W, npairs) from a result block filled by Box.energy_async."""
    lib = _load()
    p, _ = _ptr(out)
    u, k, w = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    npairs = ctypes.c_int64()
    _check(lib.lc_result_decode(p, ctypes.byref(u), ctypes.byref(k), ctypes.byref(w), ctypes.byref(npairs)),
           "lc_result_decode")
    return u.value, k.value, w.value, npairs.value


def probe_fp32(iters=1 << 16, stream=None):
    """(flops, seconds) of the library's FP32 FMA throughput probe on the
    current device (lc_probe_fp32)."""
    lib_ = _load()
    f, sec = ctypes.c_double(), ctypes.c_double()
    _check(lib_.lc_probe_fp32(int(iters), ctypes.byref(f), ctypes.byref(sec), _stream(stream)), "lc_probe_fp32")
    return f.value, sec.value


def dag_plan(nc, order="loopex", perm=None):
    """(tasks, edges, critical path) of the task DAG of a grid of nc cells
    (nc[2] == 1 or a 2-tuple: the 2D grid), built on the host by the library
    (no GPU needed).  perm: the stencil order inside a cell for the cell
    order (entry 0 intra, k >= 1 the k-th forward offset)."""
    lib_ = _load()
    nc = list(nc) + [1] * (3 - len(nc))
    arr = (ctypes.c_int32 * 3)(*[int(x) for x in nc])
    p, np_ = _perm(perm)
    t, e, cp = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib_.lc_dag_plan(arr, ORDER[order], p, np_, ctypes.byref(t), ctypes.byref(e), ctypes.byref(cp)),
           "lc_dag_plan")
    return t.value, e.value, cp.value


class Box:
    """One periodic box on the GPU (an lc_ctx).  dims=2: a 2D box
    (box = (Lx, Ly); positions keep three components, z ignored)."""

    def __init__(self, box, rc, n, precision="mixed", dims=3):
        self._lib = _load()
        self.n = int(n)
        self.dims = dims
        self.box = np.ascontiguousarray(np.broadcast_to(np.asarray(box, np.float64), (dims,)))
        self.rc = float(rc)
        self.precision = precision
        h = ctypes.c_void_p()
        create = self._lib.lc_create_2d if dims == 2 else self._lib.lc_create
        _check(create(self.box.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.rc, self.n,
                      PREC[precision], ctypes.byref(h)), "lc_create")
        self._h = h

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.lc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls -------------------------------------------------------------
    def set_state(self, pos, vel=None, stream=None):
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, dtype=np.float64)
            vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64)
        p, dev = _ptr(pos)
        v, _ = _ptr(vel)
        _check(self._lib.lc_set_state(self._h, p, v, None, dev, _stream(stream)), "lc_set_state")

    def stage_state(self, pos, vel=None, slot=0, copy_stream=None):
        """Queue the copy of a later state (host arrays, page-locked to
        overlap) into staging slot 0 or 1 on copy_stream; returns at once."""
        if isinstance(pos, np.ndarray):
            raise TypeError("stage_state needs page-locked host tensors (torch .pin_memory())")
        p, dev = _ptr(pos)
        v, _ = _ptr(vel)
        if dev:
            raise TypeError("stage_state takes host memory")
        _check(self._lib.lc_stage_state(self._h, p, v, int(slot), _stream(copy_stream)), "lc_stage_state")

    def set_state_staged(self, slot=0, stream=None):
        """Make staging slot `slot` the current state, after its copy."""
        _check(self._lib.lc_set_state_staged(self._h, int(slot), _stream(stream)), "lc_set_state_staged")

    def bin(self, stream=None):
        _check(self._lib.lc_bin(self._h, _stream(stream)), "lc_bin")

    def forces(self, schedule="colour", stream=None):
        _check(self._lib.lc_forces(self._h, SCHED[schedule], _stream(stream)), "lc_forces")

    def verlet(self, dt, nsteps, schedule="colour", stream=None):
        _check(self._lib.lc_verlet_step(self._h, float(dt), int(nsteps), SCHED[schedule], _stream(stream)),
               "lc_verlet_step")

    def energy(self, stream=None):
        """(U, K, W, npairs) of the current state."""
        u, k, w = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        npairs = ctypes.c_int64()
        _check(self._lib.lc_energy_virial(self._h, ctypes.byref(u), ctypes.byref(k), ctypes.byref(w),
                                          ctypes.byref(npairs), _stream(stream)), "lc_energy_virial")
        return u.value, k.value, w.value, npairs.value

    def energy_async(self, out, stream=None):
        """Queue the energies into `out` (48 bytes of page-locked host
        memory: a pinned torch tensor or a numpy array) without waiting;
        read them with decode(out) once the stream has passed this point."""
        p, dev = _ptr(out)
        if dev:
            raise TypeError("out must be host memory")
        _check(self._lib.lc_energy_virial_async(self._h, p, _stream(stream)), "lc_energy_virial_async")

    def grid(self):
        nc = (ctypes.c_int32 * 3)()
        ncol, nph = ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.lc_grid(self._h, nc, ctypes.byref(ncol), ctypes.byref(nph)), "lc_grid")
        return np.array(list(nc), np.int32), ncol.value, nph.value

    def ncell(self):
        nb, np_, nc = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        _check(self._lib.lc_batch_info(self._h, ctypes.byref(nb), ctypes.byref(np_), ctypes.byref(nc)),
               "lc_batch_info")
        return int(nc.value)

    def get(self, what, out=None, stream=None):
        """Copy an array out; returns a numpy array unless `out` (host
        numpy array or CUDA torch tensor of the right size) is given."""
        ncell = self.ncell()
        shapes = {"cell_count": ((ncell,), np.int32), "cell_start": ((ncell,), np.int32),
                  "perm": ((self.n,), np.int32), "colour": ((ncell,), np.int8),
                  "forces": ((self.n, 3), np.float64), "pos": ((self.n, 3), np.float64),
                  "vel": ((self.n, 3), np.float64)}
        shape, dtype = shapes[what]
        if out is None:
            out = np.empty(shape, dtype)
        p, dev = _ptr(out)
        _check(self._lib.lc_get(self._h, GET[what], p, dev, _stream(stream)), f"lc_get({what})")
        return out

    def schedule_check(self, schedule, stream=None):
        conflicts, cover = ctypes.c_int64(), ctypes.c_int64()
        code = self._lib.lc_schedule_check(self._h, SCHED[schedule], ctypes.byref(conflicts), ctypes.byref(cover),
                                           _stream(stream))
        if code not in (0, 8):
            _check(code, "lc_schedule_check")
        return conflicts.value, cover.value

    def dag_build(self, order="loopex"):
        """(tasks, edges, critical path) of the task DAG of a creation order."""
        t, e, cp = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(self._lib.lc_dag_build(self._h, ORDER[order], ctypes.byref(t), ctypes.byref(e), ctypes.byref(cp)),
               "lc_dag_build")
        return t.value, e.value, cp.value

    def dag_stencil_order(self, perm=None):
        """Stencil order inside a cell for the cell creation order (None:
        table order)."""
        p, np_ = _perm(perm)
        _check(self._lib.lc_dag_stencil_order(self._h, p, np_), "lc_dag_stencil_order")

    def dag_forces(self, order="loopex", trace=None, wait_seconds=0.0, withhold=False, stream=None):
        """Forces by running the task DAG on the device; trace: None or a CUDA
        int32 tensor of 2 * tasks (start / end stamps)."""
        tp, dev = _ptr(trace)
        if trace is not None and not dev:
            raise TypeError("trace must be a CUDA tensor")
        _check(self._lib.lc_dag_forces(self._h, ORDER[order], float(wait_seconds), DAG_WITHHOLD if withhold else 0,
                                       tp, _stream(stream)), "lc_dag_forces")

    def set_skin(self, skin=0.4, kmax=0):
        """Skin of the Verlet lists (schedule "list"); kmax = 0: row capacity
        sized from the first build."""
        _check(self._lib.lc_set_skin(self._h, float(skin), int(kmax)), "lc_set_skin")

    def list_info(self, stream=None):
        """dict of the list counters: builds, long_rows, longest_row,
        rebuild_steps, entries (over all builds), kmax."""
        v = [ctypes.c_int64() for _ in range(5)]
        km = ctypes.c_int32()
        _check(self._lib.lc_list_info(self._h, *(ctypes.byref(x) for x in v), ctypes.byref(km), _stream(stream)),
               "lc_list_info")
        return {"builds": v[0].value, "long_rows": v[1].value, "longest_row": v[2].value,
                "rebuild_steps": v[3].value, "entries": v[4].value, "kmax": km.value}

    def set_queue_wait(self, seconds=2.0, withhold=False):
        """Limit of one wait of the colour schedule's queue; withhold: no task
        publishes its completion (a test of the bounded waits)."""
        _check(self._lib.lc_set_queue_wait(self._h, float(seconds), QUEUE_WITHHOLD if withhold else 0),
               "lc_set_queue_wait")

    def set_tile(self, ni=0, warps=0):
        _check(self._lib.lc_set_tile(self._h, int(ni), int(warps)), "lc_set_tile")

    def launch_counts(self):
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.lc_launch_counts(self._h, ctypes.byref(a), ctypes.byref(b)), "lc_launch_counts")
        return a.value, b.value

    def launch_counts_graphs(self):
        """(kernels of the one-step graph, kernels of the two-step graph)."""
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.lc_launch_counts_graphs(self._h, ctypes.byref(a), ctypes.byref(b)),
               "lc_launch_counts_graphs")
        return a.value, b.value


class Batch(Box):
    """Independent periodic boxes in one context (lc_batch_create): particles
    numbered box after box; every schedule but the lists."""

    def __init__(self, boxes, rcs, ns, precision="mixed"):
        self._lib = _load()
        boxes = np.ascontiguousarray(np.asarray(boxes, np.float64).reshape(-1, 3))
        rcs = np.ascontiguousarray(np.broadcast_to(np.asarray(rcs, np.float64), (boxes.shape[0],)))
        ns = np.ascontiguousarray(np.asarray(ns, np.int64))
        self.nbox = boxes.shape[0]
        self.rcs = rcs
        self.ns = ns
        self.offsets = np.concatenate([[0], np.cumsum(ns)])
        self.n = int(ns.sum())
        self.box = boxes
        self.precision = precision
        h = ctypes.c_void_p()
        _check(self._lib.lc_batch_create(self.nbox, boxes.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         rcs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         PREC[precision], ctypes.byref(h)), "lc_batch_create")
        self._h = h

    def step(self, dt, nsteps, stream=None):
        """lc_batch_step: Verlet steps of every box, colour schedule on the
        device work queue."""
        _check(self._lib.lc_batch_step(self._h, float(dt), int(nsteps), _stream(stream)), "lc_batch_step")

    def energies(self, stream=None):
        """Per-box (U, K, W, npairs) arrays."""
        u, k, w = (np.zeros(self.nbox) for _ in range(3))
        p = np.zeros(self.nbox, np.int64)
        dp = ctypes.POINTER(ctypes.c_double)
        _check(self._lib.lc_batch_energies(self._h, u.ctypes.data_as(dp), k.ctypes.data_as(dp), w.ctypes.data_as(dp),
                                           p.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _stream(stream)),
               "lc_batch_energies")
        return u, k, w, p
