"""lc_bin_noalloc: binning without device allocation, through the C ABI.

Callers that cannot allocate device memory (work issued while another
component captures a CUDA graph, code limited to a memory pool it was
given) use lc_bin_noalloc; it must give the same cell counts, cell starts
and permutation as the allocating path (lc_create + lc_set_state + lc_bin +
lc_get), bit for bit, on consecutive calls that reuse its internal scratch.
"""
import ctypes

import numpy as np
import pytest

from paper_1401_4441_gb300 import inputs

pytestmark = pytest.mark.gpu
RC = 2.5


def noalloc_fn(lc):
    fn = lc.lib().lc_bin_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def run_noalloc(lc, torch, pos, box):
    fn = noalloc_fn(lc)
    nc = np.floor(np.asarray(box) / RC).astype(np.int64)
    ncell = int(nc.prod())
    dpos = torch.from_numpy(np.ascontiguousarray(pos, dtype=np.float64)).cuda()
    count = torch.full((ncell,), -7, dtype=torch.int32, device="cuda")
    start = torch.full((ncell,), -7, dtype=torch.int32, device="cuda")
    perm = torch.full((max(pos.shape[0], 1),), -7, dtype=torch.int32, device="cuda")
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = fn(ctypes.c_void_p(dpos.data_ptr()), pos.shape[0], b, RC, ctypes.c_void_p(count.data_ptr()),
              ctypes.c_void_p(start.data_ptr()), ctypes.c_void_p(perm.data_ptr()), stream)
    torch.cuda.synchronize()
    return code, count.cpu().numpy(), start.cpu().numpy(), perm.cpu().numpy()[:pos.shape[0]]


def run_allocating(lc, pos, box):
    with lc.Box(box, RC, pos.shape[0], "mixed") as g:
        g.set_state(pos)
        g.bin()
        return g.get("cell_count"), g.get("cell_start"), g.get("perm")


def test_noalloc_matches_allocating_path_on_consecutive_calls(lc):
    torch = pytest.importorskip("torch")
    a = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    n = 30000
    box_b = np.array([40.0, 31.0, 27.5])
    pos_b = inputs.uniform(21, 0, 3 * n).reshape(n, 3) * box_b * 1.5 - 0.25 * box_b   # outside [0, L) too
    for pos, box in ((a["pos"], a["box"]), (pos_b, box_b), (a["pos"], a["box"])):
        code, count, start, perm = run_noalloc(lc, torch, pos, box)
        assert code == 0
        ref_count, ref_start, ref_perm = run_allocating(lc, pos, box)
        assert np.array_equal(count, ref_count)
        assert np.array_equal(start, ref_start)
        assert np.array_equal(perm, ref_perm)


def test_noalloc_rejects_sizes_beyond_its_scratch(lc):
    torch = pytest.importorskip("torch")
    fn = noalloc_fn(lc)
    dummy = torch.zeros(8, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    box = (ctypes.c_double * 3)(100.0, 100.0, 100.0)
    assert fn(p, (1 << 20) + 1, box, RC, p, p, p, None) == 9          # too many particles
    big = (ctypes.c_double * 3)(300.0, 300.0, 300.0)                   # 120^3 cells
    assert fn(p, 10, big, RC, p, p, p, None) == 9
    small = (ctypes.c_double * 3)(7.0, 100.0, 100.0)
    assert fn(p, 10, small, RC, p, p, p, None) == 2


def test_noalloc_empty_and_no_device_allocation(lc):
    """n = 0 gives all-zero counts and starts; after a first call, further
    calls leave the device's free memory unchanged (nothing is allocated)."""
    torch = pytest.importorskip("torch")
    a = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    run_noalloc(lc, torch, a["pos"], a["box"])          # first call: symbol look-up, kernels loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        code, count, start, perm = run_noalloc(lc, torch, a["pos"], a["box"])
        assert code == 0
    code, count, start, _ = run_noalloc(lc, torch, np.zeros((0, 3)), a["box"])
    assert code == 0
    assert not count.any() and not start.any()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # the test's own output tensors come from torch's cache, not new driver memory
    assert free1 == free0
