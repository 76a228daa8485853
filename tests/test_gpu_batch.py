"""Batches of independent boxes (lc_batch_create) against the FP64 oracle,
box by box: bit-exact binning and pair counts, forces within the same
tolerances as single boxes, per-box energies, Verlet trajectories."""
import math

import numpy as np
import pytest

import oracle
from paper_1401_4441_gb300 import inputs

pytestmark = pytest.mark.gpu
RC = 2.5
TOL = {"fp64": 1e-10, "mixed": 1e-5}


def small_batch(nbox=9, seed=5):
    # the configuration's smallest box (N = 500 at density 0.9) still has 3 cells
    return inputs.batch_boxes(nbox=nbox, n_min=500, n_max=6000, seed=seed)


def concat(boxes, key):
    return np.concatenate([b[key] for b in boxes])


def make_batch(lc, boxes, prec, with_vel=False):
    g = lc.Batch([b["box"] for b in boxes], RC, [b["pos"].shape[0] for b in boxes], prec)
    g.set_state(concat(boxes, "pos"), concat(boxes, "vel") if with_vel else None)
    return g


def test_batch_binning_bit_exact(lc):
    boxes = small_batch()
    with make_batch(lc, boxes, "mixed") as g:
        g.bin()
        count, start, perm = g.get("cell_count"), g.get("cell_start"), g.get("perm")
    coff = 0
    for b, bx in enumerate(boxes):
        p = bx["pos"]
        ref = oracle.bin(p[:, 0], p[:, 1], p[:, 2], bx["box"], RC)
        nc = ref["count"].shape[0]
        assert np.array_equal(count[coff:coff + nc], ref["count"])
        off = g.offsets[b]
        assert np.array_equal(start[coff:coff + nc] - off, ref["start"])
        assert np.array_equal(perm[off:off + p.shape[0]] - off, ref["perm"])
        coff += nc


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("sched", ["atomic", "fullshell", "buffer"])
def test_batch_forces_per_box(lc, prec, sched):
    boxes = small_batch()
    with make_batch(lc, boxes, prec) as g:
        g.forces(sched)
        f = g.get("forces")
        u, k, w, npairs = g.energies()
        U, K, W, NP = g.energy()
    assert U == pytest.approx(u.sum(), rel=1e-12) and NP == npairs.sum()
    for b, bx in enumerate(boxes):
        p = bx["pos"]
        fref, Ur, Wr, npr = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], bx["box"], RC)
        fb = f[g.offsets[b]:g.offsets[b + 1]]
        rms = math.sqrt(float((fref ** 2).sum(1).mean()))
        err = float(np.sqrt(((fb - fref) ** 2).sum(1)).max()) / rms
        assert npairs[b] == npr
        assert err <= TOL[prec], (b, err)
        assert u[b] == pytest.approx(Ur, rel=TOL[prec])
        assert w[b] == pytest.approx(Wr, rel=TOL[prec])


def test_batch_verlet(lc):
    boxes = small_batch(nbox=5, seed=9)
    with make_batch(lc, boxes, "fp64", with_vel=True) as g:
        g.verlet(0.005, 5, "atomic")
        pos = g.get("pos")
        u, k, w, npairs = g.energies()
    for b, bx in enumerate(boxes):
        x, v, f, e = oracle.verlet(bx["pos"], bx["vel"], bx["box"], RC, 0.005, 5)
        d = pos[g.offsets[b]:g.offsets[b + 1]] - x
        d -= bx["box"] * np.rint(d / bx["box"])
        assert np.abs(d).max() < 1e-9
        assert u[b] == pytest.approx(e[-1, 0], rel=1e-9)
        assert k[b] == pytest.approx(e[-1, 1], rel=1e-9)


def test_batch_rejects_colour_schedule(lc):
    boxes = small_batch(nbox=2)
    with make_batch(lc, boxes, "mixed") as g:
        with pytest.raises(lc.LCError) as e:
            g.forces("colour")
        assert e.value.code == 1
