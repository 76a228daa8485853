"""Batches of independent boxes (lc_batch_create) against the FP64 oracle,
box by box: bit-exact binning and pair counts, forces within the same
tolerances as single boxes, per-box energies, Verlet trajectories; the
colour schedule's device work queue over (colour, box, cells): the batched
configuration's spread of box sizes and densities, lc_batch_step, bounded
waits."""
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
@pytest.mark.parametrize("sched", ["colour", "atomic", "fullshell", "buffer"])
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


def spread_batch():
    """The batched configuration's spread: N log-uniform in [500, 50000],
    density U[0.5, 0.9], T U[0.7, 1.2], FCC + jitter 0.05, 12 boxes, plus the
    two extremes (N = 500 at density 0.9: 3 cells per side; N = 50000 at 0.5)."""
    boxes = inputs.batch_boxes(nbox=12, seed=77)
    boxes.append(inputs.fcc_box(500, 0.9, 1.2, seed=5, jitter=0.05))
    boxes.append(inputs.fcc_box(50000, 0.5, 0.7, seed=6, jitter=0.05))
    return boxes


def test_batch_colour_queue_config_spread(lc):
    boxes = spread_batch()
    ns = [b["pos"].shape[0] for b in boxes]
    assert min(ns) == 500 and max(ns) == 50000
    with make_batch(lc, boxes, "mixed") as g:
        g.forces("colour")
        f = g.get("forces")
        u, k, w, npairs = g.energies()
        g.forces("colour")                  # the same bits on a second evaluation
        assert np.array_equal(g.get("forces"), f)
        assert np.array_equal(g.energies()[0], u)
    for b, bx in enumerate(boxes):
        p = bx["pos"]
        fref, Ur, Wr, npr = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], bx["box"], RC)
        fb = f[g.offsets[b]:g.offsets[b + 1]]
        rms = math.sqrt(float((fref ** 2).sum(1).mean()))
        err = float(np.sqrt(((fb - fref) ** 2).sum(1)).max()) / rms
        assert npairs[b] == npr, b
        assert err <= TOL["mixed"], (b, ns[b], err)
        assert u[b] == pytest.approx(Ur, rel=TOL["mixed"])
        assert w[b] == pytest.approx(Wr, rel=TOL["mixed"])


def test_batch_step_against_oracle(lc):
    """lc_batch_step (colour queue) against the oracle's FP64 Verlet run of
    every box, FP64 path; and the mixed path against the atomic schedule."""
    boxes = small_batch(nbox=5, seed=9)
    with make_batch(lc, boxes, "fp64", with_vel=True) as g:
        g.step(0.005, 5)
        pos = g.get("pos")
        u, k, w, npairs = g.energies()
    for b, bx in enumerate(boxes):
        x, v, f, e = oracle.verlet(bx["pos"], bx["vel"], bx["box"], RC, 0.005, 5)
        d = pos[g.offsets[b]:g.offsets[b + 1]] - x
        d -= bx["box"] * np.rint(d / bx["box"])
        assert np.abs(d).max() < 1e-9
        assert u[b] == pytest.approx(e[-1, 0], rel=1e-9)
        assert k[b] == pytest.approx(e[-1, 1], rel=1e-9)
    with make_batch(lc, boxes, "mixed", with_vel=True) as g1, make_batch(lc, boxes, "mixed", with_vel=True) as g2:
        g1.step(0.005, 6)
        g2.verlet(0.005, 6, "atomic")
        d = g1.get("pos") - g2.get("pos")
        assert np.abs(d).max() < 1e-7


def test_batch_colour_queue_bounded_wait(lc):
    """With no task publishing its completion every wait for an
    earlier-coloured task runs out: LC_ERR_TIMEOUT, and the context stays
    usable once the flag is cleared."""
    boxes = small_batch(nbox=3)
    with make_batch(lc, boxes, "mixed") as g:
        g.set_queue_wait(0.05, withhold=True)
        g.forces("colour")
        with pytest.raises(lc.LCError) as e:
            g.energies()
        assert e.value.code == 6
        g.set_queue_wait(2.0)
        g.set_state(concat(boxes, "pos"))
        g.forces("colour")
        u, k, w, npairs = g.energies()
        p = boxes[0]["pos"]
        _, Ur, _, npr = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], boxes[0]["box"], RC)
        assert npairs[0] == npr and u[0] == pytest.approx(Ur, rel=1e-5)
