"""2D link-cell force sweep (Sec. IV, Fig. 3a: the 5-cell stencil) against
the FP64 oracle, whose 3D routines compute the 2D system for particles in
the z = 0 plane of a box with a z side of 3 r_c (pinned by 2D lattice sums
in the oracle tests); and the 2D task DAG on the device (Sec. V, Fig. 5)."""
import math

import numpy as np
import pytest

import oracle
from oracle import dag as odag
from paper_1401_4441_gb300 import inputs
from test_colour_cells import colours as schedule_colours

pytestmark = pytest.mark.gpu

RC = 2.5
SCHEDS = ["colour", "atomic", "fullshell", "buffer"]
TOL = {"fp64": 1e-10, "mixed": 1e-5}


def embed(pos, box2):
    return np.array([box2[0], box2[1], 3.0 * RC])


def reference(pos, box2):
    L = embed(pos, box2)
    return oracle.lc_forces(pos[:, 0], pos[:, 1], np.zeros(pos.shape[0]), L, RC)


def check(lc, pos, box2, prec, sched):
    fref, U, W, npairs = reference(pos, box2)
    with lc.Box(box2, RC, pos.shape[0], prec, dims=2) as g:
        g.set_state(pos)
        g.forces(sched)
        f = g.get("forces")
        u, k, w, np_ = g.energy()
        p = g.get("pos")
    rms = math.sqrt(float((fref ** 2).sum(1).mean()))
    assert np_ == npairs
    assert float(np.sqrt(((f - fref) ** 2).sum(1)).max()) / rms <= TOL[prec]
    assert np.all(f[:, 2] == 0.0) and np.all(p[:, 2] == 0.0)
    assert u == pytest.approx(U, rel=TOL[prec])
    assert w == pytest.approx(W, rel=TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("sched", SCHEDS)
def test_2d_liquid_forces(lc, prec, sched):
    """Jitter 0.05 as the 2D workload, and 0.15 (forces to 14x the RMS)."""
    for jitter in (0.05, 0.15):
        b = inputs.tri_box(120, 100, 0.7, 0.5, seed=4, jitter=jitter)
        check(lc, b["pos"], b["box"], prec, sched)


@pytest.mark.parametrize("sched", SCHEDS)
def test_2d_uniform_odd_grids(lc, sched):
    for box2 in (np.array([7.6, 9.1]), np.array([12.7, 7.9]), np.array([31.0, 23.3])):
        n = int(0.6 * box2.prod())
        u = inputs.uniform(21, 0, 2 * n).reshape(n, 2) * box2
        pos = np.zeros((n, 3))
        pos[:, :2] = u
        from scipy.spatial import cKDTree
        pairs = cKDTree(np.mod(u, box2), boxsize=box2).query_pairs(0.8, output_type="ndarray")
        keep = np.ones(n, bool)
        keep[np.unique(pairs[:, 1])] = False
        for prec in ("fp64", "mixed"):
            check(lc, pos[keep], box2, prec, sched)


def test_2d_perfect_lattice_and_grid(lc):
    b = inputs.tri_box(64, 64, 0.7, 0.5)
    with lc.Box(b["box"], RC, b["pos"].shape[0], "mixed", dims=2) as g:
        g.set_state(b["pos"])
        nc, ncol, nph = g.grid()
        assert nc[2] == 1 and ncol == 4 and nph == schedule_colours(nc, dims=2)
        for sched in SCHEDS:
            g.forces(sched)
            f = g.get("forces")
            _, _, _, np_ = g.energy()
            assert np.abs(f).max() < 1e-5
            assert np_ == b["pos"].shape[0] * 6


@pytest.mark.parametrize("sched", SCHEDS)
def test_2d_schedule_check(lc, sched):
    for box2 in (np.array([16.8, 16.8]), np.array([7.6, 12.7]), np.array([10.2, 17.6])):
        with lc.Box(box2, RC, 10, "mixed", dims=2) as b:
            assert b.schedule_check(sched) == (0, 0)


def test_2d_verlet_against_oracle(lc):
    b = inputs.tri_box(40, 40, 0.7, 0.5, seed=6, jitter=0.05)
    pos, vel, box2 = b["pos"], b["vel"], b["box"]
    x, v, f, e = oracle.verlet(pos, vel, embed(pos, box2), RC, 0.005, 7)
    with lc.Box(box2, RC, pos.shape[0], "fp64", dims=2) as g:
        g.set_state(pos, vel)
        g.verlet(0.005, 7, "atomic")
        p = g.get("pos")
        vv = g.get("vel")
        u, k, w, _ = g.energy()
    dx = p[:, :2] - x[:, :2]
    dx -= box2 * np.rint(dx / box2)
    assert np.abs(dx).max() < 1e-9
    assert np.abs(vv - v).max() < 1e-8
    assert u == pytest.approx(e[-1, 0], rel=1e-9)
    assert k == pytest.approx(e[-1, 1], rel=1e-9)


# The library's 2D stencil entries: 0 intra, then the forward offsets
# (1,0), (-1,1), (0,1), (1,1) in (y, x) order.
LIB_2D = [(0, 0), (1, 0), (-1, 1), (0, 1), (1, 1)]


@pytest.mark.parametrize("perm", [(0, 1, 2, 3, 4), (0, 2, 3, 1, 4), (0, 2, 3, 4, 1), (1, 0, 4, 3, 2)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_2d_dag_on_device(lc, perm, prec):
    """Stencil orders of the cell creation order (their DAG speedups span the
    Fig. 5 range: 2.43, 1.24, 1.00, 4.80 on 50 x 50 cells) and the loop
    exchange run by the device queue: forces as the oracle's, every DAG edge
    respected."""
    import torch
    b = inputs.tri_box(60, 60, 0.7, 0.5, seed=8, jitter=0.05)
    pos, box2 = b["pos"], b["box"]
    fref, U, W, npairs = reference(pos, box2)
    rms = math.sqrt(float((fref ** 2).sum(1).mean()))
    with lc.Box(box2, RC, pos.shape[0], prec, dims=2) as g:
        g.set_state(pos)
        nc, _, _ = g.grid()
        dims = (int(nc[0]), int(nc[1]))
        g.dag_stencil_order(perm)
        for order in ("cell", "loopex"):
            t, e, cp = g.dag_build(order)
            trace = torch.full((2 * t,), -1, dtype=torch.int32, device="cuda")
            g.dag_forces(order, trace=trace)
            f = g.get("forces")
            _, _, _, np_ = g.energy()
            assert np_ == npairs
            assert float(np.sqrt(((f - fref) ** 2).sum(1)).max()) / rms <= TOL[prec]
            if order == "cell":
                tasks = odag.basic_order_tasks(dims, [LIB_2D[k] for k in perm])
            else:
                cells = list(odag._cells(dims))
                key = lambda c: c[0] + 3 * c[1]
                cols = sorted(set(odag._colour(c, dims) for c in cells), key=key)
                tasks = [odag.lc_task(c, o, dims) for o in LIB_2D for k in cols for c in cells
                         if odag._colour(c, dims) == k]
            parents = odag.build_dag(tasks)
            assert cp == odag.critical_path(parents) and t == len(parents)
            tr = trace.cpu().numpy().reshape(-1, 2)
            assert np.array_equal(np.sort(tr.ravel()), np.arange(2 * t))
            src = np.array([p for s, ps in enumerate(parents) for p in ps])
            dst = np.array([s for s, ps in enumerate(parents) for _ in ps])
            assert np.all(tr[src, 1] < tr[dst, 0])
