"""The force sweep as a task DAG executed on the device (Sec. III, Sec. V,
Sec. VI Strategy 2): the library's DAG against the oracle's address-based
DAG builder, the execution order against the DAG's edges, the forces against
the FP64 oracle, and the bounded waits."""
import math

import numpy as np
import pytest

import oracle
from oracle import dag as odag
from paper_1401_4441_gb300 import inputs

pytestmark = pytest.mark.gpu

RC = 2.5
TOL = {"fp64": 1e-10, "mixed": 1e-5}


def creation_order(dims, order):
    """The library's two creation orders written with the oracle's task
    helper: cells x fastest; stencil = intra + the 13 forward offsets in
    (z, y, x) order; loop exchange visits colours ordered by their class
    code class_x + 3 class_y + 9 class_z."""
    stencil = [(0, 0, 0)] + odag.half_shell_3d()
    cells = list(odag._cells(dims))
    if order == "cell":
        return [odag.lc_task(c, o, dims) for c in cells for o in stencil]
    key = lambda k: k[0] + 3 * k[1] + 9 * k[2]
    colours = sorted(set(odag._colour(c, dims) for c in cells), key=key)
    return [odag.lc_task(c, o, dims) for o in stencil for k in colours for c in cells
            if odag._colour(c, dims) == k]


def box_for(dims, rho=0.8, seed=11):
    """Uniform random particles (near-overlaps removed) in a box of
    dims cells of side 2.56."""
    box = np.array(dims, float) * 2.56
    n = int(rho * box.prod())
    pos = inputs.uniform(seed, 0, 3 * n).reshape(n, 3) * box
    from scipy.spatial import cKDTree
    pairs = cKDTree(np.mod(pos, box), boxsize=box).query_pairs(0.8, output_type="ndarray")
    keep = np.ones(n, bool)
    keep[np.unique(pairs[:, 1])] = False
    return pos[keep], box


@pytest.mark.parametrize("dims", [(6, 6, 6), (3, 4, 5), (10, 10, 30)])
@pytest.mark.parametrize("order", ["cell", "loopex"])
def test_dag_matches_oracle(lc, dims, order):
    pos, box = box_for(dims)
    with lc.Box(box, RC, pos.shape[0]) as g:
        nc, _, _ = g.grid()
        assert tuple(nc) == dims
        ntasks, nedges, cp = g.dag_build(order)
    parents = odag.build_dag(creation_order(dims, order))
    assert ntasks == len(parents) == 14 * int(np.prod(dims))
    assert nedges == sum(len(p) for p in parents)
    assert cp == odag.critical_path(parents)


def test_dag_critical_paths_paper_domain(lc):
    """A 30 x 10 x 10 cell domain: with the intra-cell task first the cell
    order's speedup bound stays below the 7 of Sec. V (14 stencil tasks,
    displacement at least 2), while loop exchange with colouring has a
    critical path of 27 tasks whatever the domain size (Sec. VI: not
    limited by the stencil)."""
    pos, box = box_for((30, 10, 10), rho=0.05)
    with lc.Box(box, RC, pos.shape[0]) as g:
        t, _, cp_cell = g.dag_build("cell")
        _, _, cp_lx = g.dag_build("loopex")
    assert t == 42000
    assert 6.0 < t / cp_cell <= 7.0
    assert cp_lx == 27


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("order", ["cell", "loopex"])
def test_dag_forces_and_trace(lc, prec, order):
    import torch
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    pos, box = b["pos"], b["box"]
    fref, U, W, npairs = oracle.lc_forces(pos[:, 0], pos[:, 1], pos[:, 2], box, RC)
    with lc.Box(box, RC, pos.shape[0], prec) as g:
        g.set_state(pos)
        nc, _, _ = g.grid()
        ntasks, _, _ = g.dag_build(order)
        trace = torch.full((2 * ntasks,), -1, dtype=torch.int32, device="cuda")
        g.dag_forces(order, trace=trace)
        f = g.get("forces")
        u, k, w, np_ = g.energy()
        # a second evaluation without a trace gives the same result
        g.dag_forces(order)
        f2 = g.get("forces")
    rms = math.sqrt(float((fref ** 2).sum(1).mean()))
    assert float(np.sqrt(((f - fref) ** 2).sum(1)).max()) / rms <= TOL[prec]
    assert float(np.sqrt(((f2 - fref) ** 2).sum(1)).max()) / rms <= TOL[prec]
    assert np_ == npairs
    assert u == pytest.approx(U, rel=TOL[prec])
    assert w == pytest.approx(W, rel=TOL[prec])
    tr = trace.cpu().numpy().reshape(-1, 2)
    # every task ran exactly once, stamps are a permutation of 0 .. 2T-1
    assert np.array_equal(np.sort(tr.ravel()), np.arange(2 * ntasks))
    assert np.all(tr[:, 0] < tr[:, 1])
    # every dependency edge of the oracle's DAG was respected
    parents = odag.build_dag(creation_order(tuple(int(x) for x in nc), order))
    src = np.array([p for t, ps in enumerate(parents) for p in ps])
    dst = np.array([t for t, ps in enumerate(parents) for _ in ps])
    assert np.all(tr[src, 1] < tr[dst, 0])


def test_dag_wait_times_out_and_context_recovers(lc):
    """With no task published every wait for a queue slot runs out: the call
    returns LC_ERR_TIMEOUT after about the limit, and the next call works."""
    import time
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    pos, box = b["pos"], b["box"]
    with lc.Box(box, RC, pos.shape[0], "mixed") as g:
        g.set_state(pos)
        g.dag_build("loopex")
        t0 = time.time()
        with pytest.raises(lc.LCError) as e:
            g.dag_forces("loopex", wait_seconds=0.05, withhold=True)
        assert e.value.code == 6
        assert time.time() - t0 < 30
        g.dag_forces("loopex")
        u, k, w, np_ = g.energy()
        g.forces("atomic")
        u2, _, _, np2 = g.energy()
    assert np_ == np2 and u == pytest.approx(u2, rel=1e-5)
