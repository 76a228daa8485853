"""Verlet neighbour lists (schedule "list": not the paper's method, an
extension built on its link cells) against the FP64 oracle.

Fresh builds: forces within 1e-5 of the RMS force, energy and virial within
1e-5, the exact pair count.  Rows longer than the list capacity (swept from
the cells instead) give the same result.  Trajectories that reuse the lists
follow the oracle's, and the number of rebuilds the device decides equals
the displacement rule (2 max |x - x_build| > skin) applied to the oracle's
own trajectory.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1401_4441_gb300 import inputs

pytestmark = pytest.mark.gpu

RC = 2.5
TOL = 1e-5


def rel_err(f, fref):
    rms = math.sqrt(float((fref ** 2).sum(1).mean()))
    return float(np.sqrt(((f - fref) ** 2).sum(1)).max()) / rms


def list_case(lc, pos, box, skin=0.3, kmax=0, max_tol=TOL):
    fref, U, W, npairs = oracle.lc_forces(pos[:, 0], pos[:, 1], pos[:, 2], box, RC)
    with lc.Box(box, RC, pos.shape[0], "mixed") as g:
        g.set_state(pos)
        g.set_skin(skin, kmax)
        g.forces("list")
        f = g.get("forces")
        u, k, w, np_ = g.energy()
        info = g.list_info()
    assert np_ == npairs
    assert rel_err(f, fref) <= max_tol
    assert u == pytest.approx(U, rel=TOL)
    assert w == pytest.approx(W, rel=TOL)
    assert info["builds"] == 1
    return f, info


def test_list_forces_4k(lc):
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    _, info = list_case(lc, b["pos"], b["box"])
    # FCC + small jitter: 78 partners within rc + skin on average
    assert 60 <= info["longest_row"] <= 120 and info["long_rows"] == 0
    assert info["kmax"] == info["longest_row"] + info["longest_row"] // 4 + 8
    # every pair within rc + skin in two rows: brute force over the box
    from scipy.spatial import cKDTree
    pos, box = b["pos"], b["box"]
    n_rl = len(cKDTree(np.mod(pos, box), boxsize=box).query_pairs(RC + 0.3))
    assert abs(info["entries"] - 2 * n_rl) <= 2 * 1e-3 * n_rl   # FP32 test with a 2e-5 margin on (rc + skin)^2


def test_list_forces_liquid_like(lc):
    """Strong jitter: close pairs, many pairs near rc (gate as the link-cell
    schedules on this input)."""
    b = inputs.fcc_box(20000, 0.8442, 1.0, seed=3, jitter=0.12)
    list_case(lc, b["pos"], b["box"], max_tol=2e-5)


@pytest.mark.parametrize("kmax", [1, 8, 70])
def test_list_long_rows_swept_from_cells(lc, kmax):
    """Rows longer than the capacity are swept from the 27 list cells: same
    pairs, same forces as rows that fit."""
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    f_full, _ = list_case(lc, b["pos"], b["box"])
    f, info = list_case(lc, b["pos"], b["box"], kmax=kmax)
    assert info["kmax"] == kmax and info["long_rows"] > 0
    assert np.abs(f - f_full).max() <= 1e-5 * np.abs(f_full).max()


def test_list_overlap_stress(lc):
    """Overlapping particles (min distance 0.46 sigma, forces up to 1e6): the
    exact pair set, and the error bound the link-cell schedules meet on this
    input (FP32 pair math keeps about 1e-6 of each particle's own force)."""
    b = inputs.fcc_box(20000, 0.8442, 1.0, seed=3, jitter=0.25)
    pos, box = b["pos"], b["box"]
    fref, U, W, npairs = oracle.lc_forces(pos[:, 0], pos[:, 1], pos[:, 2], box, RC)
    with lc.Box(box, RC, pos.shape[0], "mixed") as g:
        g.set_state(pos)
        g.forces("list")
        f = g.get("forces")
        u, k, w, np_ = g.energy()
    assert np_ == npairs
    assert rel_err(f, fref) <= 1e-4
    assert u == pytest.approx(U, rel=1e-4)


def test_list_odd_grids_and_skins(lc):
    for box, skin in ((np.array([9.1, 8.5, 12.7]), 0.3), (np.array([10.2, 15.3, 8.6]), 0.1),
                      (np.array([7.6, 7.6, 7.6]), 0.0)):
        n = int(0.7 * box.prod())
        pos = inputs.uniform(9, 0, 3 * n).reshape(n, 3) * box
        from scipy.spatial import cKDTree
        pairs = cKDTree(np.mod(pos, box), boxsize=box).query_pairs(0.8, output_type="ndarray")
        keep = np.ones(n, bool)
        keep[np.unique(pairs[:, 1])] = False
        list_case(lc, pos[keep], box, skin=skin)


def test_list_box_too_small_for_skin(lc):
    """7.6 / (2.5 + 0.3) < 3 list cells: reported, the context stays usable."""
    box = np.array([7.6, 7.6, 7.6])
    pos = inputs.uniform(9, 0, 300).reshape(100, 3) * box
    with lc.Box(box, RC, 100, "mixed") as g:
        g.set_state(pos)
        with pytest.raises(lc.LCError) as ei:
            g.forces("list")
        assert ei.value.code == 2   # LC_ERR_BOX_TOO_SMALL
        g.set_skin(0.0)
        g.forces("list")
        g.forces("atomic")


def test_list_dense_cells(lc):
    """Crowded cells: more than 32 particles per list cell and candidate
    lists beyond one batch."""
    n = 1500
    box = np.array([10.0, 10.0, 10.0])
    u = inputs.uniform(8, 0, 3 * n).reshape(n, 3)
    pos = np.where(np.arange(n)[:, None] < 900, u * 4.9 + 0.05, u * box)
    from scipy.spatial import cKDTree
    pairs = cKDTree(np.mod(pos, box), boxsize=box).query_pairs(0.35, output_type="ndarray")
    keep = np.ones(n, bool)
    keep[np.unique(pairs[:, 1])] = False
    _, info = list_case(lc, pos[keep], box)
    assert info["longest_row"] > 300


def test_list_empty_and_tiny(lc):
    box = np.array([12.0, 12.0, 12.0])
    with lc.Box(box, RC, 0, "mixed") as g:
        g.set_state(np.zeros((0, 3)))
        g.forces("list")
        u, k, w, np_ = g.energy()
        assert (u, k, w, np_) == (0.0, 0.0, 0.0, 0)
        g.verlet(0.005, 3, "list")
    pos = np.array([[1.0, 1.0, 1.0], [2.2, 1.0, 1.0], [11.5, 1.0, 1.0]])   # one pair across the boundary
    list_case(lc, pos, box)


def test_list_1m(lc):
    b = inputs.workload("liquid1m")
    list_case(lc, b["pos"], b["box"])


def test_list_rejects(lc):
    box = np.array([16.8, 16.8, 16.8])
    with lc.Box(box, RC, 10, "mixed") as g:
        for bad in ((-0.1, 0), (float("nan"), 0), (0.3, -1)):
            with pytest.raises(lc.LCError):
                g.set_skin(*bad)
    with lc.Box(box, RC, 10, "fp64") as g:
        g.set_state(inputs.uniform(1, 0, 30).reshape(10, 3) * box)
        with pytest.raises(lc.LCError):
            g.forces("list")
    with lc.Batch([box, box], RC, [5, 5]) as g:
        g.set_state(inputs.uniform(1, 0, 30).reshape(10, 3) * 16.8)
        with pytest.raises(lc.LCError):
            g.forces("list")
        with pytest.raises(lc.LCError):
            g.verlet(0.005, 2, "list")


def oracle_rebuild_steps(pos, vel, box, dt, nsteps, skin):
    """Steps at which the displacement rule asks for a rebuild, on the
    oracle's trajectory, and the smallest distance of the rule's maximum to
    its threshold (near-ties could go either way in the mixed path)."""
    x, v = pos.copy(), vel.copy()
    f = None
    ref = np.mod(pos, box)
    thr = 0.5 * skin - 1e-6
    steps, margin = [], np.inf
    for s in range(nsteps):
        x, v, f, _ = oracle.verlet(x, v, box, RC, dt, 1, f=f)
        d = x - ref
        d -= box * np.rint(d / box)
        dmax = float(np.sqrt((d ** 2).sum(1)).max())
        margin = min(margin, abs(dmax - thr))
        if dmax > thr:
            steps.append(s)
            ref = x.copy()
    return steps, margin


@pytest.mark.parametrize("skin", [0.3, 0.08])
def test_list_verlet_matches_oracle(lc, skin):
    """Reused lists and device-decided rebuilds: the trajectory and energies
    of the oracle, and its rebuild count."""
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    nsteps = 40
    x, v, f, e = oracle.verlet(b["pos"], b["vel"], b["box"], RC, 0.005, nsteps)
    with lc.Box(b["box"], RC, 4000, "mixed") as g:
        g.set_state(b["pos"], b["vel"])
        g.set_skin(skin)
        g.verlet(0.005, 17, "list")   # graphs of two steps and one step
        g.verlet(0.005, 23, "list")
        u, k, w, np_ = g.energy()
        p = g.get("pos")
        vel = g.get("vel")
        info = g.list_info()
        g.forces("list")              # the lists are still valid: no build
        f_now = g.get("forces")
        _, _, _, np_now = g.energy()
        assert g.list_info()["builds"] == info["builds"]
    fref, _, _, npairs_now = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], b["box"], RC)
    assert np_now == npairs_now
    assert rel_err(f_now, fref) <= TOL
    dx = p - x
    dx -= b["box"] * np.rint(dx / b["box"])
    assert np.abs(dx).max() < 1e-5
    assert np.abs(vel - v).max() < 1e-4
    assert np.all((p >= 0) & (p < b["box"]))
    assert u == pytest.approx(e[-1, 0], rel=1e-5)
    assert k == pytest.approx(e[-1, 1], rel=1e-5)
    steps, margin = oracle_rebuild_steps(b["pos"], b["vel"], b["box"], 0.005, nsteps, skin)
    assert info["builds"] == 1 + info["rebuild_steps"]
    if margin > 1e-4:
        assert info["rebuild_steps"] == len(steps)
    else:
        assert abs(info["rebuild_steps"] - len(steps)) <= 1
    if skin < 0.1:
        assert len(steps) >= 3


def test_list_verlet_mixed_with_link_cells(lc):
    """List steps, link-cell steps and list steps again on one context: the
    lists are rebuilt after the link-cell binning re-sorted the state."""
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    x, v, f, e = oracle.verlet(b["pos"], b["vel"], b["box"], RC, 0.005, 9)
    with lc.Box(b["box"], RC, 4000, "mixed") as g:
        g.set_state(b["pos"], b["vel"])
        g.verlet(0.005, 3, "list")
        g.verlet(0.005, 1, "atomic")
        g.verlet(0.005, 2, "list")
        g.forces("atomic")
        g.verlet(0.005, 3, "list")
        p = g.get("pos")
        u, k, w, np_ = g.energy()
        with pytest.raises(lc.LCError):
            g.get("cell_count")   # the link-cell binning is stale after list steps
        g.bin()
        g.get("cell_count")
    dx = p - x
    dx -= b["box"] * np.rint(dx / b["box"])
    assert np.abs(dx).max() < 1e-5
    assert u == pytest.approx(e[-1, 0], rel=1e-5)


def test_list_2d(lc):
    """2D context: the 9-cell list stencil against the oracle's 2D system."""
    b = inputs.tri_box(120, 100, 0.7, 0.5, seed=4, jitter=0.05)
    pos, box2 = b["pos"], b["box"]
    L = np.array([box2[0], box2[1], 3.0 * RC])
    fref, U, W, npairs = oracle.lc_forces(pos[:, 0], pos[:, 1], np.zeros(pos.shape[0]), L, RC)
    with lc.Box(box2, RC, pos.shape[0], "mixed", dims=2) as g:
        g.set_state(pos)
        g.forces("list")
        f = g.get("forces")
        u, k, w, np_ = g.energy()
        g.verlet(0.005, 5, "list")
        p = g.get("pos")
    assert np_ == npairs
    assert rel_err(f, fref) <= TOL
    assert np.all(f[:, 2] == 0.0) and np.all(p[:, 2] == 0.0)
    assert u == pytest.approx(U, rel=TOL)


def test_list_energy_drift_1m(lc):
    """Liquid, 1M particles, 100 list steps: the energy drift of the
    link-cell path on the same run (both mixed precision)."""
    b = inputs.workload("liquid1m")
    drift = {}
    for sched in ("atomic", "list"):
        with lc.Box(b["box"], RC, b["pos"].shape[0], "mixed") as g:
            g.set_state(b["pos"], b["vel"])
            g.forces(sched)
            u0, k0, _, _ = g.energy()
            g.verlet(0.005, 100, sched)
            u1, k1, _, _ = g.energy()
            if sched == "list":
                info = g.list_info()
        drift[sched] = abs((u1 + k1) - (u0 + k0)) / abs(u0 + k0)
    assert info["long_rows"] == 0 and info["builds"] >= 2
    assert drift["list"] <= 3 * drift["atomic"] + 1e-6, drift


def test_list_16m_sampled(lc):
    """The 16.7M-particle box from fresh lists: per-particle oracle sums on a
    sample, and the pair count of the link-cell sweep on the same state."""
    b = inputs.workload("fcc16m")
    pos, box = b["pos"], b["box"]
    with lc.Box(box, RC, pos.shape[0], "mixed") as g:
        g.set_state(pos)
        g.forces("list")
        f = g.get("forces")
        _, _, _, np_list = g.energy()
        info = g.list_info()
        g.forces("atomic")
        _, _, _, np_lc = g.energy()
    ids = np.linspace(0, pos.shape[0] - 1, 3000).astype(np.int64)
    fref, _ = oracle.forces_sample(pos[:, 0], pos[:, 1], pos[:, 2], box, RC, ids)
    scale = max(1e-3, math.sqrt(float((fref ** 2).sum(1).mean())))
    assert np.abs(f[ids] - fref).max() <= 1e-5 * scale + 1e-9
    assert np_list == np_lc
    assert info["long_rows"] == 0 and info["builds"] == 1


def test_list_verlet_skin_change_and_long_rows(lc):
    """Skin changed between calls (the lists and step graphs are rebuilt),
    and steps whose rows mostly exceed the capacity (swept from the cells
    inside the captured step): the oracle's trajectory."""
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    x, v, f, e = oracle.verlet(b["pos"], b["vel"], b["box"], RC, 0.005, 12)
    with lc.Box(b["box"], RC, 4000, "mixed") as g:
        g.set_state(b["pos"], b["vel"])
        g.set_skin(0.3)
        g.verlet(0.005, 4, "list")
        g.set_skin(0.1, 40)                 # rows of ~55: most are swept from the cells
        g.verlet(0.005, 5, "list")
        info = g.list_info()
        g.set_skin(0.5)
        g.verlet(0.005, 3, "list")
        p = g.get("pos")
        u, k, w, np_ = g.energy()
    assert info["kmax"] == 40 and info["long_rows"] > 0 and info["builds"] >= 1
    dx = p - x
    dx -= b["box"] * np.rint(dx / b["box"])
    assert np.abs(dx).max() < 1e-5
    assert u == pytest.approx(e[-1, 0], rel=1e-5)
