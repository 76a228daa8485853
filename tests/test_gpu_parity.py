"""GPU path (C ABI via the ctypes binding) against the FP64 oracle.

Bit-exact: cell counts, cell starts, the slot -> ID permutation, colours and
the number of pairs inside r_c.  Floating point: FP64 path within 1e-10 of
the RMS force; mixed path within 1e-5 (max over particles of |dF| / RMS |F|),
energy and virial within 1e-5 relative.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1401_4441_gb300 import inputs
from test_colour_cells import colours as schedule_colours

pytestmark = pytest.mark.gpu

RC = 2.5
# "rows": the atomic schedule through its row-group kernel (tile setting
# ni = 16, warps = 16; mixed precision, single 3D boxes)
SCHEDS = ["colour", "atomic", "fullshell", "buffer", "rows"]
TOL = {"fp64": 1e-10, "mixed": 1e-5}


def run(b, sched):
    """The schedule's force evaluation ("rows": the row-group kernel)."""
    if sched == "rows":
        b.set_tile(16, 16)
        sched = "atomic"
    b.forces(sched)


def rel_force_err(f, fref):
    rms = math.sqrt(float((fref ** 2).sum(1).mean()))
    return float(np.sqrt(((f - fref) ** 2).sum(1)).max()) / rms, rms


def make(lc, pos, box, prec, vel=None):
    b = lc.Box(box, RC, pos.shape[0], prec)
    b.set_state(pos, vel)
    return b


def check_bin(lc, pos, box):
    ref = oracle.bin(pos[:, 0], pos[:, 1], pos[:, 2], box, RC)
    with make(lc, pos, box, "mixed") as b:
        b.bin()
        assert np.array_equal(b.get("cell_count"), ref["count"])
        assert np.array_equal(b.get("cell_start"), ref["start"])
        assert np.array_equal(b.get("perm"), ref["perm"])
        assert np.array_equal(b.get("colour"), ref["colour"])
        nc, ncol, nph = b.grid()
        assert np.array_equal(nc, ref["nc"]) and ncol == ref["ncolours"] and nph == schedule_colours(nc)
        p = b.get("pos")
        for i in range(0, pos.shape[0], max(1, pos.shape[0] // 50)):
            for d in range(3):
                assert p[i, d] == oracle.wrap(pos[i, d], box[d])


def test_binning_bit_exact_small(lc):
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    check_bin(lc, b["pos"], b["box"])
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.0)
    check_bin(lc, b["pos"], b["box"])


def test_binning_bit_exact_uneven_and_outside(lc):
    n = 3000
    box = np.array([9.1, 7.6, 12.7])        # 3 x 3 x 5 cells: 27 colours... odd dims
    pos = inputs.uniform(5, 0, 3 * n).reshape(n, 3) * box * 3.0 - box   # spans [-L, 2L)
    check_bin(lc, pos, box)


def test_binning_dense_cells(lc):
    """Cells holding far more than a warp of particles (ragged, > 32 and > 512)."""
    n = 2500
    box = np.array([10.0, 10.0, 10.0])
    u = inputs.uniform(6, 0, 3 * n).reshape(n, 3)
    pos = np.where(np.arange(n)[:, None] < 1800, u * 2.4 + 0.05, u * box)
    check_bin(lc, pos, box)


def test_binning_bit_exact_many_scan_tiles(lc):
    """A dilute gas over 165^3 = 4.49M cells: 1097 scan tiles of 4096 cells,
    more than the 1024 threads of the block that scans the tile totals (its
    carry loop runs twice); most cells are empty."""
    n = 200000
    box = np.array([412.5, 412.5, 412.5])
    pos = inputs.uniform(8, 0, 3 * n).reshape(n, 3) * box
    check_bin(lc, pos, box)


def test_binning_bit_exact_1m(lc):
    b = inputs.workload("liquid1m")
    check_bin(lc, b["pos"], b["box"])


def forces_case(lc, pos, box, prec, sched):
    """Forces, pair count, energy and virial of one evaluation against the
    oracle: the max over particles and the RMS over particles of |dF| / RMS |F|
    are both held to TOL."""
    fref, U, W, npairs = oracle.lc_forces(pos[:, 0], pos[:, 1], pos[:, 2], box, RC)
    with make(lc, pos, box, prec) as b:
        run(b, sched)
        f = b.get("forces")
        u, k, w, np_ = b.energy()
    err, rms = rel_force_err(f, fref)
    rms_err = math.sqrt(float(((f - fref) ** 2).sum(1).mean())) / rms
    assert np_ == npairs
    assert rms_err <= TOL[prec], (prec, sched, rms_err)
    assert err <= TOL[prec], (prec, sched, err)
    assert u == pytest.approx(U, rel=TOL[prec], abs=1e-12)
    assert w == pytest.approx(W, rel=TOL[prec], abs=1e-12)
    return err


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("sched", SCHEDS)
def test_forces_4k_jittered(lc, prec, sched):
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    forces_case(lc, b["pos"], b["box"], prec, sched)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("sched", SCHEDS)
def test_forces_liquid_like(lc, prec, sched):
    """Strong jitter (RMS force 86, harsher than an equilibrium liquid at
    T = 0.72): close pairs, uneven occupancy, many pairs near r_c.  The
    largest per-particle errors come from the closest pairs, whose FP32 r^2
    rounding the r^-14 of the force amplifies; those pairs (r < 0.95) are
    computed in FP64, so the mixed path meets 1e-5 (max over particles)."""
    b = inputs.fcc_box(20000, 0.8442, 1.0, seed=3, jitter=0.12)
    err = forces_case(lc, b["pos"], b["box"], prec, sched)
    print(f"liquid-like {prec} {sched}: max |dF| / RMS {err:.2e}")


@pytest.mark.parametrize("sched", SCHEDS)
def test_forces_overlap_stress(lc, sched):
    """Overlapping particles (min distance 0.46 sigma, forces up to 1e6,
    heavy-tailed): the pairs closer than 0.95 sigma, which carry the large
    forces, are computed in FP64, so the mixed path meets the same 1e-5 of
    the RMS force as on the workloads, with the exact pair set; the FP64 path
    meets 1e-10."""
    b = inputs.fcc_box(20000, 0.8442, 1.0, seed=3, jitter=0.25)
    pos, box = b["pos"], b["box"]
    fref, U, W, npairs = oracle.lc_forces(pos[:, 0], pos[:, 1], pos[:, 2], box, RC)
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-5)):
        with make(lc, pos, box, prec) as g:
            run(g, sched)
            f = g.get("forces")
            u, k, w, np_ = g.energy()
        err, rms = rel_force_err(f, fref)
        print(f"overlap stress {prec} {sched}: max |dF| / RMS {err:.2e}")
        assert np_ == npairs
        assert err <= tol, (prec, err)
        assert u == pytest.approx(U, rel=tol)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("sched", SCHEDS)
def test_forces_odd_and_minimal_grids(lc, prec, sched):
    for box in (np.array([7.6, 7.6, 7.6]), np.array([9.1, 7.6, 12.7]), np.array([10.2, 15.3, 7.9])):
        n = int(0.7 * box.prod())
        pos = inputs.uniform(9, 0, 3 * n).reshape(n, 3) * box
        # keep the uniform random positions but drop near-overlaps
        keep = np.ones(n, bool)
        from scipy.spatial import cKDTree
        pairs = cKDTree(np.mod(pos, box), boxsize=box).query_pairs(0.8, output_type="ndarray")
        keep[np.unique(pairs[:, 1])] = False
        forces_case(lc, pos[keep], box, prec, sched)


def test_forces_dense_cells(lc):
    """Particles crowded into few cells (> 32 and > NI per cell, j lists over
    512 entries), all schedules agree with the oracle."""
    n = 1500
    box = np.array([10.0, 10.0, 10.0])
    u = inputs.uniform(8, 0, 3 * n).reshape(n, 3)
    pos = np.where(np.arange(n)[:, None] < 900, u * 4.9 + 0.05, u * box)
    from scipy.spatial import cKDTree
    pairs = cKDTree(np.mod(pos, box), boxsize=box).query_pairs(0.35, output_type="ndarray")
    keep = np.ones(n, bool)
    keep[np.unique(pairs[:, 1])] = False
    pos = pos[keep]
    for prec in ("fp64", "mixed"):
        for sched in SCHEDS:
            forces_case(lc, pos, box, prec, sched)


@pytest.mark.parametrize("sched", SCHEDS)
def test_forces_1m_mixed(lc, sched):
    b = inputs.workload("liquid1m")
    err = forces_case(lc, b["pos"], b["box"], "mixed", sched)
    print(f"1M {sched}: max |dF|/rms = {err:.3e}")


def test_rows_unstaged_runs(lc):
    """Row-group kernel with r_c = 4 (54 particles per cell): a group's rows
    hold more particles than a shared-memory slot, so its later runs are
    read from global memory; forces and the pair set as the oracle's."""
    b = inputs.fcc_box(4 * 38 ** 3, 0.8442, 0.72, seed=12, jitter=0.08)
    pos, box = b["pos"], b["box"]
    rc = 4.0
    assert np.floor(box / rc).min() >= 15
    fref, U, W, npairs = oracle.lc_forces(pos[:, 0], pos[:, 1], pos[:, 2], box, rc)
    with lc.Box(box, rc, pos.shape[0], "mixed") as g:
        g.set_state(pos)
        g.set_tile(16, 16)
        g.forces("atomic")
        f = g.get("forces")
        u, k, w, np_ = g.energy()
    err, rms = rel_force_err(f, fref)
    assert np_ == npairs
    assert err <= TOL["mixed"], err
    assert u == pytest.approx(U, rel=1e-5) and w == pytest.approx(W, rel=1e-5)


def test_rows_verlet_agrees_with_atomic(lc):
    """Mixed Verlet steps through the row-group kernel (captured step graphs)
    follow the per-warp atomic kernel's trajectory."""
    b = inputs.fcc_box(32000, 0.8442, 0.72, seed=5, jitter=0.05)
    with make(lc, b["pos"], b["box"], "mixed", b["vel"]) as g1, \
            make(lc, b["pos"], b["box"], "mixed", b["vel"]) as g2:
        g1.set_tile(16, 16)
        for g in (g1, g2):
            g.verlet(0.005, 3, "atomic")
            g.verlet(0.005, 4, "atomic")
        d = g1.get("pos") - g2.get("pos")
        d -= b["box"] * np.rint(d / b["box"])
        assert np.abs(d).max() < 1e-7
        e1, e2 = g1.energy(), g2.energy()
        assert e1[3] == e2[3]
        assert e1[0] == pytest.approx(e2[0], rel=1e-6)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_buffer_schedule_reproducible(lc, prec):
    """Buffer schedule (Sec. VI, Strategy 3): every partial force has its own
    buffer entry and the reduce sums them in a fixed order, so repeated
    evaluations and a fresh context give bit-identical forces and energies
    (the atomic schedule's FP64 atomics make no such promise)."""
    b = inputs.fcc_box(200_000, 0.8442, 0.72, seed=5, jitter=0.05)
    runs = []
    for _ in range(2):
        with make(lc, b["pos"], b["box"], prec) as g:
            for _ in range(2):
                g.forces("buffer")
                runs.append((g.get("forces"), g.energy()))
    for f, e in runs[1:]:
        assert np.array_equal(f, runs[0][0])
        assert e == runs[0][1]
    fref, U, W, npairs = oracle.lc_forces(b["pos"][:, 0], b["pos"][:, 1], b["pos"][:, 2], b["box"], RC)
    err, _ = rel_force_err(runs[0][0], fref)
    assert err <= TOL[prec]


@pytest.mark.parametrize("sched", SCHEDS)
def test_schedule_check(lc, sched):
    # cells per dimension: 6^3, 3^3, (5, 4, 7), (42, 11, 3), (9, 13, 5): one, two, odd and even block counts
    for box in (np.array([16.8, 16.8, 16.8]), np.array([7.6, 7.6, 7.6]), np.array([12.7, 10.2, 17.6]),
                np.array([105.0, 27.6, 8.1]), np.array([22.6, 32.6, 12.6])):
        with lc.Box(box, RC, 10, "mixed") as b:
            conflicts, cover = b.schedule_check("atomic" if sched == "rows" else sched)
            assert conflicts == 0 and cover == 0


def test_empty_and_single(lc):
    box = np.array([8.0, 8.0, 8.0])
    for n in (0, 1):
        pos = np.full((n, 3), 1.0)
        with make(lc, pos, box, "mixed") as b:
            for s in SCHEDS:
                run(b, s)
                u, k, w, np_ = b.energy()
                assert (u, w, np_) == (0.0, 0.0, 0)
                if n:
                    assert np.all(b.get("forces") == 0.0)


def test_errors(lc):
    with pytest.raises(lc.LCError) as e:
        lc.Box([7.4, 8.0, 8.0], RC, 10)
    assert e.value.code == 2
    box = np.array([8.0, 8.0, 8.0])
    pos = np.full((5, 3), 1.0)
    pos[3, 1] = np.nan
    with make(lc, pos, box, "mixed") as b:
        b.forces("atomic")
        with pytest.raises(lc.LCError) as e:
            b.energy()
        assert e.value.code == 5
    with lc.Box(box, RC, 5) as b:
        with pytest.raises(lc.LCError) as e:
            b.forces("colour")
        assert e.value.code == 7


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_verlet_4k(lc, prec):
    b = inputs.workload("fcc4k")
    x, v, f, e = oracle.verlet(b["pos"], b["vel"], b["box"], RC, 0.005, 10)
    with make(lc, b["pos"], b["box"], prec, b["vel"]) as g:
        g.forces("colour")
        u0, k0, w0, _ = g.energy()
        assert u0 == pytest.approx(e[0, 0], rel=TOL[prec])
        assert k0 == pytest.approx(e[0, 1], rel=1e-12)
        g.verlet(0.005, 10, "colour")
        u, k, w, np_ = g.energy()
        p = g.get("pos")
        vel = g.get("vel")
    dx = p - x
    dx -= b["box"] * np.rint(dx / b["box"])
    tol = 1e-9 if prec == "fp64" else 1e-6
    assert np.abs(dx).max() < tol
    assert np.abs(vel - v).max() < tol * 10
    assert u == pytest.approx(e[-1, 0], rel=tol)
    assert k == pytest.approx(e[-1, 1], rel=tol)


@pytest.mark.parametrize("prec,sched", [("fp64", "atomic"), ("mixed", "colour"), ("mixed", "list")])
def test_kinetic_from_the_kick(lc, prec, sched):
    """K after an odd step count comes from the one-step graph's closing
    kick (fused partials and a last-block sum), after an even count and
    after list steps from a pass over the velocities, after lc_set_state
    from the set-up pass: each equal to 1/2 sum v^2 of the velocities read
    back, and the same from lc_energy_virial and the asynchronous result
    block."""
    import torch
    b = inputs.fcc_box(4000, 0.8442, 0.72, seed=3, jitter=0.05)
    res = torch.zeros(6, dtype=torch.float64).pin_memory()

    def half_v2(v):
        return 0.5 * math.fsum((v.astype(np.float64) ** 2).ravel())

    with make(lc, b["pos"], b["box"], prec, b["vel"]) as g:
        g.forces(sched)
        assert g.energy()[1] == pytest.approx(half_v2(b["vel"]), rel=1e-13)
        for nsteps in (3, 2, 1):
            g.verlet(0.005, nsteps, sched)
            u, k, w, np_ = g.energy()
            assert k == pytest.approx(half_v2(g.get("vel")), rel=1e-13)
            g.energy_async(res)
            torch.cuda.synchronize()
            assert lc.decode(res) == (u, k, w, np_)
        g.set_state(g.get("pos"), g.get("vel"))
        g.forces("atomic" if sched == "list" else sched)
        assert g.energy()[1] == pytest.approx(half_v2(g.get("vel")), rel=1e-13)


def test_kinetic_magnitudes(lc):
    """K of velocities with components far from unit size (3e13, 2e-15,
    7e-13, zero) among ordinary ones, through the set-up pass, the kinetic
    pass (two steps of dt = 0) and the kick of a one-step graph (dt = 0):
    1/2 sum v^2 to 1e-13; all-zero velocities: exactly 0."""
    b = inputs.fcc_box(4000, 0.8442, 0.72, seed=5, jitter=0.05)
    v = b["vel"].copy()
    v[0, 0] = 3.0e13
    v[1, 1] = -2.0e-15
    v[2, :] = 0.0
    v[3, 2] = 7.0e-13
    want = 0.5 * math.fsum((v ** 2).ravel())
    with make(lc, b["pos"], b["box"], "mixed", v) as g:
        g.forces("atomic")
        assert g.energy()[1] == pytest.approx(want, rel=1e-13)
        g.verlet(0.0, 2, "atomic")
        assert g.energy()[1] == pytest.approx(want, rel=1e-13)
        g.verlet(0.0, 1, "atomic")
        assert g.energy()[1] == pytest.approx(want, rel=1e-13)
    with make(lc, b["pos"], b["box"], "mixed") as g:
        g.forces("atomic")
        assert g.energy()[1] == 0.0
        g.verlet(0.0, 1, "atomic")
        assert g.energy()[1] == 0.0


@pytest.mark.parametrize("sched", SCHEDS)
def test_verlet_schedules_agree(lc, sched):
    """Odd step counts (graph of two steps + one direct step) and repeated
    calls give the oracle's trajectory."""
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    x, v, f, e = oracle.verlet(b["pos"], b["vel"], b["box"], RC, 0.005, 7)
    with make(lc, b["pos"], b["box"], "fp64", b["vel"]) as g:
        if sched == "rows":   # no effect in FP64 (the row kernel is mixed only)
            g.set_tile(16, 16)
            sched = "atomic"
        g.verlet(0.005, 3, sched)
        g.verlet(0.005, 1, sched)
        g.verlet(0.005, 3, sched)
        p = g.get("pos")
        u, k, w, _ = g.energy()
    dx = p - x
    dx -= b["box"] * np.rint(dx / b["box"])
    assert np.abs(dx).max() < 1e-9
    assert u == pytest.approx(e[-1, 0], rel=1e-9)


def test_16m_sampled(lc):
    """Full 16.7M-particle box, mixed colour schedule, against per-particle
    oracle sums on a sample of particles, plus pair-count and Newton-3 checks."""
    b = inputs.workload("fcc16m")
    pos, box = b["pos"], b["box"]
    with make(lc, pos, box, "mixed") as g:
        g.forces("colour")
        f = g.get("forces")
        u, k, w, np_ = g.energy()
    ids = np.linspace(0, pos.shape[0] - 1, 3000).astype(np.int64)
    fref, nn = oracle.forces_sample(pos[:, 0], pos[:, 1], pos[:, 2], box, RC, ids)
    scale = max(1e-3, math.sqrt(float((fref ** 2).sum(1).mean())))
    assert np.abs(f[ids] - fref).max() <= 1e-5 * scale + 1e-9
    assert np_ > 0
    # Newton's third law: the net force per particle vanishes (lattice
    # rounding is coherent across cells, so bound the mean, not sqrt(N))
    assert np.abs(f.sum(0)).max() < 1e-6 * pos.shape[0]


def test_set_state_host_paths(lc):
    """Pageable host arrays (copied), page-locked host arrays (read in place
    by the set-up kernel) and device arrays give the same binned state and
    forces, bit for bit."""
    import torch
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    pos, vel = b["pos"], b["vel"]
    outs = []
    for kind in ("pageable", "pinned", "device"):
        if kind == "pageable":
            p, v = pos, vel
        elif kind == "pinned":
            p, v = torch.from_numpy(pos).pin_memory(), torch.from_numpy(vel).pin_memory()
        else:
            p, v = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
        with lc.Box(b["box"], RC, pos.shape[0], "mixed") as g:
            g.set_state(p, v)
            g.forces("buffer")
            outs.append((g.get("perm"), g.get("forces"), g.get("vel")))
    for perm, f, v in outs[1:]:
        assert np.array_equal(perm, outs[0][0])
        assert np.array_equal(f, outs[0][1])
        assert np.array_equal(v, outs[0][2])


def test_staged_host_input(lc):
    """Host input staged ahead on a copy stream (two slots) gives the same
    state and forces as lc_set_state, and slots can be refilled while the
    other one is in use."""
    import torch
    b1 = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    b2 = inputs.fcc_box(4000, 0.8442, 0.72, seed=9, jitter=0.05)
    h = [(torch.from_numpy(b["pos"]).pin_memory(), torch.from_numpy(b["vel"]).pin_memory()) for b in (b1, b2)]
    ref = []
    with lc.Box(b1["box"], RC, 4000, "mixed") as g:
        for p, v in h:
            g.set_state(p, v)
            g.forces("buffer")
            ref.append((g.get("forces"), g.get("vel")))
    cs = torch.cuda.Stream()
    with lc.Box(b1["box"], RC, 4000, "mixed") as g:
        with pytest.raises(lc.LCError):
            g.set_state_staged(1)                 # never staged
        g.stage_state(*h[0], slot=0, copy_stream=cs.cuda_stream)
        for k in range(4):
            g.set_state_staged(k % 2)
            g.stage_state(*h[(k + 1) % 2], slot=(k + 1) % 2, copy_stream=cs.cuda_stream)
            g.forces("buffer")
            f, v = g.get("forces"), g.get("vel")
            assert np.array_equal(f, ref[k % 2][0])
            assert np.array_equal(v, ref[k % 2][1])
        torch.cuda.synchronize()


def test_energy_async_pipelined(lc):
    """Result blocks read back without waiting: decoded one step later they
    equal lc_energy_virial's values, with staged host input on a copy stream
    (the pipelined end-to-end loop of the benchmark)."""
    import torch
    boxes = [inputs.fcc_box(4000, 0.8442, 0.72, seed=s, jitter=0.05) for s in (1, 2)]
    h = [(torch.from_numpy(b["pos"]).pin_memory(), torch.from_numpy(b["vel"]).pin_memory()) for b in boxes]
    ref = []
    with lc.Box(boxes[0]["box"], RC, 4000, "mixed") as g:
        for p, v in h:
            g.set_state(p, v)
            g.forces("buffer")
            ref.append(g.energy())
        res = [torch.zeros(6, dtype=torch.float64).pin_memory() for _ in range(2)]
        done = [torch.cuda.Event(), torch.cuda.Event()]
        cs = torch.cuda.Stream()
        st = torch.cuda.current_stream()
        got = []
        g.stage_state(*h[0], slot=0, copy_stream=cs.cuda_stream)
        for k in range(6):
            g.set_state_staged(k % 2)
            if k + 1 < 6:
                g.stage_state(*h[(k + 1) % 2], slot=(k + 1) % 2, copy_stream=cs.cuda_stream)
            g.forces("buffer")
            g.energy_async(res[k % 2])
            done[k % 2].record(st)
            if k >= 1:
                done[(k - 1) % 2].synchronize()
                got.append(lc.decode(res[(k - 1) % 2]))
        done[1].synchronize()
        got.append(lc.decode(res[1]))
        for k, e in enumerate(got):
            assert e == ref[k % 2]
        g.set_state(*h[0])
        with pytest.raises(lc.LCError) as ei:
            g.energy_async(res[0])          # no forces for this state yet
        assert ei.value.code == 7
    with lc.Batch([boxes[0]["box"]] * 2, RC, [10, 10]) as g:
        with pytest.raises(lc.LCError):
            g.energy_async(res[0])
