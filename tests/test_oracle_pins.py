"""Pins of the FP64 oracle against facts fixed by mathematics, not by itself.

Each test would catch a plausible slip in the oracle: a dropped factor or
sign in the pair force (closed form, finite differences), a wrong image or
wrap (boundary pair, translation invariance, O(N^2) == link-cell), a missed or
doubled neighbour cell (FCC shell sums, pair counts), an asymmetric update
(Newton's third law), a wrong integrator step (energy conservation,
time reversibility, a two-body trajectory against an independent ODE solver), a wrong sort (binning invariants), an unsafe colouring
(phase write sets).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1401_4441_gb300 import inputs

RC = 2.5


def lj_u(r):
    """Closed form U(r) = 4 (r^-12 - r^-6) (sigma = epsilon = 1)."""
    return 4.0 * (r ** -12 - r ** -6)


def lj_du(r):
    """dU/dr = 4 (-12 r^-13 + 6 r^-7)."""
    return 4.0 * (-12.0 * r ** -13 + 6.0 * r ** -7)


def two(r, L=10.0, x0=3.0, direction=(1.0, 0.0, 0.0)):
    e = np.asarray(direction, float)
    e = e / np.linalg.norm(e)
    p = np.array([[x0, 4.0, 5.0], [x0, 4.0, 5.0]]) + np.array([np.zeros(3), r * e])
    return p, np.array([L, L, L])


@pytest.mark.parametrize("r", [0.95, 1.0, 2 ** (1 / 6), 1.5, 2.2, 2.5 - 1e-9])
@pytest.mark.parametrize("fn", ["lc_forces", "nsq_forces"])
def test_two_particle_closed_form(r, fn):
    for direction in [(1, 0, 0), (1, 1, 0), (1, 2, 3)]:
        p, L = two(r, direction=direction)
        f, U, W, npairs = getattr(oracle, fn)(p[:, 0], p[:, 1], p[:, 2], L, RC)
        e = np.asarray(direction, float) / np.linalg.norm(direction)
        assert npairs == 1
        assert U == pytest.approx(lj_u(r), rel=1e-12, abs=1e-14)
        # particle 0 sits at -r e from particle 1: F_0 = -dU/dx_0 = dU/dr * e
        np.testing.assert_allclose(f[0], lj_du(r) * e, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(f[1], -lj_du(r) * e, rtol=1e-10, atol=1e-12)
        # virial W = r . F = -r dU/dr for one pair
        assert W == pytest.approx(-r * lj_du(r), rel=1e-10, abs=1e-12)


def test_two_particle_special_values():
    p, L = two(2 ** (1 / 6))
    f, U, W, _ = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], L, RC)
    assert U == pytest.approx(-1.0, abs=1e-14)
    assert np.abs(f).max() < 1e-12
    p, L = two(1.0)
    f, U, W, _ = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], L, RC)
    assert U == pytest.approx(0.0, abs=1e-14)
    assert f[0, 0] == pytest.approx(-24.0, rel=1e-14)


@pytest.mark.parametrize("fn", ["lc_forces", "nsq_forces"])
def test_cutoff_is_strict_and_truncated(fn):
    p, L = two(2.5 + 1e-9)
    f, U, W, npairs = getattr(oracle, fn)(p[:, 0], p[:, 1], p[:, 2], L, RC)
    assert npairs == 0 and U == 0.0 and np.abs(f).max() == 0.0
    p, L = two(2.5 - 1e-9)
    f, U, W, npairs = getattr(oracle, fn)(p[:, 0], p[:, 1], p[:, 2], L, RC)
    assert npairs == 1 and U == pytest.approx(lj_u(2.5), rel=1e-8)


@pytest.mark.parametrize("fn", ["lc_forces", "nsq_forces"])
def test_pair_across_periodic_boundary(fn):
    L = np.array([10.0, 11.0, 12.0])
    for d in range(3):
        p = np.array([[5.0, 5.5, 6.0], [5.0, 5.5, 6.0]])
        p[0, d] = 0.2
        p[1, d] = L[d] - 0.8            # 1.0 apart through the boundary
        f, U, W, npairs = getattr(oracle, fn)(p[:, 0], p[:, 1], p[:, 2], L, RC)
        assert npairs == 1
        assert U == pytest.approx(0.0, abs=1e-12)
        e = np.zeros(3); e[d] = 1.0       # particle 0 is +1 from the image of 1
        np.testing.assert_allclose(f[0], -lj_du(1.0) * e, rtol=1e-10, atol=1e-12)


def fcc_shells(a):
    """FCC neighbour shells inside r = 2.5 at lattice constant a: (count, distance).
    Counts from the lattice vectors a/2 (h, k, l) with h + k + l even."""
    shells = {}
    for h, k, l in itertools.product(range(-6, 7), repeat=3):
        if (h + k + l) % 2 or (h, k, l) == (0, 0, 0):
            continue
        r = 0.5 * a * math.sqrt(h * h + k * k + l * l)
        if r < RC:
            key = h * h + k * k + l * l
            shells[key] = (shells.get(key, (0, r))[0] + 1, r)
    return sorted(shells.values(), key=lambda t: t[1])


def test_fcc_lattice_shell_sums():
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.0)
    p, L = b["pos"], b["box"]
    a = L[0] / 10
    shells = fcc_shells(a)
    assert [z for z, _ in shells] == [12, 6, 24, 12]
    f, U, W, npairs = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], L, RC)
    n = p.shape[0]
    assert np.abs(f).max() < 1e-10          # every force vanishes by symmetry
    assert npairs == n * 54 // 2
    u_site = 0.5 * sum(z * lj_u(r) for z, r in shells)
    w_site = 0.5 * sum(z * (-r * lj_du(r)) for z, r in shells)
    assert U / n == pytest.approx(u_site, rel=1e-12)
    assert W / n == pytest.approx(w_site, rel=1e-12)


def jittered(n, rho=0.8442, jitter=0.2, seed=7):
    b = inputs.fcc_box(n, rho, 1.0, seed=seed, jitter=jitter)
    return b["pos"], b["box"]


def test_newton_third_law_and_nsq_equals_lc():
    for n, rho in [(250, 0.5), (500, 0.8442), (4000, 0.8442)]:
        p, L = jittered(n, rho)
        f1, U1, W1, n1 = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], L, RC)
        f2, U2, W2, n2 = oracle.nsq_forces(p[:, 0], p[:, 1], p[:, 2], L, RC)
        rms = math.sqrt((f2 ** 2).sum(1).mean())
        assert n1 == n2
        assert np.abs(f1 - f2).max() < 1e-11 * rms
        assert U1 == pytest.approx(U2, rel=1e-12)
        assert W1 == pytest.approx(W2, rel=1e-12)
        assert np.abs(f1.sum(0)).max() < 1e-11 * rms * math.sqrt(n)


def test_uneven_box_and_odd_grids():
    rng_pos = inputs.uniform(3, 0, 3 * 300).reshape(300, 3)
    L = np.array([9.1, 7.6, 12.7])           # 3 x 3 x 5 cells
    p = rng_pos * L
    f1, U1, W1, n1 = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], L, RC)
    f2, U2, W2, n2 = oracle.nsq_forces(p[:, 0], p[:, 1], p[:, 2], L, RC)
    assert n1 == n2
    rms = math.sqrt((f2 ** 2).sum(1).mean())
    assert np.abs(f1 - f2).max() < 1e-10 * rms


def test_translation_invariance():
    p, L = jittered(4000)
    f1, U1, W1, _ = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], L, RC)
    q = p + np.array([0.37, -1.1, 2.9])
    f2, U2, W2, _ = oracle.lc_forces(q[:, 0], q[:, 1], q[:, 2], L, RC)
    rms = math.sqrt((f1 ** 2).sum(1).mean())
    assert np.abs(f1 - f2).max() < 1e-9 * rms
    assert U1 == pytest.approx(U2, rel=1e-11)


def test_wrap_against_exact_modulo():
    """orc_wrap returns a value in [0, L) within a couple of units in the last
    place (of max(|x|, L)) of the exact real x mod L (rational arithmetic),
    and x itself for x already in [0, L)."""
    from fractions import Fraction
    for L in (10.0, 7.6, 107.49419, 2.5 * 165):
        xs = [0.0, -0.0, 1e-300, -1e-300, L, math.nextafter(L, 0.0), -L, 3.0 * L + 0.5, -2.5 * L, 0.5 * L,
              1e6 + 0.123, -1e6 - 0.123, L * 1e-17, -L * 1e-17]
        for x in xs:
            y = oracle.wrap(x, L)
            assert 0.0 <= y < L
            if 0.0 <= x < L:
                assert y == x
                continue
            ex = Fraction(x) - Fraction(L) * math.floor(Fraction(x) / Fraction(L))
            tol = 2.0 * math.ulp(max(abs(x), L))
            err = abs(Fraction(y) - ex)
            err = min(err, abs(Fraction(L) - err))   # the same point of the circle
            assert float(err) <= tol


def test_grid_is_the_floor_of_l_over_rc():
    """Cells per axis = floor(L / r_c) (exact for these values), refused when
    an axis has fewer than 3 cells."""
    from fractions import Fraction
    for L, rc in (([10.0, 7.6, 12.7], 2.5), ([107.49419, 107.49419, 107.49419], 2.5), ([7.5, 7.5, 30.0], 2.5),
                  ([7.4999, 9.0, 9.0], 2.5), ([485.29, 121.32, 121.32], 3.0)):
        nc, bad = oracle.grid(np.array(L), rc)
        ref = [math.floor(Fraction(v) / Fraction(rc)) for v in L]
        assert list(nc) == ref
        assert bad == (min(ref) < 3)


def test_forces_sample_equals_the_definition():
    """The sampled per-particle sums (the 27 cells around the particle's own
    cell) against a numpy brute force of the definition: every j != i under
    the minimum image, r < r_c, F_i = sum 24 (2 r^-14 - r^-8) d_ij; on an
    uneven box with positions outside [0, L) (wrapped by the oracle), with
    the neighbour counts compared exactly."""
    n = 600
    L = np.array([9.1, 7.6, 12.7])
    p = inputs.uniform(9, 0, 3 * n).reshape(n, 3) * L * 3.0 - L
    ids = np.array([0, 1, 17, 123, 300, 444, 599], np.int64)
    f, nn = oracle.forces_sample(p[:, 0], p[:, 1], p[:, 2], L, RC, ids)
    for s, i in enumerate(ids):
        d = p[i] - p
        d -= L * np.rint(d / L)
        r2 = (d * d).sum(1)
        m = r2 < RC * RC
        m[i] = False
        fij = (24.0 * (2.0 * r2[m] ** -7 - r2[m] ** -4))[:, None] * d[m]
        assert nn[s] == int(m.sum())
        scale = np.abs(fij).sum() + 1e-300
        assert np.abs(f[s] - fij.sum(0)).max() <= 1e-12 * scale


def test_force_is_minus_gradient_of_energy():
    p, L = jittered(300, rho=0.6, jitter=0.3, seed=11)
    f, U, W, _ = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], L, RC)
    h = 1e-6
    for i in [0, 17, 123]:
        for d in range(3):
            q = p.copy(); q[i, d] += h
            _, Up, _, np_p = oracle.lc_forces(q[:, 0], q[:, 1], q[:, 2], L, RC)
            q[i, d] -= 2 * h
            _, Um, _, np_m = oracle.lc_forces(q[:, 0], q[:, 1], q[:, 2], L, RC)
            assert np_p == np_m                 # no pair crossed the cutoff
            grad = (Up - Um) / (2 * h)
            assert -grad == pytest.approx(f[i, d], rel=1e-5, abs=2e-5)


def test_virial_equals_sum_r_dot_f():
    """W = sum over pairs r_ij . F_ij equals sum_i r_i . F_i for a cluster
    that does not touch the periodic boundary (no image terms)."""
    p, L = jittered(300, rho=0.8442, jitter=0.1, seed=5)
    box = L * 3.0
    q = p + L                                   # centre the cluster in a 3x box
    f, U, W, _ = oracle.lc_forces(q[:, 0], q[:, 1], q[:, 2], box, RC)
    assert W == pytest.approx(float((q * f).sum()), rel=1e-10)


def test_verlet_energy_conservation_and_reversibility():
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.0)
    x, v, f, e = oracle.verlet(b["pos"], b["vel"], b["box"], RC, 0.005, 10)
    E = e[:, 0] + e[:, 1]
    drift = np.abs(E - E[0]).max() / abs(E[0])
    assert drift < 1e-3
    # Second order: over the first 0.025 time units (before pairs cross the
    # truncated, unshifted cutoff, whose energy jumps do not depend on dt)
    # halving dt quarters the energy error.
    _, _, _, e_half = oracle.verlet(b["pos"], b["vel"], b["box"], RC, 0.0025, 10)
    E_half = e_half[:, 0] + e_half[:, 1]
    ratio = np.abs(E[:6] - E[0]).max() / np.abs(E_half - E_half[0]).max()
    assert 3.5 < ratio < 4.5
    assert e[0, 1] == pytest.approx(0.5 * 3 * (4000 - 1) * 0.72, rel=1e-12)
    # run back: velocity Verlet is time reversible
    x2, v2, f2, e2 = oracle.verlet(x, -v, b["box"], RC, 0.005, 10)
    dx = x2 - np.mod(b["pos"], b["box"])
    dx -= b["box"] * np.rint(dx / b["box"])
    assert np.abs(dx).max() < 1e-9
    assert np.abs(-v2 - b["vel"]).max() < 1e-9


def test_verlet_two_body_trajectory_converges_at_second_order():
    """Two particles far from every image (box 10, r_c 2.5): the oracle's
    velocity Verlet trajectory approaches the solution of Newton's equations
    for the closed-form pair force, integrated by scipy's DOP853 (8th order,
    rtol 1e-13), with the error falling four-fold per halved step.  A kick of
    dt instead of dt/2, a stale force in the closing kick or a sign slip gives
    order one or a diverging error."""
    from scipy.integrate import solve_ivp

    L = np.array([10.0, 10.0, 10.0])
    p = np.array([[4.4, 5.0, 5.0], [5.7, 5.1, 5.0]])
    v = np.array([[0.3, 0.1, 0.0], [-0.3, -0.1, 0.05]])

    def rhs(t, y):
        d = y[0:3] - y[3:6]
        r = np.linalg.norm(d)
        f0 = -lj_du(r) * d / r
        return np.concatenate([y[6:], f0, -f0])

    T = 0.6
    ref = solve_ivp(rhs, (0.0, T), np.concatenate([p.ravel(), v.ravel()]), method="DOP853",
                    rtol=1e-13, atol=1e-14).y[:, -1]
    errs = []
    for n in (150, 300, 600):
        x, vv, _, _ = oracle.verlet(p, v, L, RC, T / n, n)
        errs.append(max(np.abs(x.ravel() - ref[:6]).max(), np.abs(vv.ravel() - ref[6:]).max()))
    assert errs[0] < 2e-4
    for a, b in zip(errs, errs[1:]):
        assert 3.8 < a / b < 4.2


def test_binning_invariants():
    for n, L in [(4000, None), (777, np.array([9.1, 7.6, 12.7]))]:
        if L is None:
            p, L = jittered(n)
        else:
            p = inputs.uniform(9, 0, 3 * n).reshape(n, 3) * L * 1.7 - 0.3 * L   # outside [0, L) too
        r = oracle.bin(p[:, 0], p[:, 1], p[:, 2], L, RC)
        nc, count, start, perm = r["nc"], r["count"], r["start"], r["perm"]
        assert count.sum() == n
        assert np.array_equal(start, np.concatenate([[0], np.cumsum(count)[:-1]]))
        assert np.array_equal(np.sort(perm), np.arange(n))
        h = L / nc
        pw = np.mod(p, L)
        for c in range(count.shape[0]):
            ids = perm[start[c]:start[c] + count[c]]
            assert np.all(np.diff(ids) > 0)          # ascending ID inside a cell
            cz, rem = divmod(c, nc[0] * nc[1])
            cy, cx = divmod(rem, nc[0])
            cc = np.array([cx, cy, cz])
            assert np.all(pw[ids] >= cc * h - 1e-12) and np.all(pw[ids] < (cc + 1) * h + 1e-12)
        assert np.array_equal(r["cell_of"][perm], np.repeat(np.arange(count.shape[0]), count))


def test_binning_tiny_by_hand():
    L = np.array([7.5, 7.5, 7.5])     # 3 cells of side 2.5 per dimension
    p = np.array([[0.1, 0.1, 0.1],     # cell 0
                  [7.4, 0.1, 0.1],     # cell 2
                  [2.6, 5.1, 0.1],     # cell 1 + 3*2 = 7
                  [-0.1, 0.1, 0.1],    # wraps to x = 7.4 -> cell 2
                  [0.2, 0.2, 5.0]])    # cell 0 + 9*2 = 18  (5.0 / 2.5 = 2 exactly)
    r = oracle.bin(p[:, 0], p[:, 1], p[:, 2], L, RC)
    assert list(r["cell_of"]) == [0, 2, 7, 2, 18]
    assert list(r["perm"]) == [0, 1, 3, 2, 4]
    assert r["ncolours"] == 27


def phase_schedule(nc):
    """Enumerate the colour phases from the oracle's own definitions."""
    n = int(nc[0] * nc[1] * nc[2])
    p = np.zeros((max(n, 1), 3))
    r = oracle.bin(p[:1, 0], p[:1, 1], p[:1, 2], nc * 2.5, RC)
    colour, ncol = r["colour"], r["ncolours"]
    hs, groups = oracle.half_shell(), oracle.offset_groups()
    phases = []
    for g in range(4):
        offs = [tuple(hs[k]) for k in range(13) if groups[k] == g]
        for k in range(ncol):
            tasks = []
            for c in range(n):
                if colour[c] != k:
                    continue
                cz, rem = divmod(c, nc[0] * nc[1])
                cy, cx = divmod(rem, nc[0])
                pairs = [(c, c)] if g == 0 else []
                for o in offs:
                    b = ((cx + o[0]) % nc[0]) + nc[0] * (((cy + o[1]) % nc[1]) + nc[1] * ((cz + o[2]) % nc[2]))
                    pairs.append((c, int(b)))
                tasks.append(pairs)
            phases.append(tasks)
    return phases, ncol


@pytest.mark.parametrize("nc", [(4, 4, 4), (6, 6, 6), (3, 3, 3), (5, 4, 3), (7, 3, 4), (3, 8, 5)])
def test_colour_phases_disjoint_and_complete(nc):
    nc = np.array(nc)
    phases, ncol = phase_schedule(nc)
    odd = int((nc % 2 == 1).sum())
    assert ncol == 2 ** (3 - odd) * 3 ** odd
    hs = oracle.half_shell()
    covered = {}
    for tasks in phases:
        written = set()
        for pairs in tasks:
            cells = {c for pr in pairs for c in pr}
            assert written.isdisjoint(cells)         # no cell written twice in a phase
            written |= cells
            for pr in pairs:
                covered[pr] = covered.get(pr, 0) + 1
    n = int(nc.prod())
    expect = {}
    for c in range(n):
        cz, rem = divmod(c, nc[0] * nc[1]); cy, cx = divmod(rem, nc[0])
        expect[(c, c)] = 1
        for o in hs:
            b = ((cx + o[0]) % nc[0]) + nc[0] * (((cy + o[1]) % nc[1]) + nc[1] * ((cz + o[2]) % nc[2]))
            expect[(c, int(b))] = expect.get((c, int(b)), 0) + 1
    assert covered == expect
    # every unordered neighbour pair is visited once: no cell pair appears in both orders
    for (a, b) in covered:
        if a != b:
            assert (b, a) not in covered


def test_half_shell_is_a_half():
    hs = [tuple(o) for o in oracle.half_shell()]
    assert len(hs) == 13 and len(set(hs)) == 13
    for o in hs:
        assert tuple(-x for x in o) not in hs
    assert set(hs) | {tuple(-x for x in o) for o in hs} == set(itertools.product((-1, 0, 1), repeat=3)) - {(0, 0, 0)}


def test_force_scale():
    """S_i = sum_j |F_ij|: equals |F| for an isolated pair, the shell sum
    z |F(r_s)| on a perfect FCC lattice, and bounds |F_i| everywhere."""
    p, L = two(1.05)
    s = oracle.force_scale(p[:, 0], p[:, 1], p[:, 2], L, RC)
    assert s == pytest.approx([abs(lj_du(1.05))] * 2, rel=1e-12)
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.0)
    s = oracle.force_scale(b["pos"][:, 0], b["pos"][:, 1], b["pos"][:, 2], b["box"], RC)
    shells = fcc_shells(b["box"][0] / 10)
    assert np.allclose(s, sum(z * abs(lj_du(r)) for z, r in shells), rtol=1e-12)
    q, Lq = jittered(4000)
    f, _, _, _ = oracle.lc_forces(q[:, 0], q[:, 1], q[:, 2], Lq, RC)
    s = oracle.force_scale(q[:, 0], q[:, 1], q[:, 2], Lq, RC)
    assert np.all(np.sqrt((f ** 2).sum(1)) <= s * (1 + 1e-12))


# ---- 2D (Sec. IV, Fig. 3a): the oracle's 3D routines on particles in the
# z = 0 plane of a box whose z side is 3 r_c (every z image farther than
# r_c) compute the 2D Lennard-Jones system; pinned here by 2D lattice sums.

def embed_2d(pos, box2):
    return pos, np.array([box2[0], box2[1], 3.0 * RC])


def test_triangular_lattice_shell_sums_2d():
    b = inputs.tri_box(16, 16, 0.7, 0.5)
    p, L = embed_2d(b["pos"], b["box"])
    a = b["a"]
    # shells of the triangular lattice within r_c = 2.5: 6 at a, 6 at a sqrt(3)
    assert math.sqrt(3.0) * a < RC < 2.0 * a
    shells = [(6, a), (6, math.sqrt(3.0) * a)]
    f, U, W, npairs = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], L, RC)
    n = p.shape[0]
    assert np.abs(f).max() < 1e-10          # every force vanishes by symmetry
    assert npairs == n * 12 // 2
    u_site = 0.5 * sum(z * lj_u(r) for z, r in shells)
    w_site = 0.5 * sum(z * (-r * lj_du(r)) for z, r in shells)
    assert U / n == pytest.approx(u_site, rel=1e-12)
    assert W / n == pytest.approx(w_site, rel=1e-12)


def test_2d_forces_stay_in_plane_and_lc_equals_nsq():
    b = inputs.tri_box(12, 10, 0.7, 0.5, jitter=0.2)
    p, L = embed_2d(b["pos"], b["box"])
    f1, U1, W1, n1 = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], L, RC)
    f2, U2, W2, n2 = oracle.nsq_forces(p[:, 0], p[:, 1], p[:, 2], L, RC)
    rms = math.sqrt((f2 ** 2).sum(1).mean())
    assert n1 == n2 and n1 > 0
    assert np.abs(f1 - f2).max() < 1e-11 * rms
    assert np.all(f1[:, 2] == 0.0)
    assert U1 == pytest.approx(U2, rel=1e-12)
