"""Seeded synthetic inputs for the link-cell Lennard-Jones sweep.

This module feeds both the CUDA path and the CPU oracle, so it holds none of
the method's arithmetic (no binning, no cells, no forces): only particle
positions, velocities and box sizes.  Random numbers come from a
counter-based SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): value i of stream s is the
SplitMix64 output function applied to key(seed, s) + (i + 1) * 0x9E3779B97F4A7C15,
so every draw is reproducible on any machine and independent of call order.

Workloads (reduced LJ units, sigma = epsilon = m = 1):
  fcc_box       FCC lattice at density rho in a cubic periodic box, optional
                uniform jitter, Maxwell velocities at T.  N != 4 n^3 leaves
                uniformly chosen vacancies (seeded partial Fisher-Yates).
  slab_box      liquid slab (density 0.80) filling the first third of x of a
                4:1:1 box, vapour (0.02) elsewhere, uniform random positions,
                redrawn until no pair is closer than r_min.
  batch_boxes   independent cubic boxes with log-uniform N, uniform density
                and temperature, FCC plus jitter starts.
  tri_box       2D: triangular lattice (rows of spacing a, alternate rows
                shifted by a/2, row pitch a sqrt(3)/2) filling a periodic
                rectangle commensurate with it, optional jitter, 2D Maxwell
                velocities; positions keep three components with z = 0.
"""
import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
DEFAULT_SEED = 20140117


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed, stream):
    s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    t = np.array([stream & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(_mix(s) ^ (t * np.uint64(0xD1B54A32D192ED03)))[0]


def u64(seed, stream, n, offset=0):
    """n raw 64-bit draws of stream `stream`, counters offset .. offset+n-1."""
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(_key(seed, stream) + i * GOLDEN)


def uniform(seed, stream, n, offset=0):
    """Doubles in [0, 1) with 53 random bits."""
    return (u64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian(seed, stream, n):
    """Standard normals by the Box-Muller transform of two uniform streams."""
    u1 = 1.0 - uniform(seed, stream, n)          # (0, 1]
    u2 = uniform(seed, stream + 1, n)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def maxwell(n, T, seed, stream=100):
    """Velocities (n, 3): normal with variance T per component, zero total
    momentum, rescaled so that sum v^2 = 3 (n - 1) T."""
    v = np.stack([gaussian(seed, stream + 2 * d, n) for d in range(3)], axis=1) * math.sqrt(T)
    if n > 1:
        v -= v.mean(axis=0, keepdims=True)
        s2 = float((v * v).sum())
        if s2 > 0:
            v *= math.sqrt(3.0 * (n - 1) * T / s2)
    return v


def cube_side(n, rho):
    """Edge of a cubic box holding n particles at number density rho."""
    return (n / rho) ** (1.0 / 3.0)


def fcc_cells_per_side(n):
    """Smallest n_uc with 4 n_uc^3 >= n (integer search, no pow rounding)."""
    m = 1
    while 4 * m * m * m < n:
        m += 1
    return m


def fcc_positions(n, L, seed, jitter=0.0, stream=10):
    """FCC sites (i + b) a + a/4 with a = L / n_uc, x fastest then y then z,
    basis b in {0, (1/2,1/2,0), (1/2,0,1/2), (0,1/2,1/2)}; the a/4 offset keeps
    sites off the cell faces.  If 4 n_uc^3 > n, a seeded partial Fisher-Yates
    picks the vacancies.  Jitter adds U[-jitter, +jitter) per coordinate."""
    m = fcc_cells_per_side(n)
    a = L / m
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    iz, iy, ix = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    pos = sites * a + a / 4.0
    total = pos.shape[0]
    if total > n:
        nvac = total - n
        idx = np.arange(total, dtype=np.int64)
        u = uniform(seed, stream, nvac)
        for k in range(nvac):
            j = k + int(u[k] * (total - k))
            idx[k], idx[j] = idx[j], idx[k]
        keep = np.sort(idx[nvac:])
        pos = pos[keep]
    if jitter > 0.0:
        for d in range(3):
            pos[:, d] += (2.0 * uniform(seed, stream + 1 + d, n) - 1.0) * jitter
    return np.ascontiguousarray(pos)


def fcc_box(n, rho, T, seed=DEFAULT_SEED, jitter=0.0):
    """Cubic periodic FCC box: returns dict(pos (n,3), vel (n,3), box (3,))."""
    L = cube_side(n, rho)
    pos = fcc_positions(n, L, seed, jitter)
    vel = maxwell(n, T, seed)
    return dict(pos=pos, vel=vel, box=np.array([L, L, L]), rho=rho, T=T, seed=seed)


def slab_box(n=2_000_000, rho_liq=0.80, rho_vap=0.02, T=0.85, seed=DEFAULT_SEED,
             r_min=0.01, aspect=4.0):
    """Liquid slab in x in [0, Lx/3), vapour elsewhere, Ly = Lz, Lx = aspect Ly.
    Uniform random positions in each region; any particle closer than r_min to
    an earlier one is redrawn (fresh counters) until no such pair is left."""
    V = n / (rho_liq / 3.0 + rho_vap * 2.0 / 3.0)
    Ly = (V / aspect) ** (1.0 / 3.0)
    Lx = aspect * Ly
    box = np.array([Lx, Ly, Ly])
    n_liq = int(round(rho_liq * V / 3.0))
    n_vap = n - n_liq
    lo = np.concatenate([np.zeros(n_liq), np.full(n_vap, Lx / 3.0)])
    width = np.concatenate([np.full(n_liq, Lx / 3.0), np.full(n_vap, 2.0 * Lx / 3.0)])

    def draw(ids, rnd):
        off = int(rnd) * n
        p = np.empty((ids.shape[0], 3))
        p[:, 0] = lo[ids] + width[ids] * uniform(seed, 40, n, off)[ids]
        p[:, 1] = Ly * uniform(seed, 41, n, off)[ids]
        p[:, 2] = Ly * uniform(seed, 42, n, off)[ids]
        return p

    pos = draw(np.arange(n), 0)
    redraws = 0
    from scipy.spatial import cKDTree  # scipy is present on both machines
    for rnd in range(1, 64):
        pos_w = np.mod(pos, box)
        pos_w[pos_w >= box] = 0.0
        pairs = cKDTree(pos_w, boxsize=box).query_pairs(r_min, output_type="ndarray")
        if pairs.shape[0] == 0:
            break
        bad = np.unique(pairs.max(axis=1))
        pos[bad] = draw(bad, rnd)
        redraws += bad.shape[0]
    vel = maxwell(n, T, seed)
    return dict(pos=np.ascontiguousarray(pos), vel=vel, box=box, n_liq=n_liq,
                T=T, seed=seed, redraws=redraws)


def batch_boxes(nbox=512, n_min=500, n_max=50_000, rho=(0.5, 0.9), T=(0.7, 1.2),
                seed=DEFAULT_SEED, jitter=0.05):
    """Independent cubic boxes; box b uses seed + b for its own lattice and
    velocities.  N is log-uniform in [n_min, n_max], density and temperature
    uniform in their ranges."""
    un = uniform(seed, 60, nbox)
    ur = uniform(seed, 61, nbox)
    ut = uniform(seed, 62, nbox)
    ns = np.rint(np.exp(math.log(n_min) + un * (math.log(n_max) - math.log(n_min)))).astype(np.int64)
    rhos = rho[0] + ur * (rho[1] - rho[0])
    Ts = T[0] + ut * (T[1] - T[0])
    boxes = []
    for b in range(nbox):
        boxes.append(fcc_box(int(ns[b]), float(rhos[b]), float(Ts[b]), seed=seed + 1 + b, jitter=jitter))
    return boxes


def maxwell2d(n, T, seed, stream=120):
    """In-plane velocities (n, 3) with vz = 0: normal with variance T per
    component, zero total momentum, rescaled so that sum v^2 = 2 (n - 1) T."""
    v = np.zeros((n, 3))
    v[:, :2] = np.stack([gaussian(seed, stream + 2 * d, n) for d in range(2)], axis=1) * math.sqrt(T)
    if n > 1:
        v[:, :2] -= v[:, :2].mean(axis=0, keepdims=True)
        s2 = float((v * v).sum())
        if s2 > 0:
            v *= math.sqrt(2.0 * (n - 1) * T / s2)
    return v


def tri_box(nx, ny, rho, T, seed=DEFAULT_SEED, jitter=0.0, stream=30):
    """2D triangular lattice of nx particles per row and ny rows (ny even, so
    the periodic box is commensurate): spacing a from the number density rho
    (area per particle a^2 sqrt(3)/2), box (nx a, ny a sqrt(3)/2).  Jitter
    adds U[-jitter, +jitter) to x and y.  Returns dict(pos (n, 3) with z = 0,
    vel (n, 3) with vz = 0, box (2,))."""
    if ny % 2:
        raise ValueError("ny must be even for a periodic triangular lattice")
    a = math.sqrt(2.0 / (math.sqrt(3.0) * rho))
    h = a * math.sqrt(3.0) / 2.0
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    x = (ix + 0.5 * (iy % 2) + 0.25) * a
    y = (iy + 0.25) * h
    n = nx * ny
    pos = np.zeros((n, 3))
    pos[:, 0] = x.ravel()
    pos[:, 1] = y.ravel()
    if jitter > 0.0:
        for d in range(2):
            pos[:, d] += (2.0 * uniform(seed, stream + 1 + d, n) - 1.0) * jitter
    return dict(pos=np.ascontiguousarray(pos), vel=maxwell2d(n, T, seed), box=np.array([nx * a, ny * h]),
                rho=rho, T=T, seed=seed, a=a)


# Named workloads (sizes of the single-box configurations).
WORKLOADS = {
    "fcc4k": dict(n=4000, rho=0.8442, T=0.72, rc=2.5, jitter=0.0),
    "liquid1m": dict(n=1_048_576, rho=0.8442, T=0.72, rc=2.5, jitter=0.05),
    "fcc16m": dict(n=16_777_216, rho=0.8442, T=0.72, rc=2.5, jitter=0.0),
    "slab2m": dict(n=2_000_000, rho=None, T=0.85, rc=3.0, jitter=0.0, kind="slab"),
    # 2D liquid: 1024 x 1024 triangular lattice at area density 0.7, jittered
    "liquid2d": dict(n=1024 * 1024, nx=1024, ny=1024, rho=0.7, T=0.5, rc=2.5, jitter=0.05, kind="2d"),
}


def workload(name, seed=DEFAULT_SEED):
    w = WORKLOADS[name]
    if w.get("kind") == "2d":
        b = tri_box(w["nx"], w["ny"], w["rho"], w["T"], seed=seed, jitter=w["jitter"])
        b["rc"] = w["rc"]
        b["name"] = name
        b["dims"] = 2
        return b
    if w.get("kind") == "slab":
        b = slab_box(n=w["n"], T=w["T"], seed=seed)
        b["rc"] = w["rc"]
        b["name"] = name
        b["rho"] = None
        return b
    b = fcc_box(w["n"], w["rho"], w["T"], seed=seed, jitter=w["jitter"])
    b["rc"] = w["rc"]
    b["name"] = name
    return b
