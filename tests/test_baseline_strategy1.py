"""The OpenMP Strategy-1 CPU baseline (loop exchange + 2-strided colouring,
Sec. VI, Fig. 6) gives the oracle's link-cell forces, energy, virial and pair
count, on even and odd grids and with several threads."""
import math

import numpy as np
import pytest

import baseline
import oracle
from paper_1401_4441_gb300 import inputs


@pytest.mark.parametrize("case", ["fcc4k", "odd", "outside"])
def test_strategy1_matches_oracle(case):
    if case == "fcc4k":
        b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
        pos, box = b["pos"], b["box"]
    else:
        box = np.array([9.1, 12.7, 17.6])            # 3 x 5 x 7 cells: odd dimensions
        n = int(0.6 * box.prod())
        pos = inputs.uniform(13, 0, 3 * n).reshape(n, 3) * box
        if case == "outside":
            pos = pos * 2.0 - 0.5 * box              # positions outside [0, L) as well
        from scipy.spatial import cKDTree
        keep = np.ones(n, bool)
        pairs = cKDTree(np.mod(pos, box), boxsize=box).query_pairs(0.8, output_type="ndarray")
        keep[np.unique(pairs[:, 1])] = False
        pos = pos[keep]
    f, U, W, npairs = baseline.forces(pos, box, 2.5)
    fref, Ur, Wr, npr = oracle.lc_forces(pos[:, 0], pos[:, 1], pos[:, 2], box, 2.5)
    rms = math.sqrt(float((fref ** 2).sum(1).mean()))
    assert npairs == npr
    assert float(np.abs(f - fref).max()) <= 1e-10 * rms
    assert U == pytest.approx(Ur, rel=1e-12) and W == pytest.approx(Wr, rel=1e-12)


def test_strategy1_threads():
    assert baseline.threads() >= 1
