"""The largest particle count a context accepts (n = 2^26 - 1, 67.1M
particles, about 12 GB on the device; 45 GB with the Verlet lists): binning
invariants, forces of the link-cell sweep and of the lists against
per-particle oracle sums on a sample, Newton's third law, the same pair count
on both paths; one particle more is refused."""
import math

import numpy as np
import pytest

import oracle
from paper_1401_4441_gb300 import inputs

pytestmark = pytest.mark.gpu

RC = 2.5


def test_max_particle_count(lc):
    n = (1 << 26) - 1
    b = inputs.fcc_box(n, 0.8442, 0.72, jitter=0.05)
    pos, box = b["pos"], b["box"]
    with pytest.raises(lc.LCError) as ei:
        lc.Box(box, RC, n + 1, "mixed")
    assert ei.value.code == 9                      # LC_ERR_TOO_LARGE
    with lc.Box(box, RC, n, "mixed") as g:
        g.set_state(pos)
        g.bin()
        counts = g.get("cell_count")
        starts = g.get("cell_start")
        perm = g.get("perm")
        g.forces("atomic")
        f = g.get("forces")
        u, k, w, npairs = g.energy()
    assert int(counts.sum()) == n
    assert starts[0] == 0 and np.array_equal(np.diff(starts), counts[:-1])   # exclusive scan, 1243 tiles
    seen = np.zeros(n, np.bool_)
    seen[perm] = True
    assert seen.all()                              # a permutation of the IDs
    ids = np.linspace(0, n - 1, 2000).astype(np.int64)
    fref, _ = oracle.forces_sample(pos[:, 0], pos[:, 1], pos[:, 2], box, RC, ids)
    scale = max(1e-3, math.sqrt(float((fref ** 2).sum(1).mean())))
    assert np.abs(f[ids] - fref).max() <= 1e-5 * scale + 1e-9
    assert np.abs(f.sum(0)).max() < 1e-6 * n       # Newton's third law
    assert npairs > 0 and math.isfinite(u) and u < 0
    # the Verlet lists at the same size: entries slot << 6 use all 32 bits
    with lc.Box(box, RC, n, "mixed") as g:
        g.set_state(pos)
        g.forces("list")
        fl = g.get("forces")
        _, _, _, npairs_list = g.energy()
        info = g.list_info()
    assert npairs_list == npairs and info["long_rows"] == 0
    assert np.abs(fl[ids] - fref).max() <= 1e-5 * scale + 1e-9
