"""Energy conservation of the large single box: 50 velocity-Verlet steps of
the 16.7M-particle FCC box (mixed precision, FP64 positions and velocities)
against the same 50 steps of the 4,000-particle box by the FP64 oracle (same
density, temperature, cutoff and dt).  The potential is truncated and not
shifted, so the total energy jumps by U(r_c) whenever a pair crosses r_c;
the relative drift of both runs is dominated by that and is intensive, so
the 16M drift must stay within 3x the oracle's."""
import math

import numpy as np
import pytest

import oracle
from paper_1401_4441_gb300 import inputs

pytestmark = pytest.mark.gpu

RC, DT, STEPS = 2.5, 0.005, 50


def test_16m_energy_drift_against_4k_oracle(lc):
    small = inputs.workload("fcc4k")
    _, _, _, e = oracle.verlet(small["pos"], small["vel"], small["box"], RC, DT, STEPS)
    E = e[:, 0] + e[:, 1]
    drift_ref = abs(E[-1] - E[0]) / abs(E[0])

    big = inputs.workload("fcc16m")
    with lc.Box(big["box"], RC, big["pos"].shape[0], "mixed") as g:
        g.set_state(big["pos"], big["vel"])
        g.forces("atomic")
        u0, k0, _, _ = g.energy()
        g.verlet(DT, STEPS, "atomic")
        u1, k1, _, _ = g.energy()
    drift = abs((u1 + k1) - (u0 + k0)) / abs(u0 + k0)
    print(f"relative energy drift over {STEPS} steps: 16.7M mixed {drift:.3e}, 4k FP64 oracle {drift_ref:.3e}")
    assert math.isfinite(drift)
    assert drift <= 3.0 * drift_ref + 1e-7
