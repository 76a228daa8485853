"""The seeded input generators shared by the CUDA path and the oracle: the
counter-based SplitMix64 against the generator's published first outputs,
reproducibility independent of call order, and the workload shapes (particle
count, density, box, temperature)."""
import math

import numpy as np

from paper_1401_4441_gb300 import inputs


def test_splitmix64_reference_outputs():
    """SplitMix64 from state 0 (Steele, Lea and Flood, OOPSLA 2014) starts
    0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f: the output
    function applied to the counters 1, 2, 3 times the golden gamma."""
    i = np.arange(1, 4, dtype=np.uint64)
    with np.errstate(over="ignore"):
        out = inputs._mix(i * inputs.GOLDEN)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_draws_do_not_depend_on_call_order():
    a = inputs.uniform(7, 3, 1000)
    b = np.concatenate([inputs.uniform(7, 3, 400), inputs.uniform(7, 3, 600, offset=400)])
    assert np.array_equal(a, b)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert not np.array_equal(a, inputs.uniform(7, 4, 1000))       # another stream
    assert not np.array_equal(a, inputs.uniform(8, 3, 1000))       # another seed
    assert abs(a.mean() - 0.5) < 0.03


def test_fcc_box_shape():
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.0)
    n = b["pos"].shape[0]
    assert n == 4000 and b["vel"].shape == (4000, 3)
    assert math.isclose(n / float(np.prod(b["box"])), 0.8442, rel_tol=1e-12)
    assert np.all(b["pos"] >= 0.0) and np.all(b["pos"] < b["box"])
    v = b["vel"]
    assert np.abs(v.sum(0)).max() < 1e-9                               # no net momentum
    assert math.isclose((v * v).sum() / (3 * (n - 1)), 0.72, rel_tol=1e-12)


def test_liquid1m_workload():
    b = inputs.workload("liquid1m")
    assert b["pos"].shape == (1_048_576, 3)
    assert math.isclose(1_048_576 / float(np.prod(b["box"])), 0.8442, rel_tol=1e-12)
    assert int(math.floor(b["box"][0] / 2.5)) == 42
