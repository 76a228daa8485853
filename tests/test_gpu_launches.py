"""Kernel accounting of the captured step graphs (lc_launch_counts_graphs):
the counts follow the step's structure, so the benchmark's gpu_launches is
the number of kernels its timed calls launch."""
import pytest

from paper_1401_4441_gb300 import inputs

pytestmark = pytest.mark.gpu

RC = 2.5
BIN = 4   # cell pass (with the kick and drift), tile scan, scatter, rank + gather


@pytest.mark.parametrize("prec,sched,one,two", [
    # mixed: the first step of a two-step graph forms no statistics; the
    # closing kick sums the statistics slots (no reduction launch)
    ("mixed", "atomic", BIN + 1 + 1, 2 * BIN + 2 + 1),
    ("mixed", "buffer", BIN + 2 + 1, 2 * BIN + 4 + 1),
    # the colour schedule's per-cell partials: two reduction kernels
    ("mixed", "colour", BIN + 1 + 2 + 1, 2 * BIN + 2 + 2 + 1),
    # FP64 forms statistics in every step: the first step's reduction is
    # its own launch (that step has no closing kick)
    ("fp64", "atomic", BIN + 1 + 1, 2 * BIN + 2 + 1 + 1),
])
def test_graph_launch_counts(lc, prec, sched, one, two):
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    with lc.Box(b["box"], RC, 4000, prec) as g:
        g.set_state(b["pos"], b["vel"])
        assert g.launch_counts_graphs() == (0, 0)
        g.verlet(0.005, 3, sched)
        assert g.launch_counts_graphs() == (one, two)
        g.verlet(0.005, 2, sched)
        assert g.launch_counts_graphs() == (one, two)
