"""Checkpoint and resume on the GPU: a run interrupted, saved, resumed in a
fresh context and continued equals the uninterrupted run bit for bit with
the deterministic schedules (colour in FP64, buffer in mixed precision)."""
import numpy as np
import pytest

from paper_1401_4441_gb300 import checkpoint, inputs

pytestmark = pytest.mark.gpu

RC = 2.5


@pytest.mark.parametrize("prec,sched", [("fp64", "colour"), ("mixed", "buffer")])
def test_resume_bit_identical(lc, tmp_path, prec, sched):
    b = inputs.fcc_box(4000, 0.8442, 0.72, jitter=0.05)
    with lc.Box(b["box"], RC, 4000, prec) as g:
        g.set_state(b["pos"], b["vel"])
        g.verlet(0.005, 10, sched)
        ref = (g.get("pos"), g.get("vel"), g.get("forces"), g.energy())
    path = str(tmp_path / "ck")
    with lc.Box(b["box"], RC, 4000, prec) as g:
        g.set_state(b["pos"], b["vel"])
        g.verlet(0.005, 5, sched)
        checkpoint.save(g, path, step=5, extra={"dt": 0.005, "schedule": sched})
    g2, header = checkpoint.resume(path)
    with g2:
        assert header["step"] == 5 and header["extra"]["schedule"] == sched
        g2.verlet(0.005, 5, sched)
        got = (g2.get("pos"), g2.get("vel"), g2.get("forces"), g2.energy())
    for a, r in zip(got[:3], ref[:3]):
        assert np.array_equal(a, r)
    assert got[3] == ref[3]


def test_resume_batch_and_2d(lc, tmp_path):
    """Batch and 2D contexts come back with their geometry and state."""
    boxes = [inputs.fcc_box(n, 0.8442, 0.72, seed=s, jitter=0.05) for n, s in ((500, 1), (864, 2))]
    pos = np.concatenate([x["pos"] for x in boxes])
    vel = np.concatenate([x["vel"] for x in boxes])
    with lc.Batch([x["box"] for x in boxes], RC, [500, 864]) as g:
        g.set_state(pos, vel)
        g.forces("atomic")
        e_ref = g.energies()
        checkpoint.save(g, str(tmp_path / "batch"))
    g2, _ = checkpoint.resume(str(tmp_path / "batch"))
    with g2:
        g2.forces("atomic")
        e = g2.energies()
        assert np.array_equal(g2.get("pos"), np.mod(pos, np.repeat([x["box"] for x in boxes], [500, 864], 0)))
    assert np.array_equal(e[3], e_ref[3])   # pair counts
    assert np.allclose(e[0], e_ref[0], rtol=1e-12)
    b2 = inputs.tri_box(40, 30, 0.7, 0.5, seed=4, jitter=0.05)
    with lc.Box(b2["box"], RC, b2["pos"].shape[0], "mixed", dims=2) as g:
        g.set_state(b2["pos"], b2["vel"])
        g.verlet(0.005, 3, "buffer")
        p_ref = g.get("pos")
        checkpoint.save(g, str(tmp_path / "two"))
    g3, h3 = checkpoint.resume(str(tmp_path / "two"))
    with g3:
        assert h3["dims"] == 2
        assert np.array_equal(g3.get("pos"), p_ref)
