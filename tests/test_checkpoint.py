"""Checkpoint files (host logic): round trip, atomic replacement, and the
consistency checks of load()."""
import json

import numpy as np
import pytest

from paper_1401_4441_gb300 import checkpoint, inputs


class FakeBox:
    """Stands in for lc.Box on the host: get() returns the arrays."""

    def __init__(self, pos, vel, box, rc, dims=3, precision="fp64"):
        self.n, self.dims, self.rc, self.precision = pos.shape[0], dims, rc, precision
        self.box = np.asarray(box, np.float64)
        self._a = {"pos": pos, "vel": vel}

    def get(self, what):
        return self._a[what]


def test_round_trip(tmp_path):
    b = inputs.fcc_box(500, 0.8442, 0.72, jitter=0.05)
    fb = FakeBox(b["pos"], b["vel"], b["box"], 2.5)
    path = str(tmp_path / "ck")
    h = checkpoint.save(fb, path, step=17, extra={"dt": 0.005})
    header, pos, vel = checkpoint.load(path)
    assert header == json.loads(json.dumps(h))
    assert header["step"] == 17 and header["extra"]["dt"] == 0.005 and header["kind"] == "box"
    assert np.array_equal(pos, b["pos"]) and np.array_equal(vel, b["vel"])   # bit for bit
    # a second save replaces both files
    fb._a["vel"] = -b["vel"]
    checkpoint.save(fb, path, step=18)
    header, pos, vel = checkpoint.load(path)
    assert header["step"] == 18 and np.array_equal(vel, -b["vel"])
    assert sorted(p.name for p in tmp_path.iterdir()) == ["ck.bin", "ck.json"]


def test_load_rejects_mismatch(tmp_path):
    b = inputs.fcc_box(108, 0.8442, 0.72)
    fb = FakeBox(b["pos"], b["vel"], b["box"], 2.5)
    path = str(tmp_path / "ck")
    checkpoint.save(fb, path)
    data = np.fromfile(path + ".bin", dtype="<f8")
    data[:-3].tofile(path + ".bin")          # truncated
    with pytest.raises(ValueError):
        checkpoint.load(path)
    with open(path + ".json", "w") as f:
        json.dump({"format": "something else", "n": 1}, f)
    with pytest.raises(ValueError):
        checkpoint.load(path)
