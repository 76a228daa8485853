"""Checkpoint files (host logic): round trip, the two data slots, the commit
by the header rename, and the consistency checks of load()."""
import json
import shutil

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
    # a second save writes the other data slot and replaces the header
    fb._a["vel"] = -b["vel"]
    h2 = checkpoint.save(fb, path, step=18)
    assert h2["data"] != h["data"]
    header, pos, vel = checkpoint.load(path)
    assert header["step"] == 18 and np.array_equal(vel, -b["vel"])
    assert sorted(p.name for p in tmp_path.iterdir()) == ["ck.a.bin", "ck.b.bin", "ck.json"]
    # a third save reuses the first slot
    assert checkpoint.save(fb, path, step=19)["data"] == h["data"]


def test_interrupted_save_keeps_previous(tmp_path):
    """A save stopped after its data file (before the header rename) leaves
    the previous checkpoint loadable and unchanged."""
    b = inputs.fcc_box(256, 0.8442, 0.72, jitter=0.05)
    fb = FakeBox(b["pos"], b["vel"], b["box"], 2.5)
    path = str(tmp_path / "ck")
    checkpoint.save(fb, path, step=5)
    saved_json = (tmp_path / "ck.json").read_text()
    fb._a["pos"] = b["pos"] + 1.0
    checkpoint.save(fb, path, step=6)
    (tmp_path / "ck.json").write_text(saved_json)   # the step-6 header never committed
    header, pos, vel = checkpoint.load(path)
    assert header["step"] == 5 and np.array_equal(pos, b["pos"])


def test_stale_header_rejected(tmp_path):
    """A header next to data written by a later save fails its digest check."""
    b = inputs.fcc_box(256, 0.8442, 0.72, jitter=0.05)
    fb = FakeBox(b["pos"], b["vel"], b["box"], 2.5)
    path = str(tmp_path / "ck")
    checkpoint.save(fb, path, step=1)
    stale = (tmp_path / "ck.json").read_text()
    for step in (2, 3):   # two more saves overwrite the slot the stale header names
        fb._a["vel"] = fb._a["vel"] * 0.5
        checkpoint.save(fb, path, step=step)
    (tmp_path / "ck.json").write_text(stale)
    with pytest.raises(ValueError, match="digest"):
        checkpoint.load(path)


def test_load_rejects_mismatch(tmp_path):
    b = inputs.fcc_box(108, 0.8442, 0.72)
    fb = FakeBox(b["pos"], b["vel"], b["box"], 2.5)
    path = str(tmp_path / "ck")
    h = checkpoint.save(fb, path)
    data = np.fromfile(str(tmp_path / h["data"]), dtype="<f8")
    shutil.copy(str(tmp_path / h["data"]), str(tmp_path / "full.bin"))
    data[:-3].tofile(str(tmp_path / h["data"]))          # truncated
    with pytest.raises(ValueError):
        checkpoint.load(path)
    shutil.copy(str(tmp_path / "full.bin"), str(tmp_path / h["data"]))
    flipped = data.copy()
    flipped[7] = np.nextafter(flipped[7], np.inf)        # same size, one bit changed
    flipped.tofile(str(tmp_path / h["data"]))
    with pytest.raises(ValueError, match="digest"):
        checkpoint.load(path)
    with open(path + ".json", "w") as f:
        json.dump({"format": "something else", "n": 1}, f)
    with pytest.raises(ValueError):
        checkpoint.load(path)
