"""Checkpoint and resume of a context's particle state.

A checkpoint is two files: `<path>.bin`, the FP64 positions and then the
FP64 velocities as [n][3] little-endian doubles in particle-ID order, and
`<path>.json`, a header with the format tag, the context's geometry (box
edges, cutoff, particle count, precision, dimensions; per-box edges, cutoffs
and counts for a batch), the step counter and any caller fields.  Both are
written to temporary names and renamed, so an interrupted save leaves the
previous checkpoint intact.

Resuming sets the saved state into a fresh context; the next force
evaluation recomputes the forces from the saved positions.  Positions are
saved wrapped into the box, as the state holds them after every binning, so
with a deterministic schedule (colour in FP64, buffer) a resumed run
continues bit for bit as the uninterrupted one would.
"""
import json
import os

import numpy as np

FORMAT = "lc-checkpoint-1"


def _write_atomic(path, write):
    tmp = f"{path}.tmp{os.getpid()}"
    write(tmp)
    os.replace(tmp, path)


def save(ctx, path, step=0, extra=None):
    """Write the state of `ctx` (an lc.Box or lc.Batch) to path.bin / path.json."""
    pos = np.ascontiguousarray(ctx.get("pos"), dtype="<f8")
    vel = np.ascontiguousarray(ctx.get("vel"), dtype="<f8")
    header = {"format": FORMAT, "n": int(ctx.n), "precision": ctx.precision, "step": int(step),
              "extra": extra or {}}
    if hasattr(ctx, "nbox"):
        header.update(kind="batch", boxes=np.asarray(ctx.box).tolist(), rcs=np.asarray(ctx.rcs).tolist(),
                      ns=[int(x) for x in ctx.ns])
    else:
        header.update(kind="box", box=np.asarray(ctx.box).tolist(), rc=float(ctx.rc), dims=int(ctx.dims))

    def write_bin(tmp):
        with open(tmp, "wb") as f:
            f.write(pos.tobytes())
            f.write(vel.tobytes())

    def write_json(tmp):
        with open(tmp, "w") as f:
            json.dump(header, f)

    _write_atomic(path + ".bin", write_bin)
    _write_atomic(path + ".json", write_json)
    return header


def load(path):
    """(header, positions [n][3], velocities [n][3]) of a checkpoint; raises
    ValueError if the files do not match each other."""
    with open(path + ".json") as f:
        header = json.load(f)
    if header.get("format") != FORMAT:
        raise ValueError(f"{path}.json: not a {FORMAT} header")
    n = int(header["n"])
    data = np.fromfile(path + ".bin", dtype="<f8")
    if data.size != 6 * n:
        raise ValueError(f"{path}.bin holds {data.size} doubles, the header says {6 * n}")
    return header, data[:3 * n].reshape(n, 3).copy(), data[3 * n:].reshape(n, 3).copy()


def resume(path):
    """A fresh context holding the saved state, and the header."""
    from . import lc
    header, pos, vel = load(path)
    if header["kind"] == "batch":
        ctx = lc.Batch(header["boxes"], header["rcs"], header["ns"], header["precision"])
    else:
        ctx = lc.Box(header["box"], header["rc"], header["n"], header["precision"], dims=header["dims"])
    ctx.set_state(pos, vel)
    return ctx, header
