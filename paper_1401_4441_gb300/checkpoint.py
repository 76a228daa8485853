"""Checkpoint and resume of a context's particle state.

A checkpoint `<path>` is a header `<path>.json` and a data file it names,
`<path>.a.bin` or `<path>.b.bin`: the FP64 positions and then the FP64
velocities as [n][3] little-endian doubles in particle-ID order.  The header
holds the format tag, the context's geometry (box edges, cutoff, particle
count, precision, dimensions; per-box edges, cutoffs and counts for a
batch), the step counter, any caller fields, and the name, size and SHA-256
digest of its data file.

A save writes the data file the current header does not name (the other
slot), then the header under a temporary name, and renames the header last:
that rename is the commit.  An interrupted save therefore leaves the
previous header and the data file it names untouched, and load() checks the
digest, so a header never pairs with data written by another save.

Resuming sets the saved state into a fresh context; the next force
evaluation recomputes the forces from the saved positions.  Positions are
saved wrapped into the box, as the state holds them after every binning, so
with a deterministic schedule (colour in FP64, buffer) a resumed run
continues bit for bit as the uninterrupted one would.
"""
import hashlib
import json
import os

import numpy as np

FORMAT = "lc-checkpoint-2"
SLOTS = ("a", "b")


def _current_slot(path):
    try:
        with open(path + ".json") as f:
            return json.load(f).get("data", "")
    except (OSError, ValueError):
        return ""


def save(ctx, path, step=0, extra=None):
    """Write the state of `ctx` (an lc.Box or lc.Batch) as checkpoint `path`."""
    pos = np.ascontiguousarray(ctx.get("pos"), dtype="<f8")
    vel = np.ascontiguousarray(ctx.get("vel"), dtype="<f8")
    payload = pos.tobytes() + vel.tobytes()
    base = os.path.basename(path)
    used = _current_slot(path)
    slot = SLOTS[1] if used == f"{base}.{SLOTS[0]}.bin" else SLOTS[0]
    data_name = f"{base}.{slot}.bin"
    header = {"format": FORMAT, "n": int(ctx.n), "precision": ctx.precision, "step": int(step),
              "extra": extra or {}, "data": data_name, "bytes": len(payload),
              "sha256": hashlib.sha256(payload).hexdigest()}
    if hasattr(ctx, "nbox"):
        header.update(kind="batch", boxes=np.asarray(ctx.box).tolist(), rcs=np.asarray(ctx.rcs).tolist(),
                      ns=[int(x) for x in ctx.ns])
    else:
        header.update(kind="box", box=np.asarray(ctx.box).tolist(), rc=float(ctx.rc), dims=int(ctx.dims))
    data_path = os.path.join(os.path.dirname(path), data_name)
    with open(data_path, "wb") as f:
        f.write(payload)
        f.flush()
        os.fsync(f.fileno())
    tmp = f"{path}.json.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(header, f)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path + ".json")   # the commit point
    return header


def load(path):
    """(header, positions [n][3], velocities [n][3]) of a checkpoint; raises
    ValueError if the header is not one of this format or its data file's
    size or digest does not match it."""
    with open(path + ".json") as f:
        header = json.load(f)
    if header.get("format") != FORMAT:
        raise ValueError(f"{path}.json: not a {FORMAT} header")
    n = int(header["n"])
    data_path = os.path.join(os.path.dirname(path), header["data"])
    with open(data_path, "rb") as f:
        payload = f.read()
    if len(payload) != int(header["bytes"]) or len(payload) != 48 * n:
        raise ValueError(f"{data_path} holds {len(payload)} bytes, the header says {header['bytes']} for n = {n}")
    if hashlib.sha256(payload).hexdigest() != header["sha256"]:
        raise ValueError(f"{data_path} does not match the digest in {path}.json (written by another save)")
    data = np.frombuffer(payload, dtype="<f8")
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
