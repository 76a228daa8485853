"""Sharding of independent boxes across ranks (one process per GPU).

The boxes of a batch are independent systems, so the batch shards with no
data-path exchange: each rank steps the boxes assigned to it, and the only
collective is the final gather of the per-box results (energies, pair
counts, drift) on rank 0.  Host logic only; the ranks communicate through
torch.distributed (NCCL between GPUs, gloo on CPU).
"""
import numpy as np


def partition_boxes(ns, world):
    """Boxes of each rank: longest-processing-time greedy on the particle
    counts (largest box first, to the rank with the fewest particles so far;
    ties to the lower rank), each rank's boxes in ascending index.  Every box
    goes to exactly one rank; deterministic."""
    ns = np.asarray(ns, np.int64)
    load = np.zeros(world, np.int64)
    owner = np.empty(ns.shape[0], np.int64)
    for b in sorted(range(ns.shape[0]), key=lambda i: (-int(ns[i]), i)):
        r = int(np.argmin(load))
        owner[b] = r
        load[r] += ns[b]
    return [np.flatnonzero(owner == r) for r in range(world)]


def gather_box_results(dist, nbox, boxes, values):
    """Per-box rows computed by this rank (values[k] belongs to box
    boxes[k]) gathered into one (nbox, ...) array on rank 0 (None on the
    other ranks).  dist: torch.distributed, initialised, or None (one rank)."""
    values = np.asarray(values, np.float64)
    if dist is None:
        out = np.zeros((nbox,) + values.shape[1:], np.float64)
        out[np.asarray(boxes, np.int64)] = values
        return out
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, (np.asarray(boxes, np.int64), values))
    if dist.get_rank() != 0:
        return None
    out = np.zeros((nbox,) + values.shape[1:], np.float64)
    seen = np.zeros(nbox, np.int64)
    for idx, vals in parts:
        out[idx] = vals
        seen[idx] += 1
    if not np.all(seen == 1):
        raise RuntimeError("the ranks' boxes do not cover every box exactly once")
    return out
