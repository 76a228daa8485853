"""Autotuner of the force sweep's launch shape.

For a given context it times one force evaluation for every candidate
(schedule x centre-cell tile x warps per block) with CUDA events on the
current stream, keeps the fastest, applies it (lc_set_tile) and caches the
choice in a JSON file keyed by (GPU name, precision, batch or single box,
mean cell occupancy bucket), so later contexts of the same kind skip the
search.  Host-side only: every timed call runs the library's kernels.
"""
import json
import math
import os

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json")

TILES = (8, 16)            # centre-cell particles held per warp
WARPS = (2, 4, 8)          # warps per thread block
ROWS = 16                  # tile setting of the atomic schedule's row-group kernel (ni 16)


def occupancy_bucket(n, ncell):
    """Mean particles per cell, rounded to a power of two (the kernels' work
    per task and their lane utilisation depend on it)."""
    ppc = n / max(1, ncell)
    return 1 << max(0, int(round(math.log2(max(ppc, 1.0)))))


def _key(box, schedules):
    import torch
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    kind = "batch" if getattr(box, "nbox", 0) else "single"
    return f"{name}|{box.precision}|{kind}|ppc{occupancy_bucket(box.n, box.ncell())}|{'+'.join(schedules)}"


def _load_cache():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(cache):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def time_forces(box, schedule, reps=3):
    """Median device time (ms) of one force evaluation on a binned state."""
    import torch
    stream = torch.cuda.current_stream()
    box.forces(schedule)
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        box.forces(schedule)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return sorted(ts)[len(ts) // 2]


def tune(box, schedules=("atomic", "buffer", "fullshell", "colour"), use_cache=True):
    """Pick (schedule, tile, warps) for `box` (state already set); applies
    the tile shape and returns dict(schedule, ni, warps, ms, table)."""
    if getattr(box, "nbox", 0):
        schedules = tuple(s for s in schedules if s != "colour")
    key = _key(box, schedules)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        best = cache[key]
        box.set_tile(best["ni"], best["warps"])
        return dict(best, cached=True)
    box.bin()
    table = []
    for sched in schedules:
        for ni in TILES:
            for warps in WARPS:
                box.set_tile(ni, warps)
                table.append({"schedule": sched, "ni": ni, "warps": warps, "ms": time_forces(box, sched)})
        if sched == "atomic" and not getattr(box, "nbox", 0) and box.precision == "mixed" \
                and getattr(box, "dims", 3) == 3:
            box.set_tile(16, ROWS)
            table.append({"schedule": sched, "ni": 16, "warps": ROWS, "ms": time_forces(box, sched)})
    best = min(table, key=lambda r: r["ms"])
    box.set_tile(best["ni"], best["warps"])
    result = {"schedule": best["schedule"], "ni": best["ni"], "warps": best["warps"], "ms": best["ms"]}
    cache[key] = result
    if use_cache:
        _save_cache(cache)
    return dict(result, table=table, cached=False)
