"""Benchmark: link-cell LJ velocity-Verlet steps on one GB300 per rank.

Workload (default): homogeneous liquid start, N = 1,048,576 particles on an
FCC lattice jittered by U[-0.05, 0.05) per coordinate, density 0.8442,
T = 0.72, r_c = 2.5, cubic periodic box, mixed precision (FP32 pair math,
FP64 cutoff decisions near r_c, Kahan / FP64 cross-cell sums, FP64 state).
A step is one full velocity-Verlet step: kick + drift, counting-sort
binning, force sweep, kick.  Metric: unique pair interactions (pairs with
r < r_c, each counted once) per second, whole job.

Arms:
  --impl gb300       the CUDA library through its C ABI (default)
  --impl reference   the FP64 CPU oracle (single host core), same workload

Multi-GPU (torchrun): every rank runs an independent replica of the box
(no data-path collective); value = pairs of all ranks / max rank time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1401_4441_gb300 import inputs  # noqa: E402

METRIC = "LJ pair interactions/s (link-cell, Newton-3, velocity-Verlet steps)"
# --schedule list: Verlet lists with a skin (an extension, not the paper's method)
METRIC_LIST = "LJ pair interactions/s (Verlet lists with skin, velocity-Verlet steps)"
UNIT = "pairs/s"
DT = 0.005
RC = 2.5
FP32_LANES_PER_SM = 128
# algorithmic bytes of one binning (lc_bin): read the FP64 state (x, v) and
# the ID (52 B), write it in cell order (52 B) and the FP32 cell-local
# coordinates (16 B) per particle; per cell its count and start
BIN_BYTES_PER_PARTICLE = 120
BIN_BYTES_PER_CELL = 8


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Dist:
    def __init__(self):
        self.rank, self.world, self.local = dist_env()
        self.pg = None
        if self.world > 1:
            import torch.distributed as td
            td.init_process_group("gloo", init_method="env://")
            self.pg = td

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x):
        if not self.pg:
            return x
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x):
        if not self.pg:
            return x
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, load, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                clk, cmax, util = float(parts[1]), float(parts[2]), float(parts[9])
            except ValueError:
                continue
            sm.append(clk)
            smax.append(cmax)
            if util >= 50.0:   # a sample taken while the GPU was busy
                load.append(clk)
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        return {"sm_mhz": statistics.median(load) if load else (statistics.median(sm) if sm else None),
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "samples_under_load": len(load)}


def half_shell_candidates(counts, nc, dims=3):
    """Candidate pairs of the half-shell sweep: intra n(n-1)/2 plus n_A n_B
    over the forward neighbour cells (periodic; 13 in 3D, 4 in 2D)."""
    c = counts.reshape(nc[2], nc[1], nc[0]).astype(np.int64)
    total = int((c * (c - 1) // 2).sum())
    for oz in ((0,) if dims == 2 else (-1, 0, 1)):
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                if not (oz > 0 or (oz == 0 and oy > 0) or (oz == 0 and oy == 0 and ox > 0)):
                    continue
                nb = np.roll(c, shift=(-oz, -oy, -ox), axis=(0, 1, 2))
                total += int((c * nb).sum())
    return total


def measured_traffic(workload, sched):
    """DRAM bytes (read + write) of one force evaluation from the committed ncu
    summary profiles/k_force_<workload>.md (k_list_force_<workload>.md for the
    lists), or None when the kernel's source changed since that capture (or
    there is none)."""
    import hashlib
    import re
    kern, cu = ("k_list_force", "lc_list.cu") if sched == "list" else ("k_force", "lc_force.cu")
    src = os.path.join(ROOT, "paper_1401_4441_gb300", "csrc", cu)
    path = os.path.join(ROOT, "profiles", f"{kern}_{workload}.md")
    try:
        cur = hashlib.sha256(open(src, "rb").read()).hexdigest()
        for line in open(path):
            m = re.match(r"traffic_bytes (\w+) (\d+) sha256 ([0-9a-f]+)", line.strip())
            if m and m.group(1) == sched and m.group(3) == cur:
                return int(m.group(2))
    except OSError:
        pass
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def oracle_box(w):
    """Box for the FP64 oracle: 2D workloads lie in the z = 0 plane of a box
    whose z side is 3 r_c (no z image within r_c), which the oracle's 3D
    routines turn into the 2D system."""
    if w.get("dims", 3) == 2:
        return np.array([w["box"][0], w["box"][1], 3.0 * w["rc"]])
    return w["box"]


def cpu_baseline(pos, box, rc, budget_s=12.0):
    """The FP64 oracle (as it stands) on this host: repeated link-cell force
    evaluations of the same box for about budget_s seconds, one core.
    Returns the baseline and the oracle's (forces, U, W, pairs) of the box,
    against which the precision report compares the GPU path."""
    import oracle
    x, y, z = (np.ascontiguousarray(pos[:, d]) for d in range(3))
    t0 = time.perf_counter()
    evals, pairs, ref = 0, 0, None
    while True:
        f, U, W, npairs = oracle.lc_forces(x, y, z, box, rc)
        if ref is None:
            ref = (f, U, W, npairs)
        evals += 1
        pairs += npairs
        if time.perf_counter() - t0 > budget_s or evals >= 8:
            break
    dt = time.perf_counter() - t0
    line = {"value": pairs / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{evals} FP64 link-cell force evaluations of the full {pos.shape[0]}-particle box "
                      f"({dt:.1f} s, single thread)"}
    line["strategy1"] = strategy1_baseline(pos, box, rc)
    return line, ref


def strategy1_baseline(pos, box, rc, budget_s=8.0):
    """The paper's Strategy 1 (Sec. VI, Fig. 6: loop exchange + 2-strided
    colouring, plain writes) in OpenMP on all host cores, FP64: repeated
    force evaluations of the same box for about budget_s seconds."""
    try:
        import baseline
        cores = baseline.threads()
        baseline.forces(pos[:1000], box, rc)          # build and first touch
        t0 = time.perf_counter()
        evals, pairs = 0, 0
        while True:
            _, _, _, npairs = baseline.forces(pos, box, rc)
            evals += 1
            pairs += npairs
            if time.perf_counter() - t0 > budget_s or evals >= 20:
                break
        dt = time.perf_counter() - t0
    except Exception as exc:   # no compiler or OpenMP on this host
        return {"unavailable": f"{type(exc).__name__}: {exc}"}
    return {"value": pairs / dt, "unit": UNIT, "cores": cores, "kind": "paper Strategy 1, OpenMP",
            "sample": f"{evals} FP64 force evaluations of the full {pos.shape[0]}-particle box ({dt:.1f} s)",
            "paper_context": "the paper reports near-perfect scaling of this strategy up to 32 threads on a "
                             "32-core Cray XE6 node (OmpSs, synthetic fixed-duration tasks, Sec. VII); it "
                             "prints no LJ throughput"}


def precision_report(f, u, w, ref):
    """Errors of one GPU force evaluation against the oracle's FP64
    evaluation of the same positions: max and RMS over particles of
    |dF_i| / RMS |F|, relative errors of U and W."""
    fref, U, W, _ = ref
    rms = math.sqrt(float((fref ** 2).sum(1).mean()))
    err = np.sqrt(((f - fref) ** 2).sum(1))
    return {"force_max_rel": float(err.max()) / rms, "force_rms_rel": math.sqrt(float((err ** 2).mean())) / rms,
            "energy_rel": abs(u - U) / abs(U), "virial_rel": abs(w - W) / abs(W),
            "against": "the oracle's FP64 link-cell evaluation of the same (initial) positions"}


def oracle_drift(nsteps, rc):
    """Relative energy drift |E(n) - E(0)| / |E(0)| of the oracle's FP64
    velocity-Verlet run of the 4,000-particle FCC box (rho 0.8442, T 0.72)."""
    import oracle
    b = inputs.fcc_box(4000, 0.8442, 0.72)
    _, _, _, e = oracle.verlet(b["pos"], b["vel"], b["box"], rc, DT, nsteps)
    E = e[:, 0] + e[:, 1]
    return abs(E[-1] - E[0]) / abs(E[0])


def run_reference(args, dist):
    """Reference arm: the FP64 CPU oracle, same workload, rank 0 only."""
    if dist.rank != 0:
        return
    import oracle
    w = inputs.workload(args.workload)
    pos, vel, box, rc = w["pos"], w["vel"], oracle_box(w), w["rc"]
    f0, U, W, npairs0 = oracle.lc_forces(pos[:, 0], pos[:, 1], pos[:, 2], box, rc)
    x, v, f = pos, vel, f0
    for _ in range(args.warmup):
        x, v, f, e = oracle.verlet(x, v, box, rc, DT, 1, f=f)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x, v, f, e = oracle.verlet(x, v, box, rc, DT, 1, f=f)
    elapsed = time.perf_counter() - t0
    _, _, _, npairs1 = oracle.lc_forces(x[:, 0], x[:, 1], x[:, 2], box, rc)
    pairs = 0.5 * (npairs0 + npairs1) * args.steps
    value = pairs / elapsed
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} FP64 velocity-Verlet steps of the full box, one host core"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args, w):
    rc = w["rc"]
    nc = [int(math.floor(L / rc)) for L in w["box"]]
    if w.get("dims", 3) == 2:
        desc = (f"{args.workload}: N={w['pos'].shape[0]} 2D triangular lattice + jitter "
                f"{inputs.WORKLOADS[args.workload]['jitter']}, area density {w['rho']}, T={w['T']}, rc={rc}, "
                f"periodic {w['box'][0]:.2f} x {w['box'][1]:.2f}, cells {nc[0]}x{nc[1]}, dt={DT}")
    elif inputs.WORKLOADS[args.workload].get("kind") == "slab":
        desc = (f"{args.workload}: N={w['pos'].shape[0]} liquid slab 0.80 in x < Lx/3, vapour 0.02 elsewhere, "
                f"uniform random positions, box {w['box'][0]:.2f} x {w['box'][1]:.2f} x {w['box'][2]:.2f}, "
                f"rc={rc}, cells {nc[0]}x{nc[1]}x{nc[2]}; step = binning + one force evaluation")
    else:
        desc = (f"{args.workload}: N={w['pos'].shape[0]} FCC+jitter {inputs.WORKLOADS[args.workload]['jitter']}, "
                f"rho={w['rho']}, T={w['T']}, rc={rc}, cubic periodic L={w['box'][0]:.4f}, "
                f"cells {nc[0]}^3, dt={DT}")
    return {"workload": desc,
            "particles": int(w["pos"].shape[0]), "cells": nc,
            "precision": args.precision if args.impl == "gb300" else "fp64 (oracle)",
            "schedule": args.schedule, "l2": "flushed (512 MiB memset) between timed iterations",
            "seed": inputs.DEFAULT_SEED}


def run_profile(args, dist):
    """Only W warm-up and K timed steps of one schedule (for ncu captures)."""
    import torch
    from paper_1401_4441_gb300 import build
    torch.cuda.set_device(dist.local)
    build.build()
    from paper_1401_4441_gb300 import lc
    w = inputs.workload(args.workload)
    g = lc.Box(w["box"], w["rc"], w["pos"].shape[0], args.precision, dims=w.get("dims", 3))
    g.set_state(torch.from_numpy(w["pos"]).cuda(), torch.from_numpy(w["vel"]).cuda())
    sched = "atomic" if args.schedule == "auto" else args.schedule
    if sched == "list":
        g.set_skin(args.skin)
    if args.tile:
        g.set_tile(*[int(v) for v in args.tile.split(",")])
    g.forces(sched)
    g.verlet(DT, args.warmup, sched)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.verlet(DT, args.steps, sched)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    u, k, wv, npairs = g.energy()
    print(json.dumps({"profile": sched, "precision": args.precision, "steps": args.steps,
                      "ms_per_step": 1e3 * dt / max(1, args.steps), "pairs": npairs, "U": u, "K": k}))
    g.close()


def run_batch(args, dist):
    """Batched configuration: 512 independent boxes (N log-uniform in
    [500, 50000], density U[0.5, 0.9], T U[0.7, 1.2], FCC + jitter 0.05)
    stepped together, mixed precision; the colour schedule runs as one
    persistent launch fed by the device work queue of cell tasks (box,
    colour, cell) (lc_batch_step), the other schedules one launch per stage; two-step CUDA
    graphs.  Compared with the plain FP64 path that steps each box alone (its
    own context, per-box launches).  Under torchrun the boxes are partitioned
    over the ranks (longest-first greedy on N) and the per-box energies are
    gathered on rank 0: the total work is fixed (strong scaling)."""
    import torch
    from paper_1401_4441_gb300 import build, shard
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    if dist.rank == 0:
        build.build()
    dist.barrier()
    from paper_1401_4441_gb300 import lc
    all_boxes = inputs.batch_boxes(seed=inputs.DEFAULT_SEED)
    mine = shard.partition_boxes([b["pos"].shape[0] for b in all_boxes], dist.world)[dist.rank]
    boxes = [all_boxes[i] for i in mine]
    pos = np.concatenate([b["pos"] for b in boxes])
    vel = np.concatenate([b["vel"] for b in boxes])
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    g = lc.Batch([b["box"] for b in boxes], RC, [b["pos"].shape[0] for b in boxes], args.precision)
    dpos, dvel = torch.from_numpy(pos).to(dev), torch.from_numpy(vel).to(dev)
    sched_ms = {}
    for sch in ("colour", "atomic", "fullshell", "buffer"):
        g.set_state(dpos, dvel)
        g.forces(sch)
        ts = []
        for _ in range(3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream); g.forces(sch); e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        sched_ms[sch] = min(ts)
    sched = min(sched_ms, key=sched_ms.get) if args.schedule == "auto" else args.schedule

    def steps(k):
        if sched == "colour":
            g.step(DT, k)            # lc_batch_step: the device work queue
        else:
            g.verlet(DT, k, sched)

    g.set_state(dpos, dvel)
    g.forces(sched)
    _, _, _, np0 = g.energies()
    steps(max(2, args.warmup))
    torch.cuda.synchronize(dev)
    calls = [2] * (args.steps // 2) + ([1] if args.steps % 2 else [])
    clocks = ClockSampler(dist.local)
    dist.barrier()
    clocks.start()
    time.sleep(0.3)
    evs = []
    for k in calls:
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream); steps(k); e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize(dev)
    ms = dist.max(sum(a.elapsed_time(b) for a, b in evs))
    u1, k1, w1, np1 = g.energies()
    # the same steps continued for about one second (clocks sampled under
    # sustained load; the line's value is the K-step region above)
    sus_steps = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t_start = time.perf_counter()
    while time.perf_counter() - t_start < 1.2:
        steps(20)
        sus_steps += 20
        torch.cuda.synchronize(dev)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_sus = e0.elapsed_time(e1)
    clk = clocks.stop()
    np_sus = g.energies()[3]
    sustained = {"steps": sus_steps, "ms_per_step": t_sus / sus_steps,
                 "value": 0.5 * (np1.sum() + np_sus.sum()) / (t_sus / sus_steps * 1e-3), "unit": UNIT,
                 "note": "the timed steps continued back to back for about one second (no L2 flush), "
                         "during which the clocks were sampled"}
    pairs = 0.5 * (np0.sum() + np1.sum()) * args.steps
    value = dist.sum(pairs) / (ms * 1e-3)
    one_step, two_steps = g.launch_counts_graphs()
    launches = two_steps * (args.steps // 2) + one_step * (args.steps % 2)
    g.close()
    # per-box results of every rank on rank 0
    rows = np.stack([u1, k1, w1, np1.astype(np.float64)], axis=1)
    gathered = shard.gather_box_results(dist.pg, len(all_boxes), mine, rows)

    # plain FP64 per-box path: every box alone, FP64, its own launches
    fp64_steps = 2
    t_fp64 = 0.0
    pairs_fp64 = 0
    for b in boxes:
        gb = lc.Box(b["box"], RC, b["pos"].shape[0], "fp64")
        gb.set_state(torch.from_numpy(b["pos"]).to(dev), torch.from_numpy(b["vel"]).to(dev))
        gb.forces("atomic")
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream); gb.verlet(DT, fp64_steps, "atomic"); e1.record(stream)
        torch.cuda.synchronize(dev)
        t_fp64 += e0.elapsed_time(e1)
        pairs_fp64 += gb.energy()[3] * fp64_steps
        gb.close()
    t_fp64 = dist.max(t_fp64)
    value_fp64 = dist.sum(pairs_fp64) / (t_fp64 * 1e-3)
    if dist.rank == 0:
        ns = [b["pos"].shape[0] for b in all_boxes]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
                "data": "synthetic",
                "config": {"workload": f"batch512: 512 periodic cubic LJ boxes, N log-uniform in [500, 50000] "
                                       f"(total {sum(ns)}), density U[0.5, 0.9], T U[0.7, 1.2], rc={RC}, "
                                       f"FCC + jitter 0.05, dt={DT}; boxes partitioned over the ranks",
                           "boxes": len(ns), "particles": int(sum(ns)), "boxes_rank0": len(mine),
                           "precision": args.precision, "l2": "flushed between timed iterations"},
                "schedule": sched, "schedule_force_ms": sched_ms, "sustained": sustained, "clocks": clk,
                "fp64_per_box": {"value": value_fp64, "unit": UNIT, "ms_per_step": t_fp64 / fp64_steps,
                                 "how": "each box alone in an FP64 context, atomic schedule, per-box launches"},
                "vs_fp64_per_box": value / value_fp64, "gpu_launches": launches,
                "energies_gathered": {"boxes": int(gathered.shape[0]),
                                      "U_total": float(gathered[:, 0].sum()),
                                      "pairs_total": int(gathered[:, 3].sum())}}
        print(json.dumps(line), flush=True)


def run_gb300(args, dist):
    import torch
    from paper_1401_4441_gb300 import build
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    if dist.rank == 0:
        build.build()
    dist.barrier()
    from paper_1401_4441_gb300 import lc
    lc.lib()

    w = inputs.workload(args.workload, seed=inputs.DEFAULT_SEED + dist.rank)
    pos, vel, box = w["pos"], w["vel"], w["box"]
    rc = w["rc"]
    forces_only = inputs.WORKLOADS[args.workload].get("kind") == "slab"
    n = pos.shape[0]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    g = lc.Box(box, rc, n, args.precision, dims=w.get("dims", 3))
    dpos = torch.from_numpy(pos).to(dev)
    dvel = torch.from_numpy(vel).to(dev)
    g.set_state(dpos, dvel)

    is_list = args.schedule == "list"
    if is_list:   # Verlet lists: no link-cell schedule or tile to choose
        g.set_skin(args.skin)
        sched, sched_ms, tile = "list", {}, None
    else:
        # schedule and tile shape: the autotuner's pick, unless fixed on the command line
        from paper_1401_4441_gb300 import autotune
        tuned = autotune.tune(g, use_cache=False)
        sched_ms = {}
        for row in tuned["table"]:
            sched_ms[row["schedule"]] = min(sched_ms.get(row["schedule"], 1e30), row["ms"])
        if args.schedule == "auto":
            sched = tuned["schedule"]
        else:
            sched = args.schedule
            best = min((r for r in tuned["table"] if r["schedule"] == sched), key=lambda r: r["ms"])
            g.set_tile(best["ni"], best["warps"])
        tile = {"ni": tuned["ni"], "warps": tuned["warps"]} if args.schedule == "auto" else \
            {"ni": best["ni"], "warps": best["warps"]}
        if args.tile:
            ni, warps = [int(v) for v in args.tile.split(",")]
            g.set_tile(ni, warps)
            tile = {"ni": ni, "warps": warps}

    # the first evaluation, at the initial positions: the precision report's sample
    g.set_state(dpos, dvel)
    g.forces(sched)
    f_first = g.get("forces")
    u0, k0, w0, npairs0 = g.energy()
    E0 = u0 + k0
    for _ in range((args.warmup + 1) // 2):
        if forces_only:
            g.forces(sched)
        else:
            g.verlet(DT, 2, sched)
    torch.cuda.synchronize(dev)

    def run_steps(k):
        if forces_only:
            # the slab's random start has near-overlaps: a step is binning +
            # one force evaluation (no dynamics)
            for _ in range(k):
                g.set_state(dpos, dvel)
                g.forces(sched)
        else:
            g.verlet(DT, k, sched)

    # timed region: K steps in graph replays of two steps, L2 flushed between
    calls = [2] * (args.steps // 2) + ([1] if args.steps % 2 else [])
    clocks = ClockSampler(dist.local)
    dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    evs = []
    for k in calls:
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run_steps(k)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize(dev)
    dist.barrier()
    elapsed_ms = sum(a.elapsed_time(b) for a, b in evs)
    _, _, _, npairs1 = g.energy()
    # the same steps continued for about one second (sampled clocks under
    # sustained load; the line's value is the K-step region above)
    sus_steps, t_sus = 0, 0.0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t_start = time.perf_counter()
    while time.perf_counter() - t_start < 1.2:
        run_steps(2 * 50)
        sus_steps += 100
        torch.cuda.synchronize(dev)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_sus = e0.elapsed_time(e1)
    # the FP32 FMA probe (lc_probe_fp32), still under the clock sampler: the
    # derived peak's check on this GPU
    probe = []
    for _ in range(5):
        f, sec = lc.probe_fp32(1 << 16)
        probe.append(f / sec / 1e12)
    clk = clocks.stop()
    u1, k1, _, npairs_sus = g.energy()
    per_force, per_step = g.launch_counts()
    one_step, two_steps = g.launch_counts_graphs()
    if forces_only:   # a step: lc_set_state (one kernel) and a force evaluation
        launches = (1 + per_force) * args.steps
    else:             # the timed calls: two-step graphs, then a one-step graph for an odd K
        launches = two_steps * (args.steps // 2) + one_step * (args.steps % 2)
    list_stats = g.list_info() if is_list else None
    elapsed_ms = dist.max(elapsed_ms)
    pairs = 0.5 * (npairs0 + npairs1) * args.steps
    total_pairs = dist.sum(pairs)
    value = total_pairs / (elapsed_ms * 1e-3)
    sustained = {"steps": sus_steps, "ms_per_step": t_sus / sus_steps,
                 "value": 0.5 * (npairs1 + npairs_sus) / (t_sus / sus_steps * 1e-3), "unit": UNIT,
                 "note": "the timed steps continued back to back for about one second (no L2 flush), "
                         "during which the clocks were sampled"}
    drift_gpu = None if forces_only else {
        "steps": args.warmup + args.steps + sus_steps,
        "rel": abs((u1 + k1) - E0) / abs(E0)}

    # dominant kernel: the force sweep of one evaluation (binned state or
    # valid lists, L2 flushed)
    if forces_only:
        g.set_state(dpos, dvel)
        g.forces(sched)
    _, _, _, npairs_now = g.energy()
    if is_list:
        # per list entry the distance test (8 flop), per pair twice the
        # one-sided pair term (21 flop less the 3 of the partner's update)
        info = g.list_info()
        cand = info["entries"] / max(1, info["builds"])
        flops = 8.0 * cand + 2 * 18.0 * npairs_now
    else:
        counts = g.get("cell_count")
        nc, _, _ = g.grid()
        cand = half_shell_candidates(counts, nc, w.get("dims", 3))
        flops = 8.0 * cand + 21.0 * npairs_now
    fts = []
    for _ in range(5):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.forces(sched)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        fts.append(e0.elapsed_time(e1))
    t_force = statistics.median(fts) * 1e-3
    achieved = flops / t_force / 1e12
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_clock = clk.get("sm_mhz") if clk.get("samples_under_load") else None
    clock_src = "median SM clock of the samples under load"
    if not sm_clock:
        sm_clock = clk.get("sm_max_mhz") or measured_peaks().get("sm_max_mhz") or 2070.0
        clock_src = "maximum SM clock (no sample under load)"
    peak = sms * FP32_LANES_PER_SM * 2 * sm_clock * 1e6 / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": measured_traffic(args.workload, sched),
                "kernel": "k_list_force (mixed): one force evaluation from the lists" if is_list else
                          f"k_force ({sched}, {args.precision}): one force evaluation",
                "flops_per_eval": flops, "candidates": cand, "pairs": npairs_now,
                "eval_ms": t_force * 1e3,
                "peak_note": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {sm_clock:.0f} MHz "
                             f"({clock_src}); MEASURED_PEAKS.json has no FP32 figure",
                "frac_by_schedule": {k: flops / (v * 1e-3) / 1e12 / peak for k, v in sched_ms.items()},
                "peak_probe": {"tflops": max(probe), "frac": achieved / max(probe),
                               "how": "lc_probe_fp32: 8 blocks of 256 threads per SM, 8 chains of 65,536 packed "
                                      "f32x2 FMAs per thread, CUDA events; best of 5, sampled with the clocks"}}

    # binning (counting sort by cell, state permuted into cell order, FP32
    # cell-local coordinates): HBM-bound
    bts = []
    for _ in range(5):
        g.set_state(dpos, dvel)
        torch.cuda.synchronize(dev)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.bin()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        bts.append(e0.elapsed_time(e1))
    t_bin = statistics.median(bts) * 1e-3
    ncell = int(np.prod(g.grid()[0]))
    bin_bytes = BIN_BYTES_PER_PARTICLE * n + BIN_BYTES_PER_CELL * ncell
    hbm = measured_peaks().get("hbm_gbs")
    roofline_bin = {"bound": "hbm", "achieved": bin_bytes / t_bin / 1e9, "unit": "GB/s",
                    "peak": hbm or 6800.0, "frac": bin_bytes / t_bin / 1e9 / (hbm or 6800.0),
                    "frac_nominal_8tbs": bin_bytes / t_bin / 8e12,
                    "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json)" if hbm else "fallback 6.8 TB/s",
                    "bytes_per_launch": bin_bytes, "ms": t_bin * 1e3,
                    "kernels": "k_cellid + k_scan_tiles_ticket + k_scatter_starts + k_rank_gather (lc_bin)",
                    "bytes_note": f"{BIN_BYTES_PER_PARTICLE} B per particle (read x, v, id: 52 B; write them in "
                                  f"cell order: 52 B; write the FP32 cell-local coordinates: 16 B) + "
                                  f"{BIN_BYTES_PER_CELL} B per cell (count, start)"}

    # end to end through the C ABI from page-locked host memory, in the unit
    # of `value` (velocity-Verlet steps): every job of K steps starts from
    # the host state (copied in) and ends with the state read back into
    # host memory, and reads each step's energies and pair count back (48
    # bytes, without waiting).  Consecutive jobs are pipelined through the
    # library's two input staging slots: the next job's input copy and this
    # job's output copy run on a copy stream while the compute stream works.
    hpos = torch.from_numpy(pos).pin_memory()
    hvel = torch.from_numpy(vel).pin_memory()
    out_pos = [torch.empty_like(hpos).pin_memory() for _ in range(2)]
    out_vel = [torch.empty_like(hvel).pin_memory() for _ in range(2)]
    dout = [(torch.empty_like(dpos), torch.empty_like(dvel)) for _ in range(2)]
    copy_stream = torch.cuda.Stream(dev)
    jobs = 5
    res = [[torch.zeros(6, dtype=torch.float64).pin_memory() for _ in range(args.steps)] for _ in range(jobs)]

    def e2e_jobs(njobs):
        cs = copy_stream.cuda_stream
        g.stage_state(hpos, hvel, slot=0, copy_stream=cs)
        for j in range(njobs):
            b = j % 2
            g.set_state_staged(b)
            if j + 1 < njobs:
                g.stage_state(hpos, hvel, slot=(j + 1) % 2, copy_stream=cs)
            if forces_only:
                for k in range(args.steps):
                    if k:
                        g.set_state_staged(b)   # the job's input again
                    g.forces(sched)
                    g.energy_async(res[j][k])
            else:
                g.forces(sched)
                for k in range(args.steps):
                    g.verlet(DT, 1, sched)
                    g.energy_async(res[j][k])
            g.get("pos", out=dout[b][0])
            g.get("vel", out=dout[b][1])
            done = torch.cuda.Event()
            done.record(stream)
            copy_stream.wait_event(done)
            with torch.cuda.stream(copy_stream):
                out_pos[b].copy_(dout[b][0], non_blocking=True)
                out_vel[b].copy_(dout[b][1], non_blocking=True)
        torch.cuda.synchronize(dev)
        return sum(lc.decode(res[j][k])[3] for j in range(njobs) for k in range(args.steps))

    e2e_jobs(2)
    t0 = time.perf_counter()
    e2e_pairs = e2e_jobs(jobs)
    e2e_s = dist.max(time.perf_counter() - t0)
    state_bytes = int(hpos.numel() * 8 + hvel.numel() * 8)
    e2e = {"value": dist.sum(e2e_pairs) / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": state_bytes / args.steps,
           "d2h_bytes_per_step": 48 + state_bytes / args.steps,
           "jobs": jobs,
           "step": ("jobs of K steps through the C ABI: host state (page-locked) copied in through a staging "
                    "slot (lc_stage_state on a copy stream, lc_set_state_staged), lc_forces, K x (lc_verlet_step "
                    "of one step + lc_energy_virial_async of its 48-byte result), lc_get of positions and "
                    "velocities, copied out on the copy stream; the next job's input copy and this job's "
                    "output copy overlap the compute; bytes per step are a job's divided by K")
           if not forces_only else
                   ("jobs of K x (lc_set_state_staged + lc_forces + lc_energy_virial_async), host state copied "
                    "in through a staging slot and out on a copy stream, overlapping the compute")}
    g.close()

    if dist.rank == 0:
        cpu, errors = None, None
        if dist.world == 1 and not args.no_cpu_baseline:
            cpu, ref = cpu_baseline(pos, oracle_box(w), rc)
            u_first = u0
            errors = precision_report(f_first, u_first, w0, ref)
            if drift_gpu is not None:
                errors["drift"] = {"gpu_rel": drift_gpu["rel"], "gpu_steps": drift_gpu["steps"],
                                   "oracle_4k_fp64_rel": oracle_drift(drift_gpu["steps"], rc),
                                   "note": "relative energy drift of this run vs the oracle's FP64 run of the "
                                           "4,000-particle FCC box over the same number of steps"}
        line = {"metric": METRIC_LIST if is_list else METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
                "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
                "data": "synthetic", "config": workload_config(args, w),
                "steps_per_s": args.steps / (elapsed_ms * 1e-3) * dist.world,
                "schedule": sched, "schedule_force_ms": sched_ms, "tile": tile,
                "roofline": roofline, "roofline_bin": roofline_bin, "cpu_baseline": cpu, "errors": errors,
                "e2e": e2e, "sustained": sustained, "clocks": clk,
                "gpu_launches": launches}
        if is_list:
            line["list"] = {"skin": args.skin, "builds": list_stats["builds"],
                            "rebuild_steps": list_stats["rebuild_steps"], "kmax": list_stats["kmax"],
                            "entries_per_build": cand,
                            "note": "not the paper's method; rebuilds are decided on the device and not "
                                    "counted in gpu_launches"}
        print(json.dumps(line), flush=True)


def run_dag(args, dist):
    """The force sweep as the paper's task program on the device (Sec. III,
    Sec. V, Sec. VI Strategy 2): the DAG of each task-creation order executed
    by the dependency-counted device queue, next to the atomic schedule; for
    a 2D workload also the cell creation order under the three stencil
    orders of Fig. 5.  Prints one JSON line (an auxiliary measurement, not
    the headline)."""
    import torch
    from paper_1401_4441_gb300 import build
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    if dist.rank == 0:
        build.build()
    dist.barrier()
    from paper_1401_4441_gb300 import lc
    b = inputs.workload(args.workload, seed=inputs.DEFAULT_SEED + 1000 * dist.rank)
    pos, box, rc = b["pos"], b["box"], b["rc"]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    g = lc.Box(box, rc, pos.shape[0], args.precision, dims=b.get("dims", 3))
    g.set_state(torch.from_numpy(pos).to(dev))

    def timed(fn, reps=3):
        fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream); fn(); e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        return min(ts)

    g.forces("atomic")
    _, _, _, npairs = g.energy()
    rows = {"atomic": {"ms": timed(lambda: g.forces("atomic"))}}
    for order in ("loopex", "cell"):
        t, e, cp = g.dag_build(order)
        ms = timed(lambda: g.dag_forces(order))
        _, _, _, np_ = g.energy()
        assert np_ == npairs
        rows[f"dag_{order}"] = {"ms": ms, "tasks": t, "edges": e, "critical_path": cp,
                                "speedup_bound": t / cp, "us_per_critical_task": 1e3 * ms / cp}
    for r in rows.values():
        r["pairs_per_s"] = npairs / (r["ms"] * 1e-3)
    fig5 = None
    if b.get("dims", 3) == 2:
        # Fig. 5 on the device: the cell creation order under the paper's three
        # stencil orders (in this library's stencil orientation), on a smaller
        # 2D box (256 x 256 particles, 131 x 113 cells, 74k tasks) so that the
        # serial order stays near one second per evaluation
        s5 = inputs.tri_box(256, 256, 0.7, 0.5, seed=inputs.DEFAULT_SEED + 5, jitter=0.05)
        g5 = lc.Box(s5["box"], rc, s5["pos"].shape[0], args.precision, dims=2)
        try:
            g5.set_state(torch.from_numpy(s5["pos"]).to(dev))
            g5.forces("atomic")
            _, _, _, np5 = g5.energy()
            nc5, _, _ = g5.grid()
            fig5 = {"cells": [int(nc5[0]), int(nc5[1])], "pairs": int(np5), "orders": {}}
            for name, perm in (("naive", (0, 2, 3, 1, 4)), ("bad", (0, 2, 3, 4, 1)), ("opt", (1, 0, 4, 3, 2))):
                g5.dag_stencil_order(perm)
                t, e, cp = g5.dag_build("cell")
                ms = timed(lambda: g5.dag_forces("cell"), reps=2)
                _, _, _, np_ = g5.energy()
                assert np_ == np5
                fig5["orders"][name] = {"stencil_perm": list(perm), "ms": ms, "tasks": t, "critical_path": cp,
                                        "speedup_bound": t / cp, "us_per_critical_task": 1e3 * ms / cp}
            bad_ms = fig5["orders"]["bad"]["ms"]
            for r in fig5["orders"].values():
                r["measured_speedup_vs_bad"] = bad_ms / r["ms"]
        finally:
            g5.close()
    if dist.rank == 0:
        line = {"metric": "force evaluation time by task-DAG creation order", "unit": "ms",
                "higher_is_better": False, "n_gpus": dist.world, "precision": args.precision,
                "config": {"workload": b["name"], "particles": int(pos.shape[0]),
                           "l2": "flushed (512 MiB memset) before each timed call"},
                "pairs": int(npairs), "results": rows}
        if fig5 is not None:
            line["fig5_stencil_orders"] = fig5
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--schedule", default="auto", choices=["auto", "colour", "atomic", "fullshell", "buffer", "list"],
                    help="list: Verlet lists with a skin (not the paper's method; auxiliary line)")
    ap.add_argument("--skin", type=float, default=0.4, help="skin of --schedule list")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="liquid1m", choices=sorted(inputs.WORKLOADS) + ["batch512"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", default=None,
                    help="NI,WARPS: the force kernels' tile shape instead of the autotuner's choice "
                         "(16,16: the atomic schedule's row-group kernel)")
    ap.add_argument("--profile", action="store_true",
                    help="only warm-up + timed steps of one schedule (for ncu captures)")
    ap.add_argument("--dag", action="store_true",
                    help="time the task-DAG execution of each creation order (auxiliary line)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        elif args.profile:
            run_profile(args, dist)
        elif args.dag:
            run_dag(args, dist)
        elif args.workload == "batch512":
            run_batch(args, dist)
        else:
            run_gb300(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
