"""Multi-rank host logic on CPU with the gloo backend, world size 2: the
bench's barrier, max and sum over ranks, and the sharding of a batch of
independent boxes (partition, gather of the per-box results on rank 0)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    d = bench.Dist()
    d.barrier()
    out[rank] = (d.rank, d.world, d.max(10.0 * (rank + 1)), d.sum(rank + 1.5))
    d.close()


def test_dist_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == (0, 2, 20.0, 4.0)
    assert out[1] == (1, 2, 20.0, 4.0)


def test_autotune_occupancy_bucket():
    from paper_1401_4441_gb300 import autotune
    assert autotune.occupancy_bucket(1048576, 74088) == 16
    assert autotune.occupancy_bucket(100, 1000) == 1
    assert autotune.occupancy_bucket(2000000, 257600) == 8


def test_partition_covers_every_box_once_and_balances():
    from paper_1401_4441_gb300 import inputs, shard
    boxes = inputs.batch_boxes(nbox=512)
    ns = [b["pos"].shape[0] for b in boxes]
    for world in (1, 2, 3, 4, 8):
        parts = shard.partition_boxes(ns, world)
        allb = np.sort(np.concatenate(parts))
        assert np.array_equal(allb, np.arange(512))
        loads = [sum(ns[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(ns)        # greedy LPT bound
        assert max(loads) <= 1.02 * sum(ns) / world      # and tight on this mix


def _shard_worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as td
    import oracle
    from paper_1401_4441_gb300 import inputs, shard
    td.init_process_group("gloo", init_method="env://")
    boxes = inputs.batch_boxes(nbox=6, n_min=300, n_max=900)
    ns = [b["pos"].shape[0] for b in boxes]
    mine = shard.partition_boxes(ns, world)[rank]
    rows = []
    for bi in mine:    # each rank evaluates its boxes (the oracle stands in for the GPU)
        p = boxes[bi]["pos"]
        _, U, W, npairs = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], boxes[bi]["box"], 2.5)
        rows.append([U, W, float(npairs)])
    got = shard.gather_box_results(td, len(boxes), mine, np.array(rows).reshape(-1, 3))
    out[rank] = None if got is None else got.tolist()
    td.destroy_process_group()


def test_sharded_batch_gathers_single_rank_totals():
    """Two gloo ranks each evaluate their boxes; rank 0's gathered per-box
    energies, virials and pair counts equal those of one rank doing all."""
    import oracle
    from paper_1401_4441_gb300 import inputs, shard
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    assert out[1] is None
    boxes = inputs.batch_boxes(nbox=6, n_min=300, n_max=900)
    rows = []
    for b in boxes:
        p = b["pos"]
        _, U, W, npairs = oracle.lc_forces(p[:, 0], p[:, 1], p[:, 2], b["box"], 2.5)
        rows.append([U, W, float(npairs)])
    single = shard.gather_box_results(None, len(boxes), np.arange(len(boxes)), np.array(rows))
    assert np.array_equal(np.array(out[0]), single)
