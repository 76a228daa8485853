"""The multi-rank bench path (torchrun, one replica per rank) on CPU with
the gloo backend, world size 2: barrier, max and sum over ranks."""
import os
import socket

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
