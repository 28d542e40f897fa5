"""The benchmark's multi-rank aggregation (replicas, one per rank) on two gloo ranks on CPU:
the job time is the slowest rank's time and the work is the sum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, units = bench.aggregate(0.5 + rank, 1000.0 * (rank + 1), dist, "cpu")
    out[rank] = (t, units)
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r] == (1.5, 3000.0)


def test_aggregate_single_process_is_identity():
    import bench
    assert bench.aggregate(2.0, 7.0, None) == (2.0, 7.0)
