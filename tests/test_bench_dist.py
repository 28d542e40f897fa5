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


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints one JSON line with the
    contract's keys, the same metric, unit and config as the GPU arm, and a zero-copy e2e."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=root, check=True, capture_output=True, text=True, timeout=600)
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, root)
    import bench
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling", "vs_baseline",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GDOF/s"
    assert d["higher_is_better"] is True and d["value"] > 0
    E = 32 ** 3
    assert d["config"] == bench.arm_config(32, E, E * 512, (32 * 7 + 1) ** 3, 1)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
