"""The N > 1 path of bench.py on CPU: two gloo ranks stand in for two GPUs running
independent replicas; the whole-job throughput takes the slowest rank's time and counts
every rank's zones, with no data-path collective."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 250.0][rank]
    zu, t = bench.replica_throughput(4096 * 4096, 3, 10, local_ms, world)
    q.put((rank, zu, t))
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29517
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    expect = 4096 * 4096 * 3 * 10 * 2 / 0.25
    for rank, zu, t in res:
        assert t == 250.0
        assert zu == pytest.approx(expect, rel=1e-12)


def test_single_rank_is_local_time():
    sys.path.insert(0, ROOT)
    import bench
    zu, t = bench.replica_throughput(1000, 2, 5, 50.0, 1)
    assert t == 50.0 and zu == pytest.approx(1000 * 2 * 5 / 0.05)
