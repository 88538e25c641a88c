"""The bench's multi-rank bookkeeping (replicas: max over ranks, whole-job
throughput) on CPU with two gloo ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [100.0, 250.0][rank]   # the second rank is the slowest
    value, slowest = bench.job_throughput(ms, 1000, 4, 10, world, dist)
    out[rank] = (value, slowest)
    dist.destroy_process_group()


def test_two_rank_throughput_takes_the_slowest_rank():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in (0, 1):
        value, slowest = out[rank]
        assert slowest == 250.0
        assert abs(value - 2 * 1000 * 4 * 10 / 0.25) < 1e-6


def test_single_rank():
    import bench
    value, slowest = bench.job_throughput(50.0, 2000, 4, 5, 1)
    assert slowest == 50.0 and abs(value - 2000 * 4 * 5 / 0.05) < 1e-6
