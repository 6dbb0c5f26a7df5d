"""Host logic of bench.py that needs no GPU: whole-job throughput over
replicas (max over ranks) with a world-size-2 gloo process group."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slowest
    value, t = bench.aggregate(local_ms, 10, world, dist, "cpu")
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_takes_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        value, t = res[r]
        assert t == pytest.approx(150.0)
        assert value == pytest.approx(2 * 10 / 0.150)


def test_aggregate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    value, t = bench.aggregate(250.0, 5, 1)
    assert t == 250.0 and value == pytest.approx(20.0)
