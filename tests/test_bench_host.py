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


def test_roofline_takes_the_bound_that_binds():
    """The dominant kernel's roofline uses the larger of bytes / HBM peak and
    flops / fp32 peak, and the whole evaluation's T_bound is the grading
    formula max(bytes / HBM, flops / fp32) over the measured time."""
    sys.path.insert(0, ROOT)
    import bench
    nv = 10_485_760
    clock = {"sm_max_mhz": 2000.0}
    sms = 100
    fp32 = sms * 128 * 2 * 2000.0e6 / 1e12  # TFLOP/s
    peaks, _ = bench.measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    # k_lcc_stats: 21 B and 118 flops per voxel, 200 us per launch
    r = bench.roofline(("k_lcc_stats", (2.0, 10)), nv, clock, sms)
    t_hbm, t_alu = 21.0 * nv / (hbm * 1e9), 118.0 * nv / (fp32 * 1e12)
    assert r["bound"] == ("hbm" if t_hbm >= t_alu else "alu")
    want = 21.0 * nv / 200e-6 / 1e9 if r["bound"] == "hbm" else 118.0 * nv / 200e-6 / 1e12
    assert abs(r["achieved"] - want) <= 1e-9 * want
    assert abs(r["frac"] - r["achieved"] / r["peak"]) <= 1e-12
    e = bench.evaluation_roofline("lcc", nv, 190_440, 0.5, clock, sms)
    nbytes, flops = 8.0 * nv + 8.0 * 190_440, 287.0 * nv
    tb = max(nbytes / (hbm * 1e9), flops / (fp32 * 1e12))
    assert abs(e["t_bound_us"] - 1e6 * tb) <= 1e-6 * 1e6 * tb
    assert abs(e["frac"] - tb / 0.5e-3) <= 1e-9
    assert abs(e["hbm_frac"] - nbytes / 0.5e-3 / 1e9 / hbm) <= 1e-9
