#!/usr/bin/env python
"""Benchmark of the fused forward+adjoint objective on GB300.

One step = one evaluation of J = S_LCC + lambda*R_diff and dJ/dc
(al_objective_grad) on the 256x256x160 CT-like pair: local NCC with a 7^3
window, cubic B-spline spacing 6 (46x46x30 control points), lambda = 0.1,
control coefficients ~ N(0, 3^2) voxels. Inputs are seeded synthetic volumes
(the paper's CT data is not available) already resident in HBM; the L2 cache
is flushed by a 256 MiB write before every timed step.

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded slab of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+adjoint objective evals/s at 256×256×160; HBM GB/s vs peak; time-to-MSE"
UNIT = "evals/s"
SHAPE = (160, 256, 256)
SPACING = 6
LAMBDA = 0.1
WINDOW = 7
CTRL_SIGMA = 3.0
WORKLOAD = ("3D 256x256x160 fp32 CT-like pair (ellipsoids in [-1000,1500] HU + N(0,20^2) noise), "
            "LCC 7^3 + 0.1 diffusion, cubic B-spline spacing 6 (46x46x30 points), "
            "c ~ N(0, 3^2) voxels; one fused forward+adjoint evaluation per step")
FLUSH_BYTES = 256 << 20

# Algorithmic work of each kernel per voxel: the bytes its contract must move
# and the flops the method needs (an FMA counts 2), without tiling, halo or
# shift overhead. A kernel's roofline bound is the larger of bytes / HBM peak
# and flops / fp32 peak.
#  - k_lcc_stats: reads F, W (4 + 4 B) and the mask (1 B), writes the
#    coefficients (a', b, c) (12 B); the local sums of five fields (F, W,
#    F^2, W^2, FW) by separable 7-tap sums along three axes, 5 x 3 x 6 = 90
#    adds, 3 products, 25 for the statistics and coefficients: 118 flops;
#  - k_lcc_grad: reads the coefficients (12 B), F, W, mask (9 B), writes
#    dS/dW (4 B); box sums of three fields (3 x 18) and their combination
#    (4): 58 flops;
#  - k_fused_fwd: reads M, writes W, mask and dM~/dy (21 B); separable
#    B-spline expansion (28) and trilinear value and gradient (55): 83 flops;
#  - k_fused_gw: reads dS/dW and dM~/dy (16 B); products (3) and the
#    transposed expansion (28): 31 flops;
#  - the point-wise fused MSE / NCC kernels: read F and M (8 B); expansion,
#    warp and its adjoint, transposed expansion, the similarity terms:
#    150 / 160 flops (120-180 by a per-step count for the MSE path).
KERNEL_WORK = {  # name: (bytes per voxel, flops per voxel)
    "k_lcc_stats": (21.0, 118.0), "k_lcc_grad": (25.0, 58.0), "k_fused_fwd": (21.0, 83.0),
    "k_fused_gw": (16.0, 31.0), "k_fused_mse": (8.0, 150.0), "k_fused_ncc": (8.0, 160.0),
}
# Whole evaluation (roofline of one objective evaluation): algorithmic bytes 8 B per
# voxel (F and M read once) + 8 B per control coefficient (c in, dJ/dc out);
# algorithmic flops per voxel: expansion and transposed expansion (2 x 28),
# trilinear value and gradient (55), and the similarity: MSE 40 / NCC 50 /
# LCC 176 (forward box sums, statistics, adjoint box sums: 118 + 58), the
# regulariser on the lattice (Gram form) being negligible per voxel.
EVAL_FLOPS = {"mse": 151.0, "ncc": 161.0, "lcc": 287.0}
FP32_LANES = 128


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--sim", choices=["lcc", "mse", "ncc"], default="lcc")
    p.add_argument("--shape", type=str, default=None, help="Z,Y,X (default 160,256,256)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--learned-pairs", type=int, default=20000,
                   help="training pairs of the learned initialisation (0: skip it)")
    p.add_argument("--learned-test", type=int, default=8,
                   help="held-out pairs of the time-to-MSE comparison")
    p.add_argument("--no-registration", action="store_true",
                   help="skip the optimisation-loop timings (registration object)")
    p.add_argument("--cpu-budget", type=float, default=20.0,
                   help="seconds of oracle work for the cpu_baseline sample")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def workload(shape):
    from paper_1806_09907_gb300 import synth
    F, M = synth.ct_pair(shape)
    nd = len(shape)
    lat = tuple((s - 1) // SPACING + 4 for s in shape)
    c = synth.random_ctrl(lat, nd, CTRL_SIGMA, synth.FIELD_SEED)
    return F, M, c


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_slab(job):
    """One FP64 oracle forward+adjoint on a z-slab (a worker of the pool)."""
    import oracle
    kind, F, M, c = job
    t0 = time.perf_counter()
    oracle.objective_grad(kind, F, M, c, SPACING, LAMBDA, 1e-5, WINDOW)
    return time.perf_counter() - t0


def _slab(F, M, c, depth):
    nz = (depth - 1) // SPACING + 4
    return (np.ascontiguousarray(F[:depth]), np.ascontiguousarray(M[:depth]),
            np.ascontiguousarray(c[:, :nz]))


def oracle_sample(F, M, c, sim, budget_s, depth=None):
    """Time the oracle (single-threaded, as it stands) on a z-slab of the
    workload whose depth is chosen so one evaluation takes about budget_s
    (or of the given depth). Returns (evals/s of the full workload scaled by
    voxel count, seconds, slab depth)."""
    import oracle
    kind = {"mse": oracle.MSE, "ncc": oracle.NCC, "lcc": oracle.LCC}[sim]
    Z = F.shape[0]

    def run(depth):
        return _oracle_slab((kind,) + _slab(F, M, c, depth))

    if depth is not None:
        t = run(depth)
        return (depth / Z) / t, t, depth
    probe = min(4, Z)
    t_probe = run(probe)
    depth = int(max(2, min(Z, budget_s / max(t_probe / probe, 1e-9))))
    t = run(depth) if depth != probe else t_probe
    return (depth / Z) / t, t, depth


class OraclePool:
    """The oracle on every host core: a pool of worker processes (started with
    spawn, so no CUDA state is inherited) that evaluate z-slabs at once. The
    oracle itself is unchanged (each worker runs it single-threaded on its
    slab); covering the volume with one slab per core is the all-core timing
    of one evaluation's work."""

    def __init__(self, workers):
        import multiprocessing as mp
        self.workers = max(1, int(workers))
        self.pool = mp.get_context("spawn").Pool(self.workers)

    def close(self):
        self.pool.close()
        self.pool.join()

    def run(self, F, M, c, sim, depth):
        """`workers` slabs of `depth` slices at once: (evals/s of the full
        workload, wall seconds, fraction of the volume covered)."""
        import oracle
        kind = {"mse": oracle.MSE, "ncc": oracle.NCC, "lcc": oracle.LCC}[sim]
        job = (kind,) + _slab(F, M, c, depth)
        t0 = time.perf_counter()
        self.pool.map(_oracle_slab, [job] * self.workers, chunksize=1)
        wall = time.perf_counter() - t0
        frac = self.workers * depth / F.shape[0]
        return frac / wall, wall, frac


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(local_ms, units_per_rank, world, dist=None, device=None):
    """Whole-job throughput over `world` replicas: all units processed divided by
    the slowest rank's time (max over ranks). Returns (units/s, max_ms)."""
    t = float(local_ms)
    if dist is not None and world > 1:
        import torch
        x = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return world * units_per_rank / (t / 1000.0), t


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as fh:
                d = json.load(fh)
            return d, "measured"
        except (OSError, ValueError):
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_traffic(name, nv):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel's sources changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh).get(name)
    except (OSError, ValueError):
        return None
    if not t:
        return None
    h = hashlib.sha1()
    for f in t["sources"]:
        with open(os.path.join(ROOT, "paper_1806_09907_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return t["bytes_per_voxel"] * nv if h.hexdigest() == t["sources_sha1"] else None


def fp32_peak_tflops(clock_info, sms):
    mhz = (clock_info or {}).get("sm_max_mhz") or 2070.0
    note = f"fp32 FMA peak derived: {sms} SMs x {FP32_LANES} lanes x 2 flop x {mhz:.0f} MHz"
    return sms * FP32_LANES * 2 * mhz * 1e6 / 1e12, note


def roofline(dom, nv, clock_info, sms):
    """Roofline of the dominant kernel: its algorithmic bytes and flops per
    launch over its average launch time (library CUDA events on the launching
    stream), against the bound that binds it."""
    name, (ms_tot, launches) = dom
    per_launch_s = ms_tot / max(launches, 1) / 1000.0
    if name not in KERNEL_WORK:
        return None
    bpv, fpv = KERNEL_WORK[name]
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    fp32, fnote = fp32_peak_tflops(clock_info, sms)
    t_hbm, t_alu = bpv * nv / (hbm * 1e9), fpv * nv / (fp32 * 1e12)
    traffic = kernel_traffic(name, nv)
    if t_hbm >= t_alu:
        bound, achieved, peak, unit = "hbm", bpv * nv / per_launch_s / 1e9, hbm, "GB/s"
        note = f"HBM copy bandwidth, {src} ({fnote} does not bind)"
    else:
        bound, achieved, peak, unit = "alu", fpv * nv / per_launch_s / 1e12, fp32, "TFLOP/s"
        note = f"{fnote} (HBM copy bandwidth, {src}, does not bind)"
    out = {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
           "frac": achieved / peak, "traffic": traffic, "peak_source": note,
           "algorithmic_bytes_per_voxel": bpv, "algorithmic_flops_per_voxel": fpv,
           "launch_ms": per_launch_s * 1000.0,
           "hbm_frac": bpv * nv / per_launch_s / 1e9 / hbm,
           "alu_frac": fpv * nv / per_launch_s / 1e12 / fp32}
    if traffic is not None:
        out["traffic_gbs"] = traffic / per_launch_s / 1e9
    return out


def evaluation_roofline(sim, nv, nparams, ms_per_eval, clock_info, sms):
    """The whole evaluation against T_bound = max(bytes / HBM peak,
    flops / fp32 peak) with its algorithmic bytes and flops."""
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    fp32, fnote = fp32_peak_tflops(clock_info, sms)
    nbytes = 8.0 * nv + 8.0 * nparams
    flops = EVAL_FLOPS[sim] * nv
    t_hbm, t_alu = nbytes / (hbm * 1e9), flops / (fp32 * 1e12)
    t = ms_per_eval / 1000.0
    return {"algorithmic_bytes": nbytes, "algorithmic_flops": flops,
            "flops_per_voxel": EVAL_FLOPS[sim],
            "t_bound_us": 1e6 * max(t_hbm, t_alu), "bound": "hbm" if t_hbm >= t_alu else "alu",
            "t_hbm_us": 1e6 * t_hbm, "t_alu_us": 1e6 * t_alu, "t_measured_us": 1e6 * t,
            "frac": max(t_hbm, t_alu) / t,
            "hbm_gbs": nbytes / t / 1e9, "hbm_frac": nbytes / t / 1e9 / hbm,
            "peaks": f"HBM {hbm:.0f} GB/s ({src}); {fnote}"}


def run_reference(args, shape):
    """The reference arm: the FP64 oracle, as it stands, on the host's cores.
    Each step evaluates the full volume as one z-slab per core, all at once
    (a slab's halo is not shared, so the covered work is at least the
    volume's); when the requested steps would not fit in a few minutes, each
    step covers a bounded fraction of the volume instead and the throughput
    is scaled by voxel count."""
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    F, M, c = workload(shape)
    steps, warmup = max(1, args.steps), max(0, args.warmup)
    cores = cpu_cores()
    pool = OraclePool(cores)
    try:
        depth = -(-shape[0] // cores)  # one slab per core covers the volume
        _, t1, _ = pool.run(F, M, c, args.sim, depth)
        budget = 150.0  # seconds for the whole run
        if (steps + warmup) * t1 > budget:
            depth = max(2, int(depth * budget / ((steps + warmup) * t1)))
        vals, walls = [], []
        for i in range(warmup + steps):
            v, wall, frac = pool.run(F, M, c, args.sim, depth)
            if i >= warmup:
                vals.append(v)
                walls.append(wall / frac)  # seconds per full-volume evaluation
    finally:
        pool.close()
    total = sum(walls)
    value = steps / total
    covered = min(1.0, cores * depth / shape[0])
    sample = (f"each step: {cores} z-slabs of {shape[2]}x{shape[1]}x{depth} voxels, one FP64 "
              f"oracle forward+adjoint per slab, all at once on {cores} worker processes "
              f"({covered:.0%} of the volume per step" +
              ("" if covered >= 1.0 else ", scaled by voxel count") + ")")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": 1000.0 * total / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "shape_zyx": list(shape), "spacing": SPACING,
                   "similarity": f"{args.sim}{WINDOW if args.sim == 'lcc' else ''}",
                   "lambda": LAMBDA, "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "cpu": cpu_model(), "host_cores": cpu_cores(), "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def registration_runs(F, M, c, dev):
    """Optimisation-loop timings, outside the headline timed region: the
    three-level LCC pyramid on the headline pair (one CUDA graph per level)
    and 200 Adam iterations on the 128^3 blob pair through the autograd
    Function. Device times from CUDA events on the launching stream."""
    import torch
    from paper_1806_09907_gb300 import airgb, registration, synth

    Fd, Md = torch.from_numpy(F).to(dev), torch.from_numpy(M).to(dev)
    kw = dict(spacing=SPACING, sim="lcc", lam=LAMBDA, factors=(4, 2, 1), iterations=150)
    registration.register(Fd, Md, **kw)  # warm-up (pyramid buffers, attributes)
    r = registration.register(Fd, Md, **kw)
    levels = []
    for lv in r.levels:
        v = lv.values.cpu().numpy()
        levels.append({"factor": lv.factor, "shape_zyx": list(lv.shape), "iterations": lv.iterations,
                       "device_ms": lv.ms, "ms_per_iteration": lv.ms / lv.iterations,
                       "J_start": float(v[0, 0]), "J_end": float(v[-1, 0])})
    ev = registration.Evaluator(tuple(F.shape), SPACING, "lcc", LAMBDA, device=dev)
    v0 = torch.empty(4, dtype=torch.float64, device=dev)
    ev.evaluate(Fd, Md, torch.zeros_like(r.ctrl), v0)
    pyramid = {
        "workload": "the headline CT pair; LCC 7^3 + 0.1 diffusion, spacing 6; Gaussian pyramid "
                    "factors 4/2/1 x 150 Adam iterations (lr 0.01 in normalised units), "
                    "exact B-spline refinement between levels, one CUDA graph per level",
        "device_ms": sum(lv["device_ms"] for lv in levels), "wall_s": r.seconds,
        "levels": levels, "S_unregistered": float(v0[1]),
        "S_registered": float(r.levels[-1].values[-1, 1])}

    Fb, Mb = synth.blobs_3d_128()
    shape = tuple(Fb.shape)
    Fb, Mb = torch.from_numpy(Fb).to(dev), torch.from_numpy(Mb).to(dev)
    evb = registration.Evaluator(shape, 8, "mse", LAMBDA, device=dev)

    def adam_run(n, graphed):
        c = torch.zeros(evb.lattice, dtype=torch.float32, device=dev, requires_grad=True)
        opt = registration.BsplineAdam([c], shape, 8, lr=0.01)
        if graphed:
            it = registration.GraphedIteration(c, evb, Fb, Mb, opt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e0.record()
        for _ in range(n):
            if graphed:
                it()
            else:
                opt.zero_grad()
                J = registration.objective(c, evb, Fb, Mb)
                J.backward()
                opt.step()
        e1.record()
        torch.cuda.synchronize(dev)
        return c, e0.elapsed_time(e1), time.perf_counter() - t0

    adam_run(5, False)
    adam_run(5, True)
    _, eager_ms, eager_wall = adam_run(200, False)
    cb, dev_ms, wall = adam_run(200, True)
    vb = torch.empty((2, 4), dtype=torch.float64, device=dev)
    evb.evaluate(Fb, Mb, torch.zeros_like(cb), vb[0])
    evb.evaluate(Fb, Mb, cb.detach(), vb[1])
    vb = vb.cpu().numpy()
    adam = {
        "workload": "3D 128^3 blob pair (60 blobs, sigma 3-12), MSE + 0.1 diffusion, spacing 8 "
                    "(19^3 points), 200 Adam iterations (lr 0.01 in normalised units) through "
                    "ObjectiveFunction.backward and BsplineAdam, one iteration captured in a "
                    "CUDA graph and replayed",
        "device_ms": dev_ms, "wall_s": wall, "ms_per_iteration": dev_ms / 200,
        "eager_ms_per_iteration": eager_ms / 200,
        "mse_start": float(vb[0, 1]), "mse_end": float(vb[1, 1])}
    # 64 uneven pairs, 100 iterations: the persistent batch kernel (tuned
    # work order, all iterations in one CUDA graph) against the same
    # registrations one pair after another with plain launches
    pairs = synth.batch_pairs(32, 32, device=dev)
    iters = 100
    registration.register_batch(pairs, 8, LAMBDA, iterations=3, graph=False, tune=False)
    rb = registration.register_batch(pairs, 8, LAMBDA, iterations=iters, graph=True, tune=True)
    registration.register_sequential(pairs[:2], 8, LAMBDA, 3)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    cs, hs, seq_ms = registration.register_sequential(pairs, 8, LAMBDA, iters)
    seq_wall = time.perf_counter() - t0
    same = all(torch.equal(a, c) for a, c in zip(cs, rb.batch.ctrl))
    nvox = sum(int(np.prod(tuple(f.shape))) for f, _ in pairs)
    total, per_kind = rb.batch.items()
    batch = {
        "workload": "64 blob pairs of uneven sizes (32 2D from 96^2 to 512^2, 32 3D from 64^3 "
                    "to 192^3), MSE + 0.1 diffusion, spacing 8, 100 Adam iterations each",
        "voxels": nvox, "work_items_per_iteration": total,
        "items_bricks_tiles_chunks": list(per_kind),
        "batched_device_ms": rb.device_ms, "batched_ms_per_iteration": rb.device_ms / iters,
        "batched_order": rb.policy, "batched_tile": rb.tile,
        "batched_tile_cells": list(rb.tile_cells),
        "tuning_ms_per_iteration": rb.tuning_ms,
        "default_tile_ms_per_iteration": min(rb.tuning_ms[0]) if rb.tuning_ms else None,
        "sequential_device_ms": seq_ms, "sequential_wall_s": seq_wall,
        "speedup": seq_ms / rb.device_ms, "coefficients_bit_identical": bool(same)}
    # the diffeomorphic model on the headline pair: one forward+adjoint
    # evaluation through the step kernels, 6 squarings
    pr = airgb.make_problem(tuple(F.shape), SPACING, "lcc", LAMBDA, 1e-5, WINDOW)
    K = 6
    cd = torch.from_numpy(c).to(dev)
    wsd = torch.empty(airgb.objective_diffeo_workspace_bytes(pr, K), dtype=torch.uint8, device=dev)
    vd = torch.empty(4, dtype=torch.float64, device=dev)
    gd = torch.empty_like(cd)
    for _ in range(2):
        airgb.al_objective_grad_diffeo(pr, Fd, Md, cd, K, vd, gd, wsd)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_eval = 5
    e0.record()
    for _ in range(n_eval):
        airgb.al_objective_grad_diffeo(pr, Fd, Md, cd, K, vd, gd, wsd)
    e1.record()
    e1.synchronize()
    diffeo = {
        "workload": "the headline pair and coefficients, diffeomorphic model f = exp(v) with 6 "
                    "squarings; LCC 7^3 + 0.1 diffusion of u_6; one forward+adjoint evaluation",
        "ms_per_eval": e0.elapsed_time(e1) / n_eval,
        "evals_per_s": 1000.0 * n_eval / e0.elapsed_time(e1),
        "workspace_bytes": int(wsd.numel()), "J": float(vd[0])}
    # the other objective configurations, one forward+adjoint evaluation each:
    # MSE on the headline pair, the 128^3 blob pair (spacing 8, MSE), and the
    # 2D 128^2 blob pair (spacing 8, MSE; L2-resident and launch-latency
    # bound, so timed as CUDA-graph replays of 100 evaluations)
    def timed(ev, Fx, Mx, cx, n, graph=False):
        val = torch.empty(4, dtype=torch.float64, device=dev)
        gr = torch.empty_like(cx)
        for _ in range(3):
            ev.evaluate(Fx, Mx, cx, val, gr)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if graph:
            gph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gph, capture_error_mode="thread_local"):
                for _ in range(n):
                    ev.evaluate(Fx, Mx, cx, val, gr)
            a.record()
            gph.replay()
            b.record()
        else:
            a.record()
            for _ in range(n):
                ev.evaluate(Fx, Mx, cx, val, gr)
            b.record()
        b.synchronize()
        return a.elapsed_time(b) / n

    others = {}
    ev_mse = registration.Evaluator(tuple(F.shape), SPACING, "mse", LAMBDA, device=dev)
    ms = timed(ev_mse, Fd, Md, cd, 20)
    others["mse_ct"] = {"workload": "the headline pair and coefficients, MSE + 0.1 diffusion",
                        "ms_per_eval": ms, "evals_per_s": 1000.0 / ms}
    Fb3, Mb3 = (torch.from_numpy(a).to(dev) for a in synth.blobs_3d_128())
    c3 = torch.from_numpy(synth.random_ctrl((19, 19, 19), 3, 1.0, synth.FIELD_SEED)).to(dev)
    ms = timed(registration.Evaluator((128, 128, 128), 8, "mse", LAMBDA, device=dev), Fb3, Mb3,
               c3, 50)
    others["blobs_3d_128"] = {"workload": "3D 128^3 blob pair, MSE + 0.1 diffusion, spacing 8, "
                                          "c ~ N(0, 1)", "ms_per_eval": ms,
                              "evals_per_s": 1000.0 / ms}
    Fb2, Mb2 = (torch.from_numpy(a).to(dev) for a in synth.blobs_2d_128())
    c2 = torch.from_numpy(synth.random_ctrl((19, 19), 2, 1.0, synth.FIELD_SEED)).to(dev)
    ms = timed(registration.Evaluator((128, 128), 8, "mse", LAMBDA, device=dev), Fb2, Mb2, c2,
               100, graph=True)
    others["blobs_2d_128"] = {"workload": "2D 128^2 blob pair, MSE + 0.1 diffusion, spacing 8, "
                                          "c ~ N(0, 1); CUDA-graph replay of 100 evaluations",
                              "us_per_eval": 1000.0 * ms}
    return {"pyramid_ct": pyramid, "adam_blobs_128": adam, "batch_64": batch,
            "diffeo_ct": diffeo, "objective_configs": others}


def learned_init_runs(dev, pairs, n_test):
    """Learned initialisation: train the encoder-decoder on `pairs`
    method-generated 128^3 pairs (batch 16), then on `n_test` held-out pairs
    compare the plain optimiser (200 Adam iterations from zero) with the
    network's prediction refined by the same optimiser until it reaches the
    plain method's final MSE."""
    from paper_1806_09907_gb300 import airgb, learned_init

    shape, batch = (128, 128, 128), 16
    net = learned_init.InitNet(shape, batch, dev, seed=1806)
    # warm-up: kernel attributes and one step of every launch
    learned_init.train(learned_init.InitNet(shape, batch, dev, seed=1), pairs=batch)
    tr = learned_init.train(net, pairs=pairs, lr=1e-3, sigma=4.0, seed=0)
    # one training step's kernels (library event timing, a separate network)
    prof = learned_init.InitNet(shape, batch, dev, seed=7)
    learned_init.train(prof, pairs=batch, seed=5, graph=False)
    airgb.profile_reset()
    airgb.profile_enable(True)
    n_prof = 5
    # eager, so every launch is timed (graph replays are not)
    learned_init.train(prof, pairs=n_prof * batch, seed=5, graph=False)
    step_kernels = {k: {"us_per_step": 1000.0 * t / n_prof, "launches_per_step": n // n_prof}
                    for k, (t, n) in airgb.profile_collect().items()}
    airgb.profile_enable(False)
    airgb.profile_reset()
    # algorithmic tensor work of the layers per step: forward, input adjoint
    # (not for the first layer) and weight adjoint, 2 flop per multiply-add
    conv_flop = 0.0
    for k, cv in enumerate(prof.convs):
        cin, cout = learned_init.LAYERS[k][0], learned_init.LAYERS[k][2]
        osz = airgb.conv_output_size(cv)
        per_pass = 2.0 * batch * np.prod(osz) * cout * 27 * cin
        conv_flop += per_pass * (3 if k > 0 else 2)
    conv_us = sum(v["us_per_step"] for k, v in step_kernels.items() if k.startswith("k_conv"))
    peaks, psrc = measured_peaks()
    peak = peaks.get("bf16_tflops")
    tensor = {"flop_per_step": conv_flop, "conv_us_per_step": conv_us,
              "achieved_tflops": conv_flop / conv_us / 1e6 if conv_us else None,
              "peak_tflops": peak, "unit": "TFLOP/s",
              "peak_source": f"bf16 dense, burst ({psrc})",
              "frac": (conv_flop / conv_us / 1e6 / peak) if (conv_us and peak) else None}
    one = learned_init.InitNet(shape, 1, dev, seed=1806)
    one.params.copy_(net.params)
    one.pack()
    src = learned_init.PairSource(shape, 1, 4.0, seed=424242, device=dev)
    reports = []
    for i in range(n_test):
        F, M, ct = src.make(i)
        reports.append(learned_init.evaluate_pair(one, F[0].clone(), M[0].clone(),
                                                  ct[0].clone()))
    ok = [r for r in reports if r.iterations_to_plain >= 0]
    okJ = [r for r in reports if r.iterations_to_plain_J >= 0]

    def mean(key, rs=reports):
        return float(np.mean([getattr(r, key) for r in rs])) if rs else None

    L = tr.losses
    return {
        "workload": "3D 128^3 blob pairs (60 blobs, sigma 3-12), c* ~ N(0, 4^2) voxels at "
                    "spacing 8, F = M o (x + B c*); encoder-decoder 16/32/48/64 channels, bf16 "
                    "weights and activations, fp32 accumulation (tcgen05); plain optimiser: MSE + "
                    "0.1 diffusion, Adam lr 0.01 (normalised units), 200 iterations from zero",
        "train": {"pairs": tr.pairs, "steps": tr.steps, "batch": batch, "seconds": tr.seconds,
                  "ms_per_step": 1000.0 * tr.seconds / tr.steps,
                  "loss_first_50": float(np.mean(L[:50])), "loss_last_50": float(np.mean(L[-50:]))},
        "step_kernels": step_kernels,
        "conv_tensor": tensor,
        "test_pairs": n_test,
        "reached_plain_mse": len(ok),
        "fallbacks": int(sum(r.fallback for r in reports)),
        "plain_ms_mean": mean("plain_ms"),
        "infer_ms_mean": mean("infer_ms"),
        "learned_ms_mean": mean("learned_ms", ok),
        "iterations_to_plain_mean": mean("iterations_to_plain", ok),
        "speedup": (float(np.mean([r.plain_ms for r in ok]) / np.mean([r.learned_ms for r in ok]))
                    if ok else None),
        "iterations_to_plain_best_mse": [r.iterations_to_best for r in reports],
        "objective_J": {
            "reached_plain_J": len(okJ),
            "iterations_to_plain_J_mean": mean("iterations_to_plain_J", okJ),
            "learned_ms_J_mean": mean("learned_ms_J", okJ),
            "speedup_J": (float(np.mean([r.plain_ms for r in okJ]) /
                                np.mean([r.learned_ms_J for r in okJ])) if okJ else None),
            "plain_final_J": mean("plain_final_J"), "refined_final_J": mean("refined_final_J")},
        "mse": {"zero": mean("zero_mse"), "prediction": mean("init_mse"),
                "plain_final": mean("plain_final_mse"), "plain_best": mean("plain_best_mse"),
                "refined_final": mean("refined_final_mse")},
        "field_rmse_vox": {"zero": mean("field_rmse_zero"), "prediction": mean("field_rmse_pred"),
                           "plain_final": mean("field_rmse_plain"),
                           "refined_final": mean("field_rmse_refined")},
        "pairs": [dataclasses.asdict(r) for r in reports],
    }


def main():
    args = parse()
    shape = tuple(int(s) for s in args.shape.split(",")) if args.shape else SHAPE
    if args.impl == "reference":
        return run_reference(args, shape)

    import torch
    from paper_1806_09907_gb300 import airgb
    from paper_1806_09907_gb300 import build as airgb_build

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    if rank == 0:
        airgb_build.build()
    if pg:
        pg.barrier()
    airgb.load()

    F, M, c = workload(shape)
    Fd, Md, cd = (torch.from_numpy(a).to(dev) for a in (F, M, c))
    obj = airgb.Objective(shape, SPACING, args.sim, LAMBDA, 1e-5, WINDOW, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize(dev)

    warmup = max(3, args.warmup)
    steps = max(1, args.steps)
    for _ in range(warmup):
        flush.zero_()
        obj(Fd, Md, cd)
    torch.cuda.synchronize(dev)

    # ---- timed region: K steps, per-step CUDA events, L2 flushed before each
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    clocks = ClockSampler(torch.cuda.get_device_properties(dev).index
                          if hasattr(torch.cuda.get_device_properties(dev), "index") else local_rank)
    airgb.profile_reset()
    airgb.profile_enable(True)
    clocks.start()
    barrier()
    for k in range(steps):
        flush.zero_()
        starts[k].record(stream)
        obj(Fd, Md, cd)
        ends[k].record(stream)
    barrier()
    clock_info = clocks.stop()
    airgb.profile_enable(False)
    kernels = airgb.profile_collect()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    value, total_ms = aggregate(sum(step_ms), steps, world, pg, dev)

    # ---- end to end through the public API with host buffers: every step
    #      uploads its inputs from pinned host memory and reads J and dJ/dc
    #      back. The upload of step k+1 runs on a copy stream while step k
    #      computes (two device input buffers, ordered by events), as a
    #      serving loop would run it.
    Fh, Mh, ch = (torch.from_numpy(a).pin_memory() for a in (F, M, c))
    vh = [torch.empty(4, dtype=torch.float64).pin_memory() for _ in range(2)]
    gh = [torch.empty(tuple(cd.shape), dtype=torch.float32).pin_memory() for _ in range(2)]
    bufs = [(torch.empty_like(Fd), torch.empty_like(Md), torch.empty_like(cd)) for _ in range(2)]
    copy_stream = torch.cuda.Stream(dev)
    ready = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]
    e2e_steps = max(3, min(steps, 50))

    def e2e_loop(n):
        for k in range(n):
            b = k % 2
            Fe, Me, ce = bufs[b]
            with torch.cuda.stream(copy_stream):
                if k >= 2:
                    copy_stream.wait_event(freed[b])  # step k-2 is done with these buffers
                Fe.copy_(Fh, non_blocking=True)
                Me.copy_(Mh, non_blocking=True)
                ce.copy_(ch, non_blocking=True)
                ready[b].record(copy_stream)
            stream.wait_event(ready[b])
            v, g = obj(Fe, Me, ce)
            vh[b].copy_(v, non_blocking=True)
            gh[b].copy_(g, non_blocking=True)
            freed[b].record(stream)

    e2e_loop(2)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    copy_stream.wait_event(e0)
    e2e_loop(e2e_steps)
    e1.record(stream)
    barrier()
    e2e_value, e2e_ms = aggregate(e0.elapsed_time(e1), e2e_steps, world, pg, dev)
    h2d = F.nbytes + M.nbytes + c.nbytes
    d2h = vh[0].numel() * 8 + gh[0].numel() * 4

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel and of the whole evaluation
    nv = int(np.prod(shape))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    dom = max(kernels.items(), key=lambda kv: kv[1][0]) if kernels else None
    roof = roofline(dom, nv, clock_info, sms) if dom else None
    if roof is not None:
        roof["evaluation"] = evaluation_roofline(args.sim, nv, c.size, total_ms / steps,
                                                 clock_info, sms)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        # the oracle on every host core (one z-slab per core, all at once),
        # and single-threaded on a slab of about --cpu-budget seconds
        cores = cpu_cores()
        pool = OraclePool(cores)
        try:
            _, t1, _ = pool.run(F, M, c, args.sim, 2)
            per_slice = t1 / 2.0
            depth = int(max(2, min(shape[0], args.cpu_budget / max(per_slice, 1e-9))))
            v_all, wall, frac = pool.run(F, M, c, args.sim, depth)
        finally:
            pool.close()
        v1, t, depth1 = oracle_sample(F, M, c, args.sim, args.cpu_budget)
        cpu = {"value": v_all, "unit": UNIT, "cores": cores, "kind": "oracle",
               "cpu": cpu_model(), "host_cores": cpu_cores(),
               "sample": f"{cores} z-slabs of {shape[2]}x{shape[1]}x{depth} voxels, one FP64 "
                         f"oracle forward+adjoint per slab, all at once on {cores} worker "
                         f"processes ({wall:.1f} s for {frac:.2f} volumes), scaled by voxel count",
               "single_thread": {"value": v1, "cores": 1,
                                 "sample": f"one evaluation on a {shape[2]}x{shape[1]}x{depth1} "
                                           f"z-slab ({t:.1f} s), scaled by voxel count"}}
    reg = None
    if world == 1 and not args.no_registration:
        reg = registration_runs(F, M, c, dev)
        if args.learned_pairs > 0:
            reg["learned_init"] = learned_init_runs(dev, args.learned_pairs, args.learned_test)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "shape_zyx": list(shape), "spacing": SPACING,
                   "similarity": f"{args.sim}{WINDOW if args.sim == 'lcc' else ''}",
                   "lambda": LAMBDA, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed by a 256 MiB write before every timed step",
                   "timing": "per-step CUDA events on the launching stream"},
        "step_ms": {"median": statistics.median(step_ms), "min": min(step_ms),
                    "max": max(step_ms), "p10": float(np.percentile(step_ms, 10)),
                    "p90": float(np.percentile(step_ms, 90))},
        # algorithmic bytes of one evaluation (read F and M once, c in and
        # dJ/dc out) over the step time
        "effective_gbs": (8.0 * nv + 8.0 * c.size) / (total_ms / steps) / 1e6,
        "kernels": {k: {"total_ms": v[0], "launches": v[1], "avg_us": 1000.0 * v[0] / max(v[1], 1)}
                    for k, v in kernels.items()},
        "gpu_launches": int(sum(v[1] for v in kernels.values())),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps": e2e_steps,
                "pipeline": "step k+1's upload overlaps step k's compute (copy stream, two "
                            "device input buffers)"},
        "clocks": clock_info,
        "registration": reg,
    }
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
