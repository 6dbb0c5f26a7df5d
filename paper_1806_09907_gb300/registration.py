"""Gradient-based registration around the objective (Sec. II-A, Optimization;
Adam as in Sec. III-G and the usage example of Sec. IV; multi-resolution as in
the FFD experiment of Sec. IV-A).

Three pieces, all driving kernels of libairgb through the binding:

* :class:`ObjectiveFunction` -- J(c) as a ``torch.autograd.Function`` with a
  hand-written backward. Forward runs the fused forward+adjoint kernels when
  the control points need a gradient and keeps only dJ/dc (lattice sized);
  the displacement, warped image and per-voxel gradients are never stored.
  With ``recompute=True`` forward evaluates J alone and backward runs the
  whole evaluation again, recomputing the displacement field.
* :class:`BsplineAdam` -- a ``torch.optim.Optimizer`` whose step is the Adam
  kernel of the library, in the paper's normalised coordinates.
* :func:`register` -- coarse-to-fine registration: Gaussian pyramid levels
  of both images, Adam iterations of the objective per level (captured in one
  CUDA graph per level by default) and exact B-spline refinement of the
  coefficients between levels. With ``checkpoint`` it writes the state after
  every level (:class:`Checkpoint`, an ``.npz`` file), and ``resume`` starts
  from such a file at the next level.
"""
from __future__ import annotations

import dataclasses
import os
import time

import numpy as np
import torch

from . import airgb


class Evaluator:
    """The problem and workspace of one objective (shared by calls on the
    same stream; calls must not overlap on the GPU). diffeo_steps: None for
    the plain B-spline model, else the number of squarings of the
    diffeomorphic model f = exp(v) (Sec. III-D)."""

    def __init__(self, shape, spacing, sim="mse", lam=0.1, eps=1e-5, window=7, device="cuda",
                 fused=True, diffeo_steps=None):
        self.shape = tuple(shape)
        self.spacing = int(spacing)
        self.problem = airgb.make_problem(shape, spacing, sim, lam, eps, window)
        self.fused = fused
        self.diffeo_steps = None if diffeo_steps is None else int(diffeo_steps)
        self.lattice = (len(shape),) + airgb.lattice_shape(shape, spacing)
        nbytes = (airgb.objective_workspace_bytes(self.problem, fused) if self.diffeo_steps is None
                  else airgb.objective_diffeo_workspace_bytes(self.problem, self.diffeo_steps))
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.last_value = None  # {J, S, R, n_mask} of the latest forward

    def evaluate(self, fixed, moving, ctrl, value, grad=None):
        if self.diffeo_steps is not None:
            airgb.al_objective_grad_diffeo(self.problem, fixed, moving, ctrl, self.diffeo_steps,
                                           value, grad, self.workspace,
                                           want_grad=grad is not None)
        else:
            airgb.al_objective_grad(self.problem, fixed, moving, ctrl, value, grad,
                                    self.workspace, want_grad=grad is not None, fused=self.fused)


class ObjectiveFunction(torch.autograd.Function):
    """J(c) = S + lambda R (Eq. objective) with dJ/dc from the library's
    adjoint kernels. Returns a 0-d float64 tensor."""

    @staticmethod
    def forward(ctx, ctrl, evaluator: Evaluator, fixed, moving, recompute=False):
        value = torch.empty(4, dtype=torch.float64, device=ctrl.device)
        need = ctx.needs_input_grad[0]
        ctx.evaluator, ctx.fixed, ctx.moving = evaluator, fixed, moving
        ctx.recompute = bool(recompute)
        if need and not recompute:
            grad = torch.empty_like(ctrl)
            evaluator.evaluate(fixed, moving, ctrl, value, grad)
            ctx.save_for_backward(grad)
        else:
            evaluator.evaluate(fixed, moving, ctrl, value, None)
            if need:
                ctx.save_for_backward(ctrl)
        evaluator.last_value = value
        return value[0]

    @staticmethod
    def backward(ctx, grad_out):
        (saved,) = ctx.saved_tensors
        if ctx.recompute:  # evaluate again: u, W and dS/dW are recomputed
            grad = torch.empty_like(saved)
            scratch = torch.empty(4, dtype=torch.float64, device=saved.device)
            ctx.evaluator.evaluate(ctx.fixed, ctx.moving, saved, scratch, grad)
        else:
            grad = saved
        # chain rule with the upstream scalar (1 for loss.backward())
        return grad * grad_out.to(grad.dtype), None, None, None, None


def objective(ctrl, evaluator: Evaluator, fixed, moving, recompute=False):
    """J(c) through :class:`ObjectiveFunction`."""
    return ObjectiveFunction.apply(ctrl, evaluator, fixed, moving, recompute)


class BsplineAdam(torch.optim.Optimizer):
    """Adam on B-spline control coefficients (voxel units, shape
    (d, nz, ny, nx)) in the paper's normalised coordinates, stepped by the
    library's Adam kernel. lr = 0.01 is the usage example's value."""

    def __init__(self, params, shape, spacing, lr=0.01, betas=(0.9, 0.999), eps=1e-8):
        super().__init__(params, dict(lr=lr, betas=betas, eps=eps))
        self.shape, self.spacing = tuple(shape), int(spacing)

    @torch.no_grad()
    def init_state(self):
        """Create the moments and the device step counter of every parameter
        now (zero), so that a CUDA-graph capture of step() contains no
        initialisation."""
        for group in self.param_groups:
            for p in group["params"]:
                st = self.state[p]
                if not st:
                    st["exp_avg"] = torch.zeros_like(p)
                    st["exp_avg_sq"] = torch.zeros_like(p)
                    st["step"] = torch.zeros(1, dtype=torch.int64, device=p.device)

    @torch.no_grad()
    def step(self, closure=None):
        loss = None
        if closure is not None:
            with torch.enable_grad():
                loss = closure()
        for group in self.param_groups:
            for p in group["params"]:
                if p.grad is None:
                    continue
                st = self.state[p]
                if not st:
                    self.init_state()
                airgb.al_adam_step(self.shape, self.spacing, p, p.grad.contiguous(),
                                   st["exp_avg"], st["exp_avg_sq"], st["step"], lr=group["lr"],
                                   betas=group["betas"], eps=group["eps"])
        return loss


class GraphedIteration:
    """One optimisation iteration -- J through :class:`ObjectiveFunction`,
    its backward and a :class:`BsplineAdam` step -- captured once in a CUDA
    graph and replayed, so each iteration costs one graph launch instead of
    the Python and autograd work of an eager iteration. `ctrl` is updated in
    place on every replay; ``self.J`` holds the J of the latest replay (taken
    before its step)."""

    def __init__(self, ctrl, evaluator: Evaluator, fixed, moving, optimizer: BsplineAdam,
                 recompute=False):
        optimizer.init_state()
        # one eager evaluation outside the capture (sets kernel attributes)
        evaluator.evaluate(fixed, moving, ctrl.detach(),
                           torch.empty(4, dtype=torch.float64, device=ctrl.device))
        self.graph = torch.cuda.CUDAGraph()
        optimizer.zero_grad(set_to_none=True)
        with torch.cuda.graph(self.graph, capture_error_mode="thread_local"):
            self.J = objective(ctrl, evaluator, fixed, moving, recompute)
            self.J.backward()
            optimizer.step()

    def __call__(self):
        self.graph.replay()
        return self.J


@dataclasses.dataclass
class Level:
    factor: int
    shape: tuple
    iterations: int
    values: torch.Tensor  # (iterations + 1, 4) float64: {J, S, R, n_mask} before each step
    ms: float             # device time of the level's iterations (CUDA events)


@dataclasses.dataclass
class Result:
    ctrl: torch.Tensor    # finest-level coefficients, voxel units
    levels: list
    seconds: float        # wall time of the whole registration, pyramid included


def _level_loop(ev: Evaluator, F, M, c, iterations, lr, betas, eps, values, final=True):
    """`iterations` Adam steps of the objective; values[i] receives J before
    step i (and, with final=True, values[iterations] the final J)."""
    m = torch.zeros_like(c)
    v = torch.zeros_like(c)
    step = torch.zeros(1, dtype=torch.int64, device=c.device)
    grad = torch.empty_like(c)

    def run():
        for i in range(iterations):
            ev.evaluate(F, M, c, values[i], grad)
            airgb.al_adam_step(ev.shape, ev.spacing, c, grad, m, v, step, lr=lr, betas=betas,
                               eps=eps)
        if final:
            ev.evaluate(F, M, c, values[iterations], None)

    return run


@dataclasses.dataclass
class Checkpoint:
    """State of a coarse-to-fine registration after `levels_done` levels: the
    coefficients of the last finished level (voxel units, on that level's
    grid) and what they belong to. Adam's moments restart at every level, so
    nothing else is needed to continue."""
    levels_done: int
    factors: tuple
    shape: tuple          # grid of the last finished level (z, y, x)
    spacing: int
    ctrl: np.ndarray      # float32 (d, nz, ny, nx)

    def save(self, path):
        tmp = f"{path}.{os.getpid()}.tmp.npz"
        np.savez(tmp, levels_done=self.levels_done, factors=np.asarray(self.factors),
                 shape=np.asarray(self.shape), spacing=self.spacing, ctrl=self.ctrl)
        os.replace(tmp, path)

    @staticmethod
    def load(path):
        with np.load(path) as z:
            return Checkpoint(int(z["levels_done"]), tuple(int(f) for f in z["factors"]),
                              tuple(int(n) for n in z["shape"]), int(z["spacing"]),
                              np.array(z["ctrl"], dtype=np.float32))


def register(fixed, moving, spacing=6, sim="lcc", lam=0.1, factors=(4, 2, 1), iterations=150,
             lr=0.01, betas=(0.9, 0.999), eps=1e-8, sim_eps=1e-5, window=7, ctrl=None,
             graph=True, diffeo_steps=None, checkpoint=None, resume=None, max_levels=None):
    """Coarse-to-fine B-spline registration of `moving` onto `fixed`.

    factors: pyramid factors from coarse to fine, each twice the next, ending
    at 1. iterations: Adam steps per level (an int or one per level). The
    coefficients start at zero on the coarsest level (or at `ctrl` for a
    single-level registration) and are refined exactly between levels. With
    graph=True each level's iterations are captured in one CUDA graph and
    replayed once; graph=False issues the same launches directly.
    diffeo_steps: None for the plain B-spline model, else the squarings of
    the diffeomorphic model (the coefficients then parametrise the velocity).
    checkpoint: path of an .npz file rewritten after every finished level.
    resume: a Checkpoint (or its path) of the same factors and spacing; the
    registration continues at the level after its last finished one, from
    its coefficients, and returns only the levels it ran.
    max_levels: stop after running this many levels in this call (the rest
    can follow later from the checkpoint).
    """
    factors = tuple(int(f) for f in factors)
    if factors[-1] != 1 or any(a != 2 * b for a, b in zip(factors, factors[1:])):
        raise ValueError("factors must halve from level to level and end at 1")
    if ctrl is not None and len(factors) != 1:
        raise ValueError("an initial ctrl is only taken by a single-level registration")
    iters = [int(iterations)] * len(factors) if isinstance(iterations, int) else \
        [int(i) for i in iterations]
    dev = fixed.device
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    levels, c = [], None
    prev_shape = None
    first = 0
    if resume is not None:
        ck = Checkpoint.load(resume) if isinstance(resume, (str, os.PathLike)) else resume
        if ck.factors != factors or ck.spacing != int(spacing):
            raise ValueError("the checkpoint belongs to other pyramid factors or spacing")
        first = ck.levels_done
        c = torch.from_numpy(ck.ctrl).to(dev)
        prev_shape = ck.shape
    for li, (f, n_it) in enumerate(zip(factors, iters)):
        if li < first:
            continue
        if max_levels is not None and len(levels) >= int(max_levels):
            break
        F = airgb.al_pyramid_level(fixed, f)
        M = airgb.al_pyramid_level(moving, f)
        shape = tuple(F.shape)
        ev = Evaluator(shape, spacing, sim, lam, sim_eps, window, device=dev,
                       diffeo_steps=diffeo_steps)
        if c is None:
            c = ctrl.clone() if ctrl is not None else torch.zeros(ev.lattice, dtype=torch.float32,
                                                                  device=dev)
        else:
            c = airgb.al_bspline_refine(prev_shape, shape, spacing, c)
        values = torch.empty((n_it + 1, 4), dtype=torch.float64, device=dev)
        run = _level_loop(ev, F, M, c, n_it, lr, betas, eps, values)
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if graph:
            # J at the start, eagerly (kernel attributes get set outside the
            # capture); the capture only records the launches, the replay runs
            # them
            ev.evaluate(F, M, c, values[0], None)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, capture_error_mode="thread_local"):
                run()
            start.record()
            g.replay()
            stop.record()
        else:
            start.record()
            run()
            stop.record()
        stop.synchronize()
        levels.append(Level(f, shape, n_it, values, start.elapsed_time(stop)))
        prev_shape = shape
        if checkpoint is not None:
            Checkpoint(li + 1, factors, shape, int(spacing), c.cpu().numpy()).save(checkpoint)
    torch.cuda.synchronize(dev)
    return Result(c, levels, time.perf_counter() - t0)


@dataclasses.dataclass
class BatchResult:
    batch: airgb.Batch    # ctrl[i]: final coefficients; values[i]: J history
    device_ms: float      # the iterations' device time (CUDA events)
    policy: int           # work-item order in use
    tuning_ms: list       # ms per iteration of each (tile, order) (empty if not tuned)
    tile: int = 0         # brick tile in use
    tile_cells: tuple = ()  # control cells per block in x and y of that tile


def register_batch(pairs, spacing=8, lam=0.1, iterations=100, lr=0.01, betas=(0.9, 0.999),
                   eps=1e-8, graph=True, tune=True):
    """Single-level MSE registration of many (fixed, moving) pairs at once:
    every iteration of every pair is one launch of the persistent batch
    kernel; with graph=True all iterations are captured in one CUDA graph and
    replayed once. values[i][k] holds {J, S, R, n_mask} before step k + 1."""
    b = airgb.Batch(pairs, spacing, lam, history=iterations)
    tile, policy, tms = b.tile, b.policy, []
    if tune:
        tile, policy, tms = b.tune(3, lr, betas, eps)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if graph:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            for k in range(iterations):
                b.step(k + 1, k, lr, betas, eps)
        start.record()
        g.replay()
        stop.record()
    else:
        start.record()
        for k in range(iterations):
            b.step(k + 1, k, lr, betas, eps)
        stop.record()
    stop.synchronize()
    st = b.status()
    if st != 0:
        raise airgb.AirgbError("al_batch_status", st)
    return BatchResult(b, start.elapsed_time(stop), policy, tms, tile, b.tiles()[tile])


def register_sequential(pairs, spacing=8, lam=0.1, iterations=100, lr=0.01, betas=(0.9, 0.999),
                        eps=1e-8):
    """The same registrations one pair after another with the single-problem
    calls (al_objective_grad + al_adam_step per iteration, plain launches).
    Returns (coefficients, value histories, device ms)."""
    ctrls, hists = [], []
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    runs = []
    for F, M in pairs:
        ev = Evaluator(tuple(F.shape), spacing, "mse", lam, device=F.device)
        c = torch.zeros(ev.lattice, dtype=torch.float32, device=F.device)
        vals = torch.empty((iterations + 1, 4), dtype=torch.float64, device=F.device)
        runs.append((_level_loop(ev, F, M, c, iterations, lr, betas, eps, vals, final=False), c,
                     vals))
    start.record()
    for run, _, _ in runs:
        run()
    stop.record()
    stop.synchronize()
    return [c for _, c, _ in runs], [v for _, _, v in runs], start.elapsed_time(stop)

