"""ctypes binding of libairgb.so (include/airgb.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library. PyTorch supplies device memory (tensors) and the
current CUDA stream. The library must have been built (``build()`` in
``__graft_entry__`` or ``python -m paper_1806_09907_gb300.build``); loading
fails loudly otherwise, and every call raises ``AirgbError`` on a non-zero
status.

Layouts (see the header): volumes are float32 tensors shaped (Z, Y, X) or
(Y, X); vector fields and control coefficients are (d, Z, Y, X) /
(d, nz, ny, nx) with component 0 = x.
"""
from __future__ import annotations

import ctypes
import functools
import threading
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# AIRGB_CHECKED=1 loads the bounds-checked build (libairgb_check.so) instead
LIB_PATH = os.path.join(_HERE, "libairgb_check.so" if os.environ.get("AIRGB_CHECKED") == "1"
                        else "libairgb.so")

AL_SIM_MSE, AL_SIM_NCC, AL_SIM_LCC = 0, 1, 2
SIM_KINDS = {"mse": AL_SIM_MSE, "ncc": AL_SIM_NCC, "lcc": AL_SIM_LCC}

# Entry points declared in include/airgb.h.
EXPORTS = (
    "al_status_string", "al_bspline_init", "al_displacement", "al_displacement_adjoint",
    "al_displacement_adjoint_workspace_bytes", "al_warp", "al_warp_adjoint", "al_similarity",
    "al_similarity_workspace_bytes", "al_regulariser", "al_regulariser_workspace_bytes",
    "al_objective_grad", "al_objective_workspace_bytes", "al_objective_warped_offsets",
    "al_objective_grad_unfused",
    "al_objective_unfused_workspace_bytes", "al_get_device_error", "al_profile_enable",
    "al_profile_collect", "al_profile_reset", "al_similarity_noalloc", "al_noalloc_scratch_bytes",
    "al_adam_step", "al_pyramid_grid", "al_pyramid_level", "al_pyramid_workspace_bytes",
    "al_bspline_refine", "al_batch_create", "al_batch_destroy", "al_batch_workspace_bytes", "al_batch_set_tile",
    "al_batch_tiles",
    "al_batch_items", "al_batch_bind", "al_batch_step", "al_batch_tune", "al_batch_set_policy",
    "al_batch_set_wait", "al_batch_status", "al_exp_field", "al_exp_field_workspace_bytes",
    "al_exp_field_adjoint", "al_exp_field_adjoint_workspace_bytes", "al_objective_grad_diffeo",
    "al_objective_diffeo_workspace_bytes", "al_conv3d_output_size", "al_conv3d_packed_bytes",
    "al_conv3d_pack", "al_conv3d_forward", "al_conv3d_forward_workspace_bytes",
    "al_conv3d_backward_data",
    "al_conv3d_backward_weight_workspace_bytes", "al_conv3d_backward_weight", "al_initnet_input",
    "al_initnet_upcat", "al_initnet_upcat_adjoint", "al_initnet_head_to_ctrl",
    "al_initnet_head_adjoint", "al_field_loss_workspace_bytes", "al_field_loss", "al_adam_flat",
    "al_adam_flat_pack", "al_initnet_pair_input",
    "al_render_blobs", "al_lcc_set_wait", "al_fused_set_wait", "al_warp_ctrl",
)


class AirgbError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__(f"{fn} failed: status {status} ({status_string(status)})")


class al_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("size", ctypes.c_int64 * 3)]


class al_bspline(ctypes.Structure):
    _fields_ = [("grid", al_grid), ("spacing", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n", ctypes.c_int64 * 3)]


class al_sim_params(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("lcc_window", ctypes.c_int32),
                ("eps", ctypes.c_double)]


class al_problem(ctypes.Structure):
    _fields_ = [("bs", al_bspline), ("sim", al_sim_params), ("lam", ctypes.c_double)]


class al_conv3d(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("cin", ctypes.c_int32), ("cout", ctypes.c_int32),
                ("stride", ctypes.c_int32), ("size", ctypes.c_int64 * 3)]


class al_adam_params(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double)]


_lib = None


def load():
    """Load libairgb.so (once). Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libairgb.so not found at {LIB_PATH}: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, SZ, VP = ctypes.POINTER, ctypes.c_int32, ctypes.c_size_t, ctypes.c_void_p
    D = ctypes.c_double
    sig = {
        "al_status_string": ([I32], ctypes.c_char_p),
        "al_bspline_init": ([P(al_bspline), P(al_grid), I32], I32),
        "al_displacement": ([P(al_bspline), VP, VP, VP], I32),
        "al_warp_ctrl": ([P(al_bspline), I32, VP, VP, VP, VP, VP], I32),
        "al_initnet_pair_input": ([P(al_bspline), I32, VP, VP, VP, VP], I32),
        "al_displacement_adjoint": ([P(al_bspline), VP, VP, VP, SZ, VP], I32),
        "al_displacement_adjoint_workspace_bytes": ([P(al_bspline)], SZ),
        "al_warp": ([P(al_grid), VP, VP, VP, VP, VP], I32),
        "al_warp_adjoint": ([P(al_grid), VP, VP, VP, VP, VP, I32, VP], I32),
        "al_similarity": ([P(al_grid), P(al_sim_params), VP, VP, VP, VP, VP, VP, SZ, VP], I32),
        "al_similarity_workspace_bytes": ([P(al_grid), P(al_sim_params)], SZ),
        "al_regulariser": ([P(al_grid), VP, D, VP, VP, VP, SZ, VP], I32),
        "al_regulariser_workspace_bytes": ([P(al_grid)], SZ),
        "al_objective_grad": ([P(al_problem), VP, VP, VP, VP, VP, VP, SZ, VP], I32),
        "al_objective_workspace_bytes": ([P(al_problem)], SZ),
        "al_objective_warped_offsets": ([P(al_problem), P(SZ), P(SZ)], I32),
        "al_objective_grad_unfused": ([P(al_problem), VP, VP, VP, VP, VP, VP, SZ, VP], I32),
        "al_objective_unfused_workspace_bytes": ([P(al_problem)], SZ),
        "al_get_device_error": ([VP], I32),
        "al_lcc_set_wait": ([I32], I32),
        "al_fused_set_wait": ([I32], I32),
        "al_profile_enable": ([I32], I32),
        "al_profile_collect": ([ctypes.c_char_p, SZ, P(D), P(ctypes.c_int64), I32], I32),
        "al_profile_reset": ([], I32),
        "al_similarity_noalloc": ([P(al_grid), P(al_sim_params), VP, VP, VP, VP, VP, VP], I32),
        "al_noalloc_scratch_bytes": ([], SZ),
        "al_adam_step": ([P(al_bspline), P(al_adam_params), VP, VP, VP, VP, VP, VP], I32),
        "al_pyramid_grid": ([P(al_grid), I32, P(al_grid)], I32),
        "al_pyramid_level": ([P(al_grid), VP, I32, VP, VP, SZ, VP], I32),
        "al_pyramid_workspace_bytes": ([P(al_grid), I32], SZ),
        "al_bspline_refine": ([P(al_bspline), VP, P(al_bspline), VP, VP], I32),
        "al_batch_create": ([P(al_problem), I32, P(VP)], I32),
        "al_batch_destroy": ([VP], None),
        "al_batch_workspace_bytes": ([VP], SZ),
        "al_batch_items": ([VP, P(I32)], I32),
        "al_batch_bind": ([VP, P(VP), P(VP), P(VP), P(VP), P(VP), P(VP), VP, SZ], I32),
        "al_batch_step": ([VP, P(al_adam_params), ctypes.c_int64, I32, VP], I32),
        "al_batch_tune": ([VP, P(al_adam_params), I32, P(D), P(I32), P(I32), VP], I32),
        "al_batch_set_policy": ([VP, I32], I32),
        "al_batch_set_tile": ([VP, I32], I32),
        "al_batch_tiles": ([VP, P(I32)], I32),
        "al_batch_set_wait": ([VP, I32, ctypes.c_int64], I32),
        "al_batch_status": ([VP, VP], I32),
        "al_exp_field": ([P(al_grid), I32, VP, VP, VP, VP, SZ, VP], I32),
        "al_exp_field_workspace_bytes": ([P(al_grid)], SZ),
        "al_exp_field_adjoint": ([P(al_grid), I32, VP, VP, VP, VP, SZ, VP], I32),
        "al_exp_field_adjoint_workspace_bytes": ([P(al_grid)], SZ),
        "al_objective_grad_diffeo": ([P(al_problem), I32, VP, VP, VP, VP, VP, VP, SZ, VP], I32),
        "al_objective_diffeo_workspace_bytes": ([P(al_problem), I32], SZ),
        "al_conv3d_output_size": ([P(al_conv3d), P(ctypes.c_int64)], I32),
        "al_conv3d_packed_bytes": ([P(al_conv3d), I32], SZ),
        "al_conv3d_pack": ([P(al_conv3d), VP, VP, VP, VP], I32),
        "al_conv3d_forward": ([P(al_conv3d), VP, VP, VP, I32, I32, VP, VP, SZ, VP], I32),
        "al_conv3d_forward_workspace_bytes": ([P(al_conv3d)], SZ),
        "al_conv3d_backward_data": ([P(al_conv3d), VP, VP, VP, VP, I32, I32, VP, VP], I32),
        "al_conv3d_backward_weight_workspace_bytes": ([P(al_conv3d)], SZ),
        "al_conv3d_backward_weight": ([P(al_conv3d), VP, VP, VP, VP, VP, SZ, VP], I32),
        "al_initnet_input": ([I32, P(ctypes.c_int64), VP, VP, VP, VP], I32),
        "al_initnet_upcat": ([I32, P(ctypes.c_int64), I32, I32, VP, VP, VP, VP], I32),
        "al_initnet_upcat_adjoint": ([I32, P(ctypes.c_int64), I32, I32, VP, VP, VP, VP], I32),
        "al_initnet_head_to_ctrl": ([P(al_bspline), I32, P(ctypes.c_int64), I32, VP, VP, VP],
                                    I32),
        "al_initnet_head_adjoint": ([P(al_bspline), I32, P(ctypes.c_int64), I32, VP, VP, VP],
                                    I32),
        "al_field_loss_workspace_bytes": ([I32], SZ),
        "al_field_loss": ([P(al_bspline), I32, VP, VP, VP, VP, VP, SZ, VP], I32),
        "al_adam_flat": ([P(al_adam_params), ctypes.c_int64, VP, VP, VP, VP, VP, VP], I32),
        "al_adam_flat_pack": ([P(al_adam_params), ctypes.c_int64, VP, VP, VP, VP, VP, I32,
                               P(al_conv3d), P(ctypes.c_int64), P(VP), P(VP), VP], I32),
        "al_render_blobs": ([P(ctypes.c_int64), I32, I32, VP, VP, VP], I32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().al_status_string(int(status)).decode()


# The device of the tensors of the call being marshalled: set by _ptr, read
# by _stream (the default stream is that device's current stream) and by
# _call, which runs the C call with that device current.
_tls = threading.local()


def _call(name, *args):
    dev = getattr(_tls, "dev", None)
    _tls.dev = None
    fn = getattr(load(), name)
    if dev is not None:
        with torch.cuda.device(dev):
            st = fn(*args)
    else:
        st = fn(*args)
    if st != 0:
        raise AirgbError(name, st)


# ---------------------------------------------------------------- helpers --

def make_grid(shape) -> al_grid:
    g = al_grid()
    if len(shape) == 3:
        g.ndim, g.size[0], g.size[1], g.size[2] = 3, shape[2], shape[1], shape[0]
    elif len(shape) == 2:
        g.ndim, g.size[0], g.size[1], g.size[2] = 2, shape[1], shape[0], 1
    else:
        raise ValueError(f"volume shape must be (Z,Y,X) or (Y,X), got {tuple(shape)}")
    return g


def bspline_init(shape, spacing: int) -> al_bspline:
    bs = al_bspline()
    _call("al_bspline_init", ctypes.byref(bs), ctypes.byref(make_grid(shape)), int(spacing))
    return bs


def lattice_shape(shape, spacing: int):
    """Control-lattice shape in volume order: (nz, ny, nx) or (ny, nx)."""
    bs = bspline_init(shape, spacing)
    return (bs.n[2], bs.n[1], bs.n[0]) if len(shape) == 3 else (bs.n[1], bs.n[0])


def make_problem(shape, spacing: int, sim: str = "mse", lam: float = 0.1, eps: float = 1e-5,
                 window: int = 7) -> al_problem:
    pr = al_problem()
    pr.bs = bspline_init(shape, spacing)
    pr.sim.kind = SIM_KINDS[sim] if isinstance(sim, str) else int(sim)
    pr.sim.lcc_window = int(window)
    pr.sim.eps = float(eps)
    pr.lam = float(lam)
    return pr


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensors must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    dev = getattr(_tls, "dev", None)
    if dev is None:
        _tls.dev = t.device
    elif dev != t.device:
        _tls.dev = None
        raise ValueError(f"the tensors of one call must share a device ({dev} and {t.device})")
    return ctypes.c_void_p(t.data_ptr())


def _f32(t, shape, what):
    if t.dtype != torch.float32 or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what}: expected float32 {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")
    return _ptr(t)


def _stream(stream=None):
    if stream is None:
        dev = getattr(_tls, "dev", None)
        stream = torch.cuda.current_stream(dev) if dev is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _workspace(nbytes, device, ws=None):
    if ws is not None:
        if ws.numel() * ws.element_size() < nbytes:
            raise ValueError("workspace too small")
        return ws
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _ndim_of(shape):
    return len(shape)


# ------------------------------------------------------------ entry points --

def al_displacement(shape, spacing, ctrl, disp=None, stream=None):
    """A1: B-spline expansion u = sum_j c_j k(x_j, x)."""
    bs = bspline_init(shape, spacing)
    d = _ndim_of(shape)
    _f32(ctrl, (d,) + lattice_shape(shape, spacing), "ctrl")
    if disp is None:
        disp = torch.empty((d,) + tuple(shape), dtype=torch.float32, device=ctrl.device)
    _f32(disp, (d,) + tuple(shape), "disp")
    _call("al_displacement", ctypes.byref(bs), _ptr(ctrl), _ptr(disp), _stream(stream))
    return disp


def al_warp_ctrl(shape, spacing, moving, ctrl, warped=None, mask=None, stream=None):
    """A1 + A2 for a batch: warped[v] = moving[v] o (x + B ctrl[v]) without
    materialising the field. moving: (count, *shape), ctrl: (count, ndim,
    *lattice); mask (optional, uint8, (count, *shape)) receives the mask."""
    bs = bspline_init(shape, spacing)
    d = _ndim_of(shape)
    count = int(moving.shape[0])
    _f32(moving, (count,) + tuple(shape), "moving")
    _f32(ctrl, (count, d) + lattice_shape(shape, spacing), "ctrl")
    if warped is None:
        warped = torch.empty_like(moving)
    _f32(warped, (count,) + tuple(shape), "warped")
    if mask is not None and (mask.dtype != torch.uint8 or tuple(mask.shape) != (count,) + tuple(shape)
                             or not mask.is_contiguous()):
        raise ValueError(f"mask: expected uint8 {(count,) + tuple(shape)}")
    _call("al_warp_ctrl", ctypes.byref(bs), count, _ptr(moving), _ptr(ctrl), _ptr(warped),
          _ptr(mask), _stream(stream))
    return warped


def al_displacement_adjoint(shape, spacing, grad_disp, grad_ctrl=None, workspace=None,
                            stream=None):
    """A6: transpose of the expansion, g_c = B^T g_u."""
    bs = bspline_init(shape, spacing)
    d = _ndim_of(shape)
    _f32(grad_disp, (d,) + tuple(shape), "grad_disp")
    if grad_ctrl is None:
        grad_ctrl = torch.empty((d,) + lattice_shape(shape, spacing), dtype=torch.float32,
                                device=grad_disp.device)
    nb = load().al_displacement_adjoint_workspace_bytes(ctypes.byref(bs))
    ws = _workspace(nb, grad_disp.device, workspace)
    _call("al_displacement_adjoint", ctypes.byref(bs), _ptr(grad_disp), _ptr(grad_ctrl),
          _ptr(ws), ctypes.c_size_t(ws.numel()), _stream(stream))
    return grad_ctrl


def al_warp(moving, disp, warped=None, mask=None, stream=None):
    """A2: backward warp with mask. Returns (warped, mask uint8)."""
    shape = tuple(moving.shape)
    g = make_grid(shape)
    _f32(moving, shape, "moving")
    _f32(disp, (len(shape),) + shape, "disp")
    if warped is None:
        warped = torch.empty(shape, dtype=torch.float32, device=moving.device)
    if mask is None:
        mask = torch.empty(shape, dtype=torch.uint8, device=moving.device)
    _call("al_warp", ctypes.byref(g), _ptr(moving), _ptr(disp), _ptr(warped), _ptr(mask),
          _stream(stream))
    return warped, mask


def al_warp_adjoint(moving, disp, mask, grad_warped, grad_disp=None, accumulate=False,
                    stream=None):
    """A5: grad_disp = mask * grad_warped * dM~/dy (optionally accumulated)."""
    shape = tuple(moving.shape)
    g = make_grid(shape)
    if grad_disp is None:
        if accumulate:
            raise ValueError("accumulate needs grad_disp")
        grad_disp = torch.empty((len(shape),) + shape, dtype=torch.float32, device=moving.device)
    _call("al_warp_adjoint", ctypes.byref(g), _ptr(moving), _ptr(disp), _ptr(mask),
          _ptr(grad_warped), _ptr(grad_disp), int(bool(accumulate)), _stream(stream))
    return grad_disp


def al_similarity(sim, fixed, warped, mask, eps=1e-5, window=7, grad=True, workspace=None,
                  stream=None):
    """A3: similarity value {S, n_mask} (float64 device tensor) and dS/dW."""
    shape = tuple(fixed.shape)
    g = make_grid(shape)
    p = al_sim_params()
    p.kind = SIM_KINDS[sim] if isinstance(sim, str) else int(sim)
    p.lcc_window = int(window)
    p.eps = float(eps)
    value = torch.empty(2, dtype=torch.float64, device=fixed.device)
    gw = torch.empty(shape, dtype=torch.float32, device=fixed.device) if grad else None
    nb = load().al_similarity_workspace_bytes(ctypes.byref(g), ctypes.byref(p))
    if nb == 0:
        raise AirgbError("al_similarity_workspace_bytes", 1)
    ws = _workspace(nb, fixed.device, workspace)
    _call("al_similarity", ctypes.byref(g), ctypes.byref(p), _ptr(fixed), _ptr(warped),
          _ptr(mask), _ptr(value), _ptr(gw), _ptr(ws), ctypes.c_size_t(ws.numel()),
          _stream(stream))
    return value, gw


def al_similarity_noalloc(sim, fixed, warped, mask, eps=1e-5, window=7, grad=True, stream=None):
    """A3 without a workspace: the library's built-in scratch array is used
    (for callers that cannot allocate device memory; see the header)."""
    shape = tuple(fixed.shape)
    g = make_grid(shape)
    p = al_sim_params()
    p.kind = SIM_KINDS[sim] if isinstance(sim, str) else int(sim)
    p.lcc_window = int(window)
    p.eps = float(eps)
    value = torch.empty(2, dtype=torch.float64, device=fixed.device)
    gw = torch.empty(shape, dtype=torch.float32, device=fixed.device) if grad else None
    _call("al_similarity_noalloc", ctypes.byref(g), ctypes.byref(p), _ptr(fixed), _ptr(warped),
          _ptr(mask), _ptr(value), _ptr(gw), _stream(stream))
    return value, gw


def al_regulariser(disp, weight=1.0, grad=True, workspace=None, stream=None):
    """A4: R_diff (float64 device tensor of 1) and weight * dR/du."""
    shape = tuple(disp.shape[1:])
    g = make_grid(shape)
    value = torch.empty(1, dtype=torch.float64, device=disp.device)
    gu = torch.empty_like(disp) if grad else None
    nb = load().al_regulariser_workspace_bytes(ctypes.byref(g))
    ws = _workspace(nb, disp.device, workspace)
    _call("al_regulariser", ctypes.byref(g), _ptr(disp), ctypes.c_double(weight), _ptr(value),
          _ptr(gu), _ptr(ws), ctypes.c_size_t(ws.numel()), _stream(stream))
    return value, gu


def objective_workspace_bytes(problem: al_problem, fused=True) -> int:
    fn = "al_objective_workspace_bytes" if fused else "al_objective_unfused_workspace_bytes"
    n = getattr(load(), fn)(ctypes.byref(problem))
    if n == 0:
        raise AirgbError(fn, 1)
    return int(n)


def objective_warped_offsets(problem: al_problem):
    """Byte offsets (W, mask) of the warped image a fused LCC evaluation
    keeps in its workspace (al_objective_warped_offsets)."""
    w, m = ctypes.c_size_t(), ctypes.c_size_t()
    _call("al_objective_warped_offsets", ctypes.byref(problem), ctypes.byref(w), ctypes.byref(m))
    return int(w.value), int(m.value)


def al_objective_grad(problem: al_problem, fixed, moving, ctrl, value=None, grad_ctrl=None,
                      workspace=None, want_grad=True, fused=True, stream=None):
    """A7: value {J, S, R, n_mask} (float64 device tensor) and dJ/dc."""
    shape = tuple(fixed.shape)
    d = len(shape)
    _f32(fixed, shape, "fixed")
    _f32(moving, shape, "moving")
    lat = (problem.bs.n[2], problem.bs.n[1], problem.bs.n[0]) if d == 3 else \
        (problem.bs.n[1], problem.bs.n[0])
    _f32(ctrl, (d,) + lat, "ctrl")
    if value is None:
        value = torch.empty(4, dtype=torch.float64, device=fixed.device)
    if want_grad and grad_ctrl is None:
        grad_ctrl = torch.empty_like(ctrl)
    ws = _workspace(objective_workspace_bytes(problem, fused), fixed.device, workspace)
    fn = "al_objective_grad" if fused else "al_objective_grad_unfused"
    _call(fn, ctypes.byref(problem), _ptr(fixed), _ptr(moving), _ptr(ctrl), _ptr(value),
          _ptr(grad_ctrl if want_grad else None), _ptr(ws), ctypes.c_size_t(ws.numel()),
          _stream(stream))
    return value, (grad_ctrl if want_grad else None)


def al_adam_step(shape, spacing, ctrl, grad_ctrl, m, v, step, lr=0.01, betas=(0.9, 0.999),
                 eps=1e-8, stream=None):
    """One Adam step on the control points in normalised units, in place on
    ctrl, m, v; step is a 1-element int64 device tensor (steps taken so far),
    advanced by the call."""
    bs = bspline_init(shape, spacing)
    want = (len(shape),) + lattice_shape(shape, spacing)
    for t, name in ((ctrl, "ctrl"), (grad_ctrl, "grad_ctrl"), (m, "m"), (v, "v")):
        _f32(t, want, name)
    if step.dtype != torch.int64 or step.numel() != 1:
        raise ValueError("step: expected a 1-element int64 tensor")
    p = al_adam_params(float(lr), float(betas[0]), float(betas[1]), float(eps))
    _call("al_adam_step", ctypes.byref(bs), ctypes.byref(p), _ptr(ctrl), _ptr(grad_ctrl), _ptr(m),
          _ptr(v), _ptr(step), _stream(stream))


def pyramid_shape(shape, factor: int):
    """Shape of a pyramid level (every factor-th voxel from voxel 0)."""
    g = make_grid(shape)
    out = al_grid()
    _call("al_pyramid_grid", ctypes.byref(g), int(factor), ctypes.byref(out))
    return (out.size[2], out.size[1], out.size[0]) if len(shape) == 3 else \
        (out.size[1], out.size[0])


def al_pyramid_level(image, factor: int, level=None, workspace=None, stream=None):
    """One Gaussian pyramid level of `image` (sigma = factor/2, subsampled by
    factor)."""
    shape = tuple(image.shape)
    g = make_grid(shape)
    _f32(image, shape, "image")
    out_shape = pyramid_shape(shape, factor)
    if level is None:
        level = torch.empty(out_shape, dtype=torch.float32, device=image.device)
    _f32(level, out_shape, "level")
    nb = load().al_pyramid_workspace_bytes(ctypes.byref(g), int(factor))
    ws = _workspace(nb, image.device, workspace) if nb > 0 else None
    _call("al_pyramid_level", ctypes.byref(g), _ptr(image), int(factor), _ptr(level), _ptr(ws),
          ctypes.c_size_t(ws.numel() if ws is not None else 0), _stream(stream))
    return level


def al_bspline_refine(coarse_shape, fine_shape, spacing, ctrl_coarse, ctrl_fine=None,
                      stream=None):
    """Coefficients on the finer level with the same displacement (fine voxel
    units); coarse_shape must be pyramid_shape(fine_shape, 2)."""
    bc, bf = bspline_init(coarse_shape, spacing), bspline_init(fine_shape, spacing)
    d = len(fine_shape)
    _f32(ctrl_coarse, (d,) + lattice_shape(coarse_shape, spacing), "ctrl_coarse")
    if ctrl_fine is None:
        ctrl_fine = torch.empty((d,) + lattice_shape(fine_shape, spacing), dtype=torch.float32,
                                device=ctrl_coarse.device)
    _f32(ctrl_fine, (d,) + lattice_shape(fine_shape, spacing), "ctrl_fine")
    _call("al_bspline_refine", ctypes.byref(bc), _ptr(ctrl_coarse), ctypes.byref(bf),
          _ptr(ctrl_fine), _stream(stream))
    return ctrl_fine


def al_exp_field(velocity, steps=6, trajectory=False, stream=None):
    """f = exp(v) by scaling and squaring: the displacement u (d, *shape);
    with trajectory=True also u_0 .. u_{K-1} (K, d, *shape) for the adjoint."""
    shape = tuple(velocity.shape[1:])
    g = make_grid(shape)
    _f32(velocity, (len(shape),) + shape, "velocity")
    u = torch.empty_like(velocity)
    traj = (torch.empty((max(int(steps), 1),) + tuple(velocity.shape), dtype=torch.float32,
                        device=velocity.device) if trajectory else None)
    ws = None
    if not trajectory and steps > 0:
        ws = _workspace(load().al_exp_field_workspace_bytes(ctypes.byref(g)), velocity.device)
    _call("al_exp_field", ctypes.byref(g), int(steps), _ptr(velocity), _ptr(u), _ptr(traj),
          _ptr(ws), ctypes.c_size_t(ws.numel() if ws is not None else 0), _stream(stream))
    return (u, traj[:int(steps)]) if trajectory else u


def al_exp_field_adjoint(trajectory, grad_disp, steps=6, stream=None):
    """(d u_K / d v)^T grad_disp from the trajectory of al_exp_field."""
    shape = tuple(grad_disp.shape[1:])
    g = make_grid(shape)
    gv = torch.empty_like(grad_disp)
    ws = _workspace(load().al_exp_field_adjoint_workspace_bytes(ctypes.byref(g)), grad_disp.device)
    traj = trajectory.contiguous() if steps > 0 else None
    _call("al_exp_field_adjoint", ctypes.byref(g), int(steps), _ptr(traj), _ptr(grad_disp),
          _ptr(gv), _ptr(ws), ctypes.c_size_t(ws.numel()), _stream(stream))
    return gv


def objective_diffeo_workspace_bytes(problem: al_problem, steps: int) -> int:
    n = load().al_objective_diffeo_workspace_bytes(ctypes.byref(problem), int(steps))
    if n == 0:
        raise AirgbError("al_objective_diffeo_workspace_bytes", 1)
    return int(n)


def al_objective_grad_diffeo(problem: al_problem, fixed, moving, ctrl, steps=6, value=None,
                             grad_ctrl=None, workspace=None, want_grad=True, stream=None):
    """J and dJ/dc of the diffeomorphic B-spline model (f = exp(v))."""
    shape = tuple(fixed.shape)
    d = len(shape)
    _f32(fixed, shape, "fixed")
    _f32(moving, shape, "moving")
    lat = (problem.bs.n[2], problem.bs.n[1], problem.bs.n[0]) if d == 3 else \
        (problem.bs.n[1], problem.bs.n[0])
    _f32(ctrl, (d,) + lat, "ctrl")
    if value is None:
        value = torch.empty(4, dtype=torch.float64, device=fixed.device)
    if want_grad and grad_ctrl is None:
        grad_ctrl = torch.empty_like(ctrl)
    ws = _workspace(objective_diffeo_workspace_bytes(problem, steps), fixed.device, workspace)
    _call("al_objective_grad_diffeo", ctypes.byref(problem), int(steps), _ptr(fixed),
          _ptr(moving), _ptr(ctrl), _ptr(value), _ptr(grad_ctrl if want_grad else None), _ptr(ws),
          ctypes.c_size_t(ws.numel()), _stream(stream))
    return value, (grad_ctrl if want_grad else None)


class Batch:
    """Independent MSE problems (2D and 3D, one spacing) optimised together:
    each iteration of every problem is one launch of the library's
    persistent batch kernel. pairs: list of (fixed, moving) float32 CUDA
    tensors. Holds the coefficients (``ctrl[i]``, voxel units, start at
    zero), the Adam moments and, with history > 0, a (history, 4) float64
    value history per problem."""

    def __init__(self, pairs, spacing=8, lam=0.1, history=0, device=None):
        load()
        self.pairs = [(f, m) for f, m in pairs]
        n = len(self.pairs)
        dev = device or self.pairs[0][0].device
        self.shapes = [tuple(f.shape) for f, _ in self.pairs]
        self.spacing = int(spacing)
        probs = (al_problem * n)(*[make_problem(sh, spacing, "mse", lam) for sh in self.shapes])
        self._problems = probs
        h = ctypes.c_void_p()
        _call("al_batch_create", probs, n, ctypes.byref(h))
        self._h = h
        for (f, m), sh in zip(self.pairs, self.shapes):
            _f32(f, sh, "fixed")
            _f32(m, sh, "moving")
        self.lattices = [(len(sh),) + lattice_shape(sh, spacing) for sh in self.shapes]
        z = lambda ls: torch.zeros(ls, dtype=torch.float32, device=dev)
        self.ctrl = [z(ls) for ls in self.lattices]
        self.m = [z(ls) for ls in self.lattices]
        self.v = [z(ls) for ls in self.lattices]
        self.values = [torch.zeros((history, 4), dtype=torch.float64, device=dev)
                       for _ in range(n)] if history > 0 else None
        self.policy = 1  # the library's default order: largest problem first
        self.tile = 0    # the single-problem path's brick
        self.workspace = torch.empty(max(int(load().al_batch_workspace_bytes(h)), 256),
                                     dtype=torch.uint8, device=dev)
        arr = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
        self._ptrs = [arr([f for f, _ in self.pairs]), arr([m for _, m in self.pairs]),
                      arr(self.ctrl), arr(self.m), arr(self.v),
                      arr(self.values) if self.values is not None else None]
        _call("al_batch_bind", h, *self._ptrs, ctypes.c_void_p(self.workspace.data_ptr()),
              ctypes.c_size_t(self.workspace.numel()))

    def items(self):
        per = (ctypes.c_int32 * 3)()
        total = load().al_batch_items(self._h, per)
        return total, tuple(per)

    @staticmethod
    def _adam(lr, betas, eps):
        return al_adam_params(float(lr), float(betas[0]), float(betas[1]), float(eps))

    def step(self, t, record=-1, lr=0.01, betas=(0.9, 0.999), eps=1e-8, stream=None):
        """Adam iteration t (1-based) of every problem, one kernel launch."""
        p = self._adam(lr, betas, eps)
        _call("al_batch_step", self._h, ctypes.byref(p), int(t), int(record), _stream(stream))

    def tiles(self):
        """The brick tiles of the batch kernel: (cells in x, cells in y) each."""
        n = load().al_batch_tiles(self._h, None)
        cells = (ctypes.c_int32 * (2 * n))()
        load().al_batch_tiles(self._h, cells)
        return [(cells[2 * t], cells[2 * t + 1]) for t in range(n)]

    def tune(self, iterations=3, lr=0.01, betas=(0.9, 0.999), eps=1e-8, stream=None):
        """Time every (brick tile, work-item order) configuration and keep
        the fastest; returns (tile, order, ms per iteration as a
        tiles x orders list of lists)."""
        p = self._adam(lr, betas, eps)
        nt = len(self.tiles())
        ms = (ctypes.c_double * (4 * nt))()
        tile, policy = ctypes.c_int32(), ctypes.c_int32()
        _call("al_batch_tune", self._h, ctypes.byref(p), int(iterations), ms, ctypes.byref(tile),
              ctypes.byref(policy), _stream(stream))
        self.tile, self.policy = int(tile.value), int(policy.value)
        return self.tile, self.policy, [list(ms[4 * t:4 * t + 4]) for t in range(nt)]

    def set_policy(self, policy):
        _call("al_batch_set_policy", self._h, int(policy))
        self.policy = int(policy)

    def set_tile(self, tile):
        _call("al_batch_set_tile", self._h, int(tile))
        self.tile = int(tile)

    def set_wait(self, extra_items=0, max_polls=20000000):
        _call("al_batch_set_wait", self._h, int(extra_items), int(max_polls))

    def status(self, stream=None) -> int:
        return int(load().al_batch_status(self._h, _stream(stream)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.al_batch_destroy(h)
            self._h = None


def al_get_device_error(stream=None) -> int:
    return int(load().al_get_device_error(_stream(stream)))


def al_lcc_set_wait(drop_slice=-1) -> None:
    """Test hook: the TMA-staged LCC gradient skips the load of this slice of
    every block, so its bounded wait runs out (AL_ERR_TIMEOUT); -1 restores."""
    _call("al_lcc_set_wait", int(drop_slice))


def al_fused_set_wait(drop_batch=-1) -> None:
    """Test hook: the TMA-staged 3D brick kernels skip this copy batch of every
    brick, so its bounded wait runs out (AL_ERR_TIMEOUT); -1 restores."""
    _call("al_fused_set_wait", int(drop_batch))


def profile_enable(on: bool = True):
    _call("al_profile_enable", int(bool(on)))


def profile_reset():
    _call("al_profile_reset")


def profile_collect(max_kernels: int = 64):
    """Per-kernel totals since the last reset: {name: (total_ms, launches)}."""
    buf = ctypes.create_string_buffer(8192)
    ms = (ctypes.c_double * max_kernels)()
    cnt = (ctypes.c_int64 * max_kernels)()
    n = load().al_profile_collect(buf, ctypes.c_size_t(8192), ms, cnt, max_kernels)
    names = buf.value.decode().split("\n")[:min(n, max_kernels)]
    return {names[i]: (ms[i], int(cnt[i])) for i in range(len(names))}


class Objective:
    """Preallocated evaluator of J and dJ/dc for one problem: holds the
    workspace and output buffers so repeated calls allocate nothing."""

    def __init__(self, shape, spacing, sim="mse", lam=0.1, eps=1e-5, window=7, device="cuda",
                 fused=True):
        self.shape = tuple(shape)
        self.problem = make_problem(shape, spacing, sim, lam, eps, window)
        self.fused = fused
        d = len(shape)
        self.lattice = lattice_shape(shape, spacing)
        self.value = torch.empty(4, dtype=torch.float64, device=device)
        self.grad = torch.empty((d,) + self.lattice, dtype=torch.float32, device=device)
        self.workspace = torch.empty(objective_workspace_bytes(self.problem, fused),
                                     dtype=torch.uint8, device=device)

    def __call__(self, fixed, moving, ctrl, want_grad=True, stream=None):
        return al_objective_grad(self.problem, fixed, moving, ctrl, self.value,
                                 self.grad if want_grad else None, self.workspace,
                                 want_grad=want_grad, fused=self.fused, stream=stream)


# ---------------------------------------------- learned initialisation ----
# Activations are torch.bfloat16 tensors shaped (batch, D, H, W, C), channels
# last; weights are float32 (cout, 27, cin) masters.

def make_conv(batch, size, cin, cout, stride) -> al_conv3d:
    cv = al_conv3d()
    cv.batch, cv.cin, cv.cout, cv.stride = int(batch), int(cin), int(cout), int(stride)
    for k in range(3):
        cv.size[k] = int(size[k])
    return cv


def conv_output_size(cv: al_conv3d):
    out = (ctypes.c_int64 * 3)()
    _call("al_conv3d_output_size", ctypes.byref(cv), out)
    return tuple(int(v) for v in out)


def _i64x3(v):
    a = (ctypes.c_int64 * 3)()
    for k in range(3):
        a[k] = int(v[k])
    return a


def _act(t, shape, what, dtype=torch.bfloat16):
    if t.dtype != dtype or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what}: expected {dtype} {tuple(shape)}, got {t.dtype} "
                         f"{tuple(t.shape)}")
    return _ptr(t)


def al_conv3d_pack(cv, weight, fwd=True, dgrad=True, stream=None, out=None):
    """bf16 weight copies in the layer kernels' layout: (packed_fwd, packed_dgrad).
    out: a previous result to write into (no allocation)."""
    _f32(weight, (cv.cout, 27, cv.cin), "weight")
    pf = pd = None
    if fwd:
        nf = load().al_conv3d_packed_bytes(ctypes.byref(cv), 0)
        pf = out[0] if out is not None and out[0] is not None else None
        if pf is None or pf.numel() != nf:
            pf = torch.empty(nf, dtype=torch.uint8, device=weight.device)
    if dgrad:
        n = load().al_conv3d_packed_bytes(ctypes.byref(cv), 1)
        if n == 0:
            raise ValueError("dgrad packing needs cin a multiple of 16")
        pd = out[1] if out is not None and out[1] is not None else None
        if pd is None or pd.numel() != n:
            pd = torch.empty(n, dtype=torch.uint8, device=weight.device)
    _call("al_conv3d_pack", ctypes.byref(cv), _ptr(weight), _ptr(pf), _ptr(pd), _stream(stream))
    return pf, pd


def conv_forward_workspace_bytes(cv) -> int:
    return int(load().al_conv3d_forward_workspace_bytes(ctypes.byref(cv)))


def al_conv3d_forward(cv, x, packed_fwd, bias=None, relu=True, out_f32=False, out=None,
                      workspace=None, split=True, stream=None):
    """split=True passes a workspace (the given one, else a new one) so that
    layers with few output tiles split their K sum over more CTAs."""
    osz = conv_output_size(cv)
    _act(x, (cv.batch,) + tuple(cv.size) + (cv.cin,), "input")
    shape = (cv.batch,) + osz + (cv.cout,)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32 if out_f32 else torch.bfloat16,
                          device=x.device)
    _act(out, shape, "output", torch.float32 if out_f32 else torch.bfloat16)
    if bias is not None:
        _f32(bias, (cv.cout,), "bias")
    ws, nbytes = None, 0
    if split:
        nbytes = conv_forward_workspace_bytes(cv)
        if nbytes:
            ws = _workspace(nbytes, x.device, workspace)
    _call("al_conv3d_forward", ctypes.byref(cv), _ptr(x), _ptr(packed_fwd), _ptr(bias),
          int(bool(relu)), int(bool(out_f32)), _ptr(out), _ptr(ws),
          ctypes.c_size_t(ws.numel() if ws is not None else 0), _stream(stream))
    return out


def al_conv3d_backward_data(cv, grad_out, packed_dgrad, relu_input=None, addend=None,
                            addend_offset=0, grad_in=None, stream=None):
    osz = conv_output_size(cv)
    _act(grad_out, (cv.batch,) + osz + (cv.cout,), "grad_output")
    shape = (cv.batch,) + tuple(cv.size) + (cv.cin,)
    if relu_input is not None:
        _act(relu_input, shape, "relu_input")
    stride = 0
    if addend is not None:
        if addend.dtype != torch.bfloat16 or tuple(addend.shape[:4]) != shape[:4]:
            raise ValueError("addend: bf16 on the input grid expected")
        stride = int(addend.shape[4])
    if grad_in is None:
        grad_in = torch.empty(shape, dtype=torch.bfloat16, device=grad_out.device)
    _act(grad_in, shape, "grad_input")
    _call("al_conv3d_backward_data", ctypes.byref(cv), _ptr(grad_out), _ptr(packed_dgrad),
          _ptr(relu_input), _ptr(addend), int(stride), int(addend_offset), _ptr(grad_in),
          _stream(stream))
    return grad_in


def al_conv3d_backward_weight(cv, x, grad_out, grad_weight=None, grad_bias=None, workspace=None,
                              stream=None):
    osz = conv_output_size(cv)
    _act(x, (cv.batch,) + tuple(cv.size) + (cv.cin,), "input")
    _act(grad_out, (cv.batch,) + osz + (cv.cout,), "grad_output")
    if grad_weight is None:
        grad_weight = torch.empty((cv.cout, 27, cv.cin), dtype=torch.float32, device=x.device)
    if grad_bias is None:
        grad_bias = torch.empty(cv.cout, dtype=torch.float32, device=x.device)
    nb = load().al_conv3d_backward_weight_workspace_bytes(ctypes.byref(cv))
    ws = _workspace(nb, x.device, workspace)
    _call("al_conv3d_backward_weight", ctypes.byref(cv), _ptr(x), _ptr(grad_out),
          _ptr(grad_weight), _ptr(grad_bias), _ptr(ws), ctypes.c_size_t(ws.numel()),
          _stream(stream))
    return grad_weight, grad_bias


def conv_wgrad_workspace_bytes(cv) -> int:
    return int(load().al_conv3d_backward_weight_workspace_bytes(ctypes.byref(cv)))


def al_initnet_input(fixed, moving, out=None, stream=None):
    """(batch, D, H, W) fp32 pair -> (batch, D, H, W, 2) bf16."""
    shape = tuple(fixed.shape)
    _f32(fixed, shape, "fixed")
    _f32(moving, shape, "moving")
    if out is None:
        out = torch.empty(shape + (2,), dtype=torch.bfloat16, device=fixed.device)
    _call("al_initnet_input", int(shape[0]), _i64x3(shape[1:]), _ptr(fixed), _ptr(moving),
          _ptr(out), _stream(stream))
    return out


def al_initnet_pair_input(shape, spacing, moving, ctrl, out=None, stream=None):
    """Network input (count, *shape, 2) bf16 of the pairs F = M o (x + B c):
    moving (count, *shape) fp32, ctrl (count, 3, nz, ny, nx) fp32."""
    bs = bspline_init(shape, spacing)
    count = int(moving.shape[0])
    _f32(moving, (count,) + tuple(shape), "moving")
    _f32(ctrl, (count, 3) + lattice_shape(shape, spacing), "ctrl")
    if out is None:
        out = torch.empty((count,) + tuple(shape) + (2,), dtype=torch.bfloat16,
                          device=moving.device)
    if out.dtype != torch.bfloat16 or tuple(out.shape) != (count,) + tuple(shape) + (2,):
        raise ValueError("out: expected bf16 (count, *shape, 2)")
    _call("al_initnet_pair_input", ctypes.byref(bs), count, _ptr(moving), _ptr(ctrl), _ptr(out),
          _stream(stream))
    return out


def al_initnet_upcat(e4, e3, out=None, stream=None):
    nb, n3, c3, c4 = e3.shape[0], tuple(e3.shape[1:4]), e3.shape[4], e4.shape[4]
    if out is None:
        out = torch.empty((nb,) + n3 + (c4 + c3,), dtype=torch.bfloat16, device=e3.device)
    _call("al_initnet_upcat", int(nb), _i64x3(n3), int(c4), int(c3), _ptr(e4), _ptr(e3),
          _ptr(out), _stream(stream))
    return out


def al_initnet_upcat_adjoint(grad_cat, e4, out=None, stream=None):
    nb, n3 = grad_cat.shape[0], tuple(grad_cat.shape[1:4])
    c4 = e4.shape[4]
    c3 = grad_cat.shape[4] - c4
    if out is None:
        out = torch.empty_like(e4)
    _call("al_initnet_upcat_adjoint", int(nb), _i64x3(n3), int(c4), int(c3), _ptr(grad_cat),
          _ptr(e4), _ptr(out), _stream(stream))
    return out


def al_initnet_head_to_ctrl(shape, head, out=None, stream=None):
    """head (batch, n3z, n3y, n3x, C) fp32 -> (batch, 3, nz, ny, nx) at spacing 8."""
    bs = bspline_init(shape, 8)
    nb = head.shape[0]
    if out is None:
        out = torch.empty((nb, 3) + lattice_shape(shape, 8), dtype=torch.float32,
                          device=head.device)
    _call("al_initnet_head_to_ctrl", ctypes.byref(bs), int(nb), _i64x3(head.shape[1:4]),
          int(head.shape[4]), _ptr(head), _ptr(out), _stream(stream))
    return out


def al_initnet_head_adjoint(shape, grad_ctrl, head_shape, out=None, stream=None):
    bs = bspline_init(shape, 8)
    nb = grad_ctrl.shape[0]
    if out is None:
        out = torch.empty(tuple(head_shape), dtype=torch.bfloat16, device=grad_ctrl.device)
    _call("al_initnet_head_adjoint", ctypes.byref(bs), int(nb), _i64x3(head_shape[1:4]),
          int(head_shape[4]), _ptr(grad_ctrl), _ptr(out), _stream(stream))
    return out


def field_loss_workspace_bytes(batch) -> int:
    return int(load().al_field_loss_workspace_bytes(int(batch)))


def al_field_loss(shape, ctrl, ctrl_true, loss=None, grad=None, workspace=None, stream=None):
    """Mean squared displacement-field difference (spacing 8) and its gradient."""
    bs = bspline_init(shape, 8)
    nb = ctrl.shape[0]
    if loss is None:
        loss = torch.empty(1, dtype=torch.float64, device=ctrl.device)
    if grad is None:
        grad = torch.empty_like(ctrl)
    ws = _workspace(load().al_field_loss_workspace_bytes(int(nb)), ctrl.device, workspace)
    _call("al_field_loss", ctypes.byref(bs), int(nb), _ptr(ctrl), _ptr(ctrl_true), _ptr(loss),
          _ptr(grad), _ptr(ws), ctypes.c_size_t(ws.numel()), _stream(stream))
    return loss, grad


def al_adam_flat(param, grad, m, v, step, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, stream=None):
    p = al_adam_params()
    p.lr, p.beta1, p.beta2, p.eps = float(lr), float(betas[0]), float(betas[1]), float(eps)
    _call("al_adam_flat", ctypes.byref(p), ctypes.c_int64(param.numel()), _ptr(step),
          _ptr(param), _ptr(grad), _ptr(m), _ptr(v), _stream(stream))


def al_adam_flat_pack(param, grad, m, v, step, layers, lr=1e-3, betas=(0.9, 0.999), eps=1e-8,
                      stream=None):
    """al_adam_flat plus the refresh of packed weights: layers is a list of
    (cv, weight_offset, packed_fwd, packed_dgrad), the packed tensors (either
    None) holding an al_conv3d_pack result of that layer."""
    n = param.numel()
    for t, what in ((param, "param"), (grad, "grad"), (m, "m"), (v, "v")):
        _f32(t, (n,), what)
    for cv, _, f, d in layers:
        # the kernel writes every slot of a real weight: the copies must be
        # whole al_conv3d_pack results of this layer
        for t, kind in ((f, 0), (d, 1)):
            if t is not None and t.numel() * t.element_size() != \
                    load().al_conv3d_packed_bytes(ctypes.byref(cv), kind):
                raise ValueError("packed weights: expected an al_conv3d_pack result of the layer")
    p = al_adam_params()
    p.lr, p.beta1, p.beta2, p.eps = float(lr), float(betas[0]), float(betas[1]), float(eps)
    nl = len(layers)
    cvs = (al_conv3d * max(nl, 1))(*[l[0] for l in layers])
    offs = (ctypes.c_int64 * max(nl, 1))(*[int(l[1]) for l in layers])
    pf = (ctypes.c_void_p * max(nl, 1))(*[_ptr(l[2]) for l in layers])
    pd = (ctypes.c_void_p * max(nl, 1))(*[_ptr(l[3]) for l in layers])
    _call("al_adam_flat_pack", ctypes.byref(p), ctypes.c_int64(n), _ptr(step),
          _ptr(param), _ptr(grad), _ptr(m), _ptr(v), nl, cvs, offs, pf, pd, _stream(stream))


def al_render_blobs(shape, table, out=None, stream=None):
    """table (count, n_blobs, 5) fp32 on the device -> (count, *shape) fp32 volumes."""
    count, nbl = int(table.shape[0]), int(table.shape[1])
    if out is None:
        out = torch.empty((count,) + tuple(shape), dtype=torch.float32, device=table.device)
    _call("al_render_blobs", _i64x3(shape), count, nbl, _ptr(table), _ptr(out), _stream(stream))
    return out


def _fresh_call_state(fn):
    """Entry points start with no device recorded (a call that failed while
    marshalling must not leave its device behind)."""
    @functools.wraps(fn)
    def wrapped(*a, **k):
        _tls.dev = None
        return fn(*a, **k)
    return wrapped


for _name in [n for n in list(globals())
              if n.startswith("al_") and type(globals()[n]) is type(_fresh_call_state)]:
    globals()[_name] = _fresh_call_state(globals()[_name])
