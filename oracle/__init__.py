"""FP64 CPU oracle for the B-spline registration objective (arXiv 1806.09907).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this module; the library itself never does. The
arithmetic lives in ``airgb_oracle.c`` (plain C, double precision); this
module builds it with gcc and wraps it with ctypes. It shares no code with the
CUDA path.

Every array argument is widened to float64 (exact for the fp32 arrays the GPU
path consumes). Shapes follow the library's layout: scalar volumes are
``(Z, Y, X)`` (``(Y, X)`` in 2D), vector fields and control coefficients are
component planes ``(d, Z, Y, X)`` / ``(d, nz, ny, nx)`` with component 0 = x.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "airgb_oracle.c"), os.path.join(_HERE, "initnet_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

MSE, NCC, LCC = 0, 1, 2


_CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared"]


def _digest() -> str:
    """SHA-256 of the oracle's sources and flags (a library built from other
    sources, or copied from another machine, is rebuilt)."""
    h = hashlib.sha256(" ".join(_CFLAGS).encode())
    for src in _SRCS:
        with open(src, "rb") as f:
            h.update(os.path.basename(src).encode() + b"\0" + f.read())
    return h.hexdigest()


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` with gcc (portable C11)."""
    stamp = _LIB + ".sha256"
    digest = _digest()
    stale = not os.path.exists(_LIB) or not os.path.exists(stamp) or open(stamp).read().strip() != digest
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc"] + _CFLAGS + ["-o", tmp] + _SRCS + ["-lm"], check=True)
        os.replace(tmp, _LIB)
        with open(stamp + ".tmp", "w") as f:
            f.write(digest + "\n")
        os.replace(stamp + ".tmp", stamp)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    i64p = ctypes.POINTER(ctypes.c_int64)
    dp = ctypes.POINTER(ctypes.c_double)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    ci, cd = ctypes.c_int, ctypes.c_double
    lib.alref_kernel_b3.argtypes = [cd]
    lib.alref_kernel_b3.restype = cd
    lib.alref_lattice_size.argtypes = [ci, i64p, ci, i64p]
    lib.alref_displacement.argtypes = [ci, i64p, ci, dp, dp]
    lib.alref_displacement_adjoint.argtypes = [ci, i64p, ci, dp, dp]
    lib.alref_warp.argtypes = [ci, i64p, dp, dp, dp, u8p, dp]
    lib.alref_mse.argtypes = [i64p, dp, dp, u8p, dp, dp]
    lib.alref_ncc.argtypes = [i64p, dp, dp, u8p, cd, dp, dp]
    lib.alref_lcc.argtypes = [ci, i64p, dp, dp, u8p, ci, cd, dp, dp]
    lib.alref_diffusion.argtypes = [ci, i64p, dp, dp, dp]
    lib.alref_objective_grad.argtypes = [ci, i64p, ci, ci, ci, cd, cd, dp, dp, dp, dp, dp]
    lib.alref_objective_grad_ex.argtypes = [ci, i64p, ci, ci, ci, cd, cd, dp, dp, dp, dp, dp, dp,
                                            dp]
    lib.alref_adam_step.argtypes = [ci, i64p, ci, cd, cd, cd, cd, ctypes.c_int64, dp, dp, dp, dp]
    lib.alref_pyramid_level.argtypes = [ci, i64p, dp, ci, dp]
    lib.alref_bspline_refine.argtypes = [ci, i64p, i64p, ci, dp, dp]
    lib.alref_exp_field.argtypes = [ci, i64p, ci, dp, dp, dp]
    lib.alref_exp_field_adjoint.argtypes = [ci, i64p, ci, dp, dp, dp]
    lib.alref_objective_grad_diffeo.argtypes = [ci, i64p, ci, ci, ci, ci, cd, cd, dp, dp, dp, dp,
                                                dp]
    lib.alref_conv3d.argtypes = [ci, i64p, ci, ci, ci, dp, dp, dp, ci, dp]
    lib.alref_conv3d_dgrad.argtypes = [ci, i64p, ci, ci, ci, dp, dp, dp]
    lib.alref_conv3d_wgrad.argtypes = [ci, i64p, ci, ci, ci, dp, dp, dp, dp]
    for name in ("alref_lattice_size", "alref_displacement", "alref_displacement_adjoint",
                 "alref_warp", "alref_mse", "alref_ncc", "alref_lcc", "alref_diffusion",
                 "alref_objective_grad", "alref_objective_grad_ex", "alref_adam_step",
                 "alref_pyramid_level", "alref_bspline_refine", "alref_exp_field",
                 "alref_exp_field_adjoint", "alref_objective_grad_diffeo", "alref_conv3d",
                 "alref_conv3d_dgrad", "alref_conv3d_wgrad"):
        getattr(lib, name).restype = ci
    _lib = lib
    return lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a, t=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _grid(shape):
    """Volume shape (Z,Y,X) or (Y,X) -> (ndim, int64[3] sizes X,Y,Z)."""
    if len(shape) == 3:
        return 3, np.array([shape[2], shape[1], shape[0]], dtype=np.int64)
    if len(shape) == 2:
        return 2, np.array([shape[1], shape[0], 1], dtype=np.int64)
    raise ValueError(f"bad volume shape {shape}")


def _check(st, what):
    if st != 0:
        raise ValueError(f"oracle {what} rejected its arguments (status {st})")


def kernel_b3(r: float) -> float:
    """k_B1D(r) of the cubic B-spline kernel (Sec. III-C)."""
    return _load().alref_kernel_b3(float(r))


def lattice_shape(shape, delta: int):
    """Control-lattice shape in volume order ((nz,ny,nx) or (ny,nx))."""
    nd, N = _grid(shape)
    n = np.zeros(3, dtype=np.int64)
    _check(_load().alref_lattice_size(nd, _p(N, ctypes.c_int64), int(delta), _p(n, ctypes.c_int64)),
           "lattice_size")
    return (int(n[2]), int(n[1]), int(n[0])) if nd == 3 else (int(n[1]), int(n[0]))


def displacement(shape, delta, ctrl):
    """u = sum_j c_j k(x_j, x), Eq. (kernel_basis) with the B-spline basis."""
    nd, N = _grid(shape)
    c = _d(ctrl)
    assert c.shape == (nd,) + lattice_shape(shape, delta), c.shape
    u = np.zeros((nd,) + tuple(shape), dtype=np.float64)
    _check(_load().alref_displacement(nd, _p(N, ctypes.c_int64), int(delta), _p(c), _p(u)),
           "displacement")
    return u


def displacement_adjoint(shape, delta, g_disp):
    """g_c = B^T g_u, the transpose of :func:`displacement`."""
    nd, N = _grid(shape)
    g = _d(g_disp)
    assert g.shape == (nd,) + tuple(shape)
    gc = np.zeros((nd,) + lattice_shape(shape, delta), dtype=np.float64)
    _check(_load().alref_displacement_adjoint(nd, _p(N, ctypes.c_int64), int(delta), _p(g), _p(gc)),
           "displacement_adjoint")
    return gc


def warp(moving, disp, with_grad=False):
    """Backward warp with mask and linear interpolation (Sec. III-C, Image Warping).

    Returns (W, mask[, dM~/dy]) with W = 0 and grad = 0 outside the mask."""
    m = _d(moving)
    nd, N = _grid(m.shape)
    u = _d(disp)
    assert u.shape == (nd,) + m.shape
    w = np.zeros(m.shape, dtype=np.float64)
    mask = np.zeros(m.shape, dtype=np.uint8)
    gy = np.zeros((nd,) + m.shape, dtype=np.float64) if with_grad else None
    _check(_load().alref_warp(nd, _p(N, ctypes.c_int64), _p(m), _p(u), _p(w),
                              _p(mask, ctypes.c_uint8), _p(gy) if with_grad else None), "warp")
    return (w, mask, gy) if with_grad else (w, mask)


def similarity(kind, fixed, warped, mask, eps=1e-5, window=7):
    """S and dS/dW for MSE / NCC / LCC (Sec. III-B)."""
    f, w = _d(fixed), _d(warped)
    mk = np.ascontiguousarray(mask, dtype=np.uint8)
    nd, N = _grid(f.shape)
    S = np.zeros(1, dtype=np.float64)
    g = np.zeros(f.shape, dtype=np.float64)
    lib = _load()
    if kind == MSE:
        st = lib.alref_mse(_p(N, ctypes.c_int64), _p(f), _p(w), _p(mk, ctypes.c_uint8), _p(S), _p(g))
    elif kind == NCC:
        st = lib.alref_ncc(_p(N, ctypes.c_int64), _p(f), _p(w), _p(mk, ctypes.c_uint8), float(eps),
                           _p(S), _p(g))
    elif kind == LCC:
        st = lib.alref_lcc(nd, _p(N, ctypes.c_int64), _p(f), _p(w), _p(mk, ctypes.c_uint8),
                           int(window), float(eps), _p(S), _p(g))
    else:
        raise ValueError(kind)
    _check(st, "similarity")
    return float(S[0]), g


def diffusion(disp):
    """R_diff and dR/du, Eq. (diffusion_regularizer)."""
    u = _d(disp)
    nd = u.shape[0]
    _, N = _grid(u.shape[1:])
    R = np.zeros(1, dtype=np.float64)
    g = np.zeros_like(u)
    _check(_load().alref_diffusion(nd, _p(N, ctypes.c_int64), _p(u), _p(R), _p(g)), "diffusion")
    return float(R[0]), g


def objective_grad(kind, fixed, moving, ctrl, delta, lam, eps=1e-5, window=7, grad=True,
                   intermediates=False):
    """J = S + lam*R, Eq. (objective), and dJ/dc.

    Returns ({"J","S","R","n_mask"}, g_ctrl or None); with intermediates=True
    the dict also holds the displacement "u" and the per-voxel "dS_dW"."""
    f, m, c = _d(fixed), _d(moving), _d(ctrl)
    nd, N = _grid(f.shape)
    assert c.shape == (nd,) + lattice_shape(f.shape, delta), c.shape
    out = np.zeros(4, dtype=np.float64)
    gc = np.zeros_like(c) if grad else None
    u = np.zeros((nd,) + f.shape) if intermediates else None
    gw = np.zeros(f.shape) if intermediates else None
    _check(_load().alref_objective_grad_ex(nd, _p(N, ctypes.c_int64), int(delta), int(kind),
                                           int(window), float(eps), float(lam), _p(f), _p(m),
                                           _p(c), _p(out), _p(gc) if grad else None,
                                           _p(u) if intermediates else None,
                                           _p(gw) if intermediates else None), "objective_grad")
    vals = {"J": float(out[0]), "S": float(out[1]), "R": float(out[2]), "n_mask": float(out[3])}
    if intermediates:
        vals["u"], vals["dS_dW"] = u, gw
    return vals, gc


def adam_step(shape, delta, ctrl, grad, m, v, step, lr=0.01, betas=(0.9, 0.999), eps=1e-8):
    """One Adam step on the control points in normalised units (Sec. II-A,
    Optimization; Kingma and Ba's update). Returns new (ctrl, m, v) arrays."""
    nd, N = _grid(shape)
    c, g, mm, vv = _d(ctrl).copy(), _d(grad), _d(m).copy(), _d(v).copy()
    want = (nd,) + lattice_shape(shape, delta)
    assert c.shape == want and g.shape == want and mm.shape == want and vv.shape == want
    _check(_load().alref_adam_step(nd, _p(N, ctypes.c_int64), int(delta), float(lr),
                                   float(betas[0]), float(betas[1]), float(eps), int(step),
                                   _p(c), _p(g), _p(mm), _p(vv)), "adam_step")
    return c, mm, vv


def level_shape(shape, factor):
    """Grid of a pyramid level: every factor-th voxel from voxel 0."""
    return tuple((n - 1) // factor + 1 for n in shape)


def pyramid_level(image, factor):
    """Gaussian-smoothed (sigma = factor/2, |t| <= 3 sigma, clamped edges),
    subsampled image of one pyramid level (Sec. IV-A, multi-resolution)."""
    im = _d(image)
    nd, N = _grid(im.shape)
    out = np.zeros(level_shape(im.shape, factor), dtype=np.float64)
    _check(_load().alref_pyramid_level(nd, _p(N, ctypes.c_int64), _p(im), int(factor), _p(out)),
           "pyramid_level")
    return out


def bspline_refine(coarse_shape, fine_shape, delta, ctrl_coarse):
    """Fine-level coefficients whose displacement equals the coarse one
    (two-scale relation of the cubic B-spline), in fine voxel units."""
    nd, Nc = _grid(coarse_shape)
    _, Nf = _grid(fine_shape)
    c = _d(ctrl_coarse)
    assert c.shape == (nd,) + lattice_shape(coarse_shape, delta), c.shape
    out = np.zeros((nd,) + lattice_shape(fine_shape, delta), dtype=np.float64)
    _check(_load().alref_bspline_refine(nd, _p(Nc, ctypes.c_int64), _p(Nf, ctypes.c_int64),
                                        int(delta), _p(c), _p(out)), "bspline_refine")
    return out


def exp_field(velocity, steps=6, trajectory=False):
    """f = exp(v) by scaling and squaring (Sec. III-D): the displacement u_K
    of the diffeomorphism, (d, *shape); with trajectory=True also the inputs
    u_0 .. u_{K-1} of the squarings, (K, d, *shape)."""
    v = _d(velocity)
    nd, N = _grid(v.shape[1:])
    u = np.zeros_like(v)
    traj = np.zeros((max(int(steps), 1),) + v.shape) if trajectory else None
    _check(_load().alref_exp_field(nd, _p(N, ctypes.c_int64), int(steps), _p(v), _p(u),
                                   _p(traj) if trajectory else None), "exp_field")
    return (u, traj[:int(steps)]) if trajectory else u


def exp_field_adjoint(trajectory, grad_u, steps=6):
    """(d u_K / d v)^T grad_u from the trajectory of :func:`exp_field`."""
    g = _d(grad_u)
    nd, N = _grid(g.shape[1:])
    t = _d(trajectory) if int(steps) > 0 else np.zeros((1,) + g.shape)
    gv = np.zeros_like(g)
    _check(_load().alref_exp_field_adjoint(nd, _p(N, ctypes.c_int64), int(steps), _p(t), _p(g),
                                           _p(gv)), "exp_field_adjoint")
    return gv


def objective_grad_diffeo(kind, fixed, moving, ctrl, delta, lam, steps=6, eps=1e-5, window=7,
                          grad=True):
    """J = S(M o exp(v), F) + lam R_diff(u_K), v the B-spline field of c, and
    dJ/dc. Returns ({"J","S","R","n_mask"}, g_ctrl or None)."""
    f, m, c = _d(fixed), _d(moving), _d(ctrl)
    nd, N = _grid(f.shape)
    assert c.shape == (nd,) + lattice_shape(f.shape, delta), c.shape
    out = np.zeros(4, dtype=np.float64)
    gc = np.zeros_like(c) if grad else None
    _check(_load().alref_objective_grad_diffeo(nd, _p(N, ctypes.c_int64), int(delta), int(steps),
                                               int(kind), int(window), float(eps), float(lam),
                                               _p(f), _p(m), _p(c), _p(out),
                                               _p(gc) if grad else None), "objective_grad_diffeo")
    return {"J": float(out[0]), "S": float(out[1]), "R": float(out[2]),
            "n_mask": float(out[3])}, gc

