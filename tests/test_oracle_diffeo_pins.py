"""Pins of the oracle's diffeomorphic transformation (Sec. III-D): f = exp(v)
by scaling and squaring, its adjoint, and the objective built on it.

Each pin comes from outside the oracle's code: exact results for zero,
constant and affine velocity fields (the affine one in closed form through
a matrix power), inverse consistency exp(-v) o exp(v) ~ id, a dot-product
test of the adjoint against central differences of the exponential, and
central differences of the whole objective.
"""
import numpy as np
import pytest

import oracle
from paper_1806_09907_gb300 import synth


def smooth_velocity(shape, rms, seed):
    return synth.smooth_field(shape, rms, seed, min_wavelength=12.0)


@pytest.mark.parametrize("shape", [(9, 11), (6, 7, 8)])
@pytest.mark.parametrize("steps", [0, 3, 6])
def test_exp_of_constant_field_is_the_translation(shape, steps):
    nd = len(shape)
    t = np.array([0.75, -1.25, 0.5][:nd])
    v = np.broadcast_to(t.reshape((nd,) + (1,) * nd), (nd,) + shape).copy()
    u = oracle.exp_field(v, steps)
    np.testing.assert_array_equal(u, v)
    assert np.all(oracle.exp_field(np.zeros_like(v), steps) == 0.0)


def test_exp_with_no_squaring_is_the_velocity():
    v = smooth_velocity((8, 9, 10), 1.5, 3)
    np.testing.assert_array_equal(oracle.exp_field(v, 0), v)


@pytest.mark.parametrize("nd", [2, 3])
def test_exp_of_affine_field_closed_form(nd):
    """v(x) = A x + b: linear interpolation reproduces affine fields, so
    every squaring maps (A_k, b_k) to I + A_{k+1} = (I + A_k)^2 and
    b_{k+1} = (2 I + A_k) b_k, i.e. I + A_K = (I + A/2^K)^(2^K). Checked at
    points whose samples stay inside the grid at every step."""
    shape = (31, 33) if nd == 2 else (21, 23, 25)
    rng = np.random.default_rng(5)
    A = rng.normal(0, 0.03, (nd, nd))
    b = rng.normal(0, 0.5, nd)
    axes = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    xs = [axes[nd - 1 - k] for k in range(nd)]  # x first
    v = np.stack([sum(A[i, k] * xs[k] for k in range(nd)) + b[i] for i in range(nd)])
    K = 5
    u = oracle.exp_field(v, K)
    Ak, bk = A / 2 ** K, b / 2 ** K
    for _ in range(K):
        Ak, bk = 2 * Ak + Ak @ Ak, (2 * np.eye(nd) + Ak) @ bk
    want = np.stack([sum(Ak[i, k] * xs[k] for k in range(nd)) + bk[i] for i in range(nd)])
    # interior: samples near a face are clamped in some squaring, and the
    # difference this makes reaches inwards by about the summed per-step
    # displacement (|v| < 1.5 voxels here); 5 voxels from every face it is gone
    inner = tuple(slice(5, n - 5) for n in shape)
    np.testing.assert_allclose(u[(slice(None),) + inner], want[(slice(None),) + inner],
                               rtol=0, atol=1e-12)
    ref = np.linalg.matrix_power(np.eye(nd) + A / 2 ** K, 2 ** K) - np.eye(nd)
    np.testing.assert_allclose(Ak, ref, rtol=1e-12, atol=1e-15)


def test_inverse_is_exp_of_minus_v():
    """f^-1 = exp(-v): x + u+(x) + u-(x + u+(x)) stays within a small
    fraction of the displacement of x in the interior (the discrete
    exponential is inverse consistent up to its interpolation error)."""
    shape = (24, 26, 28)
    v = smooth_velocity(shape, 1.0, 7)
    up = oracle.exp_field(v, 6)
    um = oracle.exp_field(-v, 6)
    nd = 3
    axes = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    xs = [axes[nd - 1 - k] for k in range(nd)]
    p = [xs[k] + up[k] for k in range(nd)]
    from scipy.ndimage import map_coordinates
    coords = np.stack([p[2], p[1], p[0]])  # z, y, x for map_coordinates
    back = [p[k] + map_coordinates(um[k], coords, order=1, mode="nearest") for k in range(nd)]
    inner = tuple(slice(4, n - 4) for n in shape)
    err = max(np.abs(back[k] - xs[k])[inner].max() for k in range(nd))
    assert err < 0.02 * np.abs(v).max(), err


@pytest.mark.parametrize("shape", [(10, 12), (7, 8, 9)])
def test_exp_adjoint_dot_product(shape):
    """<(exp(v + h dv) - exp(v - h dv)) / 2h, g> = <dv, adjoint(g)>."""
    nd = len(shape)
    v = smooth_velocity(shape, 1.3, 11)
    dv = smooth_velocity(shape, 1.0, 12)
    g = np.random.default_rng(13).normal(size=(nd,) + shape)
    K, h = 4, 1e-6
    _, traj = oracle.exp_field(v, K, trajectory=True)
    gv = oracle.exp_field_adjoint(traj, g, K)
    fd = (oracle.exp_field(v + h * dv, K) - oracle.exp_field(v - h * dv, K)) / (2 * h)
    lhs, rhs = float(np.sum(fd * g)), float(np.sum(dv * gv))
    assert abs(lhs - rhs) <= 1e-6 * abs(rhs), (lhs, rhs)


@pytest.mark.parametrize("shape,delta,kind", [((11, 13), 4, oracle.MSE), ((7, 8, 9), 3, oracle.MSE),
                                              ((9, 10, 8), 3, oracle.LCC)])
def test_diffeo_objective_central_differences(shape, delta, kind):
    nd = len(shape)
    sc = synth.blob_scene(shape, 4, (2.0, 4.0), 21)
    F = synth.render_blobs(shape, sc)
    M = synth.render_blobs(shape, sc, synth.smooth_field(shape, 1.0, 22, min_wavelength=8.0))
    rng = np.random.default_rng(23)
    c = rng.normal(0, 0.6, (nd,) + oracle.lattice_shape(shape, delta))
    K, lam, h = 3, 0.1, 1e-6
    _, g = oracle.objective_grad_diffeo(kind, F, M, c, delta, lam, K, window=3)
    fd = np.zeros_like(c)
    for idx in np.ndindex(c.shape):
        cp, cm = c.copy(), c.copy()
        cp[idx] += h
        cm[idx] -= h
        jp, _ = oracle.objective_grad_diffeo(kind, F, M, cp, delta, lam, K, window=3, grad=False)
        jm, _ = oracle.objective_grad_diffeo(kind, F, M, cm, delta, lam, K, window=3, grad=False)
        fd[idx] = (jp["J"] - jm["J"]) / (2 * h)
    err = np.linalg.norm(fd - g) / np.linalg.norm(g)
    assert err <= 1e-6, err


def test_diffeo_objective_reduces_to_the_plain_model_at_small_fields():
    """exp(v) = v + O(|v| |grad v|): for a tiny velocity the diffeomorphic J
    approaches the plain B-spline J, with a difference of second order."""
    shape, delta = (12, 14, 10), 3
    sc = synth.blob_scene(shape, 4, (2.0, 4.0), 31)
    F = synth.render_blobs(shape, sc)
    M = synth.render_blobs(shape, sc, synth.smooth_field(shape, 1.0, 32, min_wavelength=8.0))
    c = np.random.default_rng(33).normal(0, 1.0, (3,) + oracle.lattice_shape(shape, delta))
    diffs = []
    for s in (1e-2, 5e-3):
        jd, _ = oracle.objective_grad_diffeo(oracle.MSE, F, M, s * c, delta, 0.1, 6, grad=False)
        jp, _ = oracle.objective_grad(oracle.MSE, F, M, s * c, delta, 0.1, grad=False)
        diffs.append(abs(jd["J"] - jp["J"]))
    assert diffs[1] < 0.35 * diffs[0]  # second order: halving s quarters it
