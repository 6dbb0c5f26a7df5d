"""Pins of the oracle's optimisation-loop routines: Adam on the control
points, the Gaussian pyramid level and the dyadic B-spline refinement.

Each pin comes from outside the oracle's own code: closed forms of Adam's
update, PyTorch's Adam and SciPy's Gaussian filter as independent library
routines, and the exactness of B-spline refinement checked through the
oracle's definitional displacement sum.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- Adam ------

@pytest.mark.parametrize("shape,delta", [((20, 17), 4), ((9, 12, 10), 3)])
def test_adam_first_step_closed_form(shape, delta):
    """t = 1 from zero moments: m^ = g~, v^ = g~^2, so each normalised
    coordinate moves by -lr g~/(|g~| + eps)."""
    rng = _rng(1)
    nd = len(shape)
    ls = (nd,) + oracle.lattice_shape(shape, delta)
    c0 = rng.normal(0, 2, ls)
    g = rng.normal(0, 1e-3, ls)
    g.reshape(nd, -1)[:, ::7] = 0.0  # zero gradients stay put
    lr, eps = 0.01, 1e-8
    c1, m1, v1 = oracle.adam_step(shape, delta, c0, g, np.zeros(ls), np.zeros(ls), 1, lr=lr,
                                  eps=eps)
    N = shape[::-1]  # x, y, z sizes; component i belongs to axis i
    for i in range(nd):
        h = (N[i] - 1) / 2.0  # voxel units per normalised unit
        gn = g[i] * h
        want = c0[i] - h * lr * gn / (np.abs(gn) + eps)
        np.testing.assert_allclose(c1[i], want, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(m1[i], 0.1 * gn, rtol=1e-13, atol=0)
        np.testing.assert_allclose(v1[i], 0.001 * gn * gn, rtol=1e-13, atol=0)


def test_adam_constant_gradient_closed_form():
    """With a constant gradient the bias-corrected moments are exactly g~ and
    g~^2 at every step, so T steps move by T times the first step."""
    shape, delta = (11, 13, 12), 4
    rng = _rng(2)
    ls = (3,) + oracle.lattice_shape(shape, delta)
    c = rng.normal(0, 1, ls)
    c0 = c.copy()
    g = rng.normal(0, 1e-2, ls)
    m, v = np.zeros(ls), np.zeros(ls)
    T, lr, eps = 25, 0.02, 1e-8
    for t in range(1, T + 1):
        c, m, v = oracle.adam_step(shape, delta, c, g, m, v, t, lr=lr, eps=eps)
    N = shape[::-1]
    for i in range(3):
        h = (N[i] - 1) / 2.0
        gn = g[i] * h
        np.testing.assert_allclose(c[i], c0[i] - T * h * lr * gn / (np.abs(gn) + eps),
                                   rtol=1e-10, atol=1e-12)


def test_adam_matches_torch_adam():
    """Against torch.optim.Adam (float64, CPU) run on c~ = c * 2/(N-1) with
    the normalised gradient, over varying gradients and betas."""
    torch = pytest.importorskip("torch")
    shape, delta = (10, 14, 9), 3
    rng = _rng(3)
    nd = 3
    ls = (nd,) + oracle.lattice_shape(shape, delta)
    N = shape[::-1]
    to_norm = np.array([2.0 / (N[i] - 1) for i in range(nd)]).reshape(nd, 1, 1, 1)
    c = rng.normal(0, 2, ls)
    p = torch.tensor(c * to_norm, dtype=torch.float64, requires_grad=True)
    lr, betas, eps = 0.03, (0.8, 0.99), 1e-6
    opt = torch.optim.Adam([p], lr=lr, betas=betas, eps=eps)
    m, v = np.zeros(ls), np.zeros(ls)
    for t in range(1, 8):
        g = rng.normal(0, 10.0 ** rng.uniform(-6, -1), ls)
        c, m, v = oracle.adam_step(shape, delta, c, g, m, v, t, lr=lr, betas=betas, eps=eps)
        p.grad = torch.tensor(g / to_norm, dtype=torch.float64)
        opt.step()
        np.testing.assert_allclose(c * to_norm, p.detach().numpy(), rtol=1e-12, atol=1e-14)
    st = opt.state[p]
    np.testing.assert_allclose(m, st["exp_avg"].numpy(), rtol=1e-12, atol=0)
    np.testing.assert_allclose(v, st["exp_avg_sq"].numpy(), rtol=1e-12, atol=0)


def test_adam_rejects_step_zero():
    shape, delta = (8, 8), 4
    ls = (2,) + oracle.lattice_shape(shape, delta)
    z = np.zeros(ls)
    with pytest.raises(ValueError):
        oracle.adam_step(shape, delta, z, z, z, z, 0)


# ------------------------------------------------------------- pyramid ------

@pytest.mark.parametrize("shape", [(37, 29), (23, 30, 19)])
def test_pyramid_factor_one_is_identity(shape):
    im = _rng(4).normal(size=shape)
    np.testing.assert_array_equal(oracle.pyramid_level(im, 1), im)


@pytest.mark.parametrize("shape", [(37, 29), (23, 30, 19)])
@pytest.mark.parametrize("factor", [2, 4])
def test_pyramid_matches_scipy_gaussian(shape, factor):
    """SciPy's Gaussian filter with clamped ('nearest') edges, truncated at
    3 sigma (its radius int(3 sigma + 0.5) equals floor(3 sigma) for
    sigma = 1 and 2), then every factor-th voxel."""
    ndimage = pytest.importorskip("scipy.ndimage")
    im = _rng(5).uniform(-1000, 1500, shape)
    ref = ndimage.gaussian_filter(im, sigma=factor / 2.0, mode="nearest", truncate=3.0)
    ref = ref[tuple(slice(None, None, factor) for _ in shape)]
    out = oracle.pyramid_level(im, factor)
    assert out.shape == oracle.level_shape(shape, factor) == ref.shape
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-9)


def test_pyramid_constant_and_shapes():
    im = np.full((160, 33, 40), 7.25)
    out = oracle.pyramid_level(im, 4)
    assert out.shape == (40, 9, 10)
    np.testing.assert_allclose(out, 7.25, rtol=1e-14)
    assert oracle.level_shape((256, 256, 160), 4) == (64, 64, 40)
    assert oracle.level_shape((256, 256, 160), 2) == (128, 128, 80)


# -------------------------------------------------------------- refine ------

def _coarse_of(fine_shape):
    return oracle.level_shape(fine_shape, 2)


@pytest.mark.parametrize("fine_shape,delta", [((31, 26), 4), ((26, 21, 17), 3), ((20, 24, 29), 6)])
def test_refine_preserves_displacement(fine_shape, delta):
    """u_fine(2x) = 2 u_coarse(x) at every coarse voxel: the refined spline
    is the coarse one, both evaluated by the definitional sum."""
    cs = _coarse_of(fine_shape)
    nd = len(fine_shape)
    cc = _rng(6).normal(0, 2, (nd,) + oracle.lattice_shape(cs, delta))
    cf = oracle.bspline_refine(cs, fine_shape, delta, cc)
    uc = oracle.displacement(cs, delta, cc)
    uf = oracle.displacement(fine_shape, delta, cf)
    sub = (slice(None),) + tuple(slice(None, None, 2) for _ in fine_shape)
    np.testing.assert_allclose(uf[sub], 2.0 * uc, rtol=0, atol=1e-12)


def test_refine_linear_closed_form():
    """Coarse coefficients c_j = A p_j + b (linear precision) refine to
    c_i = A p_i + 2 b on the fine lattice, p the point positions in each
    level's own voxels."""
    fine_shape, delta = (21, 26, 23), 4
    cs = _coarse_of(fine_shape)
    A = np.array([[0.1, -0.2, 0.05], [0.3, 0.0, -0.1], [-0.15, 0.2, 0.25]])  # A[i, axis]
    b = np.array([1.5, -2.0, 0.75])

    def linear(shape):
        ls = oracle.lattice_shape(shape, delta)
        pz, py, px = np.meshgrid(*[(np.arange(n) - 1.0) * delta for n in ls], indexing="ij")
        return ls, (px, py, pz)

    lsc, pc = linear(cs)
    cc = np.stack([A[i, 0] * pc[0] + A[i, 1] * pc[1] + A[i, 2] * pc[2] + b[i] for i in range(3)])
    lsf, pf = linear(fine_shape)
    want = np.stack([A[i, 0] * pf[0] + A[i, 1] * pf[1] + A[i, 2] * pf[2] + 2 * b[i]
                     for i in range(3)])
    np.testing.assert_allclose(oracle.bspline_refine(cs, fine_shape, delta, cc), want, rtol=0,
                               atol=1e-12)


def test_refine_rejects_mismatched_levels():
    delta = 4
    cc = np.zeros((2,) + oracle.lattice_shape((16, 16), delta))
    with pytest.raises(ValueError):
        oracle.bspline_refine((16, 16), (40, 31), delta, cc)
