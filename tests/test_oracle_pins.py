"""Pins of the FP64 oracle to facts that do not come from the oracle itself:
values worked out from the paper's formulas, closed forms, invariants,
library routines on special cases, and central finite differences.

Each test names the passage (section / equation) it follows."""
import os

import numpy as np
import pytest
from scipy import ndimage

import oracle
from paper_1806_09907_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(t) for t in line.split()])
    return rows


# ---------------------------------------------------------------- kernel ---

def test_kernel_values_match_hand_worked_fractions():
    """Sec. III-C, k_B1D: values at the printed breakpoints."""
    for r, num, den in _golden("bspline_kernel.txt"):
        assert oracle.kernel_b3(r) == pytest.approx(num / den, abs=1e-15)


def test_kernel_equals_box_convolved_four_times():
    """Sec. III-C, arbitrary order: B_3 = B_0 * B_0 * B_0 * B_0 with B_0 a unit
    box (spacing 1, normalised). Built numerically, independent of k_B1D."""
    h = 1e-3
    box = np.ones(int(round(1.0 / h)))
    b = box.copy()
    for _ in range(3):
        b = np.convolve(b, box) * h
    # b now samples B_3 on a grid of step h centred on its support [-2, 2]
    r = (np.arange(b.size) - (b.size - 1) / 2.0) * h
    for rr in (0.0, 0.3, 0.5, 1.0, 1.4, 1.9, -0.7):
        i = int(np.argmin(np.abs(r - rr)))
        assert oracle.kernel_b3(r[i]) == pytest.approx(b[i], abs=5e-6)


def test_weights_at_quarter_points():
    """Weights at t = 0 and t = 1/2 past a control point (Sec. III-C)."""
    for t, w0, w1, w2, w3, den in _golden("bspline_weights.txt"):
        got = [oracle.kernel_b3(t + 1), oracle.kernel_b3(t), oracle.kernel_b3(t - 1),
               oracle.kernel_b3(t - 2)]
        assert got == pytest.approx([w0 / den, w1 / den, w2 / den, w3 / den], abs=1e-15)


# ------------------------------------------------------- A1 displacement ---

@pytest.mark.parametrize("shape,delta", [((13, 11), 4), ((7, 9), 3), ((9, 10, 11), 4),
                                         ((5, 6, 7), 2)])
def test_partition_of_unity(shape, delta):
    """Eq. (kernel_basis) with B-splines: constant coefficients give a constant field."""
    nd = len(shape)
    ns = oracle.lattice_shape(shape, delta)
    c = np.zeros((nd,) + ns)
    for i in range(nd):
        c[i] = 1.7 - 0.9 * i
    u = oracle.displacement(shape, delta, c)
    for i in range(nd):
        np.testing.assert_allclose(u[i], 1.7 - 0.9 * i, atol=1e-13)


@pytest.mark.parametrize("shape,delta", [((13, 11), 4), ((9, 10, 11), 3)])
def test_linear_precision(shape, delta):
    """Cubic B-splines reproduce affine functions: c_j = A p_j + b with
    p_j = (j-1) delta gives u(x) = A x + b at every voxel."""
    nd = len(shape)
    ns = oracle.lattice_shape(shape, delta)
    g = np.random.default_rng(0)
    A = g.normal(size=(nd, nd))
    b = g.normal(size=nd)
    pj = np.meshgrid(*[(np.arange(n) - 1.0) * delta for n in ns], indexing="ij")  # z,y,x order
    pj = pj[::-1]  # x first
    xs = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")[::-1]
    c = np.zeros((nd,) + ns)
    want = np.zeros((nd,) + tuple(shape))
    for i in range(nd):
        c[i] = b[i] + sum(A[i, k] * pj[k] for k in range(nd))
        want[i] = b[i] + sum(A[i, k] * xs[k] for k in range(nd))
    u = oracle.displacement(shape, delta, c)
    np.testing.assert_allclose(u, want, atol=1e-12)


def test_single_control_point_placement():
    """One unit coefficient at lattice index j puts (2/3)^d at voxel (j-1) delta
    and k_B1D(r/delta) products around it (control point j sits at (j-1) delta)."""
    shape, delta = (17, 19, 21), 4
    ns = oracle.lattice_shape(shape, delta)
    c = np.zeros((3,) + ns)
    jz, jy, jx = 2, 3, 4
    c[1, jz, jy, jx] = 1.0
    u = oracle.displacement(shape, delta, c)
    z0, y0, x0 = (jz - 1) * delta, (jy - 1) * delta, (jx - 1) * delta
    assert u[1, z0, y0, x0] == pytest.approx((2.0 / 3.0) ** 3, abs=1e-15)
    assert u[1, z0, y0, x0 + 2] == pytest.approx((2.0 / 3.0) ** 2 * 23.0 / 48.0, abs=1e-15)
    assert u[1, z0 + 4, y0, x0] == pytest.approx((2.0 / 3.0) ** 2 / 6.0, abs=1e-15)
    assert u[1, z0 + 8, y0, x0] == 0.0
    assert np.all(u[0] == 0.0) and np.all(u[2] == 0.0)


def test_adjoint_is_transpose():
    """Sec. III-C: the gradient path is the transpose of the up-sampling:
    <B c, g> = <c, B^T g> for random c, g."""
    for shape, delta in (((9, 10, 11), 4), ((13, 11), 3)):
        nd = len(shape)
        ns = oracle.lattice_shape(shape, delta)
        g = np.random.default_rng(1)
        c = g.normal(size=(nd,) + ns)
        gu = g.normal(size=(nd,) + tuple(shape))
        lhs = np.sum(oracle.displacement(shape, delta, c) * gu)
        rhs = np.sum(c * oracle.displacement_adjoint(shape, delta, gu))
        assert lhs == pytest.approx(rhs, rel=1e-12)


# --------------------------------------------------------------- A2 warp ---

def test_identity_warp_is_exact():
    """Zero displacement: W = M bit for bit and every point inside."""
    g = np.random.default_rng(2)
    for shape in ((9, 10, 11), (13, 11)):
        M = g.normal(size=shape).astype(np.float32)
        W, m = oracle.warp(M, np.zeros((len(shape),) + shape))
        assert np.all(m == 1)
        assert np.array_equal(W, M.astype(np.float64))


def test_integer_shift_and_face_tie():
    """Integer shift s: W(x) = M(x+s) where 0 <= x+s <= N-1, outside otherwise.
    Points landing exactly on the last face are inside (strict test of the
    masking snippet, Sec. III-C)."""
    shape = (6, 7, 8)
    g = np.random.default_rng(3)
    M = g.normal(size=shape)
    s = (2, -1, 3)  # x, y, z
    u = np.zeros((3,) + shape)
    for k in range(3):
        u[k] = s[k]
    W, m = oracle.warp(M, u)
    Z, Y, X = shape
    for z in range(Z):
        for y in range(Y):
            for x in range(X):
                xx, yy, zz = x + s[0], y + s[1], z + s[2]
                inside = 0 <= xx <= X - 1 and 0 <= yy <= Y - 1 and 0 <= zz <= Z - 1
                assert m[z, y, x] == inside
                assert W[z, y, x] == (M[zz, yy, xx] if inside else 0.0)
    # a point a hair beyond the face is outside
    u2 = np.zeros((3,) + shape)
    u2[0, 0, 0, X - 1] = 1e-9
    _, m2 = oracle.warp(M, u2)
    assert m2[0, 0, X - 1] == 0 and m2.sum() == m2.size - 1


def test_affine_image_reproduced():
    """Linear interpolation reproduces affine images: M(p) = a.p + b gives
    W = a.(x+u) + b exactly at inside points, and dM~/dy = a."""
    shape = (8, 9, 10)
    Z, Y, X = shape
    a = np.array([0.7, -1.3, 2.1])
    zz, yy, xx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    M = a[0] * xx + a[1] * yy + a[2] * zz + 0.5
    g = np.random.default_rng(4)
    u = g.uniform(-1.5, 1.5, size=(3,) + shape)
    W, m, gy = oracle.warp(M, u, with_grad=True)
    want = a[0] * (xx + u[0]) + a[1] * (yy + u[1]) + a[2] * (zz + u[2]) + 0.5
    assert m.sum() > 0.3 * m.size
    np.testing.assert_allclose(W[m == 1], want[m == 1], atol=1e-12)
    for k in range(3):
        np.testing.assert_allclose(gy[k][m == 1], a[k], atol=1e-12)


def test_warp_matches_scipy_linear_interpolation():
    """Special case that reduces to a library routine: order-1
    map_coordinates equals the trilinear interpolant at inside points."""
    for shape in ((9, 10, 11), (13, 11)):
        nd = len(shape)
        g = np.random.default_rng(5)
        M = g.normal(size=shape)
        u = g.uniform(-2.0, 2.0, size=(nd,) + shape)
        W, m = oracle.warp(M, u)
        grids = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
        coords = [grids[a] + u[nd - 1 - a] for a in range(nd)]  # axis order z,y,x
        ref = ndimage.map_coordinates(M, coords, order=1, mode="nearest")
        np.testing.assert_allclose(W[m == 1], ref[m == 1], atol=1e-12)
        inside = np.ones(shape, dtype=bool)
        for a in range(nd):
            inside &= (coords[a] >= 0) & (coords[a] <= shape[a] - 1)
        assert np.array_equal(m == 1, inside)


# --------------------------------------------------------- A3 similarity ---

def test_mse_textbook_and_identical():
    """Eq. (mse) over the masked points; zero for identical images."""
    g = np.random.default_rng(6)
    F = g.normal(size=(9, 10, 11))
    W = g.normal(size=F.shape)
    m = (g.uniform(size=F.shape) > 0.2).astype(np.uint8)
    S, gw = oracle.similarity(oracle.MSE, F, W, m)
    assert S == pytest.approx(np.mean((W - F)[m == 1] ** 2), rel=1e-13)
    np.testing.assert_allclose(gw, 2 * m * (W - F) / m.sum(), atol=1e-15)
    S0, g0 = oracle.similarity(oracle.MSE, F, F, m)
    assert S0 == 0.0 and np.all(g0 == 0.0)


def test_ncc_matches_pearson():
    """NCC (Sec. III-B) read as Pearson over the mask: compare with numpy's
    corrcoef (eps = 0), and rho(F, aF+b) = sign(a)."""
    g = np.random.default_rng(7)
    F = g.normal(size=(9, 10, 11))
    W = 0.6 * F + g.normal(size=F.shape)
    m = (g.uniform(size=F.shape) > 0.3).astype(np.uint8)
    S, _ = oracle.similarity(oracle.NCC, F, W, m, eps=0.0)
    rho = np.corrcoef(F[m == 1], W[m == 1])[0, 1]
    assert S == pytest.approx(1.0 - rho, abs=1e-13)
    S1, g1 = oracle.similarity(oracle.NCC, F, 3.0 * F + 2.0, m, eps=0.0)
    assert S1 == pytest.approx(0.0, abs=1e-13)
    assert np.abs(g1).max() < 1e-13
    S2, _ = oracle.similarity(oracle.NCC, F, -0.5 * F + 1.0, m, eps=0.0)
    assert S2 == pytest.approx(2.0, abs=1e-13)


def test_lcc_huge_window_is_zero_padded_pearson():
    """LCC (Sec. III-B) with a window wider than twice the grid: every window
    covers the whole grid plus zero padding, so rho(x) is the Pearson
    correlation of the images extended by n - |X| zeros (numpy)."""
    g = np.random.default_rng(8)
    for shape, w in (((5, 6, 7), 15), ((9, 8), 19)):
        F = g.normal(size=shape) + 0.3
        W = 0.5 * F + g.normal(size=shape)
        m = np.ones(shape, dtype=np.uint8)
        S, _ = oracle.similarity(oracle.LCC, F, W, m, eps=0.0, window=w)
        n = w ** len(shape)
        pad = n - F.size
        rho = np.corrcoef(np.concatenate([F.ravel(), np.zeros(pad)]),
                          np.concatenate([W.ravel(), np.zeros(pad)]))[0, 1]
        assert S == pytest.approx(1.0 - rho, abs=1e-12)


def test_lcc_windows_match_pearson_brute_force():
    """LCC (Sec. III-B) on tiny grids with windows that differ from voxel to
    voxel: at every masked voxel rho is numpy's Pearson correlation of the
    w^d window samples of F and the masked W, read from zero-padded copies
    (eps = 0); S = 1 - mean over the mask. dS/dW matches central differences
    of S in W at masked voxels."""
    g = np.random.default_rng(11)
    for shape, w in (((7, 9), 3), ((7, 9), 5), ((4, 5, 6), 3)):
        r = w // 2
        F = g.normal(size=shape)
        W = 0.6 * F + g.normal(size=shape)
        m = (g.uniform(size=shape) > 0.25).astype(np.uint8)
        S, gw = oracle.similarity(oracle.LCC, F, W, m, eps=0.0, window=w)
        Fp = np.pad(F, r)
        Wp = np.pad(W * m, r)
        rhos = []
        for idx in zip(*np.nonzero(m)):
            win = tuple(slice(i, i + w) for i in idx)
            rhos.append(np.corrcoef(Fp[win].ravel(), Wp[win].ravel())[0, 1])
        assert S == pytest.approx(1.0 - np.mean(rhos), abs=1e-12)
        h = 1e-6
        for idx in list(zip(*np.nonzero(m)))[::7]:
            Wa, Wb = W.copy(), W.copy()
            Wa[idx] += h
            Wb[idx] -= h
            Sa, _ = oracle.similarity(oracle.LCC, F, Wa, m, eps=0.0, window=w)
            Sb, _ = oracle.similarity(oracle.LCC, F, Wb, m, eps=0.0, window=w)
            assert gw[idx] == pytest.approx((Sa - Sb) / (2 * h), rel=1e-5, abs=1e-8)


def test_lcc_identical_images():
    """Identical images: every local correlation is 1, S = 0, gradient 0 (eps = 0)."""
    g = np.random.default_rng(9)
    F = g.normal(size=(8, 9, 10))
    m = np.ones(F.shape, dtype=np.uint8)
    S, gw = oracle.similarity(oracle.LCC, F, F, m, eps=0.0, window=5)
    assert S == pytest.approx(0.0, abs=1e-12)
    assert np.abs(gw).max() < 1e-10


def test_lcc_window_of_one_point():
    """A 1-voxel window has zero local variance: rho = 0 / sqrt(eps) = 0."""
    g = np.random.default_rng(10)
    F = g.normal(size=(5, 6))
    m = np.ones(F.shape, dtype=np.uint8)
    S, _ = oracle.similarity(oracle.LCC, F, F + 1.0, m, eps=1e-5, window=1)
    assert S == pytest.approx(1.0, abs=1e-9)


# ------------------------------------------------------- A4 regulariser ---

def test_diffusion_constant_and_affine_closed_form():
    """Eq. (diffusion_regularizer), forward differences, Neumann end: a constant
    field gives 0; u_i = sum_k A_ik x_k gives R = sum_ik A_ik^2 (N_k-1)/N_k."""
    for shape in ((9, 10, 11), (13, 11)):
        nd = len(shape)
        R0, g0 = oracle.diffusion(np.full((nd,) + shape, 3.25))
        assert R0 == 0.0 and np.all(g0 == 0.0)
        A = np.random.default_rng(11).normal(size=(nd, nd))
        xs = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")[::-1]
        u = np.stack([sum(A[i, k] * xs[k] for k in range(nd)) for i in range(nd)])
        R, _ = oracle.diffusion(u)
        Nk = shape[::-1]
        want = sum(A[i, k] ** 2 * (Nk[k] - 1) / Nk[k] for i in range(nd) for k in range(nd))
        assert R == pytest.approx(want, rel=1e-13)


def test_diffusion_gradient_fd():
    g = np.random.default_rng(12)
    u = g.normal(size=(3, 4, 5, 6))
    R, gu = oracle.diffusion(u)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 2, 3, 4), (2, 3, 4, 5), (0, 1, 0, 5), (2, 0, 4, 0)]:
        up, um = u.copy(), u.copy()
        up[idx] += h
        um[idx] -= h
        fd = (oracle.diffusion(up)[0] - oracle.diffusion(um)[0]) / (2 * h)
        assert fd == pytest.approx(gu[idx], rel=1e-7, abs=1e-10)


# ------------------------------------------------ A5-A7 full gradient (FD) ---

def _fd_case(shape, delta, seed, sigma_c=0.35):
    nd = len(shape)
    if nd == 2:
        blobs = synth.blob_scene(shape, 6, (2.0, 4.0), seed)
    else:
        blobs = synth.blob_scene(shape, 8, (1.5, 3.0), seed)
    F = synth.render_blobs(shape, blobs)
    field = synth.smooth_field(shape, 0.8, seed + 1, min_wavelength=8.0)
    M = synth.render_blobs(shape, blobs, field)
    ns = oracle.lattice_shape(shape, delta)
    c = synth.random_ctrl(ns, nd, sigma_c, seed + 2).astype(np.float64)
    return F, M, c


def _kink_and_face_distance(shape, delta, c):
    u = oracle.displacement(shape, delta, c)
    nd = len(shape)
    xs = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")[::-1]
    dmin = np.inf
    for k in range(nd):
        y = xs[k] + u[k]
        frac = y - np.floor(y)
        dmin = min(dmin, float(np.min(np.minimum(frac, 1 - frac))))
    return dmin


@pytest.mark.parametrize("kind,shape,delta,window", [
    (oracle.MSE, (11, 13), 4, 7),
    (oracle.NCC, (11, 13), 4, 7),
    (oracle.LCC, (11, 13), 4, 5),
    (oracle.MSE, (7, 8, 9), 3, 7),
    (oracle.NCC, (7, 8, 9), 3, 7),
    (oracle.LCC, (7, 8, 9), 3, 3),
])
def test_objective_gradient_central_differences(kind, shape, delta, window):
    """Sec. III-A: the gradient is exact. Central differences of J (h = 1e-6)
    against the analytic chain rule, for every control coefficient, with the
    field kept away from interpolation kinks (no sample within 2e-5 voxel of
    an integer coordinate or face, so no sample crosses one under +-h)."""
    seed = 40 + 10 * kind
    while True:  # deterministic: first seed whose samples avoid every kink
        F, M, c = _fd_case(shape, delta, seed)
        if _kink_and_face_distance(shape, delta, c) > 2e-5:
            break
        seed += 1
    lam = 0.1
    vals, g = oracle.objective_grad(kind, F, M, c, delta, lam, eps=1e-5, window=window)
    h = 1e-6
    fd = np.zeros_like(c)
    for idx in np.ndindex(c.shape):
        cp, cm = c.copy(), c.copy()
        cp[idx] += h
        cm[idx] -= h
        jp = oracle.objective_grad(kind, F, M, cp, delta, lam, eps=1e-5, window=window, grad=False)[0]["J"]
        jm = oracle.objective_grad(kind, F, M, cm, delta, lam, eps=1e-5, window=window, grad=False)[0]["J"]
        fd[idx] = (jp - jm) / (2 * h)
    scale = np.abs(g).max()
    assert scale > 0
    assert np.abs(fd - g).max() <= 2e-6 * scale
    assert vals["J"] == pytest.approx(vals["S"] + lam * vals["R"], rel=1e-15)


def test_zero_gradient_at_identity_for_identical_images():
    """c = 0 and F = M: W = F, S_MSE = 0, R = 0 and dJ/dc = 0."""
    shape, delta = (9, 10, 11), 4
    F = np.random.default_rng(13).normal(size=shape)
    c = np.zeros((3,) + oracle.lattice_shape(shape, delta))
    vals, g = oracle.objective_grad(oracle.MSE, F, F, c, delta, 0.1)
    assert vals["J"] == 0.0 and np.all(g == 0.0)
    assert vals["n_mask"] == F.size
