"""Pins of the oracle of the learned initialisation (oracle/initnet.py and
oracle/initnet_oracle.c).

Each pin comes from outside the oracle's own code: SciPy's n-dimensional
correlation and PyTorch's conv3d (float64) for the forward layer, the
adjoint identities <A x, y> = <x, A^T y> for the input and weight adjoints,
central differences of the whole network and of the field loss, and the
partition of unity of the cubic B-spline for the loss's closed form.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
from oracle import initnet

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _rng(seed):
    return np.random.default_rng(seed)


def _layer_case(seed, nb, dims, cin, cout):
    g = _rng(seed)
    x = g.normal(0, 1, (nb,) + tuple(dims) + (cin,))
    w = g.normal(0, 1, (cout, 27, cin))
    b = g.normal(0, 1, cout)
    return x, w, b


CASES = [  # (nb, (D, H, W), cin, cout, stride)
    (1, (5, 6, 7), 2, 3, 1),
    (2, (5, 6, 7), 3, 2, 2),
    (1, (8, 4, 6), 4, 5, 2),
    (2, (3, 3, 3), 2, 2, 1),
    (1, (1, 2, 5), 3, 4, 2),
]


@pytest.mark.parametrize("nb,dims,cin,cout,stride", CASES)
def test_conv_forward_matches_scipy_correlate(nb, dims, cin, cout, stride):
    """Stride 1: the sum over input channels of SciPy's zero-padded 3x3x3
    correlation; stride 2: the same sampled at every second voxel from 0."""
    x, w, b = _layer_case(1, nb, dims, cin, cout)
    out = initnet.conv3d(x, w, b, stride, relu=False)
    for n in range(nb):
        for co in range(cout):
            acc = np.full(dims, b[co])
            for ci in range(cin):
                k = w[co, :, ci].reshape(3, 3, 3)
                acc = acc + ndi.correlate(x[n, ..., ci], k, mode="constant", cval=0.0)
            want = acc[::stride, ::stride, ::stride]
            np.testing.assert_allclose(out[n, ..., co], want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("nb,dims,cin,cout,stride", CASES)
def test_conv_forward_matches_torch_conv3d(nb, dims, cin, cout, stride):
    torch = pytest.importorskip("torch")
    x, w, b = _layer_case(2, nb, dims, cin, cout)
    out = initnet.conv3d(x, w, b, stride, relu=True)
    xt = torch.from_numpy(np.moveaxis(x, 4, 1).copy())
    wt = torch.from_numpy(np.moveaxis(w.reshape(cout, 3, 3, 3, cin), 4, 1).copy())
    ref = torch.nn.functional.conv3d(xt, wt, torch.from_numpy(b), stride=stride, padding=1)
    ref = np.moveaxis(torch.relu(ref).numpy(), 1, 4)
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_conv_output_size_and_relu():
    x, w, b = _layer_case(3, 1, (128, 9, 2), 2, 4)
    lin = initnet.conv3d(x, w, b, 2, relu=False)
    assert lin.shape == (1, 64, 5, 1, 4)
    np.testing.assert_array_equal(initnet.conv3d(x, w, b, 2, relu=True), np.maximum(lin, 0.0))


@pytest.mark.parametrize("nb,dims,cin,cout,stride", CASES)
def test_conv_dgrad_is_the_transpose(nb, dims, cin, cout, stride):
    """<conv(x) - b, y> = <x, dgrad(y)> for random x, y."""
    x, w, b = _layer_case(4, nb, dims, cin, cout)
    lin = initnet.conv3d(x, w, np.zeros(cout), stride, relu=False)
    y = _rng(5).normal(0, 1, lin.shape)
    gx = initnet.conv3d_dgrad(y, w, x.shape, stride)
    assert abs(np.sum(lin * y) - np.sum(x * gx)) <= 1e-11 * np.sum(np.abs(lin * y)) + 1e-12


@pytest.mark.parametrize("nb,dims,cin,cout,stride", CASES)
def test_conv_wgrad_is_the_transpose(nb, dims, cin, cout, stride):
    """The layer is linear in (w, b): <conv(x; w, b), y> = <w, g_w> + <b, g_b>."""
    x, w, b = _layer_case(6, nb, dims, cin, cout)
    out = initnet.conv3d(x, w, b, stride, relu=False)
    y = _rng(7).normal(0, 1, out.shape)
    g_w, g_b = initnet.conv3d_wgrad(x, y, stride)
    lhs = np.sum(out * y)
    rhs = np.sum(w * g_w) + np.sum(b * g_b)
    assert abs(lhs - rhs) <= 1e-11 * np.sum(np.abs(out * y))
    np.testing.assert_allclose(g_b, y.sum(axis=(0, 1, 2, 3)), rtol=1e-13)


def test_head_and_upsample_adjoints():
    g = _rng(8)
    e4 = g.normal(0, 1, (2, 2, 3, 2, 4))
    n3 = (3, 5, 4)
    up = initnet._upsample(e4, n3)
    assert up.shape == (2, 3, 5, 4, 4)
    assert up[1, 2, 4, 3, 1] == e4[1, 1, 2, 1, 1]
    y = g.normal(0, 1, up.shape)
    assert np.isclose(np.sum(up * y), np.sum(e4 * initnet._upsample_adjoint(y, e4.shape[1:4])))
    shape = (24, 30, 17)  # lattice (6, 7, 6) at spacing 8; h on (3, 4, 3)
    h = g.normal(0, 1, (2, 3, 4, 3, 5))
    c = initnet.head_to_ctrl(h, shape)
    assert c.shape == (2, 3) + oracle.lattice_shape(shape, 8)
    # control point j sits at voxel 8 (j - 1): h voxel j - 1, clamped
    assert c[1, 2, 1, 1, 1] == h[1, 0, 0, 0, 2] and c[0, 0, 3, 2, 4] == h[0, 2, 1, 2, 0]
    assert c[0, 1, 0, 6, 5] == h[0, 0, 3, 2, 1]
    yc = g.normal(0, 1, c.shape)
    gh = initnet.head_to_ctrl_adjoint(yc, h.shape)
    assert np.all(gh[..., 3:] == 0)
    assert np.isclose(np.sum(c * yc), np.sum(h * gh))


def test_field_loss_closed_form_and_gradient():
    """c - c* constant per component: the field error is that constant at
    every voxel (partition of unity), so L = sum_i t_i^2 / 3."""
    shape = (17, 12, 20)
    lat = oracle.lattice_shape(shape, 8)
    t = np.array([0.5, -1.25, 2.0])
    c_true = _rng(9).normal(0, 2, (1, 3) + lat)
    c = c_true + t[None, :, None, None, None]
    loss, g = initnet.field_loss(shape, c, c_true)
    assert abs(loss - np.sum(t * t) / 3.0) < 1e-12
    c = c_true + _rng(10).normal(0, 1, c.shape)
    loss, g = initnet.field_loss(shape, c, c_true)
    h = 0.1  # the loss is quadratic in c: central differences are exact up to rounding
    for idx in [(0, 0, 2, 3, 1), (0, 2, 1, 1, 4), (0, 1, 0, 0, 0)]:
        cp, cm = c.copy(), c.copy()
        cp[idx] += h
        cm[idx] -= h
        fd = (initnet.field_loss(shape, cp, c_true)[0] - initnet.field_loss(shape, cm, c_true)[0])
        assert abs(fd / (2 * h) - g[idx]) <= 1e-9 * abs(g[idx]) + 1e-15


def _net_case(seed=11, shape=(24, 20, 28), nb=2):
    from paper_1806_09907_gb300 import synth

    shapes = [(cout, 27, cin) for cin, cout, _, _ in initnet.LAYERS]
    params = [(w.astype(np.float64), _rng(seed + k).normal(0, 0.1, cout))
              for k, ((w, _), (cout, _, _)) in enumerate(zip(synth.conv_weights(shapes, seed,
                                                                                head_scale=1.0),
                                                             shapes))]
    g = _rng(seed)
    F = g.uniform(0, 1, (nb,) + shape)
    M = g.uniform(0, 1, (nb,) + shape)
    return params, F, M


def test_network_shapes():
    params, F, M = _net_case(shape=(128, 24, 40), nb=1)
    c, acts = initnet.forward(params, F, M)
    assert acts["e1"].shape == (1, 64, 12, 20, 16)
    assert acts["e3"].shape == (1, 16, 3, 5, 48)
    assert acts["e4"].shape == (1, 8, 2, 3, 64)
    assert acts["cat"].shape == (1, 16, 3, 5, 112)
    assert acts["h"].shape == (1, 16, 3, 5, 3)
    assert c.shape == (1, 3) + oracle.lattice_shape((128, 24, 40), 8) == (1, 3, 19, 6, 8)


def test_network_backward_matches_central_differences():
    """Every layer's weights and biases, a few entries each, against central
    differences of L(c(theta)) = <c, r> for a fixed random r (h = 1e-6)."""
    params, F, M = _net_case()
    c, acts = initnet.forward(params, F, M)
    r = _rng(12).normal(0, 1, c.shape)
    grads = initnet.backward(params, acts, r)
    g = _rng(13)

    def loss(ps):
        return float(np.sum(initnet.forward(ps, F, M)[0] * r))

    h = 1e-6
    for k, ((w, b), (gw, gb)) in enumerate(zip(params, grads)):
        for which, arr, garr in (("w", w, gw), ("b", b, gb)):
            for _ in range(3):
                idx = tuple(g.integers(0, n) for n in arr.shape)
                saved = arr[idx]
                arr[idx] = saved + h
                lp = loss(params)
                arr[idx] = saved - h
                lm = loss(params)
                arr[idx] = saved
                fd = (lp - lm) / (2 * h)
                assert abs(fd - garr[idx]) <= 1e-6 * max(abs(fd), 1.0), (k, which, idx, fd,
                                                                         garr[idx])


def test_adam_flat_matches_torch_adam():
    """Three steps against torch.optim.Adam in float64 (a library routine)."""
    torch = pytest.importorskip("torch")
    g = _rng(14)
    p0 = g.normal(0, 1, 50)
    grads = [g.normal(0, 1e-2, 50) for _ in range(3)]
    pt = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t, gr in enumerate(grads, start=1):
        pt.grad = torch.tensor(gr, dtype=torch.float64)
        opt.step()
        p, m, v = initnet.adam_flat(p, gr, m, v, t, 3e-3)
    np.testing.assert_allclose(p, pt.detach().numpy(), rtol=1e-13, atol=1e-15)
