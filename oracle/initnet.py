"""FP64 oracle of the learned initialisation: a 3D convolutional
encoder-decoder mapping a fixed/moving pair to cubic B-spline coefficients.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). The paper names
learning-based registration as planned work (Sec. I, Sec. V) without a
network, so this module writes out, in double precision, the network this
library trains: its layers are the plain definitions of ``initnet_oracle.c``,
its composition is written here with numpy, and its loss is the mean squared
difference of two B-spline displacement fields (Sec. III-C), computed with
the oracle's definitional expansion and its transpose.

Network (channels last, one pair = 2 input channels F, M):

    e1 = relu(conv_s2(x,  2 -> 16))      N   -> N1 = (N - 1)//2 + 1
    e2 = relu(conv_s2(e1, 16 -> 32))     N1  -> N2
    e3 = relu(conv_s2(e2, 32 -> 48))     N2  -> N3    (voxel i of e3 sits at 8 i)
    e4 = relu(conv_s2(e3, 48 -> 64))     N3  -> N4
    a  = [up(e4), e3]                    112 channels on N3; up(e4)[z] = e4[z // 2]
    d1 = relu(conv_s1(a,  112 -> 48))
    d2 = relu(conv_s1(d1, 48 -> 48))
    h  = conv_s1(d2, 48 -> 3)            3 channels on N3 (components x, y, z)
    c[i][jz][jy][jx] = h[clamp(jz-1)][clamp(jy-1)][clamp(jx-1)][i]

with clamp(j - 1) to [0, N3 - 1]: control point j of the spacing-8 lattice
sits at voxel 8 (j - 1), which is where output voxel j - 1 of h sits; the
points beyond the grid take the nearest output.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _check, _d, _load, _p, displacement, displacement_adjoint, lattice_shape

SPACING = 8
# (input channels, output channels, stride, relu) of the seven layers, in order.
LAYERS = (
    (2, 16, 2, True),
    (16, 32, 2, True),
    (32, 48, 2, True),
    (48, 64, 2, True),
    (112, 48, 1, True),
    (48, 48, 1, True),
    (48, 3, 1, False),
)


def out_size(n: int, stride: int) -> int:
    return (n - 1) // stride + 1


def _dims(x):
    return np.array(x.shape[1:4], dtype=np.int64)


def conv3d(x, w, b, stride, relu):
    """Layer forward. x: (nb, D, H, W, cin); w: (cout, 27, cin); b: (cout,)."""
    x, w, b = _d(x), _d(w), _d(b)
    nb, cin = x.shape[0], x.shape[4]
    cout = w.shape[0]
    assert w.shape == (cout, 27, cin) and b.shape == (cout,)
    dims = _dims(x)
    out = np.zeros((nb,) + tuple(out_size(int(n), stride) for n in dims) + (cout,))
    _check(_load().alref_conv3d(nb, _p(dims, ctypes.c_int64), cin, cout, stride, _p(x), _p(w),
                                _p(b), int(bool(relu)), _p(out)), "conv3d")
    return out


def conv3d_dgrad(g_out, w, in_shape, stride):
    """Input adjoint of the layer's linear part; in_shape = (nb, D, H, W, cin)."""
    g_out, w = _d(g_out), _d(w)
    nb, cin = in_shape[0], in_shape[4]
    cout = w.shape[0]
    dims = np.array(in_shape[1:4], dtype=np.int64)
    assert g_out.shape == (nb,) + tuple(out_size(int(n), stride) for n in dims) + (cout,)
    g_in = np.zeros(tuple(in_shape))
    _check(_load().alref_conv3d_dgrad(nb, _p(dims, ctypes.c_int64), cin, cout, stride, _p(g_out),
                                      _p(w), _p(g_in)), "conv3d_dgrad")
    return g_in


def conv3d_wgrad(x, g_out, stride):
    """Weight and bias adjoints of the layer: (g_w (cout, 27, cin), g_b (cout,))."""
    x, g_out = _d(x), _d(g_out)
    nb, cin = x.shape[0], x.shape[4]
    cout = g_out.shape[4]
    dims = _dims(x)
    g_w = np.zeros((cout, 27, cin))
    g_b = np.zeros(cout)
    _check(_load().alref_conv3d_wgrad(nb, _p(dims, ctypes.c_int64), cin, cout, stride, _p(x),
                                      _p(g_out), _p(g_w), _p(g_b)), "conv3d_wgrad")
    return g_w, g_b


def _upsample(e4, n3):
    """up(e4)[z][y][x] = e4[z//2][y//2][x//2] on an n3 grid."""
    iz = np.arange(n3[0]) // 2
    iy = np.arange(n3[1]) // 2
    ix = np.arange(n3[2]) // 2
    return e4[:, iz][:, :, iy][:, :, :, ix]


def _upsample_adjoint(g, n4):
    """Transpose of _upsample: each coarse voxel sums its (up to 8) copies."""
    nb, c = g.shape[0], g.shape[4]
    out = np.zeros((nb,) + tuple(n4) + (c,))
    for z in range(g.shape[1]):
        for y in range(g.shape[2]):
            for x in range(g.shape[3]):
                out[:, z // 2, y // 2, x // 2, :] += g[:, z, y, x, :]
    return out


def _lattice_index(n_lat, n3):
    return np.clip(np.arange(n_lat) - 1, 0, n3 - 1)


def head_to_ctrl(h, shape):
    """h: (nb, N3z, N3y, N3x, >=3) -> c: (nb, 3, nz, ny, nx) on the spacing-8 lattice."""
    lat = lattice_shape(shape, SPACING)
    iz = _lattice_index(lat[0], h.shape[1])
    iy = _lattice_index(lat[1], h.shape[2])
    ix = _lattice_index(lat[2], h.shape[3])
    g = h[:, iz][:, :, iy][:, :, :, ix][..., :3]  # (nb, nz, ny, nx, 3)
    return np.ascontiguousarray(np.moveaxis(g, 4, 1))


def head_to_ctrl_adjoint(g_c, h_shape):
    """Transpose of head_to_ctrl: g_h (h_shape, zero beyond channel 2)."""
    g_h = np.zeros(h_shape)
    lat = g_c.shape[2:]
    iz = _lattice_index(lat[0], h_shape[1])
    iy = _lattice_index(lat[1], h_shape[2])
    ix = _lattice_index(lat[2], h_shape[3])
    for jz in range(lat[0]):
        for jy in range(lat[1]):
            for jx in range(lat[2]):
                g_h[:, iz[jz], iy[jy], ix[jx], :3] += g_c[:, :, jz, jy, jx]
    return g_h


def forward(params, F, M):
    """params: list of (w, b) per layer; F, M: (nb, D, H, W) volumes.

    Returns (c, acts): c (nb, 3, nz, ny, nx) and every activation needed by
    :func:`backward`."""
    F, M = _d(F), _d(M)
    if F.ndim == 3:
        F, M = F[None], M[None]
    x = np.stack([F, M], axis=-1)
    acts = {"x": x}
    a = x
    for k in range(4):
        cin, cout, s, relu = LAYERS[k]
        a = conv3d(a, params[k][0], params[k][1], s, relu)
        acts[f"e{k + 1}"] = a
    n3 = acts["e3"].shape[1:4]
    cat = np.concatenate([_upsample(acts["e4"], n3), acts["e3"]], axis=-1)
    acts["cat"] = cat
    a = cat
    for k, name in zip((4, 5, 6), ("d1", "d2", "h")):
        cin, cout, s, relu = LAYERS[k]
        a = conv3d(a, params[k][0], params[k][1], s, relu)
        acts[name] = a
    return head_to_ctrl(acts["h"], F.shape[1:]), acts


def backward(params, acts, g_c):
    """Gradients [(g_w, g_b)] of every layer for the upstream gradient g_c."""
    grads = [None] * len(LAYERS)
    g = head_to_ctrl_adjoint(_d(g_c), acts["h"].shape)
    inputs = {6: "d2", 5: "d1", 4: "cat"}
    for k in (6, 5, 4):
        cin, cout, s, relu = LAYERS[k]
        x = acts[inputs[k]]
        grads[k] = conv3d_wgrad(x, g, s)
        g = conv3d_dgrad(g, params[k][0], x.shape, s)
        if k in (6, 5):  # the producing layer had a ReLU
            g = g * (x > 0)
    n4 = acts["e4"].shape[1:4]
    c4 = LAYERS[3][1]
    g_e4 = _upsample_adjoint(g[..., :c4], n4) * (acts["e4"] > 0)
    g_e3_skip = g[..., c4:]
    g = g_e4
    for k in (3, 2, 1, 0):
        cin, cout, s, relu = LAYERS[k]
        x = acts["x"] if k == 0 else acts[f"e{k}"]
        grads[k] = conv3d_wgrad(x, g, s)
        if k == 0:
            break
        g = conv3d_dgrad(g, params[k][0], x.shape, s)
        if k == 3:
            g = g + g_e3_skip
        g = g * (x > 0)
    return grads


def field_loss(shape, c, c_true):
    """Mean over the batch of (1/(3|X|)) sum_i sum_x (u_i(x) - u*_i(x))^2 with
    u = B c and u* = B c_true (the B-spline expansion of Sec. III-C), and its
    gradient with respect to c: (1/nb) (2/(3|X|)) B^T B (c - c_true)."""
    c, c_true = _d(c), _d(c_true)
    nb = c.shape[0]
    nvox = float(np.prod(shape))
    loss, g = 0.0, np.zeros_like(c)
    for b in range(nb):
        e = displacement(shape, SPACING, c[b] - c_true[b])
        loss += float(np.sum(e * e)) / (3.0 * nvox)
        g[b] = displacement_adjoint(shape, SPACING, e) * (2.0 / (3.0 * nvox))
    return loss / nb, g / nb


def adam_flat(p, g, m, v, t, lr, betas=(0.9, 0.999), eps=1e-8):
    """One Adam step (Kingma and Ba; Sec. III-G) on a flat array at step t >= 1:
    m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
    p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). Returns (p, m, v)."""
    p, g, m, v = _d(p), _d(g), _d(m), _d(v)
    b1, b2 = betas
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
