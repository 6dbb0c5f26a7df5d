"""Seeded synthetic inputs shaped like the paper's registration workloads.

This module draws the images and control-point vectors that both the CUDA
library and the FP64 oracle consume. It holds no step of the registration
method itself (no B-spline expansion, no interpolation, no similarity): the
moving image is the fixed image's *analytic* scene evaluated at displaced
coordinates x + u*(x), and u* is a band-limited random cosine field, so the
deformation never passes through either implementation under test.

Random numbers come from numpy's Philox counter-based generator, keyed by the
seed, so a seed fixes the inputs on any machine.

Scenes (the paper's DirLab / POPI CT data are not available; these stand in
for their shape class):
  * blob images: sums of isotropic Gaussian blobs with uniform random centres,
    widths and amplitudes (the 2D 128x128 and 3D 128^3 cases);
  * CT-like phantom: air at -1000 HU, a body ellipsoid at 0..40 HU, and
    rotated inner ellipsoids with values in [-1000, 1500] HU painted in order,
    plus independent N(0, noise^2) noise on each image (the 256x256x160 case).
Volumes are numpy arrays in (Z, Y, X) order ((Y, X) in 2D), x fastest.
"""
from __future__ import annotations

import numpy as np

IMAGE_SEED = 1806
FIELD_SEED = 9907


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    """Philox generator for (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=[int(seed), int(stream)]))


def _coords(shape):
    """Voxel coordinates as a list in axis order x, y[, z], each broadcastable."""
    nd = len(shape)
    axes = [np.arange(s, dtype=np.float64) for s in shape]  # (Z, Y, X) order
    grids = np.meshgrid(*axes, indexing="ij", sparse=True)
    return [grids[nd - 1 - k] for k in range(nd)]  # x first


def _field_modes(shape, seed, n_modes, min_wavelength):
    """Cosine modes of smooth_field: per component a list of (direction,
    wavelength, phase, amplitude), drawn in a fixed order."""
    nd = len(shape)
    g = rng(seed, 1)
    ext = np.array(shape[::-1], dtype=np.float64)  # sizes in x, y, z order
    modes = []
    for _ in range(nd):
        comp = []
        for _ in range(n_modes):
            direction = g.normal(size=nd)
            direction /= np.linalg.norm(direction)
            wl = g.uniform(min_wavelength, 2.0 * ext.max())
            phase = g.uniform(0.0, 2.0 * np.pi)
            amp = g.normal()
            comp.append((direction, wl, phase, amp))
        modes.append(comp)
    return modes


def smooth_field(shape, rms: float, seed: int = FIELD_SEED, n_modes: int = 8,
                 min_wavelength: float = 24.0):
    """Random smooth displacement u*(x): per component a sum of cosine modes
    with random directions, wavelengths in [min_wavelength, 2*max(shape)] and
    phases, rescaled to the requested root-mean-square (voxel units).
    Returns float64 (d, *shape), component 0 = x."""
    nd = len(shape)
    xs = _coords(shape)
    u = np.zeros((nd,) + tuple(shape), dtype=np.float64)
    for i, comp in enumerate(_field_modes(shape, seed, n_modes, min_wavelength)):
        acc = np.zeros(tuple(shape), dtype=np.float64)
        for direction, wl, phase, amp in comp:
            arg = phase
            for k in range(nd):
                arg = arg + (2.0 * np.pi / wl) * direction[k] * xs[k]
            acc = acc + amp * np.cos(arg)
        acc -= acc.mean()
        u[i] = acc * (rms / max(np.sqrt(np.mean(acc * acc)), 1e-30))
    return u


def _displaced(shape, field):
    xs = _coords(shape)
    if field is None:
        return [np.broadcast_to(x, shape) for x in xs]
    return [xs[k] + field[k] for k in range(len(shape))]


def blob_scene(shape, n_blobs: int, sigma_range, seed: int = IMAGE_SEED):
    """Parameters of a blob image: list of (centre[x,y,(z)], sigma, amplitude)."""
    g = rng(seed, 2)
    nd = len(shape)
    ext = np.array(shape[::-1], dtype=np.float64)
    blobs = []
    for _ in range(n_blobs):
        mu = g.uniform(0.0, 1.0, size=nd) * (ext - 1.0)
        sigma = g.uniform(*sigma_range)
        amp = g.uniform(0.0, 1.0)
        blobs.append((mu, sigma, amp))
    return blobs


def render_blobs(shape, blobs, field=None):
    """sum_b a_b exp(-|p - mu_b|^2 / (2 sigma_b^2)) at p = x + field(x)."""
    p = _displaced(shape, field)
    img = np.zeros(tuple(shape), dtype=np.float64)
    for mu, sigma, amp in blobs:
        r2 = 0.0
        for k in range(len(shape)):
            r2 = r2 + (p[k] - mu[k]) ** 2
        img += amp * np.exp(-r2 / (2.0 * sigma * sigma))
    return img


def _rotation(g, nd):
    q, r = np.linalg.qr(g.normal(size=(nd, nd)))
    q *= np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def ct_scene(shape, n_inner: int = 30, seed: int = IMAGE_SEED):
    """Ellipsoids of a CT-like phantom: list of (centre, semi-axes, rotation, HU),
    body first, inner ellipsoids after it in painting order. The body's
    semi-axes are (110, 90, 70) voxels on a 256x256x160 grid and scale with
    the grid; inner semi-axes are U[5, 40] voxels on that grid."""
    g = rng(seed, 3)
    nd = len(shape)
    ext = np.array(shape[::-1], dtype=np.float64)
    ref = np.array([256.0, 256.0, 160.0][:nd])
    scale = ext / ref
    centre = (ext - 1.0) / 2.0
    body_axes = np.array([110.0, 90.0, 70.0][:nd]) * scale
    items = [(centre, body_axes, np.eye(nd), g.uniform(0.0, 40.0))]
    for _ in range(n_inner):
        # centre uniformly inside 0.7 x the body ellipsoid
        while True:
            t = g.uniform(-1.0, 1.0, size=nd)
            if np.sum(t * t) <= 1.0:
                break
        c = centre + 0.7 * t * body_axes
        axes = g.uniform(5.0, 40.0, size=nd) * float(scale.min())
        rot = _rotation(g, nd)
        hu = g.uniform(-1000.0, 1500.0)
        items.append((c, axes, rot, hu))
    return items


def render_ct(shape, items, field=None, background=-1000.0):
    """Paint the ellipsoids in order at p = x + field(x)."""
    nd = len(shape)
    p = _displaced(shape, field)
    img = np.full(tuple(shape), background, dtype=np.float64)
    umax = 0.0 if field is None else float(np.abs(field).max())
    for c, axes, rot, hu in items:
        # restrict to voxels whose displaced point can reach the bounding box
        rmax = float(axes.max())
        lo = [max(0, int(np.floor(c[k] - rmax - umax)) - 1) for k in range(nd)]
        hi = [min(shape[nd - 1 - k], int(np.ceil(c[k] + rmax + umax)) + 2) for k in range(nd)]
        if any(h <= l for l, h in zip(lo, hi)):
            continue
        sl = tuple(slice(lo[k], hi[k]) for k in reversed(range(nd)))
        d = [np.broadcast_to(p[k], shape)[sl] - c[k] for k in range(nd)]
        q = 0.0
        for a in range(nd):
            comp = 0.0
            for k in range(nd):
                comp = comp + rot[k, a] * d[k]
            q = q + (comp / axes[a]) ** 2
        region = img[sl]
        region[q <= 1.0] = hu
    return img


def random_ctrl(lattice_shape, ndim: int, sigma: float, seed: int = FIELD_SEED):
    """Control coefficients ~ N(0, sigma^2) voxels, float32 (d, *lattice_shape)."""
    g = rng(seed, 4)
    return (sigma * g.standard_normal(size=(ndim,) + tuple(lattice_shape))).astype(np.float32)


# --------------------------------------------------------------------------
# Workloads. Each returns float32 (fixed, moving).
# --------------------------------------------------------------------------

def blob_pair(shape, n_blobs, sigma_range, field_rms, seed=IMAGE_SEED, field_seed=FIELD_SEED):
    blobs = blob_scene(shape, n_blobs, sigma_range, seed)
    fixed = render_blobs(shape, blobs)
    field = smooth_field(shape, field_rms, field_seed, min_wavelength=4.0 * 8)
    moving = render_blobs(shape, blobs, field)
    return fixed.astype(np.float32), moving.astype(np.float32)


def blobs_2d_128(seed=IMAGE_SEED):
    """2D 128x128, 20 blobs, sigma 4..16 px, moving deformed by ~2 px."""
    return blob_pair((128, 128), 20, (4.0, 16.0), 2.0, seed)


def blobs_3d_128(seed=IMAGE_SEED):
    """3D 128^3, 60 blobs, sigma 3..12 voxels, moving deformed by ~2 voxels."""
    return blob_pair((128, 128, 128), 60, (3.0, 12.0), 2.0, seed)


def ct_pair(shape=(160, 256, 256), noise=20.0, field_rms=3.0, seed=IMAGE_SEED,
            field_seed=FIELD_SEED, n_inner=30):
    """CT-like phantom pair (default 256x256x160): fixed = P + noise,
    moving = P(x + u*) + independent noise, u* of ~3 voxels rms."""
    items = ct_scene(shape, n_inner, seed)
    fixed = render_ct(shape, items)
    field = smooth_field(shape, field_rms, field_seed, min_wavelength=4.0 * 6)
    moving = render_ct(shape, items, field)
    g = rng(seed, 5)
    fixed += noise * g.standard_normal(size=fixed.shape)
    moving += noise * g.standard_normal(size=moving.shape)
    return fixed.astype(np.float32), moving.astype(np.float32)


def batch_sizes(n2d: int = 32, n3d: int = 32):
    """Shapes of the batched workload: n2d 2D sizes linearly spaced from 96^2
    to 512^2 (rounded to multiples of 16) and n3d 3D sizes from 64^3 to
    192^3 (rounded to multiples of 8)."""
    s2 = [int(round(v / 16.0)) * 16 for v in np.linspace(96, 512, n2d)]
    s3 = [int(round(v / 8.0)) * 8 for v in np.linspace(64, 192, n3d)]
    return [(s, s) for s in s2] + [(s, s, s) for s in s3]


def blob_pair_device(shape, n_blobs, sigma_range, field_rms, seed=IMAGE_SEED,
                     field_seed=FIELD_SEED, device="cuda"):
    """blob_pair's recipe (same parameters from the same generators),
    evaluated in float64 with torch on `device`: for workloads too large to
    render on the host in reasonable time. Returns float32 tensors."""
    import torch

    nd = len(shape)
    axes = [torch.arange(n, dtype=torch.float64, device=device) for n in shape]
    grids = torch.meshgrid(*axes, indexing="ij")
    xs = [grids[nd - 1 - k] for k in range(nd)]  # x first
    field = []
    for comp in _field_modes(shape, field_seed, 8, 4.0 * 8):
        acc = torch.zeros(tuple(shape), dtype=torch.float64, device=device)
        for direction, wl, phase, amp in comp:
            arg = torch.full(tuple(shape), phase, dtype=torch.float64, device=device)
            for k in range(nd):
                arg = arg + (2.0 * np.pi / wl) * float(direction[k]) * xs[k]
            acc = acc + amp * torch.cos(arg)
        acc = acc - acc.mean()
        field.append(acc * (field_rms / max(float(torch.sqrt(torch.mean(acc * acc))), 1e-30)))
    blobs = blob_scene(shape, n_blobs, sigma_range, seed)

    def render(p):
        img = torch.zeros(tuple(shape), dtype=torch.float64, device=device)
        for mu, sigma, amp in blobs:
            r2 = sum((p[k] - float(mu[k])) ** 2 for k in range(nd))
            img += amp * torch.exp(-r2 / (2.0 * sigma * sigma))
        return img.to(torch.float32)

    fixed = render(xs)
    moving = render([xs[k] + field[k] for k in range(nd)])
    return fixed.contiguous(), moving.contiguous()


def batch_pairs(n2d: int = 32, n3d: int = 32, seed: int = IMAGE_SEED, device="cuda"):
    """The batched workload's (fixed, moving) pairs on `device`: blob pairs
    (20 blobs, sigma 4..16 in 2D; 60 blobs, sigma 3..12 in 3D; moving
    deformed by ~2 voxels rms), one seed per pair."""
    out = []
    for i, sh in enumerate(batch_sizes(n2d, n3d)):
        nb, sig = ((20, (4.0, 16.0)) if len(sh) == 2 else (60, (3.0, 12.0)))
        out.append(blob_pair_device(sh, nb, sig, 2.0, seed + 100 * i, FIELD_SEED + 100 * i,
                                    device))
    return out



# --------------------------------------------------------------------------
# Learned initialisation: network weights and training pairs.
# --------------------------------------------------------------------------

def conv_weights(shapes, seed: int, head_scale: float = 0.1):
    """He-normal weights for 3x3x3 convolution layers, zero biases.

    shapes: [(cout, 27, cin)] per layer, in order. Weights ~ N(0, 2/(27 cin)),
    the last layer's scaled by head_scale so that the initial prediction is
    small. Returns [(w float32 (cout, 27, cin), b float32 (cout,))]."""
    g = rng(seed, 6)
    out = []
    for k, (cout, taps, cin) in enumerate(shapes):
        std = np.sqrt(2.0 / (taps * cin))
        if k == len(shapes) - 1:
            std *= head_scale
        w = (std * g.standard_normal(size=(cout, taps, cin))).astype(np.float32)
        out.append((w, np.zeros(cout, dtype=np.float32)))
    return out


def blob_table(count: int, shape, n_blobs: int = 60, sigma_range=(3.0, 12.0), seed: int = 0):
    """Blob scenes of `count` volumes as one float32 table (count, n_blobs, 5):
    centre x, y, z (uniform in the domain), sigma (uniform in sigma_range) and
    amplitude (uniform in [0, 1]) per blob, volume i drawn from stream
    (seed, 7) in order. 3D shapes (Z, Y, X) only."""
    assert len(shape) == 3
    g = rng(seed, 7)
    t = np.empty((count, n_blobs, 5), dtype=np.float64)
    hi = np.array([shape[2] - 1, shape[1] - 1, shape[0] - 1], dtype=np.float64)
    t[:, :, 0:3] = g.uniform(0.0, 1.0, size=(count, n_blobs, 3)) * hi
    t[:, :, 3] = g.uniform(sigma_range[0], sigma_range[1], size=(count, n_blobs))
    t[:, :, 4] = g.uniform(0.0, 1.0, size=(count, n_blobs))
    return t.astype(np.float32)


def render_blob_table(shape, table):
    """Host rendering of one row of blob_table in float64:
    sum_b a_b exp(-|x - mu_b|^2 / (2 sigma_b^2)) on a (Z, Y, X) grid."""
    x, y, z = _coords(shape)
    img = np.zeros(tuple(shape), dtype=np.float64)
    for mx, my, mz, s, a in np.asarray(table, dtype=np.float64):
        r2 = (x - mx) ** 2 + (y - my) ** 2 + (z - mz) ** 2
        img += a * np.exp(-r2 / (2.0 * s * s))
    return img
