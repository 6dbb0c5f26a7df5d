"""The seeded synthetic inputs follow their stated recipe (host only).

The generators stand in for the paper's CT and 2D data: blob images, a
CT-like phantom with noise, band-limited deformations and random control
coefficients. These tests pin what the recipe fixes: determinism per seed,
the value ranges and counts, the noise level and the deformation's rms."""
import numpy as np
import pytest

from paper_1806_09907_gb300 import synth


def test_generators_are_deterministic_per_seed():
    a = synth.ct_pair((12, 24, 20), n_inner=5)
    b = synth.ct_pair((12, 24, 20), n_inner=5)
    c = synth.ct_pair((12, 24, 20), n_inner=5, seed=synth.IMAGE_SEED + 1)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0])
    assert np.array_equal(synth.random_ctrl((4, 5, 6), 3, 3.0), synth.random_ctrl((4, 5, 6), 3, 3.0))
    assert np.array_equal(synth.blob_table(3, (8, 9, 10)), synth.blob_table(3, (8, 9, 10)))


@pytest.mark.parametrize("shape,rms", [((40, 48), 2.0), ((16, 20, 24), 3.0)])
def test_smooth_field_rms_and_zero_mean(shape, rms):
    u = synth.smooth_field(shape, rms, min_wavelength=24.0)
    assert u.shape == (len(shape),) + shape
    for comp in u:
        assert np.sqrt(np.mean(comp * comp)) == pytest.approx(rms, rel=1e-12)
        assert abs(comp.mean()) < 1e-12


def test_blob_scene_ranges():
    shape = (30, 40, 50)
    blobs = synth.blob_scene(shape, 60, (3.0, 12.0))
    assert len(blobs) == 60
    for mu, sigma, amp in blobs:
        assert np.all(mu >= 0) and np.all(mu <= np.array(shape[::-1]) - 1)
        assert 3.0 <= sigma <= 12.0 and 0.0 <= amp <= 1.0
    t = synth.blob_table(4, shape, 60)
    assert t.shape == (4, 60, 5) and t.dtype == np.float32
    hi = np.array([shape[2] - 1, shape[1] - 1, shape[0] - 1])
    assert np.all(t[..., :3] >= 0) and np.all(t[..., :3] <= hi)
    assert np.all((t[..., 3] >= 3.0) & (t[..., 3] <= 12.0))
    assert np.all((t[..., 4] >= 0.0) & (t[..., 4] <= 1.0))
    # the table renders to the sum of its blobs (a blob at its own centre
    # contributes its amplitude)
    one = np.zeros((1, 1, 5), dtype=np.float32)
    one[0, 0] = (7.0, 5.0, 3.0, 2.0, 0.75)
    img = synth.render_blob_table(shape, one[0])
    assert img[3, 5, 7] == pytest.approx(0.75) and img.max() == pytest.approx(0.75)


def test_ct_scene_recipe():
    items = synth.ct_scene((160, 256, 256))
    assert len(items) == 31
    c, axes, rot, hu = items[0]
    assert np.allclose(axes, (110.0, 90.0, 70.0)) and np.allclose(rot, np.eye(3))
    assert 0.0 <= hu <= 40.0
    for c, axes, rot, hu in items[1:]:
        assert -1000.0 <= hu <= 1500.0
        assert np.all((axes >= 5.0) & (axes <= 40.0))
        assert np.allclose(rot @ rot.T, np.eye(3)) and np.linalg.det(rot) == pytest.approx(1.0)


def test_ct_pair_background_and_noise():
    """Air at -1000 HU outside the body, and N(0, 20^2) noise on the fixed
    image: the corners of a small phantom are background plus noise."""
    shape = (20, 48, 40)
    F, M = synth.ct_pair(shape, n_inner=4)
    assert F.dtype == np.float32 and F.shape == shape and M.shape == shape
    P = synth.render_ct(shape, synth.ct_scene(shape, 4))
    noise = F.astype(np.float64) - P
    assert noise.mean() == pytest.approx(0.0, abs=1.0)
    assert noise.std() == pytest.approx(20.0, rel=0.05)
    corner = P[:3, :3, :3]
    assert np.all(corner == -1000.0)


def test_random_ctrl_and_batch_sizes():
    c = synth.random_ctrl((30, 46, 46), 3, 3.0)
    assert c.dtype == np.float32 and c.shape == (3, 30, 46, 46)
    assert c.std() == pytest.approx(3.0, rel=0.01) and abs(c.mean()) < 0.02
    sizes = synth.batch_sizes()
    assert len(sizes) == 64
    s2 = [s for s in sizes if len(s) == 2]
    s3 = [s for s in sizes if len(s) == 3]
    assert len(s2) == 32 and len(s3) == 32
    assert s2[0] == (96, 96) and s2[-1] == (512, 512) and all(s[0] % 16 == 0 for s in s2)
    assert s3[0] == (64, 64, 64) and s3[-1] == (192, 192, 192) and all(s[0] % 8 == 0 for s in s3)


def test_conv_weights_he_normal():
    shapes = [(16, 27, 2), (32, 27, 16), (3, 27, 48)]
    ws = synth.conv_weights(shapes, seed=5, head_scale=0.1)
    for k, ((w, b), (cout, taps, cin)) in enumerate(zip(ws, shapes)):
        assert w.shape == (cout, taps, cin) and w.dtype == np.float32
        assert np.all(b == 0)
        std = np.sqrt(2.0 / (taps * cin)) * (0.1 if k == len(shapes) - 1 else 1.0)
        assert w.std() == pytest.approx(std, rel=0.15)
