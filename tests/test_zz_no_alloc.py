"""The allocation-free similarity entry point (al_similarity_noalloc).

Callers that cannot allocate device memory (their memory belongs to another
allocator, or they have none) use this call; it takes its scratch from a
fixed array inside the library. This file runs last so that a failure here
does not hide any other test; it passes alone in a fresh process too."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1806_09907_gb300 import airgb
from paper_1806_09907_gb300 import build as airgb_build

pytestmark = pytest.mark.gpu

J_TOL, G_TOL = 1e-5, 1e-4  # the objective and gradient tolerances of the parity tests


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    airgb_build.build()
    return airgb.load()


@pytest.mark.parametrize("sim,window,shape", [
    ("mse", 7, (40, 64, 33)), ("ncc", 7, (40, 64, 33)), ("lcc", 7, (24, 40, 52)),
    ("lcc", 5, (37, 45)),
])
def test_noalloc_matches_workspace_entry_point(lib, sim, window, shape):
    """Two calls in a row through the C ABI agree with al_similarity (which
    takes a caller workspace) within the parity tolerances."""
    rng = np.random.default_rng(77)
    F = (rng.normal(size=shape) * 30.0 - 700.0).astype(np.float32)
    m = (rng.uniform(size=shape) > 0.1).astype(np.uint8)
    W = ((0.8 * F + rng.normal(size=shape) * 20.0 - 100.0) * m).astype(np.float32)
    Fd, Wd, md = (torch.from_numpy(a).cuda() for a in (F, W, m))
    v_ref, g_ref = airgb.al_similarity(sim, Fd, Wd, md, eps=1e-5, window=window)
    v_ref, g_ref = v_ref.cpu().numpy(), g_ref.cpu().numpy()
    for _ in range(2):
        v, g = airgb.al_similarity_noalloc(sim, Fd, Wd, md, eps=1e-5, window=window)
        torch.cuda.synchronize()
        v, g = v.cpu().numpy(), g.cpu().numpy()
        assert v[1] == v_ref[1]
        assert abs(v[0] - v_ref[0]) <= J_TOL * abs(v_ref[0])
        assert rel_l2(g, g_ref) <= G_TOL


def test_noalloc_rejects_problems_beyond_the_scratch(lib):
    limit = lib.al_noalloc_scratch_bytes()
    assert limit == 4 << 20
    g = airgb.make_grid((64, 128, 128))  # LCC needs 12 bytes per voxel of scratch
    p = airgb.al_sim_params()
    p.kind, p.lcc_window, p.eps = airgb.AL_SIM_LCC, 7, 1e-5
    assert lib.al_similarity_workspace_bytes(ctypes.byref(g), ctypes.byref(p)) > limit
    dummy = ctypes.c_void_p(0x10000)
    st = lib.al_similarity_noalloc(ctypes.byref(g), ctypes.byref(p), dummy, dummy, dummy, dummy,
                                   dummy, None)
    assert st == 9
    assert "scratch" in airgb.status_string(st)
