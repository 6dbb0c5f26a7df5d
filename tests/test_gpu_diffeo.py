"""The diffeomorphic B-spline model on the GPU (Sec. III-D, f = exp(v) by
scaling and squaring) against the FP64 oracle.

Tolerances: the exponential within 1e-5 * max|v| (fp32 rounding of K
squarings, each interpolating the previous field); its adjoint and the
objective's gradient within rel-L2 1e-4 and J within rel 1e-5, the hot
path's bars. The adjoint's scatter is summed in fixed point, so two runs
are bit-identical.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1806_09907_gb300 import airgb, registration, synth
from paper_1806_09907_gb300 import build as airgb_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    airgb_build.build()
    return airgb.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def velocity(shape, rms, seed):
    return synth.smooth_field(shape, rms, seed, min_wavelength=12.0).astype(np.float32)


SHAPES = [(37, 45), (64, 29), (21, 26, 40), (33, 17, 24)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("steps", [0, 1, 6])
def test_exp_field_matches_oracle(shape, steps):
    v = velocity(shape, 2.0, 3)
    u = host(airgb.al_exp_field(dev(v), steps))
    ref = oracle.exp_field(v, steps)
    assert np.abs(u - ref).max() <= 1e-5 * np.abs(v).max()
    # with a trajectory the result is the same, bit for bit
    u2, traj = airgb.al_exp_field(dev(v), steps, trajectory=True)
    np.testing.assert_array_equal(host(u2), u)
    assert traj.shape[0] == steps


@pytest.mark.parametrize("shape", SHAPES)
def test_exp_adjoint_matches_oracle_and_is_deterministic(shape):
    nd = len(shape)
    v = velocity(shape, 2.0, 5)
    g = np.random.default_rng(6).normal(size=(nd,) + shape).astype(np.float32)
    K = 6
    _, traj = airgb.al_exp_field(dev(v), K, trajectory=True)
    gv = airgb.al_exp_field_adjoint(traj, dev(g), K)
    gv2 = airgb.al_exp_field_adjoint(traj, dev(g), K)
    assert torch.equal(gv, gv2)
    _, traj_ref = oracle.exp_field(v, K, trajectory=True)
    ref = oracle.exp_field_adjoint(traj_ref, g, K)
    assert rel_l2(host(gv).astype(np.float64), ref) <= 1e-4


def test_exp_of_constant_velocity_is_the_translation():
    shape = (20, 24, 28)
    v = np.empty((3,) + shape, dtype=np.float32)
    v[0], v[1], v[2] = 1.25, -0.75, 2.5
    u = host(airgb.al_exp_field(dev(v), 6))
    assert np.abs(u - v).max() <= 1e-6


@pytest.mark.parametrize("shape,delta,sim", [((37, 45), 4, "mse"), ((24, 40, 52), 6, "mse"),
                                             ((24, 40, 52), 6, "lcc"), ((21, 26, 40), 6, "ncc")])
def test_diffeo_objective_matches_oracle(shape, delta, sim):
    nd = len(shape)
    F, M = synth.ct_pair(shape, n_inner=8) if nd == 3 else synth.blob_pair(shape, 12, (3.0, 8.0),
                                                                          2.0)
    c = synth.random_ctrl(oracle.lattice_shape(shape, delta), nd, 1.0, 41)
    pr = airgb.make_problem(shape, delta, sim, 0.1)
    K = 6
    val, g = airgb.al_objective_grad_diffeo(pr, dev(F), dev(M), dev(c), K)
    val, g = host(val), host(g).astype(np.float64)
    kind = airgb.SIM_KINDS[sim]
    ref, gref = oracle.objective_grad_diffeo(kind, F, M, c, delta, 0.1, K)
    assert abs(val[0] - ref["J"]) <= 1e-5 * abs(ref["J"]), (val[0], ref["J"])
    assert val[3] == ref["n_mask"]
    assert rel_l2(g, gref) <= 1e-4


def test_diffeo_at_zero_velocity_is_the_plain_objective():
    shape, delta = (24, 40, 52), 6
    F, M = synth.ct_pair(shape, n_inner=8)
    c = np.zeros((3,) + oracle.lattice_shape(shape, delta), dtype=np.float32)
    pr = airgb.make_problem(shape, delta, "mse", 0.1)
    vd, gd = airgb.al_objective_grad_diffeo(pr, dev(F), dev(M), dev(c), 6)
    vp, gp = airgb.al_objective_grad(pr, dev(F), dev(M), dev(c))
    assert abs(host(vd)[0] - host(vp)[0]) <= 1e-6 * abs(host(vp)[0])
    # at v = 0 the exponential's derivative is the identity
    assert rel_l2(host(gd).astype(np.float64), host(gp).astype(np.float64)) <= 1e-5


def test_diffeo_registration_descends():
    shape, delta = (40, 64, 64), 6
    F, M = synth.ct_pair(shape, seed=61, field_seed=62, n_inner=10, field_rms=2.0)
    r = registration.register(dev(F), dev(M), spacing=delta, sim="mse", factors=(2, 1),
                              iterations=(20, 20), diffeo_steps=6)
    fin = host(r.levels[-1].values)
    assert fin[-1, 0] < fin[0, 0]
