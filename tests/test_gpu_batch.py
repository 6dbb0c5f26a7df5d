"""The persistent batch kernel: many MSE registrations of uneven sizes (2D and
3D mixed) in one launch per iteration.

The batch runs the per-item arithmetic of the single-problem kernels, so
each problem's coefficients after K Adam iterations must equal, bit for
bit, those of al_objective_grad + al_adam_step run on that problem alone
(which the parity suite ties to the FP64 oracle). J is compared within
fp32 rounding only: the batch's blocks are larger, so its per-thread fp32
sums of R's tile shares group the points differently.
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


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


SHAPES = [(40, 56), (96, 72), (129, 33), (33, 40, 29), (24, 48, 64), (57, 30, 41)]


def pairs_for(shapes, seed=7):
    out = []
    for i, sh in enumerate(shapes):
        nb, sig = (8, (3.0, 10.0)) if len(sh) == 2 else (12, (3.0, 8.0))
        out.append(synth.blob_pair_device(sh, nb, sig, 2.0, seed + i, seed + 50 + i))
    return out


@pytest.mark.parametrize("spacing", [8, 6, 4])
def test_batch_equals_single_problem_path(spacing):
    shapes = SHAPES if spacing == 8 else SHAPES[::2]
    pairs = pairs_for(shapes)
    K = 4
    b = airgb.Batch(pairs, spacing, 0.1, history=K)
    for k in range(K):
        b.step(k + 1, k)
    assert b.status() == 0
    cs, hs, _ = registration.register_sequential(pairs, spacing, 0.1, K)
    for i in range(len(pairs)):
        assert torch.equal(b.ctrl[i], cs[i]), (i, shapes[i])
        vb, vs = host(b.values[i]), host(hs[i])[:K]
        np.testing.assert_array_equal(vb[:, 3], vs[:, 3])  # masked voxel counts
        np.testing.assert_allclose(vb[:, 1], vs[:, 1], rtol=1e-12, atol=0)  # S: FP64 sums
        np.testing.assert_allclose(vb[:, 0], vs[:, 0], rtol=1e-6, atol=0)   # J: R's fp32 shares


def test_batch_orders_and_graph_replay_agree():
    pairs = pairs_for(SHAPES, seed=11)
    K = 3
    ref = None
    for policy in range(4):
        b = airgb.Batch(pairs, 8, 0.1)
        b.set_policy(policy)
        for k in range(K):
            b.step(k + 1)
        assert b.status() == 0
        if ref is None:
            ref = [c.clone() for c in b.ctrl]
        else:
            assert all(torch.equal(a, c) for a, c in zip(ref, b.ctrl)), policy
    r = registration.register_batch(pairs, 8, 0.1, iterations=K, graph=True, tune=True)
    ms = np.array(r.tuning_ms)
    assert ms.shape == (len(r.batch.tiles()), 4) and np.all(ms > 0)
    assert (r.tile, r.policy) == np.unravel_index(int(np.argmin(ms)), ms.shape)
    if r.tile == 0:  # the single-problem path's brick: bit for bit
        assert all(torch.equal(a, c) for a, c in zip(ref, r.batch.ctrl))
    else:  # other bricks group the partial sums differently
        for a, c in zip(ref, r.batch.ctrl):
            assert float((a - c).abs().max()) <= 1e-4 * max(float(a.abs().max()), 1e-3)


def test_batch_timeout_is_reported_and_recoverable():
    """Control chunks told to wait for items that never come give up after a
    few polls, record AL_ERR_TIMEOUT and let the kernel finish; the next
    ordinary iteration runs normally."""
    pairs = pairs_for(SHAPES[:3], seed=13)
    b = airgb.Batch(pairs, 8, 0.1)
    c0 = [c.clone() for c in b.ctrl]
    b.set_wait(extra_items=1, max_polls=2000)
    b.step(1)
    assert b.status() == 6  # AL_ERR_TIMEOUT
    assert all(torch.equal(a, c) for a, c in zip(c0, b.ctrl))  # no chunk stepped
    b.set_wait()
    b.step(1)
    assert b.status() == 0
    assert not all(torch.equal(a, c) for a, c in zip(c0, b.ctrl))


def test_batch_final_objective_matches_oracle():
    """After 20 batched iterations the objective at each problem's
    coefficients (recorded by the batch before its last step, recomputed by
    the oracle at those coefficients) agrees within the hot path's bar."""
    shapes = [(40, 56), (24, 33, 29)]
    pairs = pairs_for(shapes, seed=17)
    K = 20
    b = airgb.Batch(pairs, 8, 0.1, history=K)
    c_prev = None
    for k in range(K):
        if k == K - 1:
            c_prev = [c.clone() for c in b.ctrl]
        b.step(k + 1, k)
    assert b.status() == 0
    for i, ((F, M), sh) in enumerate(zip(pairs, shapes)):
        ref, _ = oracle.objective_grad(oracle.MSE, host(F), host(M), host(c_prev[i]), 8, 0.1,
                                       grad=False)
        J = host(b.values[i])[K - 1, 0]
        assert abs(J - ref["J"]) <= 1e-5 * abs(ref["J"])
        assert host(b.values[i])[K - 1, 0] < host(b.values[i])[0, 0]


@pytest.mark.parametrize("spacing", [8, 6, 4])
def test_batch_tiles_gradient_matches_oracle(spacing):
    """Every brick tile of the batch kernel gives dJ/dc within rel L2 1e-4
    of the FP64 oracle (recovered from Adam's first moment after one step,
    as below), and the tiles agree with each other to fp32 rounding."""
    shapes = SHAPES[:2] + SHAPES[3:5]
    pairs = pairs_for(shapes, seed=17)
    rng = np.random.default_rng(5)
    starts = None
    grads = []
    tiles = airgb.Batch(pairs, spacing, 0.1).tiles()
    assert tiles[0] == ((8, 4) if spacing == 4 else (4, 3))
    for t in range(len(tiles)):
        b = airgb.Batch(pairs, spacing, 0.1)
        b.set_tile(t)
        if starts is None:
            starts = [(rng.normal(size=b.lattices[i]) * 0.7).astype(np.float32)
                      for i in range(len(pairs))]
        for i in range(len(pairs)):
            b.ctrl[i].copy_(torch.from_numpy(starts[i]))
        b.step(1)
        assert b.status() == 0
        omb1 = float(np.float32(1.0 - 0.9))
        gs = []
        for i, sh in enumerate(shapes):
            nd = len(sh)
            mm = host(b.m[i]).astype(np.float64)
            gs.append(np.stack([mm[k] / (omb1 * float(np.float32((sh[nd - 1 - k] - 1) / 2.0)))
                                for k in range(nd)]))
        grads.append(gs)
    for i, sh in enumerate(shapes):
        F, M = (host(x) for x in pairs[i])
        _, gref = oracle.objective_grad(oracle.MSE, F, M, starts[i], spacing, 0.1)
        for t in range(len(tiles)):
            rel = float(np.linalg.norm(grads[t][i] - gref) / np.linalg.norm(gref))
            assert rel <= 1e-4, (t, tiles[t], i, sh, rel)


def test_batch_gradient_matches_oracle():
    """dJ/dc of every problem of a batch against the FP64 oracle, rel L2 <=
    1e-4. The batch exposes its gradient through Adam's first moment: after
    one step from m = 0, m = (1 - beta1) * h * dJ/dc per component, with
    h = (N_k - 1)/2 the normalised-unit scale of that axis."""
    shapes = SHAPES
    pairs = pairs_for(shapes, seed=11)
    rng = np.random.default_rng(3)
    b = airgb.Batch(pairs, 8, 0.1)
    starts = []
    for i in range(len(pairs)):
        c0 = (rng.normal(size=b.lattices[i]) * 0.7).astype(np.float32)
        b.ctrl[i].copy_(torch.from_numpy(c0))
        starts.append(c0)
    b.step(1)
    assert b.status() == 0
    omb1 = np.float32(1.0 - 0.9)
    for i, sh in enumerate(shapes):
        nd = len(sh)
        hs = [np.float32((sh[nd - 1 - k] - 1) / 2.0) for k in range(nd)]
        mm = host(b.m[i]).astype(np.float64)
        g = np.stack([mm[k] / (float(omb1) * float(hs[k])) for k in range(nd)])
        F, M = (host(t) for t in pairs[i])
        ref, gref = oracle.objective_grad(oracle.MSE, F, M, starts[i], 8, 0.1)
        rel = float(np.linalg.norm(g - gref) / np.linalg.norm(gref))
        assert rel <= 1e-4, (i, sh, rel)
