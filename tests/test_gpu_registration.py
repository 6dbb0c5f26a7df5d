"""The optimisation loop on the GPU: Adam, pyramid and refinement kernels
against the FP64 oracle, the autograd.Function (hand-written backward against
the C-ABI gradient, the oracle gradient and central differences on 1,000
control coordinates), and coarse-to-fine registration.

Tolerances come from fp32 arithmetic and are stated per test. The objective
and gradient keep the hot path's bars: J rel 1e-5, gradient rel-L2 1e-4.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1806_09907_gb300 import airgb, registration, synth
from paper_1806_09907_gb300 import build as airgb_build

pytestmark = pytest.mark.gpu

J_TOL, G_TOL = 1e-5, 1e-4


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    airgb_build.build()
    return airgb.load()


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def blobs(shape, delta, sigma_c, seed, field_rms=2.0):
    nd = len(shape)
    sc = synth.blob_scene(shape, max(4, int(np.prod(shape) ** (1 / nd) / 3)), (2.0, 6.0), seed)
    F = synth.render_blobs(shape, sc).astype(np.float32)
    field = synth.smooth_field(shape, field_rms, seed + 1, min_wavelength=4.0 * delta)
    M = synth.render_blobs(shape, sc, field).astype(np.float32)
    c = synth.random_ctrl(oracle.lattice_shape(shape, delta), nd, sigma_c, seed + 2)
    return F, M, c


# --------------------------------------------------------------- Adam -------

@pytest.mark.parametrize("shape,delta", [((37, 45), 4), ((21, 26, 40), 6), ((64, 64, 40), 6)])
def test_adam_step_matches_oracle(shape, delta):
    """Five steps with fresh gradients (spread over five decades, some exactly
    zero); before each step both sides get the same fp32 state (c, m, v). The
    fp32 update rounds each product a few times, so per element, with
    T_m = b1 |m| + (1 - b1) |g~| and T_v = b2 v + (1 - b2) g~^2 (the terms
    being added, which may cancel in m):
      |m_gpu - m_ref| <= 4e-7 T_m,   |v_gpu - v_ref| <= 4e-7 T_v,
      |dc_gpu - dc_ref| <= lr h 4e-7 T_m / bc1 / (sqrt(v^) + eps)
                           + 1e-6 |dc_ref| + 1.2e-7 |c_new|."""
    nd = len(shape)
    ls = (nd,) + oracle.lattice_shape(shape, delta)
    rng = np.random.default_rng(21)
    c = rng.normal(0, 2, ls).astype(np.float32)
    m, v = np.zeros(ls, np.float32), np.zeros(ls, np.float32)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-8
    N = shape[::-1]
    h = np.array([(N[i] - 1) / 2.0 for i in range(nd)]).reshape((nd,) + (1,) * nd)
    for t in range(1, 6):
        g = (rng.normal(0, 1, ls) * 10.0 ** rng.uniform(-6, -1, ls)).astype(np.float32)
        g.reshape(-1)[::9] = 0.0
        cg, mg, vg = dev(c), dev(m), dev(v)
        airgb.al_adam_step(shape, delta, cg, dev(g), mg, vg, step, lr=lr, betas=(b1, b2), eps=eps)
        c64, m64, v64 = c.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
        cr, mr, vr = oracle.adam_step(shape, delta, c64, g, m64, v64, t, lr=lr, betas=(b1, b2),
                                      eps=eps)
        gn = g.astype(np.float64) * h
        Tm = b1 * np.abs(m64) + (1 - b1) * np.abs(gn)
        Tv = b2 * v64 + (1 - b2) * gn * gn
        mo, vo, co = (host(x).astype(np.float64) for x in (mg, vg, cg))
        assert np.all(np.abs(mo - mr) <= 4e-7 * Tm)
        assert np.all(np.abs(vo - vr) <= 4e-7 * Tv)
        bc1, bc2 = 1 - b1 ** t, 1 - b2 ** t
        d_ref, d_gpu = cr - c64, co - c64
        bound = (lr * h * 4e-7 * Tm / bc1 / (np.sqrt(vr / bc2) + eps) + 1e-6 * np.abs(d_ref)
                 + 1.2e-7 * np.abs(cr))
        assert np.all(np.abs(d_gpu - d_ref) <= bound), np.abs(d_gpu - d_ref).max()
        c, m, v = (x.astype(np.float32) for x in (cr, mr, vr))
    assert int(host(step)[0]) == 5


def test_adam_zero_gradient_leaves_ctrl_bit_exact():
    shape, delta = (19, 23, 29), 4
    ls = (3,) + oracle.lattice_shape(shape, delta)
    c = dev(np.random.default_rng(22).normal(0, 1, ls).astype(np.float32))
    c0 = c.clone()
    z = torch.zeros_like(c)
    m, v = torch.zeros_like(c), torch.zeros_like(c)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(3):
        airgb.al_adam_step(shape, delta, c, z, m, v, step)
    assert torch.equal(c, c0) and int(host(step)[0]) == 3


# ------------------------------------------------------------ pyramid -------

@pytest.mark.parametrize("shape", [(37, 45), (23, 30, 19), (40, 64, 64)])
@pytest.mark.parametrize("factor", [1, 2, 4])
def test_pyramid_level_matches_oracle(shape, factor):
    """fp32 separable passes of at most 13 taps per axis against the FP64
    product-kernel sum: |err| <= 4e-6 * max|image|; factor 1 is a copy."""
    im = np.random.default_rng(23).uniform(-1000, 1500, shape).astype(np.float32)
    out = host(airgb.al_pyramid_level(dev(im), factor))
    ref = oracle.pyramid_level(im, factor)
    assert out.shape == ref.shape == oracle.level_shape(shape, factor)
    if factor == 1:
        np.testing.assert_array_equal(out, im)
    else:
        assert np.abs(out - ref).max() <= 4e-6 * np.abs(im).max()


# ------------------------------------------------------------- refine -------

@pytest.mark.parametrize("fine_shape,delta", [((31, 26), 4), ((26, 21, 17), 3), ((80, 128, 128), 6)])
def test_refine_matches_oracle_and_keeps_displacement(fine_shape, delta):
    nd = len(fine_shape)
    cs = oracle.level_shape(fine_shape, 2)
    cc = np.random.default_rng(24).normal(0, 3, (nd,) + oracle.lattice_shape(cs, delta))
    cc = cc.astype(np.float32)
    cf = airgb.al_bspline_refine(cs, fine_shape, delta, dev(cc))
    ref = oracle.bspline_refine(cs, fine_shape, delta, cc)
    # at most 27 products with exact weights: a few ulps of 2 * max|c|
    assert np.abs(host(cf) - ref).max() <= 1e-6 * np.abs(cc).max()
    # the refined field equals twice the coarse one at the coarse voxels
    uc = host(airgb.al_displacement(cs, delta, dev(cc)))
    uf = host(airgb.al_displacement(fine_shape, delta, cf))
    sub = (slice(None),) + tuple(slice(None, None, 2) for _ in fine_shape)
    assert np.abs(uf[sub] - 2.0 * uc).max() <= 1e-5 * np.abs(cc).max()


# ----------------------------------------------------- autograd.Function ----

@pytest.mark.parametrize("sim", ["mse", "lcc"])
@pytest.mark.parametrize("recompute", [False, True])
def test_autograd_function_matches_abi_and_oracle(sim, recompute):
    shape, delta = (24, 40, 52), 6
    F, M = synth.ct_pair(shape, n_inner=8)
    c = synth.random_ctrl(oracle.lattice_shape(shape, delta), 3, 2.0, 9907)
    ev = registration.Evaluator(shape, delta, sim, 0.1)
    Fd, Md = dev(F), dev(M)
    cd = dev(c).requires_grad_(True)
    J = registration.objective(cd, ev, Fd, Md, recompute=recompute)
    J.backward()
    value, g_abi = airgb.al_objective_grad(ev.problem, Fd, Md, dev(c))
    assert torch.equal(J.detach(), value[0]) and torch.equal(cd.grad, g_abi)
    ref, gref = oracle.objective_grad(oracle.MSE if sim == "mse" else oracle.LCC, F, M, c,
                                      delta, 0.1)
    assert abs(float(J.detach()) - ref["J"]) <= J_TOL * abs(ref["J"])
    assert rel_l2(host(cd.grad).astype(np.float64), gref) <= G_TOL


def test_autograd_chain_rule_and_no_grad_path():
    shape, delta = (33, 70), 8
    F, M, c = blobs(shape, delta, 1.0, 35)
    ev = registration.Evaluator(shape, delta, "mse", 0.1)
    Fd, Md = dev(F), dev(M)
    cd = dev(c).requires_grad_(True)
    (3.0 * registration.objective(cd, ev, Fd, Md)).backward()
    _, g = airgb.al_objective_grad(ev.problem, Fd, Md, dev(c))
    assert torch.equal(cd.grad, 3.0 * g)
    with torch.no_grad():
        J = registration.objective(dev(c), ev, Fd, Md)
    assert J.grad_fn is None and float(J) > 0


def test_autograd_fd_on_1000_coordinates():
    """3D 128^3 blob pair, spacing 8, MSE + 0.1 diffusion: central
    differences of the GPU objective at 1,000 random control coordinates
    against the hand-written backward.

    The coordinates are drawn from control points whose support stays 8
    voxels inside the grid (|u| < 5 voxels here), so no sample crosses the
    domain boundary under the perturbation: a sample that leaves the mask
    removes its whole term from the masked mean, a jump in J that central
    differences turn into an O(jump/h) error. h = 1e-2 voxel: the fp32
    objective does not resolve a much smaller h (its noise is ~1e-4 of dJ/dc
    at this h and grows as 1/h), and samples crossing a voxel face within
    +-h bend the difference by O(h) (a few 1e-4 here). Bar: rel-L2 <= 1e-3
    over the 1,000."""
    shape, delta, h = (128, 128, 128), 8, 1e-2
    F, M = synth.blob_pair(shape, 60, (3.0, 12.0), 2.0, seed=41)
    ls = oracle.lattice_shape(shape, delta)
    c = synth.random_ctrl(ls, 3, 1.0, 42)
    ev = registration.Evaluator(shape, delta, "mse", 0.1)
    Fd, Md = dev(F), dev(M)
    u = host(airgb.al_displacement(shape, delta, dev(c)))
    assert np.abs(u).max() < 5.0
    cd = dev(c).requires_grad_(True)
    registration.objective(cd, ev, Fd, Md).backward()
    g = host(cd.grad).reshape(-1).astype(np.float64)
    # point j touches voxels ((j - 3) delta, (j + 1) delta) per axis
    inner = [np.arange(4, n - 4) for n in ls]
    cand = np.array([((i * ls[0] + jz) * ls[1] + jy) * ls[2] + jx for i in range(3)
                     for jz in inner[0] for jy in inner[1] for jx in inner[2]])
    idx = np.random.default_rng(43).choice(cand, 1000, replace=False)
    c32 = c.astype(np.float32).reshape(-1)
    flat = dev(c32.copy())
    vals = torch.empty((2 * len(idx), 4), dtype=torch.float64, device="cuda")
    steps = np.empty(len(idx))
    with torch.no_grad():
        for k, i in enumerate(idx):
            # the perturbed coordinates as the fp32 values the kernels see
            cp, cm = np.float32(c32[i] + np.float32(h)), np.float32(c32[i] - np.float32(h))
            steps[k] = float(cp) - float(cm)
            for s, ci in enumerate((cp, cm)):
                flat[i] = float(ci)
                ev.evaluate(Fd, Md, flat.view(cd.shape), vals[2 * k + s], None)
            flat[i] = float(c32[i])
    J = host(vals)[:, 0].reshape(-1, 2)
    fd = (J[:, 0] - J[:, 1]) / steps
    err = rel_l2(fd, g[idx])
    print(f"FD rel-L2 over 1000 interior coordinates: {err:.3e}")
    assert err <= 1e-3


# ------------------------------------------------------ optimiser loops ------

def test_bspline_adam_loop_equals_raw_loop_and_descends():
    """20 iterations through autograd + BsplineAdam equal the raw C-ABI loop
    bit for bit, and J decreases."""
    shape, delta = (48, 56, 64), 8
    F, M = synth.blob_pair(shape, 20, (3.0, 8.0), 2.0, seed=51)
    Fd, Md = dev(F), dev(M)
    ev = registration.Evaluator(shape, delta, "mse", 0.1)
    c1 = torch.zeros(ev.lattice, dtype=torch.float32, device="cuda", requires_grad=True)
    opt = registration.BsplineAdam([c1], shape, delta, lr=0.01)
    Js = []
    for _ in range(20):
        opt.zero_grad()
        J = registration.objective(c1, ev, Fd, Md)
        J.backward()
        opt.step()
        Js.append(J.detach())
    c2 = torch.zeros(ev.lattice, dtype=torch.float32, device="cuda")
    values = torch.empty((21, 4), dtype=torch.float64, device="cuda")
    registration._level_loop(ev, Fd, Md, c2, 20, 0.01, (0.9, 0.999), 1e-8, values)()
    assert torch.equal(c1.detach(), c2)
    Js = host(torch.stack(Js))
    assert Js[-1] < 0.9 * Js[0]
    np.testing.assert_array_equal(Js, host(values)[:20, 0])


def test_graphed_autograd_iteration_equals_eager():
    """The captured forward + backward + Adam step, replayed, gives the eager
    autograd loop's coefficients bit for bit (both recompute modes)."""
    shape, delta = (48, 56, 64), 8
    F, M = synth.blob_pair(shape, 20, (3.0, 8.0), 2.0, seed=52)
    Fd, Md = dev(F), dev(M)
    ev = registration.Evaluator(shape, delta, "mse", 0.1)
    for recompute in (False, True):
        c1 = torch.zeros(ev.lattice, dtype=torch.float32, device="cuda", requires_grad=True)
        opt1 = registration.BsplineAdam([c1], shape, delta)
        Js = []
        for _ in range(12):
            opt1.zero_grad()
            J = registration.objective(c1, ev, Fd, Md, recompute=recompute)
            J.backward()
            opt1.step()
            Js.append(J.detach().clone())
        c2 = torch.zeros(ev.lattice, dtype=torch.float32, device="cuda", requires_grad=True)
        opt2 = registration.BsplineAdam([c2], shape, delta)
        it = registration.GraphedIteration(c2, ev, Fd, Md, opt2, recompute=recompute)
        Jg = [it().clone() for _ in range(12)]
        assert torch.equal(c1.detach(), c2.detach())
        assert torch.equal(torch.stack(Js), torch.stack(Jg))
        assert int(host(opt2.state[c2]["step"])[0]) == 12


def test_register_graph_equals_eager_and_descends():
    """Three-level LCC registration of a CT-like pair: the CUDA-graph replay
    gives the eager loop's result bit for bit; the finest level lowers J; the
    registered full-resolution similarity beats the unregistered one; the
    final J agrees with the oracle's J at the final coefficients. (Adam is not
    monotone: on the smallest levels of a small image its first steps, lr in
    normalised units, can exceed the misalignment that is left.)"""
    shape, delta = (40, 64, 64), 6
    F, M = synth.ct_pair(shape, seed=61, field_seed=62, n_inner=10, field_rms=2.0)
    Fd, Md = dev(F), dev(M)
    kw = dict(spacing=delta, sim="lcc", lam=0.1, factors=(4, 2, 1), iterations=(30, 20, 10))
    rg = registration.register(Fd, Md, graph=True, **kw)
    re = registration.register(Fd, Md, graph=False, **kw)
    assert torch.equal(rg.ctrl, re.ctrl)
    assert [lv.shape for lv in rg.levels] == [(10, 16, 16), (20, 32, 32), (40, 64, 64)]
    for lg, le in zip(rg.levels, re.levels):
        np.testing.assert_array_equal(host(lg.values), host(le.values))
    fin = host(rg.levels[-1].values)
    assert fin[-1, 0] < fin[0, 0]
    ev = registration.Evaluator(shape, delta, "lcc", 0.1)
    v0 = torch.empty(4, dtype=torch.float64, device="cuda")
    ev.evaluate(Fd, Md, torch.zeros_like(rg.ctrl), v0)
    assert fin[-1, 1] < host(v0)[1]
    ref, _ = oracle.objective_grad(oracle.LCC, F, M, host(rg.ctrl), delta, 0.1, grad=False)
    assert abs(fin[-1, 0] - ref["J"]) <= J_TOL * abs(ref["J"])


def test_register_adam_200_iterations_config_128():
    """The 128^3 blob workload: 200 Adam iterations of MSE + 0.1 diffusion at
    spacing 8 reduce the similarity well below its start."""
    shape, delta = (128, 128, 128), 8
    F, M = synth.blob_pair(shape, 60, (3.0, 12.0), 2.0, seed=71)
    r = registration.register(dev(F), dev(M), spacing=delta, sim="mse", lam=0.1, factors=(1,),
                              iterations=200)
    vals = host(r.levels[0].values)
    print(f"MSE {vals[0, 1]:.4e} -> {vals[-1, 1]:.4e} in {r.levels[0].ms:.1f} ms")
    assert vals[-1, 1] < 0.5 * vals[0, 1]


def test_checkpoint_resume_is_bit_identical(tmp_path):
    """A two-level registration stopped after its first level and resumed
    from the checkpoint ends with the coefficients of the uninterrupted run."""
    F, M = (dev(a) for a in synth.ct_pair((24, 40, 36), n_inner=6))
    kw = dict(spacing=6, sim="lcc", lam=0.1, factors=(2, 1), iterations=15)
    full = registration.register(F, M, **kw)
    path = str(tmp_path / "state.npz")
    part = registration.register(F, M, checkpoint=path, max_levels=1, **kw)
    ck = registration.Checkpoint.load(path)
    assert ck.levels_done == 1 and len(part.levels) == 1 and ck.shape == part.levels[0].shape
    rest = registration.register(F, M, resume=path, checkpoint=path, **kw)
    assert len(rest.levels) == 1 and rest.levels[0].factor == 1
    assert torch.equal(rest.ctrl, full.ctrl)
    assert registration.Checkpoint.load(path).levels_done == 2
