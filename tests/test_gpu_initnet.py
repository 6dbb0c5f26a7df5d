"""GPU parity of the learned initialisation (tcgen05 convolution layers and
the network around them) against the FP64 oracle, through the C ABI.

Inputs of each layer are bf16 values (exact in float64) and its weights are
rounded to bf16 on the host before they reach the oracle, so both sides
compute the same sums; they differ only by the GPU's fp32 accumulation and,
for bf16 outputs, the final rounding. The per-element bounds used here
follow from that arithmetic:
  * accumulation: at most n * 2^-24 * S for a sum of n terms in fp32 in any
    order, S = the same sum of absolute values (computed by the oracle);
  * a bf16 output adds at most 2^-8 |ref| (round to nearest, 8 bits);
plus a relative L2 bound far below what a wrong index, tap or operand
layout produces.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import initnet as onet
from paper_1806_09907_gb300 import airgb, learned_init, synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

DEV = torch.device("cuda", 0)
U = 2.0 ** -24


def _bf16(a):
    """Round float64/float32 numpy values to bf16 and back to float64."""
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def _to_dev_bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV).to(torch.bfloat16)


def _np(t):
    return t.double().cpu().numpy()


# (batch, input D, H, W, cin, cout, stride): the seven layer shapes of the
# network at sizes that give several M tiles and ragged tails
LAYER_CASES = [
    (2, (19, 22, 27), 2, 16, 2),
    (2, (19, 22, 27), 16, 32, 2),
    (2, (11, 13, 9), 32, 48, 2),
    (2, (11, 13, 9), 48, 64, 2),
    (2, (9, 10, 11), 112, 48, 1),
    (2, (9, 10, 11), 48, 48, 1),
    (2, (9, 10, 11), 48, 16, 1),
]


def _layer(seed, nb, dims, cin, cout):
    g = np.random.default_rng(seed)
    x = _bf16(g.uniform(-1, 1, (nb,) + dims + (cin,)))
    w32 = (g.normal(0, 1, (cout, 27, cin)) / np.sqrt(27 * cin)).astype(np.float32)
    b = g.normal(0, 0.1, cout).astype(np.float32)
    return x, w32, b


@pytest.mark.parametrize("nb,dims,cin,cout,stride", LAYER_CASES)
@pytest.mark.parametrize("relu", [True, False])
def test_conv_forward_parity(nb, dims, cin, cout, stride, relu):
    x, w32, b = _layer(1, nb, dims, cin, cout)
    cv = airgb.make_conv(nb, dims, cin, cout, stride)
    wt = torch.from_numpy(w32).to(DEV)
    pf, _ = airgb.al_conv3d_pack(cv, wt, True, False)
    out_f32 = cout == 16 and cin == 48 and not relu
    y = airgb.al_conv3d_forward(cv, _to_dev_bf16(x), pf, torch.from_numpy(b).to(DEV), relu=relu,
                                out_f32=out_f32)
    torch.cuda.synchronize()
    wq = _bf16(w32)
    ref = onet.conv3d(x, wq, b.astype(np.float64), stride, relu)
    S = onet.conv3d(np.abs(x), np.abs(wq), np.abs(b.astype(np.float64)), stride, False)
    got = _np(y)
    n = 27 * cin
    bound = n * U * S + (0.0 if out_f32 else 2.0 ** -8 * np.abs(ref))
    err = np.abs(got - ref)
    assert np.all(err <= bound), (float(err.max()), float((err - bound).max()))
    rel = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
    # fp32 sums of 27 cin terms: rounding grows like sqrt(n) 2^-24, ~2e-6 here
    assert rel <= (1e-5 if out_f32 else 2.0 ** -8), rel


@pytest.mark.parametrize("nb,dims,cin,cout,stride", [c for c in LAYER_CASES if c[2] % 16 == 0])
def test_conv_dgrad_parity(nb, dims, cin, cout, stride):
    x, w32, _ = _layer(2, nb, dims, cin, cout)
    cv = airgb.make_conv(nb, dims, cin, cout, stride)
    osz = airgb.conv_output_size(cv)
    g = np.random.default_rng(3)
    gout = _bf16(g.normal(0, 1, (nb,) + osz + (cout,)))
    # addend from a wider tensor (as the skip gradient of the network), and a
    # ReLU factor from x
    extra = 16
    add = _bf16(g.normal(0, 0.5, (nb,) + dims + (cin + extra,)))
    wt = torch.from_numpy(w32).to(DEV)
    _, pd = airgb.al_conv3d_pack(cv, wt, False, True)
    got = _np(airgb.al_conv3d_backward_data(cv, _to_dev_bf16(gout), pd, relu_input=_to_dev_bf16(x),
                                            addend=_to_dev_bf16(add), addend_offset=extra))
    plain = _np(airgb.al_conv3d_backward_data(cv, _to_dev_bf16(gout), pd))
    torch.cuda.synchronize()
    wq = _bf16(w32)
    lin = onet.conv3d_dgrad(gout, wq, x.shape, stride)
    S = onet.conv3d_dgrad(np.abs(gout), np.abs(wq), x.shape, stride)
    n = 27 * cout
    # without addend or ReLU factor
    err = np.abs(plain - lin)
    assert np.all(err <= n * U * S + 2.0 ** -8 * np.abs(lin)), float(err.max())
    ref = (lin + add[..., extra:]) * (x > 0)
    bound = (n * U * S + np.abs(add[..., extra:])) * U * 4 + n * U * S + 2.0 ** -8 * np.abs(ref)
    err = np.abs(got - ref)
    assert np.all(err <= bound), float((err - bound).max())
    assert np.all(got[x <= 0] == 0.0)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 2.0 ** -8, rel


@pytest.mark.parametrize("nb,dims,cin,cout,stride", LAYER_CASES)
def test_conv_wgrad_parity(nb, dims, cin, cout, stride):
    x, _, _ = _layer(4, nb, dims, cin, cout)
    cv = airgb.make_conv(nb, dims, cin, cout, stride)
    osz = airgb.conv_output_size(cv)
    gout = _bf16(np.random.default_rng(5).normal(0, 1, (nb,) + osz + (cout,)))
    xd, gd = _to_dev_bf16(x), _to_dev_bf16(gout)
    gw, gb = airgb.al_conv3d_backward_weight(cv, xd, gd)
    gw2, gb2 = airgb.al_conv3d_backward_weight(cv, xd, gd)
    torch.cuda.synchronize()
    assert torch.equal(gw, gw2) and torch.equal(gb, gb2), "weight gradient not deterministic"
    ref_w, ref_b = onet.conv3d_wgrad(x, gout, stride)
    Sw, Sb = onet.conv3d_wgrad(np.abs(x), np.abs(gout), stride)
    nvox = nb * int(np.prod(osz))
    for got, ref, S in ((_np(gw), ref_w, Sw), (_np(gb), ref_b, Sb)):
        err = np.abs(got - ref)
        assert np.all(err <= (nvox + 1) * U * S), float((err - (nvox + 1) * U * S).max())
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= 1e-5, rel


# edge shapes: one voxel along an axis, batch 1, 8 input channels (no input
# adjoint), the largest N (128), a long K (256 input channels)
EDGE_CASES = [
    (1, (1, 5, 9), 16, 16, 2),
    (1, (2, 1, 3), 32, 16, 1),
    (3, (7, 6, 5), 8, 16, 2),
    (1, (6, 7, 9), 64, 128, 1),
    (1, (4, 5, 6), 256, 32, 2),
    (2, (13, 3, 17), 2, 32, 2),
]


@pytest.mark.parametrize("nb,dims,cin,cout,stride", EDGE_CASES)
def test_conv_edge_shapes(nb, dims, cin, cout, stride):
    test_conv_forward_parity(nb, dims, cin, cout, stride, relu=False)
    test_conv_wgrad_parity(nb, dims, cin, cout, stride)
    if cin % 16 == 0 and cin <= 128:
        test_conv_dgrad_parity(nb, dims, cin, cout, stride)


def test_glue_kernels_exact():
    g = np.random.default_rng(6)
    nb, n3 = 2, (5, 6, 7)
    n4 = tuple((n - 1) // 2 + 1 for n in n3)
    e4 = _bf16(g.normal(0, 1, (nb,) + n4 + (64,)))
    e3 = _bf16(g.normal(0, 1, (nb,) + n3 + (48,)))
    cat = airgb.al_initnet_upcat(_to_dev_bf16(e4), _to_dev_bf16(e3))
    ref = np.concatenate([onet._upsample(e4, n3), e3], axis=-1)
    assert np.array_equal(_np(cat), ref)
    gcat = _bf16(g.normal(0, 1, (nb,) + n3 + (112,)))
    ge4 = _np(airgb.al_initnet_upcat_adjoint(_to_dev_bf16(gcat), _to_dev_bf16(e4)))
    want = onet._upsample_adjoint(gcat[..., :64], n4) * (e4 > 0)
    assert np.all(np.abs(ge4 - want) <= 2.0 ** -8 * np.abs(want) + 8 * U * np.abs(want))
    # head <-> lattice of a 40 x 33 x 57 volume (n3 = 5 x 5 x 8)
    shape = (40, 33, 57)
    n3h = tuple((n - 1) // 8 + 1 for n in shape)
    h = g.normal(0, 1, (nb,) + n3h + (16,)).astype(np.float32)
    c = _np(airgb.al_initnet_head_to_ctrl(shape, torch.from_numpy(h).to(DEV)))
    assert np.array_equal(c, onet.head_to_ctrl(h.astype(np.float64), shape))
    gc = g.normal(0, 1, c.shape).astype(np.float32)
    gh = _np(airgb.al_initnet_head_adjoint(shape, torch.from_numpy(gc).to(DEV), h.shape))
    want = onet.head_to_ctrl_adjoint(gc.astype(np.float64), h.shape)
    assert np.all(np.abs(gh - want) <= 2.0 ** -8 * np.abs(want) + 1e-6 * np.abs(want).max())
    assert np.all(gh[..., 3:] == 0)
    # network input: bf16 pairs
    F = g.normal(0, 1, (nb,) + n3).astype(np.float32)
    M = g.normal(0, 1, (nb,) + n3).astype(np.float32)
    x = _np(airgb.al_initnet_input(torch.from_numpy(F).to(DEV), torch.from_numpy(M).to(DEV)))
    assert np.array_equal(x, np.stack([_bf16(F), _bf16(M)], axis=-1))


@pytest.mark.parametrize("shape", [(40, 33, 57), (128, 128, 128)])
def test_field_loss_parity(shape):
    nb = 2
    lat = oracle.lattice_shape(shape, 8)
    g = np.random.default_rng(7)
    c = g.normal(0, 2, (nb, 3) + lat).astype(np.float32)
    ct = g.normal(0, 2, (nb, 3) + lat).astype(np.float32)
    loss, grad = airgb.al_field_loss(shape, torch.from_numpy(c).to(DEV),
                                     torch.from_numpy(ct).to(DEV))
    ref, gref = onet.field_loss(shape, c, ct)
    assert abs(float(loss) - ref) <= 1e-5 * ref
    gg = grad.double().cpu().numpy()
    assert np.linalg.norm(gg - gref) <= 1e-5 * np.linalg.norm(gref)


@pytest.mark.parametrize("shape", [(21, 30, 17), (75, 19, 26)])
def test_render_blobs_parity(shape):
    """Boxes of 8 x 8 x 32 voxels, ragged in every axis, against the full sum
    over every blob (culled terms are below 1.6e-8 of their amplitude)."""
    table = synth.blob_table(3, shape, 12, seed=5)
    out = _np(airgb.al_render_blobs(shape, torch.from_numpy(table).to(DEV)))
    for v in range(3):
        ref = synth.render_blob_table(shape, table[v])
        assert np.max(np.abs(out[v] - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_adam_flat_parity():
    g = np.random.default_rng(8)
    n = 5000
    p = g.normal(0, 1, n).astype(np.float32)
    m = np.zeros(n, np.float32)
    v = np.zeros(n, np.float32)
    pt, mt, vt = (torch.from_numpy(a.copy()).to(DEV) for a in (p, m, v))
    step = torch.zeros(1, dtype=torch.int64, device=DEV)
    for t in range(1, 4):
        gr = g.normal(0, 1e-2, n).astype(np.float32)
        airgb.al_adam_flat(pt, torch.from_numpy(gr).to(DEV), mt, vt, step, lr=1e-3)
        # both sides step from the same fp32 state
        rp, rm, rv = onet.adam_flat(p, gr, m, v, t, 1e-3)
        gp, gm, gv = (_np(a) for a in (pt, mt, vt))
        assert np.all(np.abs(gm - rm) <= 4 * U * (np.abs(m) + np.abs(gr)) * 2)
        assert np.all(np.abs(gv - rv) <= 8 * U * (np.abs(v) + gr.astype(np.float64) ** 2))
        # the step is lr * O(1): compare it relative to lr
        assert np.all(np.abs(gp - rp) <= 1e-3 * 1e-4 + 4 * U * np.abs(p))
        p, m, v = gp.astype(np.float32), gm.astype(np.float32), gv.astype(np.float32)
    assert int(step) == 3


def test_adam_flat_pack_equals_adam_then_pack():
    """The Adam update that rewrites the packed weights leaves the parameters,
    moments and every layer's packed copies (forward only, stride-2 and
    stride-1 input adjoints) equal bit for bit to al_adam_flat followed by
    al_conv3d_pack, padding included, step after step."""
    net = learned_init.InitNet((40, 33, 45), 2, DEV, seed=3, head_scale=1.0)
    n = net.params.numel()
    ref = net.params.clone()
    m1, v1, m2, v2 = (torch.zeros_like(ref) for _ in range(4))
    s1, s2 = (torch.zeros(1, dtype=torch.int64, device=DEV) for _ in range(2))
    gen = np.random.default_rng(4)
    for _ in range(3):
        grad = torch.from_numpy(gen.normal(0, 1e-2, n).astype(np.float32)).to(DEV)
        airgb.al_adam_flat(ref, grad, m1, v1, s1, lr=1e-2)
        want = [airgb.al_conv3d_pack(cv, net.weight(k, ref), True, k > 0)
                for k, cv in enumerate(net.convs)]
        airgb.al_adam_flat_pack(net.params, grad, m2, v2, s2, net.packed_layers(), lr=1e-2)
        torch.cuda.synchronize()
        assert torch.equal(net.params, ref) and torch.equal(m1, m2) and torch.equal(v1, v2)
        for k in range(len(net.convs)):
            for got, exp in zip(net.packed[k], want[k]):
                assert (got is None) == (exp is None)
                if got is not None:
                    assert torch.equal(got, exp), k
    assert int(s1) == int(s2) == 3
    assert airgb.al_get_device_error() == 0
    # a packed copy that is not a whole pack result of its layer is refused
    # before anything launches
    bad = net.packed_layers()
    bad[2] = (bad[2][0], bad[2][1], bad[2][2][:-64], bad[2][3])
    with pytest.raises(ValueError):
        airgb.al_adam_flat_pack(net.params, grad, m2, v2, s2, bad, lr=1e-2)
    assert int(s2) == 3


def _small_net(nb=2, shape=(40, 33, 45), seed=9):
    net = learned_init.InitNet(shape, nb, DEV, seed=seed, head_scale=1.0)
    g = np.random.default_rng(seed)
    # biases non-zero so that every term of the layers is exercised
    net.params.copy_(net.params + torch.from_numpy(
        g.normal(0, 0.02, net.params.numel()).astype(np.float32)).to(DEV))
    for k, (cin, cout, used, _, _) in enumerate(learned_init.LAYERS):
        net.weight(k)[used:].zero_()
        net.bias(k)[used:].zero_()
    net.pack()
    F = torch.from_numpy(g.uniform(0, 1, (nb,) + shape).astype(np.float32)).to(DEV)
    M = torch.from_numpy(g.uniform(0, 1, (nb,) + shape).astype(np.float32)).to(DEV)
    return net, F, M


def test_network_layerwise_parity():
    """Forward and backward of the whole network: each layer's output checked
    against the oracle layer applied to the GPU's own (bf16) inputs, so the
    wiring (skip, up-sampling, head, ReLU factors) is checked exactly."""
    net, F, M = _small_net()
    c = net.forward(F, M)
    gc = torch.from_numpy(np.random.default_rng(10).normal(0, 1, tuple(c.shape))
                          .astype(np.float32)).to(DEV)
    net.backward(gc)
    torch.cuda.synchronize()
    A = {k: _np(v) for k, v in net.acts.items()}
    P = [(_bf16(w), b) for w, b in net.layer_params()]
    L = learned_init.LAYERS

    def fwd_check(k, x, got, relu):
        cin, cout, used, s, _ = L[k]
        ref = onet.conv3d(x, P[k][0], P[k][1], s, relu)
        S = onet.conv3d(np.abs(x), np.abs(P[k][0]), np.abs(P[k][1]), s, False)
        got = got[..., :used]
        bound = 27 * cin * U * S + (0 if k == 6 else 2.0 ** -8 * np.abs(ref))
        assert np.all(np.abs(got - ref) <= bound), k

    fwd_check(0, A["x"], A["e1"], True)
    fwd_check(1, A["e1"], A["e2"], True)
    fwd_check(2, A["e2"], A["e3"], True)
    fwd_check(3, A["e3"], A["e4"], True)
    assert np.array_equal(A["cat"], np.concatenate([onet._upsample(A["e4"], A["e3"].shape[1:4]),
                                                    A["e3"]], axis=-1))
    fwd_check(4, A["cat"], A["d1"], True)
    fwd_check(5, A["d1"], A["d2"], True)
    fwd_check(6, A["d2"], A["h"], False)
    assert np.array_equal(_np(c), onet.head_to_ctrl(A["h"], net.shape))

    G = _np(net.grad)
    gflat = {}
    for k in range(7):
        o = int(net.offsets[k])
        cin, cout = L[k][0], L[k][1]
        gflat[k] = (G[o:o + cout * 27 * cin].reshape(cout, 27, cin),
                    G[o + cout * 27 * cin:o + cout * 27 * cin + cout])

    def wcheck(k, x, g):
        cin, cout, used, s, _ = L[k]
        rw, rb = onet.conv3d_wgrad(x, g, s)
        Sw, Sb = onet.conv3d_wgrad(np.abs(x), np.abs(g), s)
        nvox = g.shape[0] * int(np.prod(g.shape[1:4]))
        gw, gb = gflat[k]
        assert np.all(np.abs(gw - rw) <= (nvox + 1) * U * Sw), k
        assert np.all(np.abs(gb - rb) <= (nvox + 1) * U * Sb), k

    def dcheck(k, g, got, x_relu=None, add=None):
        cin, cout, used, s, _ = L[k]
        lin = onet.conv3d_dgrad(g, P[k][0] if cout == used else np.pad(
            P[k][0], ((0, cout - used), (0, 0), (0, 0))), got.shape, s)
        S = onet.conv3d_dgrad(np.abs(g), np.abs(P[k][0]) if cout == used else np.pad(
            np.abs(P[k][0]), ((0, cout - used), (0, 0), (0, 0))), got.shape, s)
        ref = lin + (add if add is not None else 0.0)
        if x_relu is not None:
            ref = ref * (x_relu > 0)
        bound = 27 * cout * U * S + 2.0 ** -8 * np.abs(ref) + \
            (4 * U * np.abs(add) if add is not None else 0.0)
        assert np.all(np.abs(got - ref) <= bound), k

    gh = A["gh"]
    assert np.all(gh[..., 3:] == 0)
    want = onet.head_to_ctrl_adjoint(_np(gc), gh.shape)
    assert np.all(np.abs(gh - want) <= 2.0 ** -8 * np.abs(want) + 1e-6 * np.abs(want).max())
    wcheck(6, A["d2"], gh)
    dcheck(6, gh, A["gd2"], A["d2"])
    wcheck(5, A["d1"], A["gd2"])
    dcheck(5, A["gd2"], A["gd1"], A["d1"])
    wcheck(4, A["cat"], A["gd1"])
    dcheck(4, A["gd1"], A["gcat"])
    want = onet._upsample_adjoint(A["gcat"][..., :64], A["e4"].shape[1:4]) * (A["e4"] > 0)
    assert np.all(np.abs(A["ge4"] - want) <= 2.0 ** -8 * np.abs(want) + 8 * U * np.abs(want))
    wcheck(3, A["e3"], A["ge4"])
    dcheck(3, A["ge4"], A["ge3"], A["e3"], A["gcat"][..., 64:])
    wcheck(2, A["e2"], A["ge3"])
    dcheck(2, A["ge3"], A["ge2"], A["e2"])
    wcheck(1, A["e1"], A["ge2"])
    dcheck(1, A["ge2"], A["ge1"], A["e1"])
    wcheck(0, A["x"], A["ge1"])


def test_network_end_to_end_against_fp64_oracle():
    """The bf16 network against the all-FP64 oracle network on the same
    weights. A sanity check of the composition only (the layer-wise test is
    the exact parity): every activation and gradient is stored in bf16
    (2^-9 relative per rounding), the first layer's gradient passes through
    about a dozen such roundings, and a pre-activation within a rounding of
    zero flips its ReLU factor, so the bounds are percent-level."""
    net, F, M = _small_net(seed=11)
    c = net.forward(F, M)
    gc = torch.from_numpy(np.random.default_rng(12).normal(0, 1, tuple(c.shape))
                          .astype(np.float32)).to(DEV)
    net.backward(gc)
    torch.cuda.synchronize()
    P = [(_bf16(w), b) for w, b in net.layer_params()]
    ref, acts = onet.forward(P, _np(F), _np(M))
    rel = np.linalg.norm(_np(c) - ref) / np.linalg.norm(ref)
    assert rel <= 3e-2, rel
    grads = onet.backward(P, acts, _np(gc))
    G = _np(net.grad)
    for k, (gw, gb) in enumerate(grads):
        cin, cout, used, _, _ = learned_init.LAYERS[k]
        o = int(net.offsets[k])
        got = G[o:o + cout * 27 * cin].reshape(cout, 27, cin)[:used]
        rel = np.linalg.norm(got - gw) / np.linalg.norm(gw)
        assert rel <= 0.15, (k, rel)


def test_training_pairs_are_registered_by_their_coefficients():
    """F = M o (x + B c*): the objective at c* is zero wherever the mask keeps
    voxels (MSE over the mask), and positive at c = 0."""
    src = learned_init.PairSource((48, 40, 56), 2, sigma=3.0, seed=3, device=DEV)
    F, M, ct = src.make(0)
    pr = airgb.make_problem(src.shape, 8, "mse", 0.0)
    for b in range(2):
        val, _ = airgb.al_objective_grad(pr, F[b], M[b], ct[b].clone())
        val0, _ = airgb.al_objective_grad(pr, F[b], M[b], torch.zeros_like(ct[b]))
        assert float(val[1]) <= 1e-8 and float(val0[1]) > 1e-4, (float(val[1]), float(val0[1]))


def test_training_input_equals_the_pairs_input():
    """The training step's input (al_initnet_pair_input, no F in device
    memory) is the network input of the pairs make() returns, bit for bit,
    with the same c*."""
    src = learned_init.PairSource((48, 40, 56), 2, sigma=3.0, seed=3, device=DEV)
    F, M, ct = src.make(2)
    want_x = airgb.al_initnet_input(F, M)
    want_c = ct.clone()
    x = torch.empty_like(want_x)
    got_x, got_c = src.make_input(2, x)
    torch.cuda.synchronize()
    assert got_x is x
    assert torch.equal(x.view(torch.int16), want_x.view(torch.int16))
    assert torch.equal(got_c, want_c)


def test_short_training_lowers_the_loss():
    net = learned_init.InitNet((64, 64, 64), 4, DEV, seed=1)
    res = learned_init.train(net, pairs=4 * 200, lr=2e-3, sigma=4.0, seed=1)
    first, last = res.losses[:20].mean(), res.losses[-20:].mean()
    assert np.all(np.isfinite(res.losses)) and last < 0.95 * first, (first, last)
    assert airgb.al_get_device_error() == 0


def test_graph_replayed_training_equals_eager():
    """Training with the network part of each step replayed from a CUDA graph
    gives the eager loop's losses and parameters bit for bit."""
    runs = []
    for graph in (False, True):
        net = learned_init.InitNet((48, 48, 48), 2, DEV, seed=4)
        res = learned_init.train(net, pairs=2 * 5, lr=1e-3, sigma=3.0, seed=9, graph=graph)
        runs.append((res.losses, net.params.clone()))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert torch.equal(runs[0][1], runs[1][1])


@pytest.mark.parametrize("nb,dims,cin,cout,stride", [(1, (9, 10, 11), 112, 48, 1),
                                                     (1, (8, 8, 8), 48, 64, 2),
                                                     (1, (16, 16, 16), 32, 48, 2)])
def test_conv_forward_split_k(nb, dims, cin, cout, stride):
    """Layers with few output tiles split their K sum over up to 8 CTAs; the
    result agrees with the unsplit launch within the fp32 accumulation bound
    (both are sums of the same products in different orders)."""
    x, w32, b = _layer(9, nb, dims, cin, cout)
    cv = airgb.make_conv(nb, dims, cin, cout, stride)
    assert airgb.conv_forward_workspace_bytes(cv) > 0
    pf, _ = airgb.al_conv3d_pack(cv, torch.from_numpy(w32).to(DEV), True, False)
    xb, bd = _to_dev_bf16(x), torch.from_numpy(b).to(DEV)
    ys = _np(airgb.al_conv3d_forward(cv, xb, pf, bd, relu=False, out_f32=True, split=True))
    yu = _np(airgb.al_conv3d_forward(cv, xb, pf, bd, relu=False, out_f32=True, split=False))
    ys2 = _np(airgb.al_conv3d_forward(cv, xb, pf, bd, relu=False, out_f32=True, split=True))
    assert np.array_equal(ys, ys2), "split-K forward not deterministic"
    wq = _bf16(w32)
    S = onet.conv3d(np.abs(x), np.abs(wq), np.abs(b.astype(np.float64)), stride, False)
    ref = onet.conv3d(x, wq, b.astype(np.float64), stride, False)
    n = 27 * cin
    assert np.all(np.abs(ys - ref) <= n * U * S)
    assert np.all(np.abs(ys - yu) <= 2 * n * U * S)


def test_inference_graph_replay_equals_eager():
    """One-pair inference replayed from a CUDA graph (split-K layers
    included) gives the eager forward's coefficients bit for bit."""
    shape = (40, 33, 48)
    net = learned_init.InitNet(shape, 1, DEV, seed=4, head_scale=1.0)
    src = learned_init.PairSource(shape, 1, 3.0, seed=2, device=DEV)
    F, M, _ = src.make(0)
    lat = (3,) + airgb.lattice_shape(shape, 8)
    eager = net.forward(F, M, out=torch.empty((1,) + lat, device=DEV)).clone()
    out = torch.empty(lat, device=DEV)
    ms = learned_init.inference_ms(net, F[0].clone(), M[0].clone(), out)
    torch.cuda.synchronize()
    assert ms > 0 and torch.equal(out, eager[0])
