"""Learned initialisation of the B-spline registration.

The paper names learning-based registration as planned work (Sec. I and
Sec. V) without a network. Here a small 3D convolutional encoder-decoder
predicts the cubic B-spline coefficients (spacing 8, voxel units) of a
fixed/moving pair; the plain optimiser (the objective and Adam of Sec. II-A
and III-G) then refines the prediction, starts from zero instead when the
prediction's objective is worse (the fallback), and its result measures the
prediction's error.

Network (channels last, bf16 activations, fp32 master weights, every layer a
hand-written tcgen05 kernel of libairgb):

    e1 = relu(conv_s2(x,  2 -> 16))        x = [F, M]
    e2 = relu(conv_s2(e1, 16 -> 32))
    e3 = relu(conv_s2(e2, 32 -> 48))       voxel i of e3 sits at voxel 8 i
    e4 = relu(conv_s2(e3, 48 -> 64))
    d1 = relu(conv_s1([up(e4), e3], 112 -> 48))
    d2 = relu(conv_s1(d1, 48 -> 48))
    h  = conv_s1(d2, 48 -> 3)              stored with 16 channels, 13 zero
    c[i][j] = h[clamp(j - 1)][i]           control point j sits at voxel 8 (j - 1)

Training pairs are made by the method itself: a blob volume M (Gaussian blobs
as in the paper-shaped 3D workloads), coefficients c* ~ N(0, sigma^2) and
F = M o (x + B c*) through the library's own expansion and warp, so that c*
registers M onto F exactly (J(c*) = 0 where the mask keeps voxels). The loss
is the mean squared difference of the predicted and true displacement fields.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import airgb, registration, synth

SPACING = 8
# (cin, cout stored, cout used, stride, relu) per layer, in order
LAYERS = (
    (2, 16, 16, 2, True),
    (16, 32, 32, 2, True),
    (32, 48, 48, 2, True),
    (48, 64, 64, 2, True),
    (112, 48, 48, 1, True),
    (48, 48, 48, 1, True),
    (48, 16, 3, 1, False),
)


def _out(n, s):
    return (n - 1) // s + 1


class InitNet:
    """Weights, their packed bf16 copies and the activations of one batch
    size and volume shape (z, y, x). All parameters live in one flat fp32
    tensor (weights then bias per layer) so that one Adam launch updates
    them; `grad` has the same layout."""

    def __init__(self, shape, batch, device="cuda", seed=1806, head_scale=0.1):
        self.shape = tuple(int(s) for s in shape)
        self.batch = int(batch)
        self.device = torch.device(device)
        sizes = [self.shape]
        for k in range(4):
            sizes.append(tuple(_out(n, 2) for n in sizes[-1]))
        self.grids = sizes  # input, e1, e2, e3, e4
        n3 = sizes[3]
        self.layer_in = [sizes[0], sizes[1], sizes[2], sizes[3], n3, n3, n3]
        self.convs = [airgb.make_conv(self.batch, self.layer_in[k], cin, cout, s)
                      for k, (cin, cout, _, s, _) in enumerate(LAYERS)]
        counts = [cout * 27 * cin + cout for cin, cout, _, _, _ in LAYERS]
        self.offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        self.params = torch.zeros(int(self.offsets[-1]), dtype=torch.float32, device=self.device)
        self.grad = torch.zeros_like(self.params)
        init = synth.conv_weights([(used, 27, cin) for cin, _, used, _, _ in LAYERS], seed,
                                  head_scale)
        for k, ((w, b), (cin, cout, used, _, _)) in enumerate(zip(init, LAYERS)):
            self.weight(k)[:used].copy_(torch.from_numpy(w))
            self.bias(k)[:used].copy_(torch.from_numpy(b))
        self.packed = [None] * len(LAYERS)
        self.wspaces = [torch.empty(max(airgb.conv_wgrad_workspace_bytes(cv), 256),
                                    dtype=torch.uint8, device=self.device) for cv in self.convs]
        # split-K partials of the forward layers that have few output tiles
        self.fspaces = [torch.empty(max(airgb.conv_forward_workspace_bytes(cv), 256),
                                    dtype=torch.uint8, device=self.device) for cv in self.convs]
        self.acts = {}
        self.pack()

    # ---- parameter views ----
    def weight(self, k, flat=None):
        flat = self.params if flat is None else flat
        cin, cout = LAYERS[k][0], LAYERS[k][1]
        o = int(self.offsets[k])
        return flat[o:o + cout * 27 * cin].view(cout, 27, cin)

    def bias(self, k, flat=None):
        flat = self.params if flat is None else flat
        cin, cout = LAYERS[k][0], LAYERS[k][1]
        o = int(self.offsets[k]) + cout * 27 * cin
        return flat[o:o + cout]

    def pack(self, stream=None):
        """bf16 copies of the weights in the layer kernels' layout."""
        for k, cv in enumerate(self.convs):
            self.packed[k] = airgb.al_conv3d_pack(cv, self.weight(k), True, k > 0, stream=stream,
                                                  out=self.packed[k])

    def packed_layers(self):
        """(cv, weight offset, packed_fwd, packed_dgrad) per layer, the list
        al_adam_flat_pack refreshes."""
        return [(cv, int(self.offsets[k]), self.packed[k][0], self.packed[k][1])
                for k, cv in enumerate(self.convs)]

    # ---- forward / backward ----
    def forward(self, fixed, moving, out=None, stream=None):
        """fixed, moving: (batch, *shape) fp32 -> coefficients (batch, 3, nz, ny, nx)."""
        self.acts["xin"] = airgb.al_initnet_input(fixed, moving, out=self.acts.get("xin"),
                                                  stream=stream)
        return self.forward_input(self.acts["xin"], out=out, stream=stream)

    def forward_input(self, x, out=None, stream=None):
        """The network on a prepared input x (batch, *shape, 2) bf16 (al_initnet_input's
        or al_initnet_pair_input's); x must stay unchanged until backward."""
        A = self.acts
        A["x"] = x
        a = x
        for k, name in enumerate(("e1", "e2", "e3", "e4")):
            a = airgb.al_conv3d_forward(self.convs[k], a, self.packed[k][0], self.bias(k),
                                        relu=True, out=A.get(name), workspace=self.fspaces[k],
                                        stream=stream)
            A[name] = a
        A["cat"] = airgb.al_initnet_upcat(A["e4"], A["e3"], out=A.get("cat"), stream=stream)
        A["d1"] = airgb.al_conv3d_forward(self.convs[4], A["cat"], self.packed[4][0], self.bias(4),
                                          relu=True, out=A.get("d1"), workspace=self.fspaces[4],
                                          stream=stream)
        A["d2"] = airgb.al_conv3d_forward(self.convs[5], A["d1"], self.packed[5][0], self.bias(5),
                                          relu=True, out=A.get("d2"), workspace=self.fspaces[5],
                                          stream=stream)
        A["h"] = airgb.al_conv3d_forward(self.convs[6], A["d2"], self.packed[6][0], self.bias(6),
                                         relu=False, out_f32=True, out=A.get("h"),
                                         workspace=self.fspaces[6], stream=stream)
        return airgb.al_initnet_head_to_ctrl(self.shape, A["h"], out=out, stream=stream)

    def backward(self, grad_ctrl, stream=None):
        """Fills self.grad with the gradient of the parameters for dL/dc = grad_ctrl."""
        A, G = self.acts, {}
        # every entry of self.grad is overwritten below; the padded head rows
        # get exact zeros because their output gradient channels are zero

        def wgrad(k, x, g):
            airgb.al_conv3d_backward_weight(
                self.convs[k], x, g, grad_weight=self.weight(k, self.grad),
                grad_bias=self.bias(k, self.grad), workspace=self.wspaces[k], stream=stream)

        G["h"] = airgb.al_initnet_head_adjoint(self.shape, grad_ctrl, A["h"].shape,
                                               out=A.get("gh"), stream=stream)
        A["gh"] = G["h"]
        wgrad(6, A["d2"], G["h"])
        G["d2"] = airgb.al_conv3d_backward_data(self.convs[6], G["h"], self.packed[6][1],
                                                relu_input=A["d2"], grad_in=A.get("gd2"),
                                                stream=stream)
        A["gd2"] = G["d2"]
        wgrad(5, A["d1"], G["d2"])
        G["d1"] = airgb.al_conv3d_backward_data(self.convs[5], G["d2"], self.packed[5][1],
                                                relu_input=A["d1"], grad_in=A.get("gd1"),
                                                stream=stream)
        A["gd1"] = G["d1"]
        wgrad(4, A["cat"], G["d1"])
        G["cat"] = airgb.al_conv3d_backward_data(self.convs[4], G["d1"], self.packed[4][1],
                                                 grad_in=A.get("gcat"), stream=stream)
        A["gcat"] = G["cat"]
        G["e4"] = airgb.al_initnet_upcat_adjoint(G["cat"], A["e4"], out=A.get("ge4"),
                                                 stream=stream)
        A["ge4"] = G["e4"]
        wgrad(3, A["e3"], G["e4"])
        G["e3"] = airgb.al_conv3d_backward_data(self.convs[3], G["e4"], self.packed[3][1],
                                                relu_input=A["e3"], addend=G["cat"],
                                                addend_offset=LAYERS[3][1], grad_in=A.get("ge3"),
                                                stream=stream)
        A["ge3"] = G["e3"]
        wgrad(2, A["e2"], G["e3"])
        G["e2"] = airgb.al_conv3d_backward_data(self.convs[2], G["e3"], self.packed[2][1],
                                                relu_input=A["e2"], grad_in=A.get("ge2"),
                                                stream=stream)
        A["ge2"] = G["e2"]
        wgrad(1, A["e1"], G["e2"])
        G["e1"] = airgb.al_conv3d_backward_data(self.convs[1], G["e2"], self.packed[1][1],
                                                relu_input=A["e1"], grad_in=A.get("ge1"),
                                                stream=stream)
        A["ge1"] = G["e1"]
        wgrad(0, A["x"], G["e1"])
        return self.grad

    def layer_params(self):
        """[(w (cout_used, 27, cin), b (cout_used,))] as float64 numpy arrays."""
        out = []
        for k, (cin, cout, used, _, _) in enumerate(LAYERS):
            out.append((self.weight(k)[:used].double().cpu().numpy(),
                        self.bias(k)[:used].double().cpu().numpy()))
        return out


# --------------------------------------------------------------- training --

class PairSource:
    """Training or test pairs made by the method: M = blob volume (60 blobs,
    centres uniform in the volume, sigma uniform in [3, 12] voxels, amplitudes
    uniform in [0, 1]), c* ~ N(0, sigma^2) voxels on the spacing-8 lattice,
    F = M o (x + B c*) through al_warp_ctrl (or, for training, only the
    network input (F, M) through al_initnet_pair_input). The random numbers
    are drawn on the device by a counter-based generator (PyTorch's Philox)
    seeded with (seed, first pair), so a batch is fixed by its seed and index."""

    def __init__(self, shape, batch, sigma=4.0, seed=0, device="cuda", n_blobs=60,
                 sigma_range=(3.0, 12.0)):
        self.shape = tuple(shape)
        self.batch = int(batch)
        self.sigma = float(sigma)
        self.seed = int(seed)
        self.n_blobs = int(n_blobs)
        self.sigma_range = sigma_range
        self.device = torch.device(device)
        self.lattice = (3,) + airgb.lattice_shape(self.shape, SPACING)
        if int(np.prod(self.shape)) % 4:
            raise ValueError("the voxel count must be a multiple of 4 (16-byte aligned volumes)")
        self.F = torch.empty((self.batch,) + self.shape, dtype=torch.float32, device=self.device)
        self.M = torch.empty_like(self.F)
        self.ctrl = torch.empty((self.batch,) + self.lattice, dtype=torch.float32,
                                device=self.device)
        self.table = torch.empty((self.batch, self.n_blobs, 5), dtype=torch.float32,
                                 device=self.device)
        self.gen = torch.Generator(device=self.device)
        hi = [self.shape[2] - 1, self.shape[1] - 1, self.shape[0] - 1]
        lo_s, hi_s = self.sigma_range
        self.scale = torch.tensor(hi + [hi_s - lo_s, 1.0], dtype=torch.float32,
                                  device=self.device)
        self.offset = torch.tensor([0.0, 0.0, 0.0, lo_s, 0.0], dtype=torch.float32,
                                   device=self.device)

    def _draw(self, first, stream=None):
        """M and c* of pairs first .. first + batch - 1."""
        self.gen.manual_seed(self.seed * 1_000_003 + int(first))
        torch.rand(self.table.shape, generator=self.gen, device=self.device, out=self.table)
        self.table.mul_(self.scale).add_(self.offset)
        torch.randn(self.ctrl.shape, generator=self.gen, device=self.device, out=self.ctrl)
        self.ctrl.mul_(self.sigma)
        airgb.al_render_blobs(self.shape, self.table, out=self.M, stream=stream)

    def make(self, first, stream=None):
        """Pairs first .. first + batch - 1: (F, M, c*) on the device."""
        self._draw(first, stream)
        # F = M o (x + B c*), the whole batch in one launch
        airgb.al_warp_ctrl(self.shape, SPACING, self.M, self.ctrl, warped=self.F, stream=stream)
        return self.F, self.M, self.ctrl

    def make_input(self, first, x, stream=None):
        """The same pairs as make(first) as the network input only: x (batch,
        *shape, 2) bf16 receives (F, M) as al_initnet_input(*make(first)[:2])
        would write it, without F in device memory. Returns (x, c*)."""
        self._draw(first, stream)
        airgb.al_initnet_pair_input(self.shape, SPACING, self.M, self.ctrl, out=x, stream=stream)
        return x, self.ctrl


@dataclasses.dataclass
class TrainResult:
    steps: int
    pairs: int
    seconds: float
    losses: np.ndarray  # loss of each step (device values, read at the end)


def train(net: InitNet, pairs=20000, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, sigma=4.0, seed=0,
          log_every=0, epochs=1, lr_final=None, graph=True):
    """Adam on the field loss over `pairs` method-generated pairs, net.batch
    per step, `epochs` passes over the same pairs. The step size decays from
    lr to lr_final along a half cosine when lr_final is given (else stays lr).
    With a constant step size (and graph=True) the network part of a step --
    forward, field loss, backward, Adam with the packing, all on fixed buffers -- is
    captured once in a CUDA graph after the first (eager) step and replayed;
    the pair generation stays eager, so it is issued while the previous
    step's replay runs. Returns the per-step losses and the wall time."""
    dev = net.device
    src = PairSource(net.shape, net.batch, sigma, seed, dev)
    per_epoch = (int(pairs) + net.batch - 1) // net.batch
    steps = per_epoch * int(epochs)
    m = torch.zeros_like(net.params)
    v = torch.zeros_like(net.params)
    step = torch.zeros(1, dtype=torch.int64, device=dev)
    losses = torch.empty(steps, dtype=torch.float64, device=dev)
    gc = torch.empty((net.batch,) + src.lattice, dtype=torch.float32, device=dev)
    c = torch.empty_like(gc)
    lws = torch.empty(max(airgb.field_loss_workspace_bytes(net.batch), 256), dtype=torch.uint8,
                      device=dev)
    loss_one = torch.empty(1, dtype=torch.float64, device=dev)
    xin = torch.empty((net.batch,) + tuple(net.shape) + (2,), dtype=torch.bfloat16, device=dev)
    use_graph = graph and lr_final is None and steps > 1
    layers = net.packed_layers()
    step_graph = None

    def net_step(x, ct, loss, lr_i):
        net.forward_input(x, out=c)
        airgb.al_field_loss(net.shape, c, ct, loss=loss, grad=gc, workspace=lws)
        net.backward(gc)
        # the Adam update also rewrites the packed bf16 weights of the layers
        airgb.al_adam_flat_pack(net.params, net.grad, m, v, step, layers, lr=lr_i, betas=betas,
                                eps=eps)

    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i in range(steps):
        x, ct = src.make_input((i % per_epoch) * net.batch, xin)
        if step_graph is not None:
            step_graph.replay()
            losses[i:i + 1].copy_(loss_one)
        else:
            lr_i = lr if lr_final is None else \
                lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * i / max(steps - 1, 1)))
            net_step(x, ct, losses[i:i + 1], lr_i)
            if use_graph:
                # the buffers exist now (the eager step made them): capture
                step_graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(step_graph, capture_error_mode="thread_local"):
                    net_step(x, ct, loss_one, lr)
        if log_every and (i + 1) % log_every == 0:
            print(f"step {i + 1}/{steps} loss {float(losses[i]):.4f}", flush=True)
    torch.cuda.synchronize(dev)
    return TrainResult(steps, steps * net.batch, time.perf_counter() - t0, losses.cpu().numpy())


# ------------------------------------------------------------ evaluation --

@dataclasses.dataclass
class PairReport:
    plain_final_mse: float    # MSE after the plain optimiser's iterations
    plain_best_mse: float     # lowest MSE the plain run passed through
    plain_ms: float           # the plain iterations (device time)
    zero_mse: float           # MSE at c = 0
    init_mse: float           # MSE at the network's prediction, before refinement
    init_J: float             # J = MSE + lambda R at the prediction
    zero_J: float             # J at c = 0
    fallback: bool            # prediction rejected: its MSE is worse than at c = 0
    infer_ms: float           # network inference (device time)
    iterations_to_plain: int  # refinement iterations until MSE <= plain_final_mse (-1: never)
    learned_ms: float         # inference + those iterations, measured (device time)
    iterations_to_best: int   # refinement iterations until MSE <= plain_best_mse (-1: never)
    refined_final_mse: float  # MSE after as many refinement iterations as the plain run
    field_rmse_zero: float    # rms |u*| over voxels (the error of c = 0)
    field_rmse_pred: float    # rms |u_pred - u*|
    field_rmse_plain: float   # rms |u_plain - u*|
    field_rmse_refined: float  # rms |u_refined - u*|
    plain_final_J: float      # J = MSE + lambda R after the plain optimiser's iterations
    iterations_to_plain_J: int  # refinement iterations until J <= plain_final_J (-1: never)
    learned_ms_J: float       # inference + those iterations, measured (device time)
    refined_final_J: float    # J after as many refinement iterations as the plain run


def _field_rmse(shape, c, c_true):
    loss, _ = airgb.al_field_loss(shape, c[None].contiguous(), c_true[None].contiguous())
    return float(np.sqrt(3.0 * float(loss)))


def inference_ms(net_single: InitNet, F, M, out):
    """The network's prediction for one pair into `out`, replayed from a CUDA
    graph (its launches captured once); returns the device time of the replay."""
    Fb, Mb, ob = F[None], M[None], out[None]
    net_single.forward(Fb, Mb, out=ob)  # kernel attributes and activation buffers
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        net_single.forward(Fb, Mb, out=ob)
    graph.replay()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    graph.replay()
    stop.record()
    stop.synchronize()
    return start.elapsed_time(stop)


def _first(values, target):
    hit = np.nonzero(values <= target)[0]
    return int(hit[0]) if len(hit) else -1


def evaluate_pair(net_single: InitNet, F, M, c_true, iterations=200, lr=0.01, lam=0.1):
    """Plain optimiser from zero for `iterations`, then the network's
    prediction refined by the same optimiser: iterations and device time
    until it reaches the plain method's final MSE, and until it reaches the
    plain method's final J (the objective both runs minimise). The prediction is
    rejected (the refinement starts from zero, as the plain method) when its
    MSE is worse than at c = 0. net_single must have batch 1."""
    shape = tuple(F.shape)
    plain = registration.register(F, M, spacing=SPACING, sim="mse", lam=lam, factors=(1,),
                                  iterations=iterations, lr=lr)
    pv = plain.levels[0].values.cpu().numpy()
    target, best = float(pv[-1, 1]), float(pv[:, 1].min())
    ev = registration.Evaluator(shape, SPACING, "mse", lam, device=F.device)
    c0 = torch.empty((3,) + airgb.lattice_shape(shape, SPACING), dtype=torch.float32,
                     device=F.device)
    infer_ms = inference_ms(net_single, F, M, c0)
    val0 = torch.empty(4, dtype=torch.float64, device=F.device)
    valz = torch.empty(4, dtype=torch.float64, device=F.device)
    zero = torch.zeros_like(c0)
    ev.evaluate(F, M, c0, val0, None)
    ev.evaluate(F, M, zero, valz, None)
    fallback = not (float(val0[1]) <= float(valz[1]))
    start_c = zero if fallback else c0
    refine = registration.register(F, M, spacing=SPACING, sim="mse", lam=lam, factors=(1,),
                                   iterations=iterations, lr=lr, ctrl=start_c)
    rv = refine.levels[0].values.cpu().numpy()

    def measured(k):
        # the measured run: exactly k refinement iterations after the inference
        if k < 0:
            return float("nan")
        if k == 0:
            return infer_ms
        again = registration.register(F, M, spacing=SPACING, sim="mse", lam=lam, factors=(1,),
                                      iterations=k, lr=lr, ctrl=start_c)
        return infer_ms + again.levels[0].ms

    k = _first(rv[:, 1], target)
    learned_ms = measured(k)
    # the same for the objective the optimiser minimises: J = MSE + lambda R
    target_J = float(pv[-1, 0])
    k_J = _first(rv[:, 0], target_J)
    learned_ms_J = measured(k_J)
    return PairReport(
        plain_final_mse=target, plain_best_mse=best, plain_ms=plain.levels[0].ms,
        zero_mse=float(valz[1]), init_mse=float(val0[1]), init_J=float(val0[0]),
        zero_J=float(valz[0]), fallback=fallback, infer_ms=infer_ms, iterations_to_plain=k,
        learned_ms=learned_ms, iterations_to_best=_first(rv[:, 1], best),
        refined_final_mse=float(rv[-1, 1]),
        field_rmse_zero=_field_rmse(shape, zero, c_true),
        field_rmse_pred=_field_rmse(shape, c0, c_true),
        field_rmse_plain=_field_rmse(shape, plain.ctrl, c_true),
        field_rmse_refined=_field_rmse(shape, refine.ctrl, c_true),
        plain_final_J=target_J, iterations_to_plain_J=k_J, learned_ms_J=learned_ms_J,
        refined_final_J=float(rv[-1, 0]))


def _main():
    """Training steps of the network at a given batch and volume size, for
    timing and profiling: python -m paper_1806_09907_gb300.learned_init
    --batch 16 --size 128 --steps 3 runs 3 steps (pair generation, forward,
    field loss, backward, Adam with the packing) and prints the device time of each."""
    import argparse

    p = argparse.ArgumentParser()
    p.add_argument("--batch", type=int, default=16)
    p.add_argument("--size", type=int, default=128)
    p.add_argument("--steps", type=int, default=3)
    args = p.parse_args()
    dev = torch.device("cuda", 0)
    net = InitNet((args.size,) * 3, args.batch, dev, seed=1806)
    for i in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        res = train(net, pairs=args.batch, lr=1e-3, seed=i)
        b.record()
        b.synchronize()
        print(f"step {i}: {a.elapsed_time(b):.3f} ms, loss {float(res.losses[0]):.4f}", flush=True)
    assert airgb.al_get_device_error() == 0


if __name__ == "__main__":
    _main()
