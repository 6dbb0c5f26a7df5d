"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point the header declares, and rejects bad arguments before it
launches anything."""
import ctypes
import os
import re

import numpy as np

import pytest

from paper_1806_09907_gb300 import airgb
from paper_1806_09907_gb300 import build as airgb_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "airgb.h")


@pytest.fixture(scope="module")
def lib():
    airgb_build.build()
    return airgb.load()


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(al_[a-z0-9_]+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_binding_exports():
    assert header_functions() == sorted(airgb.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert airgb.status_string(0) == "ok"
    assert "aligned" in airgb.status_string(3)
    assert airgb.status_string(99) == "unknown status"


def test_bspline_init_lattice_sizes(lib):
    # n = (N - 1)/delta + 4 per active axis, 1 for the inactive z of 2D
    bs = airgb.bspline_init((160, 256, 256), 6)
    assert (bs.n[0], bs.n[1], bs.n[2]) == (46, 46, 30)
    bs = airgb.bspline_init((128, 128), 8)
    assert (bs.n[0], bs.n[1], bs.n[2]) == (19, 19, 1)
    assert airgb.lattice_shape((9, 10, 11), 4) == (6, 6, 6)


@pytest.mark.parametrize("ndim,size,spacing,status", [
    (4, (8, 8, 8), 4, 2),    # ndim
    (3, (1, 8, 8), 4, 2),    # axis of one voxel
    (2, (8, 8, 2), 4, 2),    # 2D with Z != 1
    (3, (8, 8, 8), 0, 1),    # spacing
    (3, (8, 8, 8), 33, 1),   # spacing above the table
    (3, (1 << 21, 2, 2), 4, 2),  # axis too long
])
def test_bspline_init_rejects(lib, ndim, size, spacing, status):
    g = airgb.al_grid()
    g.ndim = ndim
    for k in range(3):
        g.size[k] = size[k]
    bs = airgb.al_bspline()
    assert lib.al_bspline_init(ctypes.byref(bs), ctypes.byref(g), spacing) == status


def test_calls_reject_bad_pointers_before_launching(lib):
    bs = airgb.bspline_init((16, 16, 16), 4)
    # NULL arrays
    assert lib.al_displacement(ctypes.byref(bs), None, None, None) == 1
    # misaligned (never dereferenced: checked on the host)
    a, b = ctypes.c_void_p(0x10000), ctypes.c_void_p(0x10004)
    assert lib.al_displacement(ctypes.byref(bs), a, b, None) == 3
    # lattice that does not match the grid
    bad = airgb.bspline_init((16, 16, 16), 4)
    bad.n[0] += 1
    assert lib.al_displacement(ctypes.byref(bad), a, a, None) == 2


def _sim_params(kind="lcc", window=7, eps=1e-5):
    p = airgb.al_sim_params()
    p.kind, p.lcc_window, p.eps = airgb.SIM_KINDS.get(kind, 5), window, eps
    return p


def test_step_calls_reject_before_launching(lib):
    """A1-A6 step calls: NULL arrays (1), misaligned arrays (3), bad grids
    (2), short workspaces (8) and bad parameters (1) are reported on the
    host; none of these calls reaches the GPU (there is none here)."""
    P, Mis = ctypes.c_void_p(0x10000), ctypes.c_void_p(0x10004)
    big = ctypes.c_size_t(1 << 30)
    g = airgb.make_grid((16, 20, 24))
    bad = airgb.make_grid((16, 20, 24))
    bad.ndim = 4
    bs = airgb.bspline_init((16, 20, 24), 4)
    nb = lib.al_displacement_adjoint_workspace_bytes(ctypes.byref(bs))
    assert nb > 0
    assert lib.al_displacement_adjoint(ctypes.byref(bs), None, P, P, big, None) == 1
    assert lib.al_displacement_adjoint(ctypes.byref(bs), P, P, P, ctypes.c_size_t(nb - 1),
                                       None) == 8
    assert lib.al_displacement_adjoint(ctypes.byref(bs), Mis, P, P, big, None) == 3
    assert lib.al_warp(ctypes.byref(g), None, P, P, P, None) == 1
    assert lib.al_warp(ctypes.byref(g), P, Mis, P, P, None) == 3
    assert lib.al_warp(ctypes.byref(bad), P, P, P, P, None) == 2
    assert lib.al_warp_adjoint(ctypes.byref(g), P, P, None, P, P, 0, None) == 1
    assert lib.al_warp_adjoint(ctypes.byref(g), P, P, P, P, P, 2, None) == 1  # accumulate
    sp = _sim_params()
    n = lib.al_similarity_workspace_bytes(ctypes.byref(g), ctypes.byref(sp))
    assert n > 0
    assert lib.al_similarity_workspace_bytes(ctypes.byref(g), ctypes.byref(_sim_params(window=9))) == 0
    assert lib.al_similarity(ctypes.byref(g), ctypes.byref(sp), P, P, P, P, P, P,
                             ctypes.c_size_t(n - 1), None) == 8
    assert lib.al_similarity(ctypes.byref(g), ctypes.byref(sp), P, P, None, P, P, P,
                             ctypes.c_size_t(n), None) == 1
    assert lib.al_similarity(ctypes.byref(g), ctypes.byref(sp), P, Mis, P, P, P, P,
                             ctypes.c_size_t(n), None) == 3
    for badp in (_sim_params(eps=-1.0), _sim_params(kind="none")):
        assert lib.al_similarity(ctypes.byref(g), ctypes.byref(badp), P, P, P, P, P, P,
                                 ctypes.c_size_t(n), None) == 1
    nr = lib.al_regulariser_workspace_bytes(ctypes.byref(g))
    assert lib.al_regulariser(ctypes.byref(g), None, ctypes.c_double(1.0), P, P, P,
                              ctypes.c_size_t(nr), None) == 1
    assert lib.al_regulariser(ctypes.byref(g), P, ctypes.c_double(float("nan")), P, P, P,
                              ctypes.c_size_t(nr), None) == 1
    pr = airgb.make_problem((16, 20, 24), 4, "lcc", 0.1)
    nu = lib.al_objective_unfused_workspace_bytes(ctypes.byref(pr))
    assert lib.al_objective_grad_unfused(ctypes.byref(pr), P, P, P, P, P, P,
                                         ctypes.c_size_t(nu - 1), None) == 8


def test_noalloc_limits_and_pointers(lib):
    """The allocation-free similarity: a problem beyond the built-in 4 MiB
    scratch (LCC on 128x128x64) returns AL_ERR_SCRATCH_LIMIT; NULL and
    misaligned arrays are reported before the first CUDA call."""
    P, Mis = ctypes.c_void_p(0x10000), ctypes.c_void_p(0x10004)
    assert lib.al_noalloc_scratch_bytes() == 4 << 20
    sp = _sim_params()
    big = airgb.make_grid((64, 128, 128))
    assert lib.al_similarity_noalloc(ctypes.byref(big), ctypes.byref(sp), P, P, P, P, P,
                                     None) == 9
    g = airgb.make_grid((16, 20, 24))
    assert lib.al_similarity_noalloc(ctypes.byref(g), ctypes.byref(sp), None, P, P, P, P,
                                     None) == 1
    assert lib.al_similarity_noalloc(ctypes.byref(g), ctypes.byref(sp), P, P, P, P, Mis,
                                     None) == 3


def test_diffeo_calls_reject_before_launching(lib):
    """Scaling and squaring: steps outside 0..20 (1), a missing workspace or
    trajectory (8 / 1), short workspaces (8)."""
    P = ctypes.c_void_p(0x10000)
    big = ctypes.c_size_t(1 << 30)
    g = airgb.make_grid((16, 20, 24))
    assert lib.al_exp_field_workspace_bytes(ctypes.byref(g)) > 0
    for steps in (-1, 21):
        assert lib.al_exp_field(ctypes.byref(g), steps, P, P, None, P, big, None) == 1
    assert lib.al_exp_field(ctypes.byref(g), 6, P, P, None, None, ctypes.c_size_t(0), None) == 8
    assert lib.al_exp_field_adjoint(ctypes.byref(g), 6, None, P, P, P, big, None) == 1
    assert lib.al_exp_field_adjoint(ctypes.byref(g), 6, P, P, P, P, ctypes.c_size_t(1),
                                    None) == 8
    pr = airgb.make_problem((16, 20, 24), 4, "lcc", 0.1)
    nd = lib.al_objective_diffeo_workspace_bytes(ctypes.byref(pr), 6)
    assert nd > 0 and lib.al_objective_diffeo_workspace_bytes(ctypes.byref(pr), 21) == 0
    assert lib.al_objective_grad_diffeo(ctypes.byref(pr), 6, P, P, P, P, P, P,
                                        ctypes.c_size_t(nd - 1), None) == 8
    assert lib.al_objective_grad_diffeo(ctypes.byref(pr), 21, P, P, P, P, P, P,
                                        ctypes.c_size_t(nd), None) == 1


def test_workspace_checks(lib):
    pr = airgb.make_problem((24, 20, 18), 4, "lcc", 0.1)
    need = lib.al_objective_workspace_bytes(ctypes.byref(pr))
    assert need > 0
    p = ctypes.c_void_p(0x10000)
    st = lib.al_objective_grad(ctypes.byref(pr), p, p, p, p, p, p, ctypes.c_size_t(need - 1), None)
    assert st == 8
    st = lib.al_objective_grad(ctypes.byref(pr), p, p, p, p, p, None, ctypes.c_size_t(need), None)
    assert st == 8  # NULL workspace
    # unsupported LCC window and invalid eps are caught on the host
    pr.sim.lcc_window = 9
    assert lib.al_objective_workspace_bytes(ctypes.byref(pr)) == 0
    pr.sim.lcc_window = 7
    pr.sim.eps = -1.0
    st = lib.al_objective_grad(ctypes.byref(pr), p, p, p, p, p, p, ctypes.c_size_t(need), None)
    assert st == 1


def test_fused_workspace_scales_with_volume(lib):
    small = airgb.make_problem((40, 64, 64), 6, "mse")
    big = airgb.make_problem((160, 256, 256), 6, "lcc")
    a = lib.al_objective_workspace_bytes(ctypes.byref(small))
    b = lib.al_objective_workspace_bytes(ctypes.byref(big))
    # LCC keeps W, the mask and dS/dW: 9 bytes per voxel plus the partials
    assert b > 9 * 160 * 256 * 256 > a > 0


def test_pyramid_grid_and_workspace(lib):
    g = airgb.make_grid((160, 256, 256))
    out = airgb.al_grid()
    assert lib.al_pyramid_grid(ctypes.byref(g), 4, ctypes.byref(out)) == 0
    assert (out.ndim, out.size[0], out.size[1], out.size[2]) == (3, 64, 64, 40)
    assert lib.al_pyramid_grid(ctypes.byref(g), 2, ctypes.byref(out)) == 0
    assert (out.size[0], out.size[1], out.size[2]) == (128, 128, 80)
    assert lib.al_pyramid_grid(ctypes.byref(g), 0, ctypes.byref(out)) == 1
    assert lib.al_pyramid_grid(ctypes.byref(g), 9, ctypes.byref(out)) == 1
    tiny = airgb.make_grid((3, 40, 40))  # z would keep a single voxel
    assert lib.al_pyramid_grid(ctypes.byref(tiny), 4, ctypes.byref(out)) == 2
    assert lib.al_pyramid_workspace_bytes(ctypes.byref(g), 1) == 0
    assert lib.al_pyramid_workspace_bytes(ctypes.byref(g), 4) >= 4 * 64 * 256 * 160
    assert lib.al_pyramid_workspace_bytes(ctypes.byref(tiny), 4) == 0
    p = ctypes.c_void_p(0x10000)
    st = lib.al_pyramid_level(ctypes.byref(g), p, 4, p, None, ctypes.c_size_t(0), None)
    assert st == 8  # workspace needed for factor > 1
    st = lib.al_pyramid_level(ctypes.byref(g), ctypes.c_void_p(0x10008), 1, p, None,
                              ctypes.c_size_t(0), None)
    assert st == 3


def test_adam_step_rejects(lib):
    bs = airgb.bspline_init((20, 24, 28), 4)
    p = ctypes.c_void_p(0x10000)

    def call(prm, ptr=p, step=p):
        return lib.al_adam_step(ctypes.byref(bs), ctypes.byref(prm), ptr, p, p, p, step, None)

    ok = airgb.al_adam_params(0.01, 0.9, 0.999, 1e-8)
    assert call(ok, step=None) == 1
    assert call(ok, ptr=ctypes.c_void_p(0x10004)) == 3
    for bad in ((-0.1, 0.9, 0.999, 1e-8), (0.01, 1.0, 0.999, 1e-8), (0.01, 0.9, -0.5, 1e-8),
                (0.01, 0.9, 0.999, 0.0), (float("nan"), 0.9, 0.999, 1e-8)):
        assert call(airgb.al_adam_params(*bad)) == 1, bad


def test_refine_rejects(lib):
    p = ctypes.c_void_p(0x10000)
    fine = airgb.bspline_init((40, 64, 64), 6)
    coarse = airgb.bspline_init((20, 32, 32), 6)
    other = airgb.bspline_init((20, 32, 32), 4)
    wrong = airgb.bspline_init((20, 32, 31), 6)
    assert lib.al_bspline_refine(ctypes.byref(other), p, ctypes.byref(fine), p, None) == 2
    assert lib.al_bspline_refine(ctypes.byref(wrong), p, ctypes.byref(fine), p, None) == 2
    assert lib.al_bspline_refine(ctypes.byref(coarse), ctypes.c_void_p(0x10004),
                                 ctypes.byref(fine), p, None) == 3
    assert lib.al_bspline_refine(ctypes.byref(coarse), None, ctypes.byref(fine), p, None) == 1


def _batch(lib, problems):
    arr = (airgb.al_problem * len(problems))(*problems)
    h = ctypes.c_void_p()
    st = lib.al_batch_create(arr, len(problems), ctypes.byref(h))
    return st, h


def test_batch_plan_counts(lib):
    shapes = [(96, 96), (200, 136), (40, 48, 56), (64, 64, 64)]
    st, h = _batch(lib, [airgb.make_problem(s, 8, "mse", 0.1) for s in shapes])
    assert st == 0
    per = (ctypes.c_int32 * 3)()
    total = lib.al_batch_items(h, per)
    # bricks of 4 x 3 (x 4) cells of 8 voxels, Gram tiles of 16^2 / 8^3
    # points per component, chunks of 768 control points
    bricks = gram = chunks = 0
    for s in shapes:
        cells = [-(-n // 8) for n in s[::-1]]
        b = [-(-cells[0] // 4), -(-cells[1] // 3)] + ([-(-cells[2] // 4)] if len(s) == 3 else [])
        lat = [(n - 1) // 8 + 4 for n in s[::-1]]
        t = 8 if len(s) == 3 else 16
        bricks += int(np.prod(b))
        gram += len(s) * int(np.prod([-(-n // t) for n in lat]))
        chunks += -(-int(np.prod(lat)) // 768)
    assert tuple(per) == (bricks, gram, chunks) and total == bricks + gram + chunks
    assert lib.al_batch_workspace_bytes(h) > 0
    lib.al_batch_destroy(h)


def test_batch_rejects(lib):
    # one spacing per batch, MSE only, spacings with a batch kernel
    st, _ = _batch(lib, [airgb.make_problem((64, 64), 8), airgb.make_problem((64, 64), 6)])
    assert st == 7
    st, _ = _batch(lib, [airgb.make_problem((64, 64), 8, "lcc")])
    assert st == 7
    st, _ = _batch(lib, [airgb.make_problem((64, 64), 5)])
    assert st == 7
    h = ctypes.c_void_p()
    assert lib.al_batch_create(None, 1, ctypes.byref(h)) == 1
    st, h = _batch(lib, [airgb.make_problem((64, 64), 8)])
    assert st == 0
    # no workspace bound yet: nothing is launched
    p = airgb.al_adam_params(0.01, 0.9, 0.999, 1e-8)
    assert lib.al_batch_step(h, ctypes.byref(p), 1, -1, None) == 8
    bad = airgb.al_adam_params(0.01, 1.0, 0.999, 1e-8)
    assert lib.al_batch_step(h, ctypes.byref(bad), 1, -1, None) == 1
    assert lib.al_batch_step(h, ctypes.byref(p), 0, -1, None) == 1
    assert lib.al_batch_set_policy(h, 4) == 1
    assert lib.al_batch_set_wait(h, 0, 0) == 1
    lib.al_batch_destroy(h)


def test_lcc_wait_hook_rejects_bad_slice(lib):
    assert lib.al_lcc_set_wait(-2) == 1


def test_fused_wait_hook_rejects_bad_batch(lib):
    assert lib.al_fused_set_wait(-2) == 1


def test_warp_ctrl_rejects(lib):
    """al_warp_ctrl: bad count or NULL pointers 1, a spacing without a fused
    kernel 7 (unsupported), a misaligned pointer 3; nothing launches."""
    from paper_1806_09907_gb300 import airgb
    bs = airgb.bspline_init((20, 36, 48), 6)
    a = ctypes.c_void_p(0x10000)
    assert lib.al_warp_ctrl(ctypes.byref(bs), 0, a, a, a, None, None) == 1
    assert lib.al_warp_ctrl(ctypes.byref(bs), 2, None, a, a, None, None) == 1
    assert lib.al_warp_ctrl(ctypes.byref(bs), 2, a, a, ctypes.c_void_p(0x10004), None, None) == 3
    bs5 = airgb.bspline_init((20, 36, 48), 5)
    assert lib.al_warp_ctrl(ctypes.byref(bs5), 2, a, a, a, None, None) == 7


def test_initnet_pair_input_rejects(lib):
    """al_initnet_pair_input: bad count or NULL pointers 1, a 2D grid or a
    spacing without a fused kernel 7, a misaligned pointer 3; nothing launches."""
    bs = airgb.bspline_init((20, 36, 48), 8)
    a = ctypes.c_void_p(0x10000)
    assert lib.al_initnet_pair_input(ctypes.byref(bs), 0, a, a, a, None) == 1
    assert lib.al_initnet_pair_input(ctypes.byref(bs), 70000, a, a, a, None) == 1
    assert lib.al_initnet_pair_input(ctypes.byref(bs), 2, a, a, None, None) == 1
    assert lib.al_initnet_pair_input(ctypes.byref(bs), 2, a, a, ctypes.c_void_p(0x10004),
                                     None) == 3
    bs5 = airgb.bspline_init((20, 36, 48), 5)
    assert lib.al_initnet_pair_input(ctypes.byref(bs5), 2, a, a, a, None) == 7
    bs2 = airgb.bspline_init((36, 48), 8)
    assert lib.al_initnet_pair_input(ctypes.byref(bs2), 2, a, a, a, None) == 7


def test_batch_bind_tune_status_reject(lib):
    """Binding checks every device pointer (NULL 1, misaligned 3) and the
    workspace (8) on the host; tuning needs a bound workspace (8) and at
    least one iteration (1); a NULL batch is an invalid argument."""
    st, h = _batch(lib, [airgb.make_problem((64, 64), 8), airgb.make_problem((32, 40, 48), 8)])
    assert st == 0
    ws = lib.al_batch_workspace_bytes(h)
    a = ctypes.c_void_p(0x10000)
    two = ctypes.c_void_p * 2
    ok = two(0x10000, 0x20000)

    def bind(fixed=ok, workspace=a, nbytes=ws):
        return lib.al_batch_bind(h, fixed, ok, ok, ok, ok, None, workspace,
                                 ctypes.c_size_t(nbytes))

    assert bind(fixed=None) == 1
    assert bind(fixed=two(0x10000, None)) == 1
    assert bind(fixed=two(0x10000, 0x20004)) == 3
    assert bind(nbytes=ws - 1) == 8
    assert bind(workspace=None) == 8
    p = airgb.al_adam_params(0.01, 0.9, 0.999, 1e-8)
    assert lib.al_batch_tune(h, ctypes.byref(p), 5, None, None, None, None) == 8  # not bound
    assert lib.al_batch_tune(h, ctypes.byref(p), 0, None, None, None, None) == 1
    assert lib.al_batch_set_tile(h, -1) == 1
    assert lib.al_batch_set_tile(h, lib.al_batch_tiles(h, None)) == 1
    assert lib.al_batch_set_tile(h, 1) == 0  # before binding: recorded for the bind
    assert lib.al_batch_status(None, None) == 1
    assert lib.al_batch_bind(None, ok, ok, ok, ok, ok, None, a, ctypes.c_size_t(ws)) == 1
    lib.al_batch_destroy(h)


# ---- learned initialisation: layer and glue argument checks ----------------

def _conv(batch=2, size=(8, 8, 8), cin=16, cout=32, stride=2):
    return airgb.make_conv(batch, size, cin, cout, stride)


@pytest.mark.parametrize("kw,status", [
    (dict(cin=3), 2),            # channels: 2 or a multiple of 8
    (dict(cin=264), 2),          # at most 256 input channels
    (dict(cout=24), 2),          # output channels: a multiple of 16
    (dict(cout=144), 2),         # at most 128
    (dict(stride=3), 1),         # stride 1 or 2
    (dict(batch=0), 1),
    (dict(size=(0, 8, 8)), 2),
    (dict(batch=1024, size=(1024, 1024, 8)), 2),  # 2^33 voxels
    (dict(batch=1, size=(2, 8192, 8192), cin=16), 2),  # tap offsets beyond 32 bits
])
def test_conv_layer_shape_checks(lib, kw, status):
    cv = _conv(**kw)
    out = (ctypes.c_int64 * 3)()
    assert lib.al_conv3d_output_size(ctypes.byref(cv), out) == status
    assert lib.al_conv3d_packed_bytes(ctypes.byref(cv), 0) == 0


def test_conv_layer_sizes(lib):
    cv = _conv(size=(9, 12, 10))
    assert airgb.conv_output_size(cv) == (5, 6, 5)
    # forward: ceil(27 cin / 64) slices of cout x 64 bf16
    assert lib.al_conv3d_packed_bytes(ctypes.byref(cv), 0) == 7 * 32 * 64 * 2
    # stride-2 input adjoint: the 8 parity classes' own slices (1, 2, 4 or 8
    # taps of 32 channels: 1 + 3 * 1 + 3 * 2 + 4 = 14 slices of 16 x 64)
    assert lib.al_conv3d_packed_bytes(ctypes.byref(cv), 1) == 14 * 16 * 64 * 2
    assert lib.al_conv3d_packed_bytes(ctypes.byref(_conv(stride=1)), 1) == 14 * 16 * 64 * 2
    assert lib.al_conv3d_packed_bytes(ctypes.byref(_conv(cin=2)), 1) == 0  # no dgrad for 2
    assert lib.al_conv3d_backward_weight_workspace_bytes(ctypes.byref(cv)) > 0
    # split K only for layers with few output tiles and enough K slices
    few = _conv(batch=1, size=(9, 10, 11), cin=112, cout=48, stride=1)  # 8 tiles, 48 slices
    assert lib.al_conv3d_forward_workspace_bytes(ctypes.byref(few)) == 8 * 990 * 48 * 4
    many = _conv(batch=16, size=(128, 128, 128), cin=2, cout=16, stride=2)
    assert lib.al_conv3d_forward_workspace_bytes(ctypes.byref(many)) == 0


def test_conv_calls_reject_before_launching(lib):
    cv = _conv()
    p = ctypes.byref(cv)
    a, b = ctypes.c_void_p(0x10000), ctypes.c_void_p(0x10004)
    assert lib.al_conv3d_forward(p, None, a, None, 1, 0, a, None, 0, None) == 1
    assert lib.al_conv3d_forward(p, a, a, None, 1, 0, b, None, 0, None) == 3
    assert lib.al_conv3d_forward(p, a, a, None, 1, 0, a, b, 1 << 20, None) == 3
    assert lib.al_conv3d_pack(p, a, None, None, None) == 1
    assert lib.al_conv3d_pack(ctypes.byref(_conv(cin=2)), a, None, a, None) == 7
    # the input adjoint needs cin a multiple of 16
    assert lib.al_conv3d_backward_data(ctypes.byref(_conv(cin=8)), a, a, None, None, 0, 0, a,
                                       None) == 7
    # addend stride/offset must be multiples of 8 that hold the cin channels
    assert lib.al_conv3d_backward_data(p, a, a, None, a, 20, 0, a, None) == 1
    assert lib.al_conv3d_backward_data(p, a, a, None, a, 32, 24, a, None) == 1
    ws = lib.al_conv3d_backward_weight_workspace_bytes(p)
    assert lib.al_conv3d_backward_weight(p, a, a, a, None, a, ws - 1, None) == 8
    assert lib.al_conv3d_backward_weight(p, a, a, a, None, None, ws, None) == 8


def test_adam_flat_pack_rejects(lib):
    """Argument checks of the Adam update with the packing (nothing launches)."""
    a = ctypes.c_void_p(0x10000)
    mis = ctypes.c_void_p(0x10004)
    p = airgb.al_adam_params()
    p.lr, p.beta1, p.beta2, p.eps = 1e-3, 0.9, 0.999, 1e-8
    c1, c2 = _conv(cin=16, cout=32), _conv(cin=32, cout=16, stride=1)
    n1, n2 = 32 * 27 * 16, 16 * 27 * 32

    def call(n, layers, offs, pf, pd, par=p, param=a):
        k = max(len(layers), 1)
        return lib.al_adam_flat_pack(ctypes.byref(par), n, a, param, a, a, a, len(layers),
                                     (airgb.al_conv3d * k)(*layers), (ctypes.c_int64 * k)(*offs),
                                     (ctypes.c_void_p * k)(*pf), (ctypes.c_void_p * k)(*pd), None)

    n = n1 + n2 + 48
    # a valid call would launch: only rejections are exercised here
    assert call(n, [c1, c2], [0, n1 + 32], [a, a], [None, None], param=mis) == 3
    assert call(n, [], [], [], []) == 1                                   # no layer
    assert call(n, [c1] * 9, [0] * 9, [a] * 9, [a] * 9) == 1               # more than 8
    assert call(n, [c1, c2], [0, n1], [None, a], [None, a]) == 1           # neither copy
    assert call(n, [c1, c2], [0, n1 - 1], [a, a], [a, a]) == 1             # ranges overlap
    assert call(n, [c1, c2], [0, n - n2 + 1], [a, a], [a, a]) == 1         # past n
    assert call(n, [c1, c2], [-1, n1], [a, a], [a, a]) == 1                # negative offset
    assert call(n, [c1, c2], [0, n1], [a, mis], [a, a]) == 3               # packed alignment
    assert call(n, [_conv(cin=2), c2], [0, n1], [a, a], [a, a]) == 7       # no dgrad for cin 2
    assert call(n, [_conv(cout=24), c2], [0, n1], [a, a], [a, a]) == 2     # layer checks
    bad = airgb.al_adam_params()
    bad.lr, bad.beta1, bad.beta2, bad.eps = 1e-3, 1.0, 0.999, 1e-8
    assert call(n, [c1, c2], [0, n1], [a, a], [a, a], par=bad) == 1        # beta1 < 1


def test_initnet_glue_checks(lib):
    a = ctypes.c_void_p(0x10000)
    n3 = (ctypes.c_int64 * 3)(16, 16, 16)
    assert lib.al_initnet_upcat(2, n3, 64, 44, a, a, a, None) == 1      # channels % 8
    assert lib.al_initnet_upcat(0, n3, 64, 48, a, a, a, None) == 1
    bs = airgb.bspline_init((128, 128, 128), 8)
    bad = (ctypes.c_int64 * 3)(15, 16, 16)  # the head must sit on (N - 1)/8 + 1 voxels
    assert lib.al_initnet_head_to_ctrl(ctypes.byref(bs), 2, bad, 16, a, a, None) == 2
    bs6 = airgb.bspline_init((128, 128, 128), 6)
    assert lib.al_initnet_head_to_ctrl(ctypes.byref(bs6), 2, n3, 16, a, a, None) == 7
    assert lib.al_field_loss_workspace_bytes(4) == 4 * 3 * 8
    assert lib.al_field_loss(ctypes.byref(bs), 4, a, a, a, a, None, 0, None) == 8
    p = airgb.al_adam_params()
    p.lr, p.beta1, p.beta2, p.eps = 0.0, 0.9, 0.999, 1e-8
    assert lib.al_adam_flat(ctypes.byref(p), 10, a, a, a, a, a, None) == 1  # lr > 0
    sz = (ctypes.c_int64 * 3)(8, 8, 8)
    assert lib.al_render_blobs(sz, 0, 10, a, a, None) == 1
    assert lib.al_render_blobs(sz, 1, 10, a, ctypes.c_void_p(0x10004), None) == 3
    mis = ctypes.c_void_p(0x10004)
    assert lib.al_initnet_input(2, sz, None, a, a, None) == 1
    assert lib.al_initnet_input(0, sz, a, a, a, None) == 1
    assert lib.al_initnet_input(2, sz, a, mis, a, None) == 3
    assert lib.al_initnet_input(2, (ctypes.c_int64 * 3)(0, 8, 8), a, a, a, None) == 2
    assert lib.al_initnet_upcat_adjoint(2, n3, 60, 48, a, a, a, None) == 1  # channels % 8
    assert lib.al_initnet_upcat_adjoint(2, n3, 64, 48, None, a, a, None) == 1
    assert lib.al_initnet_upcat_adjoint(2, n3, 64, 48, a, mis, a, None) == 3
    assert lib.al_initnet_head_adjoint(ctypes.byref(bs), 2, n3, 6, a, a, None) == 2  # % 4
    assert lib.al_initnet_head_adjoint(ctypes.byref(bs), 2, n3, 16, None, a, None) == 1
    assert lib.al_initnet_head_adjoint(ctypes.byref(bs), 2, bad, 16, a, a, None) == 2
    assert lib.al_initnet_head_adjoint(ctypes.byref(bs6), 2, n3, 16, a, a, None) == 7


def test_registration_checkpoint_roundtrip(tmp_path):
    from paper_1806_09907_gb300 import registration

    c = np.random.default_rng(3).normal(0, 1, (3, 7, 8, 9)).astype(np.float32)
    ck = registration.Checkpoint(2, (4, 2, 1), (40, 64, 64), 6, c)
    path = str(tmp_path / "s.npz")
    ck.save(path)
    back = registration.Checkpoint.load(path)
    assert (back.levels_done, back.factors, back.shape, back.spacing) == (2, (4, 2, 1),
                                                                        (40, 64, 64), 6)
    assert back.ctrl.dtype == np.float32 and np.array_equal(back.ctrl, c)


def test_warped_offsets_only_for_fused_lcc(lib):
    """The warped image of a fused evaluation is in its workspace only for
    LCC; MSE and NCC keep it on chip."""
    pr = airgb.make_problem((40, 48, 64), 6, "lcc", 0.1, 1e-5, 7)
    w, m = airgb.objective_warped_offsets(pr)
    nv = 40 * 48 * 64
    assert w % 256 == 0 and m % 256 == 0
    assert (w + 4 * nv <= m or m + nv <= w)
    assert max(w + 4 * nv, m + nv) <= airgb.objective_workspace_bytes(pr)
    for sim in ("mse", "ncc"):
        with pytest.raises(airgb.AirgbError):
            airgb.objective_warped_offsets(airgb.make_problem((40, 48, 64), 6, sim))
