// C ABI of libairgb: argument checking, workspace layout and launches.
// Declarations and contracts: include/airgb.h.
#include <math.h>
#include <string.h>

#include "airgb.h"
#include "checks.h"
#include "launch.h"

using namespace airgb;

namespace {

__device__ int g_device_error = 0;

constexpr int64_t kMaxAxis = 1 << 20;
constexpr int64_t kMaxVoxels = ((int64_t)1 << 31) - 1;

}  // namespace

namespace airgb {

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

al_status check_grid(const al_grid *g, Grid *out)
{
    if (!g)
        return AL_ERR_INVALID_ARG;
    if (g->ndim != 2 && g->ndim != 3)
        return AL_ERR_SHAPE;
    for (int k = 0; k < 3; ++k) {
        const int64_t n = g->size[k];
        if (k < g->ndim) {
            if (n < 2 || n > kMaxAxis)
                return AL_ERR_SHAPE;
        } else if (n != 1) {
            return AL_ERR_SHAPE;
        }
    }
    const int64_t nv = g->size[0] * g->size[1] * g->size[2];
    if (nv > kMaxVoxels)
        return AL_ERR_SHAPE;
    if (out) {
        out->ndim = g->ndim;
        out->X = (int)g->size[0];
        out->Y = (int)g->size[1];
        out->Z = (int)g->size[2];
        out->nv = (int)nv;
    }
    return AL_OK;
}

int64_t lattice_n(int64_t N, int spacing) { return (N - 1) / spacing + 4; }

// Validates bs against its own grid and fills the kernel descriptor.
al_status check_bspline(const al_bspline *bs, Grid *g, Lattice *L)
{
    if (!bs)
        return AL_ERR_INVALID_ARG;
    al_status st = check_grid(&bs->grid, g);
    if (st != AL_OK)
        return st;
    if (bs->spacing < 1 || bs->spacing > kMaxDelta)
        return AL_ERR_INVALID_ARG;
    int64_t n[3];
    for (int k = 0; k < 3; ++k)
        n[k] = k < bs->grid.ndim ? lattice_n(bs->grid.size[k], bs->spacing) : 1;
    for (int k = 0; k < 3; ++k)
        if (bs->n[k] != n[k])
            return AL_ERR_SHAPE;
    if (L) {
        L->delta = bs->spacing;
        L->nx = (int)n[0];
        L->ny = (int)n[1];
        L->nz = (int)n[2];
        L->nc = (int)(n[0] * n[1] * n[2]);
        memset(L->w, 0, sizeof(L->w));
        for (int p = 0; p < bs->spacing; ++p)
            for (int a = 0; a < 4; ++a)
                L->w[p][a] = (float)bsw_d(p, a, bs->spacing);
    }
    return AL_OK;
}

al_status check_sim(const al_sim_params *p, int ndim)
{
    if (!p)
        return AL_ERR_INVALID_ARG;
    if (p->kind < AL_SIM_MSE || p->kind > AL_SIM_LCC)
        return AL_ERR_INVALID_ARG;
    if (!(p->eps >= 0.0) || !isfinite(p->eps))
        return AL_ERR_INVALID_ARG;
    if (p->kind == AL_SIM_LCC) {
        if (p->lcc_window < 1 || p->lcc_window % 2 == 0 || p->lcc_window > 15)
            return AL_ERR_INVALID_ARG;
        if (p->lcc_window < 3 || p->lcc_window > 7)
            return AL_ERR_UNSUPPORTED;
    }
    (void)ndim;
    return AL_OK;
}

al_status launched(cudaError_t e) { return e == cudaSuccess ? AL_OK : AL_ERR_CUDA; }

int device_sms()
{
    constexpr int kDevices = 64, kFallback = 152;
    static int cache[kDevices] = {};  // idempotent writes: a race stores the same value
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return kFallback;
    }
    if (dev >= 0 && dev < kDevices && cache[dev] > 0)
        return cache[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        return kFallback;
    }
    if (dev >= 0 && dev < kDevices)
        cache[dev] = n;
    return n;
}

}  // namespace airgb

namespace {

cudaStream_t S(al_stream s) { return (cudaStream_t)s; }

size_t a256(size_t b) { return (b + 255) / 256 * 256; }

// Workspace of the unfused composition: u, W, mask, gW, gu, step scratch,
// value slots.
struct UnfusedLayout {
    size_t u, W, m, gW, gu, vals, scratch, total;
};

UnfusedLayout unfused_layout(const Grid &g, const Lattice &L, int kind, int window)
{
    UnfusedLayout o{};
    size_t off = 0;
    const size_t nv = (size_t)g.nv;
    o.u = off;
    off += a256(nv * g.ndim * 4);
    o.W = off;
    off += a256(nv * 4);
    o.m = off;
    off += a256(nv);
    o.gW = off;
    off += a256(nv * 4);
    o.gu = off;
    off += a256(nv * g.ndim * 4);
    o.vals = off;
    off += 256;
    o.scratch = off;
    size_t sc = similarity_ws(g, kind, window);
    size_t r = regulariser_ws(g);
    size_t d = displacement_adjoint_ws(g, L);
    size_t mx = sc > r ? sc : r;
    mx = mx > d ? mx : d;
    off += a256(mx);
    o.total = off;
    return o;
}

}  // namespace

extern "C" {

const char *al_status_string(al_status s)
{
    switch (s) {
    case AL_OK: return "ok";
    case AL_ERR_INVALID_ARG: return "invalid argument";
    case AL_ERR_SHAPE: return "unsupported or inconsistent shape";
    case AL_ERR_ALIGN: return "pointer not 16-byte aligned";
    case AL_ERR_CUDA: return "CUDA error";
    case AL_ERR_BOUNDS: return "kernel index out of range";
    case AL_ERR_TIMEOUT: return "device wait timed out";
    case AL_ERR_UNSUPPORTED: return "not supported by this library";
    case AL_ERR_WORKSPACE: return "workspace missing or too small";
    case AL_ERR_SCRATCH_LIMIT: return "problem too large for the built-in scratch";
    }
    return "unknown status";
}

al_status al_bspline_init(al_bspline *bs, const al_grid *g, int32_t spacing)
{
    if (!bs || !g)
        return AL_ERR_INVALID_ARG;
    al_status st = check_grid(g, nullptr);
    if (st != AL_OK)
        return st;
    if (spacing < 1 || spacing > kMaxDelta)
        return AL_ERR_INVALID_ARG;
    memset(bs, 0, sizeof(*bs));
    bs->grid = *g;
    bs->spacing = spacing;
    for (int k = 0; k < 3; ++k)
        bs->n[k] = k < g->ndim ? lattice_n(g->size[k], spacing) : 1;
    return AL_OK;
}

al_status al_displacement(const al_bspline *bs, const float *ctrl, float *disp, al_stream stream)
{
    Grid g;
    Lattice L;
    al_status st = check_bspline(bs, &g, &L);
    if (st != AL_OK)
        return st;
    if (!ctrl || !disp)
        return AL_ERR_INVALID_ARG;
    if (!aligned16(ctrl) || !aligned16(disp))
        return AL_ERR_ALIGN;
    return launched(launch_displacement(g, L, ctrl, disp, S(stream)));
}

al_status al_warp_ctrl(const al_bspline *bs, int32_t count, const float *moving,
                       const float *ctrl, float *warped, uint8_t *mask, al_stream stream)
{
    Grid g;
    Lattice L;
    al_status st = check_bspline(bs, &g, &L);
    if (st != AL_OK)
        return st;
    if (count < 1 || count > 65535 || !moving || !ctrl || !warped)
        return AL_ERR_INVALID_ARG;
    if (L.delta != 4 && L.delta != 6 && L.delta != 8)
        return AL_ERR_UNSUPPORTED;
    if (!aligned16(moving) || !aligned16(ctrl) || !aligned16(warped) || (mask && !aligned16(mask)))
        return AL_ERR_ALIGN;
    return launched(launch_warp_ctrl(g, L, count, moving, ctrl, warped, mask, nullptr, S(stream)));
}

al_status al_initnet_pair_input(const al_bspline *bs, int32_t count, const float *moving,
                                const float *ctrl, void *x, al_stream stream)
{
    Grid g;
    Lattice L;
    al_status st = check_bspline(bs, &g, &L);
    if (st != AL_OK)
        return st;
    if (count < 1 || count > 65535 || !moving || !ctrl || !x)
        return AL_ERR_INVALID_ARG;
    if (g.ndim != 3 || (L.delta != 4 && L.delta != 6 && L.delta != 8))
        return AL_ERR_UNSUPPORTED;
    if (!aligned16(moving) || !aligned16(ctrl) || !aligned16(x))
        return AL_ERR_ALIGN;
    return launched(launch_warp_ctrl(g, L, count, moving, ctrl, nullptr, nullptr, x, S(stream)));
}

size_t al_displacement_adjoint_workspace_bytes(const al_bspline *bs)
{
    Grid g;
    Lattice L;
    if (check_bspline(bs, &g, &L) != AL_OK)
        return 0;
    return displacement_adjoint_ws(g, L);
}

al_status al_displacement_adjoint(const al_bspline *bs, const float *grad_disp, float *grad_ctrl,
                                  void *workspace, size_t workspace_bytes, al_stream stream)
{
    Grid g;
    Lattice L;
    al_status st = check_bspline(bs, &g, &L);
    if (st != AL_OK)
        return st;
    if (!grad_disp || !grad_ctrl)
        return AL_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < displacement_adjoint_ws(g, L))
        return AL_ERR_WORKSPACE;
    if (!aligned16(grad_disp) || !aligned16(grad_ctrl) || !aligned16(workspace))
        return AL_ERR_ALIGN;
    return launched(launch_displacement_adjoint(g, L, grad_disp, grad_ctrl, workspace, S(stream)));
}

al_status al_warp(const al_grid *gr, const float *moving, const float *disp, float *warped,
                  uint8_t *mask, al_stream stream)
{
    Grid g;
    al_status st = check_grid(gr, &g);
    if (st != AL_OK)
        return st;
    if (!moving || !disp || !warped || !mask)
        return AL_ERR_INVALID_ARG;
    if (!aligned16(moving) || !aligned16(disp) || !aligned16(warped) || !aligned16(mask))
        return AL_ERR_ALIGN;
    return launched(launch_warp(g, moving, disp, warped, mask, S(stream)));
}

al_status al_warp_adjoint(const al_grid *gr, const float *moving, const float *disp,
                          const uint8_t *mask, const float *grad_warped, float *grad_disp,
                          int32_t accumulate, al_stream stream)
{
    Grid g;
    al_status st = check_grid(gr, &g);
    if (st != AL_OK)
        return st;
    if (!moving || !disp || !mask || !grad_warped || !grad_disp)
        return AL_ERR_INVALID_ARG;
    if (accumulate != 0 && accumulate != 1)
        return AL_ERR_INVALID_ARG;
    if (!aligned16(moving) || !aligned16(disp) || !aligned16(mask) || !aligned16(grad_warped) ||
        !aligned16(grad_disp))
        return AL_ERR_ALIGN;
    return launched(
        launch_warp_adjoint(g, moving, disp, mask, grad_warped, grad_disp, accumulate, S(stream)));
}

size_t al_similarity_workspace_bytes(const al_grid *gr, const al_sim_params *p)
{
    Grid g;
    if (check_grid(gr, &g) != AL_OK || check_sim(p, g.ndim) != AL_OK)
        return 0;
    return similarity_ws(g, p->kind, p->lcc_window);
}

al_status al_similarity(const al_grid *gr, const al_sim_params *p, const float *fixed,
                        const float *warped, const uint8_t *mask, double *value_dev,
                        float *grad_warped, void *workspace, size_t workspace_bytes,
                        al_stream stream)
{
    Grid g;
    al_status st = check_grid(gr, &g);
    if (st != AL_OK)
        return st;
    if ((st = check_sim(p, g.ndim)) != AL_OK)
        return st;
    if (!fixed || !warped || !mask || !value_dev)
        return AL_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < similarity_ws(g, p->kind, p->lcc_window))
        return AL_ERR_WORKSPACE;
    if (!aligned16(fixed) || !aligned16(warped) || !aligned16(mask) || !aligned16(value_dev) ||
        !aligned16(workspace) || (grad_warped && !aligned16(grad_warped)))
        return AL_ERR_ALIGN;
    return launched(launch_similarity(g, p->kind, p->lcc_window, p->eps, fixed, warped, mask,
                                      value_dev, grad_warped, workspace, S(stream)));
}

size_t al_regulariser_workspace_bytes(const al_grid *gr)
{
    Grid g;
    if (check_grid(gr, &g) != AL_OK)
        return 0;
    return regulariser_ws(g);
}

al_status al_regulariser(const al_grid *gr, const float *disp, double weight, double *value_dev,
                         float *grad_disp, void *workspace, size_t workspace_bytes,
                         al_stream stream)
{
    Grid g;
    al_status st = check_grid(gr, &g);
    if (st != AL_OK)
        return st;
    if (!disp || !value_dev || !isfinite(weight))
        return AL_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < regulariser_ws(g))
        return AL_ERR_WORKSPACE;
    if (!aligned16(disp) || !aligned16(value_dev) || !aligned16(workspace) ||
        (grad_disp && !aligned16(grad_disp)))
        return AL_ERR_ALIGN;
    return launched(launch_regulariser(g, disp, weight, value_dev, grad_disp, workspace, S(stream)));
}

static al_status check_problem(const al_problem *pr, Grid *g, Lattice *L)
{
    if (!pr)
        return AL_ERR_INVALID_ARG;
    al_status st = check_bspline(&pr->bs, g, L);
    if (st != AL_OK)
        return st;
    if ((st = check_sim(&pr->sim, g->ndim)) != AL_OK)
        return st;
    if (!isfinite(pr->lambda))
        return AL_ERR_INVALID_ARG;
    return AL_OK;
}

size_t al_objective_unfused_workspace_bytes(const al_problem *pr)
{
    Grid g;
    Lattice L;
    if (check_problem(pr, &g, &L) != AL_OK)
        return 0;
    return unfused_layout(g, L, pr->sim.kind, pr->sim.lcc_window).total;
}

static al_status objective_unfused(const al_problem *pr, const Grid &g, const Lattice &L,
                                   const float *fixed, const float *moving, const float *ctrl,
                                   double *value_dev, float *grad_ctrl, void *workspace,
                                   cudaStream_t s)
{
    const UnfusedLayout lay = unfused_layout(g, L, pr->sim.kind, pr->sim.lcc_window);
    char *w = (char *)workspace;
    float *u = (float *)(w + lay.u), *W = (float *)(w + lay.W), *gW = (float *)(w + lay.gW);
    float *gu = (float *)(w + lay.gu);
    uint8_t *m = (uint8_t *)(w + lay.m);
    double *vals = (double *)(w + lay.vals);  // [0..1] similarity, [2] regulariser
    void *scratch = w + lay.scratch;
    if (launch_displacement(g, L, ctrl, u, s) != cudaSuccess)
        return AL_ERR_CUDA;
    if (launch_warp(g, moving, u, W, m, s) != cudaSuccess)
        return AL_ERR_CUDA;
    if (launch_similarity(g, pr->sim.kind, pr->sim.lcc_window, pr->sim.eps, fixed, W, m, vals,
                          grad_ctrl ? gW : nullptr, scratch, s) != cudaSuccess)
        return AL_ERR_CUDA;
    if (launch_regulariser(g, u, pr->lambda, vals + 2, grad_ctrl ? gu : nullptr, scratch, s) !=
        cudaSuccess)
        return AL_ERR_CUDA;
    if (grad_ctrl) {
        if (launch_warp_adjoint(g, moving, u, m, gW, gu, 1, s) != cudaSuccess)
            return AL_ERR_CUDA;
        if (launch_displacement_adjoint(g, L, gu, grad_ctrl, scratch, s) != cudaSuccess)
            return AL_ERR_CUDA;
    }
    return launched(launch_combine(vals, vals + 2, pr->lambda, value_dev, s));
}

al_status al_objective_grad_unfused(const al_problem *pr, const float *fixed, const float *moving,
                                    const float *ctrl, double *value_dev, float *grad_ctrl,
                                    void *workspace, size_t workspace_bytes, al_stream stream)
{
    Grid g;
    Lattice L;
    al_status st = check_problem(pr, &g, &L);
    if (st != AL_OK)
        return st;
    if (!fixed || !moving || !ctrl || !value_dev)
        return AL_ERR_INVALID_ARG;
    if (!workspace ||
        workspace_bytes < unfused_layout(g, L, pr->sim.kind, pr->sim.lcc_window).total)
        return AL_ERR_WORKSPACE;
    if (!aligned16(fixed) || !aligned16(moving) || !aligned16(ctrl) || !aligned16(value_dev) ||
        !aligned16(workspace) || (grad_ctrl && !aligned16(grad_ctrl)))
        return AL_ERR_ALIGN;
    return objective_unfused(pr, g, L, fixed, moving, ctrl, value_dev, grad_ctrl, workspace,
                             S(stream));
}

size_t al_objective_workspace_bytes(const al_problem *pr)
{
    Grid g;
    Lattice L;
    if (check_problem(pr, &g, &L) != AL_OK)
        return 0;
    if (fused_supported(g, L, pr->sim.kind, pr->sim.lcc_window))
        return fused_ws(g, L, pr->sim.kind, pr->sim.lcc_window);
    return unfused_layout(g, L, pr->sim.kind, pr->sim.lcc_window).total;
}

al_status al_objective_warped_offsets(const al_problem *pr, size_t *warped_offset,
                                      size_t *mask_offset)
{
    Grid g;
    Lattice L;
    al_status st = check_problem(pr, &g, &L);
    if (st != AL_OK)
        return st;
    if (!warped_offset || !mask_offset)
        return AL_ERR_INVALID_ARG;
    if (pr->sim.kind != AL_SIM_LCC || !fused_supported(g, L, pr->sim.kind, pr->sim.lcc_window))
        return AL_ERR_UNSUPPORTED;
    fused_warped_offsets(g, L, pr->sim.lcc_window, warped_offset, mask_offset);
    return AL_OK;
}

al_status al_objective_grad(const al_problem *pr, const float *fixed, const float *moving,
                            const float *ctrl, double *value_dev, float *grad_ctrl,
                            void *workspace, size_t workspace_bytes, al_stream stream)
{
    Grid g;
    Lattice L;
    al_status st = check_problem(pr, &g, &L);
    if (st != AL_OK)
        return st;
    if (!fixed || !moving || !ctrl || !value_dev)
        return AL_ERR_INVALID_ARG;
    const bool fused = fused_supported(g, L, pr->sim.kind, pr->sim.lcc_window);
    const size_t need = fused ? fused_ws(g, L, pr->sim.kind, pr->sim.lcc_window)
                              : unfused_layout(g, L, pr->sim.kind, pr->sim.lcc_window).total;
    if (!workspace || workspace_bytes < need)
        return AL_ERR_WORKSPACE;
    if (!aligned16(fixed) || !aligned16(moving) || !aligned16(ctrl) || !aligned16(value_dev) ||
        !aligned16(workspace) || (grad_ctrl && !aligned16(grad_ctrl)))
        return AL_ERR_ALIGN;
    if (!fused)  // spacings without a fused kernel run the step kernels in sequence
        return objective_unfused(pr, g, L, fixed, moving, ctrl, value_dev, grad_ctrl, workspace,
                                 S(stream));
    return launched(launch_fused(g, L, pr->sim.kind, pr->sim.lcc_window, pr->sim.eps, pr->lambda,
                                 fixed, moving, ctrl, value_dev, grad_ctrl, workspace, S(stream)));
}

al_status al_adam_step(const al_bspline *bs, const al_adam_params *p, float *ctrl,
                       const float *grad_ctrl, float *m, float *v, int64_t *step_dev,
                       al_stream stream)
{
    Grid g;
    Lattice L;
    al_status st = check_bspline(bs, &g, &L);
    if (st != AL_OK)
        return st;
    if (!p || !ctrl || !grad_ctrl || !m || !v || !step_dev)
        return AL_ERR_INVALID_ARG;
    if (!(p->lr >= 0.0) || !isfinite(p->lr) || !(p->beta1 >= 0.0 && p->beta1 < 1.0) ||
        !(p->beta2 >= 0.0 && p->beta2 < 1.0) || !(p->eps > 0.0) || !isfinite(p->eps))
        return AL_ERR_INVALID_ARG;
    if (!aligned16(ctrl) || !aligned16(grad_ctrl) || !aligned16(m) || !aligned16(v) ||
        !aligned16(step_dev))
        return AL_ERR_ALIGN;
    AdamArgs a{};
    a.beta1 = p->beta1;
    a.beta2 = p->beta2;
    a.lr = (float)p->lr;
    a.eps = (float)p->eps;
    for (int k = 0; k < 3; ++k)
        a.h[k] = k < g.ndim ? (float)((bs->grid.size[k] - 1) / 2.0) : 0.0f;
    a.nc = L.nc;
    a.ndim = g.ndim;
    return launched(launch_adam(a, step_dev, ctrl, grad_ctrl, m, v, S(stream)));
}

al_status al_pyramid_grid(const al_grid *gr, int32_t factor, al_grid *level)
{
    if (!level)
        return AL_ERR_INVALID_ARG;
    al_status st = check_grid(gr, nullptr);
    if (st != AL_OK)
        return st;
    if (factor < 1 || factor > kMaxPyramidFactor)
        return AL_ERR_INVALID_ARG;
    al_grid out = *gr;
    for (int k = 0; k < gr->ndim; ++k) {
        out.size[k] = (gr->size[k] - 1) / factor + 1;
        if (out.size[k] < 2)
            return AL_ERR_SHAPE;
    }
    *level = out;
    return AL_OK;
}

size_t al_pyramid_workspace_bytes(const al_grid *gr, int32_t factor)
{
    Grid g;
    al_grid lv;
    if (check_grid(gr, &g) != AL_OK || al_pyramid_grid(gr, factor, &lv) != AL_OK)
        return 0;
    return pyramid_ws(g, factor);
}

al_status al_pyramid_level(const al_grid *gr, const float *image, int32_t factor, float *level,
                           void *workspace, size_t workspace_bytes, al_stream stream)
{
    Grid g;
    al_grid lv;
    al_status st = check_grid(gr, &g);
    if (st != AL_OK)
        return st;
    if ((st = al_pyramid_grid(gr, factor, &lv)) != AL_OK)
        return st;
    if (!image || !level)
        return AL_ERR_INVALID_ARG;
    const size_t need = pyramid_ws(g, factor);
    if (need > 0 && (!workspace || workspace_bytes < need))
        return AL_ERR_WORKSPACE;
    if (!aligned16(image) || !aligned16(level) || (need > 0 && !aligned16(workspace)))
        return AL_ERR_ALIGN;
    // Gaussian taps, sigma = factor/2, |t| <= 3 sigma, unit sum (double, then fp32)
    GaussTaps t{};
    if (factor > 1) {
        const double sigma = factor / 2.0;
        t.r = (int)floor(3.0 * sigma);
        double w[sizeof(t.w) / sizeof(t.w[0])], sum = 0.0;
        for (int k = -t.r; k <= t.r; ++k) {
            w[k + t.r] = exp(-(double)(k * k) / (2.0 * sigma * sigma));
            sum += w[k + t.r];
        }
        for (int k = 0; k <= 2 * t.r; ++k)
            t.w[k] = (float)(w[k] / sum);
    }
    return launched(launch_pyramid(g, factor, t, image, level, workspace, S(stream)));
}

al_status al_bspline_refine(const al_bspline *coarse, const float *ctrl_coarse,
                            const al_bspline *fine, float *ctrl_fine, al_stream stream)
{
    Grid gc, gf;
    Lattice Lc, Lf;
    al_status st = check_bspline(coarse, &gc, &Lc);
    if (st != AL_OK)
        return st;
    if ((st = check_bspline(fine, &gf, &Lf)) != AL_OK)
        return st;
    if (!ctrl_coarse || !ctrl_fine)
        return AL_ERR_INVALID_ARG;
    if (gc.ndim != gf.ndim || coarse->spacing != fine->spacing)
        return AL_ERR_SHAPE;
    const int nc[3] = {Lc.nx, Lc.ny, Lc.nz}, nf[3] = {Lf.nx, Lf.ny, Lf.nz};
    for (int k = 0; k < gc.ndim; ++k) {
        if ((fine->grid.size[k] - 1) / 2 + 1 != coarse->grid.size[k])
            return AL_ERR_SHAPE;
        // taps of the last fine point: (nf - 2)/2 + 2 must be a coarse index
        // (the first point, i = 0, takes coarse 0 and 1)
        if ((nf[k] - 2) / 2 + 2 > nc[k] - 1 || nc[k] < 2)
            return AL_ERR_SHAPE;
    }
    if (!aligned16(ctrl_coarse) || !aligned16(ctrl_fine))
        return AL_ERR_ALIGN;
    return launched(launch_refine(gc.ndim, nc, nf, ctrl_coarse, ctrl_fine, S(stream)));
}

static bool steps_ok(int32_t steps) { return steps >= 0 && steps <= 20; }

al_status al_exp_field(const al_grid *gr, int32_t steps, const float *velocity, float *disp,
                       float *trajectory, void *workspace, size_t workspace_bytes,
                       al_stream stream)
{
    Grid g;
    al_status st = check_grid(gr, &g);
    if (st != AL_OK)
        return st;
    if (!steps_ok(steps))
        return AL_ERR_INVALID_ARG;
    if (!velocity || !disp)
        return AL_ERR_INVALID_ARG;
    const size_t field = (size_t)g.ndim * g.nv * sizeof(float);
    const bool need_tmp = steps > 0 && !trajectory;
    if (need_tmp && (!workspace || workspace_bytes < field))
        return AL_ERR_WORKSPACE;
    if (!aligned16(velocity) || !aligned16(disp) || (trajectory && !aligned16(trajectory)) ||
        (need_tmp && !aligned16(workspace)))
        return AL_ERR_ALIGN;
    return launched(launch_exp(g, steps, velocity, disp, trajectory,
                               need_tmp ? (float *)workspace : nullptr, S(stream)));
}

size_t al_exp_field_workspace_bytes(const al_grid *gr)
{
    Grid g;
    if (check_grid(gr, &g) != AL_OK)
        return 0;
    return (size_t)g.ndim * g.nv * sizeof(float);
}

al_status al_exp_field_adjoint(const al_grid *gr, int32_t steps, const float *trajectory,
                               const float *grad_disp, float *grad_velocity, void *workspace,
                               size_t workspace_bytes, al_stream stream)
{
    Grid g;
    al_status st = check_grid(gr, &g);
    if (st != AL_OK)
        return st;
    if (!steps_ok(steps))
        return AL_ERR_INVALID_ARG;
    if (!grad_disp || !grad_velocity || (steps > 0 && !trajectory))
        return AL_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < exp_adjoint_ws(g))
        return AL_ERR_WORKSPACE;
    if ((trajectory && !aligned16(trajectory)) || !aligned16(grad_disp) ||
        !aligned16(grad_velocity) || !aligned16(workspace))
        return AL_ERR_ALIGN;
    return launched(
        launch_exp_adjoint(g, steps, trajectory, grad_disp, grad_velocity, workspace, S(stream)));
}

size_t al_exp_field_adjoint_workspace_bytes(const al_grid *gr)
{
    Grid g;
    if (check_grid(gr, &g) != AL_OK)
        return 0;
    return exp_adjoint_ws(g);
}

namespace {

// Workspace of the diffeomorphic objective: v, the trajectory, u_K, W, mask,
// dS/dW, dJ/du, dJ/dv, value slots, and scratch shared by the step calls.
struct DiffeoLayout {
    size_t v, traj, u, W, m, gW, gu, gv, vals, scratch, total;
};

DiffeoLayout diffeo_layout(const Grid &g, const Lattice &L, int kind, int window, int K)
{
    DiffeoLayout o{};
    const size_t nv = (size_t)g.nv, field = a256(nv * g.ndim * 4);
    size_t off = 0;
    o.v = off;
    off += field;
    o.traj = off;
    off += (size_t)K * field;
    o.u = off;
    off += field;
    o.W = off;
    off += a256(nv * 4);
    o.m = off;
    off += a256(nv);
    o.gW = off;
    off += a256(nv * 4);
    o.gu = off;
    off += field;
    o.gv = off;
    off += field;
    o.vals = off;
    off += 256;
    o.scratch = off;
    size_t mx = similarity_ws(g, kind, window);
    const size_t cand[3] = {regulariser_ws(g), displacement_adjoint_ws(g, L), exp_adjoint_ws(g)};
    for (size_t c : cand)
        mx = c > mx ? c : mx;
    off += a256(mx);
    o.total = off;
    return o;
}

}  // namespace

size_t al_objective_diffeo_workspace_bytes(const al_problem *pr, int32_t steps)
{
    Grid g;
    Lattice L;
    if (check_problem(pr, &g, &L) != AL_OK || !steps_ok(steps))
        return 0;
    return diffeo_layout(g, L, pr->sim.kind, pr->sim.lcc_window, steps).total;
}

al_status al_objective_grad_diffeo(const al_problem *pr, int32_t steps, const float *fixed,
                                   const float *moving, const float *ctrl, double *value_dev,
                                   float *grad_ctrl, void *workspace, size_t workspace_bytes,
                                   al_stream stream)
{
    Grid g;
    Lattice L;
    al_status st = check_problem(pr, &g, &L);
    if (st != AL_OK)
        return st;
    if (!steps_ok(steps))
        return AL_ERR_INVALID_ARG;
    if (!fixed || !moving || !ctrl || !value_dev)
        return AL_ERR_INVALID_ARG;
    const DiffeoLayout lay = diffeo_layout(g, L, pr->sim.kind, pr->sim.lcc_window, steps);
    if (!workspace || workspace_bytes < lay.total)
        return AL_ERR_WORKSPACE;
    if (!aligned16(fixed) || !aligned16(moving) || !aligned16(ctrl) || !aligned16(value_dev) ||
        !aligned16(workspace) || (grad_ctrl && !aligned16(grad_ctrl)))
        return AL_ERR_ALIGN;
    char *w = (char *)workspace;
    float *v = (float *)(w + lay.v), *traj = steps > 0 ? (float *)(w + lay.traj) : nullptr;
    float *u = (float *)(w + lay.u), *W = (float *)(w + lay.W), *gW = (float *)(w + lay.gW);
    float *gu = (float *)(w + lay.gu), *gv = (float *)(w + lay.gv);
    uint8_t *m = (uint8_t *)(w + lay.m);
    double *vals = (double *)(w + lay.vals);
    void *scratch = w + lay.scratch;
    const cudaStream_t s = S(stream);
    if (launch_displacement(g, L, ctrl, v, s) != cudaSuccess ||
        launch_exp(g, steps, v, u, traj, nullptr, s) != cudaSuccess ||
        launch_warp(g, moving, u, W, m, s) != cudaSuccess ||
        launch_similarity(g, pr->sim.kind, pr->sim.lcc_window, pr->sim.eps, fixed, W, m, vals,
                          grad_ctrl ? gW : nullptr, scratch, s) != cudaSuccess ||
        launch_regulariser(g, u, pr->lambda, vals + 2, grad_ctrl ? gu : nullptr, scratch, s) !=
            cudaSuccess)
        return AL_ERR_CUDA;
    if (grad_ctrl) {
        if (launch_warp_adjoint(g, moving, u, m, gW, gu, 1, s) != cudaSuccess ||
            launch_exp_adjoint(g, steps, traj, gu, gv, scratch, s) != cudaSuccess ||
            launch_displacement_adjoint(g, L, gv, grad_ctrl, scratch, s) != cudaSuccess)
            return AL_ERR_CUDA;
    }
    return launched(launch_combine(vals, vals + 2, pr->lambda, value_dev, s));
}

al_status al_lcc_set_wait(int32_t drop_slice)
{
    if (drop_slice < -1)
        return AL_ERR_INVALID_ARG;
    return lcc_set_drop_slice((int)drop_slice) == cudaSuccess ? AL_OK : AL_ERR_CUDA;
}

al_status al_fused_set_wait(int32_t drop_batch)
{
    if (drop_batch < -1)
        return AL_ERR_INVALID_ARG;
    return fused_set_drop_batch((int)drop_batch) == cudaSuccess ? AL_OK : AL_ERR_CUDA;
}

al_status al_get_device_error(al_stream stream)
{
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess)
        return AL_ERR_CUDA;
    int h = 0;
    if (cudaMemcpyFromSymbol(&h, g_device_error, sizeof(int)) != cudaSuccess)
        return AL_ERR_CUDA;
    if (h != 0) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_device_error, &zero, sizeof(int)) != cudaSuccess)
            return AL_ERR_CUDA;
    }
    const int others[5] = {conv_device_error(true), unit_error_basic(true),
                           unit_error_fused(true), unit_error_conv(true), unit_error_lcc(true)};
    for (int k = 0; k < 5; ++k) {
        if (others[k] < 0)
            return AL_ERR_CUDA;
        if (h == 0)
            h = others[k];
    }
    return h == 0 ? AL_OK : (al_status)h;
}

}  // extern "C"
