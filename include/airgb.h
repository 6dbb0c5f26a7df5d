/*
 * airgb.h - C ABI of libairgb.so: the regularised B-spline registration
 * objective of AIRLab (arXiv 1806.09907) and its exact gradient with respect
 * to the control points, as hand-written CUDA kernels for sm_103a (GB300).
 *
 * The objective (Sec. II-A, Eq. objective):
 *     J(c) = S(I_M o (x + u_c), I_F) + lambda * R_diff(u_c)
 * with u_c the cubic B-spline expansion of the control coefficients c
 * (Eq. kernel_basis, Sec. III-C), the backward warp with linear
 * interpolation and the out-of-domain mask (Sec. III-C, Image Warping), the
 * MSE / NCC / LCC similarity (Eq. mse, Sec. III-B) and the diffusion
 * regulariser (Eq. diffusion_regularizer, Sec. III-F).
 *
 * Conventions shared by every call
 *  - Grid: ndim 2 or 3, sizes X, Y, Z (Z = 1 in 2D, every active size >= 2).
 *    Volumes are fp32, x fastest: element (x,y,z) at (z*Y + y)*X + x.
 *  - Vector fields (displacements and their gradients) are ndim component
 *    planes, component 0 = x: u[i*X*Y*Z + voxel]. Voxel units.
 *  - Control lattice with integer spacing delta: n_k = (N_k - 1)/delta + 4
 *    points per active axis (n_z = 1 in 2D), point j at voxel coordinate
 *    (j - 1)*delta; coefficients are ndim planes c[i][jz][jy][jx], voxel units.
 *    The kernel is k_B1D(r/delta) per axis (tensor product).
 *  - Warp: y = x + u(x); a voxel is outside the mask when some y_k < 0 or
 *    y_k > N_k - 1 (or y_k is not finite); outside voxels have W = 0.
 *    Linear interpolation uses the floor cell clamped to [0, N_k - 2].
 *  - Similarities run over the masked voxels: MSE is the mean over them, NCC
 *    is 1 - Pearson correlation over them, LCC is 1 - the mean over them of
 *    the correlation in a centred box window (zero padding, fixed count
 *    window^ndim). eps is added to var_F*var_W under the square root.
 *  - R_diff uses forward differences with the out-of-grid difference dropped,
 *    divided by the number of voxels.
 *
 * Memory and streams
 *  - Every array pointer is DEVICE memory owned by the caller, contiguous,
 *    16-byte aligned (AL_ERR_ALIGN otherwise). Results are written to device
 *    memory; nothing is copied to the host and no call synchronises, except
 *    al_get_device_error. Calls are asynchronous on `stream` (a cudaStream_t;
 *    NULL = the legacy default stream).
 *  - The library allocates no device memory. Calls that need scratch take a
 *    caller-owned workspace of at least the size the matching
 *    *_workspace_bytes function returns (AL_ERR_WORKSPACE otherwise); its
 *    contents on entry do not matter. Two calls that share a workspace or an
 *    output must be ordered on the GPU by the caller.
 *  - Gradients are overwritten, not accumulated, unless a call says so. A NULL
 *    gradient pointer means value only, where allowed.
 *  - Results are deterministic: sums use fixed-order reductions, no atomics.
 *
 * Errors
 *  - Argument, shape, alignment and workspace errors are detected on the host
 *    before anything is launched; the call returns that status and leaves
 *    every output untouched.
 *  - A failed kernel launch returns AL_ERR_CUDA (the CUDA error is left for
 *    the caller to read with cudaGetLastError).
 *  - Errors found by the kernels themselves are recorded in a per-device
 *    error word that al_get_device_error reads and clears.
 *  - No call aborts, traps or throws.
 */
#ifndef AIRGB_H
#define AIRGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AL_OK = 0,
    AL_ERR_INVALID_ARG = 1, /* NULL pointer, bad enum, bad spacing/window/eps */
    AL_ERR_SHAPE = 2,       /* grid or lattice sizes inconsistent or unsupported */
    AL_ERR_ALIGN = 3,       /* a pointer is not 16-byte aligned */
    AL_ERR_CUDA = 4,        /* a CUDA runtime call or launch failed */
    AL_ERR_BOUNDS = 5,      /* a kernel saw an index out of range (checked builds) */
    AL_ERR_TIMEOUT = 6,     /* a bounded device-side wait ran out */
    AL_ERR_UNSUPPORTED = 7, /* valid but not supported by this library */
    AL_ERR_WORKSPACE = 8,   /* workspace missing or too small */
    AL_ERR_SCRATCH_LIMIT = 9 /* problem needs more than the built-in scratch of the
                                allocation-free entry point */
} al_status;

typedef enum { AL_SIM_MSE = 0, AL_SIM_NCC = 1, AL_SIM_LCC = 2 } al_sim_kind;

/* cudaStream_t, passed as an opaque pointer so this header needs no CUDA. */
typedef void *al_stream;

/* Image grid (Sec. II-A: the regular point set X). */
typedef struct {
    int32_t ndim;    /* 2 or 3 */
    int32_t reserved;
    int64_t size[3]; /* X, Y, Z; Z = 1 when ndim = 2 */
} al_grid;

/* Cubic B-spline transformation on a control lattice (Sec. III-C). */
typedef struct {
    al_grid grid;
    int32_t spacing; /* delta, control spacing in voxels, 1..32 */
    int32_t reserved;
    int64_t n[3];    /* lattice size nx, ny, nz; filled by al_bspline_init */
} al_bspline;

/* Similarity measure (Sec. III-B). */
typedef struct {
    int32_t kind;       /* al_sim_kind */
    int32_t lcc_window; /* odd LCC window width (default 7): 3, 5 or 7; other odd
                           widths up to 15 return AL_ERR_UNSUPPORTED */
    double eps;         /* added to var_F*var_W, >= 0 (default 1e-5) */
} al_sim_params;

/* One registration objective (Eq. objective): transformation, similarity
 * and the weight lambda of the diffusion regulariser. */
typedef struct {
    al_bspline bs;
    al_sim_params sim;
    double lambda;
} al_problem;

/* Text for a status code (static storage). */
const char *al_status_string(al_status status);

/* Fill *bs for grid *g and spacing delta: checks the grid (ndim 2/3, sizes
 * >= 2 on active axes, Z = 1 in 2D, at most 2^31 voxels) and sets
 * bs->n = (N - 1)/delta + 4 per active axis (Sec. III-C; lattice placement
 * is a reading, the paper gives none). Host only, launches nothing. */
al_status al_bspline_init(al_bspline *bs, const al_grid *g, int32_t spacing);

/* A1. Displacement u = sum_j c_j k(x_j, x) (Eq. kernel_basis, Sec. III-C:
 * the control points are up-sampled with the B-spline as interpolation
 * kernel). ctrl: ndim * nz*ny*nx floats; disp: ndim * Z*Y*X floats
 * (overwritten). */
al_status al_displacement(const al_bspline *bs, const float *ctrl, float *disp, al_stream stream);

/* A1 + A2 for `count` volumes at once, without materialising the field:
 * warped[v] = moving[v] o (x + u_v), u_v = the displacement of ctrl[v] (as
 * al_displacement), with the masked trilinear warp of al_warp; mask[v]
 * written when mask is not NULL. moving, warped: count volumes of Z*Y*X
 * floats; ctrl: count lattices of ndim * nz*ny*nx floats; mask: count * Z*Y*X
 * bytes. The arithmetic is that of al_objective_grad's fused path. Spacings
 * 4, 6 and 8 (AL_ERR_UNSUPPORTED otherwise); count 1 .. 65535. */
al_status al_warp_ctrl(const al_bspline *bs, int32_t count, const float *moving,
                       const float *ctrl, float *warped, uint8_t *mask, al_stream stream);

/* A6. Adjoint of al_displacement (the transposed up-sampling):
 * grad_ctrl[i,j] = sum_x k(x_j, x) grad_disp[i](x), computed as a gather per
 * control point (fixed order, no atomics). grad_ctrl is overwritten.
 * Workspace: al_displacement_adjoint_workspace_bytes(bs). */
al_status al_displacement_adjoint(const al_bspline *bs, const float *grad_disp, float *grad_ctrl,
                                  void *workspace, size_t workspace_bytes, al_stream stream);
size_t al_displacement_adjoint_workspace_bytes(const al_bspline *bs);

/* A2. Backward warp (Sec. III-C, Image Warping): warped = m * M~(x + u),
 * mask = m (1 inside, 0 outside), both overwritten. moving, warped: Z*Y*X
 * floats; disp: ndim planes; mask: Z*Y*X bytes. */
al_status al_warp(const al_grid *g, const float *moving, const float *disp, float *warped,
                  uint8_t *mask, al_stream stream);

/* A5. Adjoint of the warp with respect to the displacement (the exact
 * gradient, Sec. III-A): grad_disp[k](x) = mask(x) * grad_warped(x) *
 * dM~/dy_k(x + u(x)), the derivative of the linear interpolant inside its
 * (clamped) floor cell. accumulate = 0 overwrites grad_disp, 1 adds to it. */
al_status al_warp_adjoint(const al_grid *g, const float *moving, const float *disp,
                          const uint8_t *mask, const float *grad_warped, float *grad_disp,
                          int32_t accumulate, al_stream stream);

/* A3. Similarity S(W, F) over the mask (Eq. mse; NCC and LCC of Sec. III-B)
 * and its gradient dS/dW (grad_warped, nullable, overwritten; zero off the
 * mask). value_dev: 2 doubles on the device, {S, number of masked voxels}.
 * Workspace: al_similarity_workspace_bytes(g, p). */
al_status al_similarity(const al_grid *g, const al_sim_params *p, const float *fixed,
                        const float *warped, const uint8_t *mask, double *value_dev,
                        float *grad_warped, void *workspace, size_t workspace_bytes,
                        al_stream stream);
size_t al_similarity_workspace_bytes(const al_grid *g, const al_sim_params *p);

/* A4. Diffusion regulariser R (Eq. diffusion_regularizer) of a displacement
 * field and weight * dR/du (grad_disp, nullable, overwritten).
 * value_dev: 1 double on the device, R (unweighted).
 * Workspace: al_regulariser_workspace_bytes(g). */
al_status al_regulariser(const al_grid *g, const float *disp, double weight, double *value_dev,
                         float *grad_disp, void *workspace, size_t workspace_bytes,
                         al_stream stream);
size_t al_regulariser_workspace_bytes(const al_grid *g);

/* A7. One evaluation of J = S + lambda R (Eq. objective) and dJ/dc, fused:
 * the displacement, warped image and per-voxel gradients stay on chip (LCC
 * keeps the warped image and its gradient in the workspace); R and dR/dc are
 * evaluated on the control lattice in Gram form, which equals the voxel sum.
 * value_dev: 4 doubles on the device, {J, S, R, number of masked voxels}.
 * grad_ctrl: ndim * nz*ny*nx floats, nullable (value only), overwritten.
 * Workspace: al_objective_workspace_bytes(pr). */
al_status al_objective_grad(const al_problem *pr, const float *fixed, const float *moving,
                            const float *ctrl, double *value_dev, float *grad_ctrl,
                            void *workspace, size_t workspace_bytes, al_stream stream);
size_t al_objective_workspace_bytes(const al_problem *pr);

/* Where a fused LCC evaluation keeps its warped image: byte offsets, inside
 * the workspace of al_objective_grad, of W (fp32, X*Y*Z values, zero off the
 * mask; Sec. III-C, Image Warping) and of the mask (one byte per voxel) that
 * the last al_objective_grad call on that workspace wrote. For inspection
 * and tests; the layout belongs to this library version. AL_ERR_UNSUPPORTED
 * when the evaluation keeps W on chip (MSE, NCC) or runs unfused. */
al_status al_objective_warped_offsets(const al_problem *pr, size_t *warped_offset,
                                      size_t *mask_offset);

/* The same evaluation as the composition of the step calls above
 * (A1 -> A2 -> A3, A4 -> A5 -> A6), with every intermediate field in the
 * workspace. Same arguments and results as al_objective_grad.
 * Workspace: al_objective_unfused_workspace_bytes(pr). */
al_status al_objective_grad_unfused(const al_problem *pr, const float *fixed, const float *moving,
                                    const float *ctrl, double *value_dev, float *grad_ctrl,
                                    void *workspace, size_t workspace_bytes, al_stream stream);
size_t al_objective_unfused_workspace_bytes(const al_problem *pr);

/* The similarity step A3 for callers that cannot allocate device memory
 * (the paper has no counterpart: it is a service of this library). Some
 * hosts cannot provide a workspace: their device memory belongs to another
 * allocator that must see every allocation (a framework's caching pool, an
 * embedded runtime that forbids allocation after start-up), or they are
 * plain C programs without a device allocator. This call takes its scratch
 * from a fixed array in the library's own device memory,
 * al_noalloc_scratch_bytes() bytes (4 MiB) held on every GPU that loads the
 * library until the process exits, and calls no allocating routine.
 * Arguments and results are those of al_similarity without the workspace.
 * A problem whose workspace (al_similarity_workspace_bytes) exceeds the
 * array returns AL_ERR_SCRATCH_LIMIT and launches nothing: MSE and NCC fit
 * at any size, LCC up to about 340,000 voxels.
 * All calls on a device share the array and leave their data in it; calls
 * whose kernels overlap on the GPU race on it, so order them. The first call
 * in each context of a device looks up the array's device address
 * (cudaGetSymbolAddress with that device current) and caches it with the
 * context's id, so a call after a device reset looks it up again: make the
 * first call of a context before any stream capture. A failed lookup
 * returns AL_ERR_CUDA and leaves no runtime error set. */
al_status al_similarity_noalloc(const al_grid *g, const al_sim_params *p, const float *fixed,
                                const float *warped, const uint8_t *mask, double *value_dev,
                                float *grad_warped, al_stream stream);
size_t al_noalloc_scratch_bytes(void);

/* ---- The optimisation loop around the objective ---------------------------
 * Gradient-based optimisation of J (Sec. II-A, Optimization) with Adam
 * (Sec. III-G; the usage example of Sec. IV sets lr = 0.01) and the
 * multi-resolution strategy of the FFD experiment (Sec. IV-A): Gaussian image
 * pyramid, coarse-to-fine levels, coefficients carried to the next level. */

/* Adam hyper-parameters. lr is in the paper's normalised coordinates, where
 * the image spans [-1, 1] per axis (Sec. III-C, Image Warping). */
typedef struct {
    double lr;    /* step size, >= 0 (0.01) */
    double beta1; /* first-moment decay, in [0, 1) (0.9) */
    double beta2; /* second-moment decay, in [0, 1) (0.999) */
    double eps;   /* added to sqrt(v^), > 0 (1e-8) */
} al_adam_params;

/* One Adam step (Kingma and Ba's update) on the control coefficients of bs,
 * taken in normalised units c~_k = c_k * 2/(N_k - 1): with g~ the normalised
 * gradient and t = *step_dev + 1,
 *   m <- beta1 m + (1 - beta1) g~,  v <- beta2 v + (1 - beta2) g~^2,
 *   c~ <- c~ - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).
 * ctrl (updated in place) and grad_ctrl are in voxel units, ndim * nz*ny*nx
 * floats; m and v (same size, zero before the first step) hold the moments
 * in normalised units. step_dev: one int64 on the device, the number of steps
 * taken so far; the call stores t there after the update, so the call can be
 * captured in a CUDA graph and replayed. Two launches, no host read. */
al_status al_adam_step(const al_bspline *bs, const al_adam_params *p, float *ctrl,
                       const float *grad_ctrl, float *m, float *v, int64_t *step_dev,
                       al_stream stream);

/* Grid of one pyramid level: every factor-th voxel from voxel 0 on each
 * active axis, size (N_k - 1)/factor + 1. factor 1..8; AL_ERR_SHAPE if an
 * active axis of the level would have fewer than 2 voxels. Host only. */
al_status al_pyramid_grid(const al_grid *g, int32_t factor, al_grid *level);

/* One pyramid level of an image (Sec. IV-A, multi-resolution; the filter is
 * a reading, the paper gives none): factor 1 copies the image; factor >= 2
 * smooths it with a Gaussian of sigma = factor/2 voxels, truncated to the
 * taps |t| <= 3 sigma, normalised to unit sum, with indices clamped to the
 * grid, and keeps every factor-th voxel from voxel 0. image: the grid *g;
 * level: the grid al_pyramid_grid returns (overwritten).
 * Workspace: al_pyramid_workspace_bytes(g, factor) (0 for factor 1). */
al_status al_pyramid_level(const al_grid *g, const float *image, int32_t factor, float *level,
                           void *workspace, size_t workspace_bytes, al_stream stream);
size_t al_pyramid_workspace_bytes(const al_grid *g, int32_t factor);

/* Coefficients of the next finer level whose displacement equals the coarse
 * one at every coarse voxel (exact dyadic refinement of the cubic B-spline
 * by its two-scale relation), in fine voxel units. coarse->grid must be
 * al_pyramid_grid(fine->grid, 2) and both lattices must have the same
 * spacing (AL_ERR_SHAPE otherwise). ctrl_coarse: ndim planes of the coarse
 * lattice; ctrl_fine: ndim planes of the fine lattice (overwritten). */
al_status al_bspline_refine(const al_bspline *coarse, const float *ctrl_coarse,
                            const al_bspline *fine, float *ctrl_fine, al_stream stream);

/* ---- Diffeomorphic B-spline transformation (Sec. III-D) ---------------------
 * f = exp(v) of the stationary velocity field v (here the B-spline field of
 * c), computed by scaling and squaring, the method of the works the section
 * cites: u_0 = v / 2^steps, u_{k+1}(x) = u_k(x) + u~_k(x + u_k(x)),
 * f = x + u_steps. u~_k is the linear interpolant of u_k at the sample
 * position clamped to the grid (a field has no mask; along a clamped axis
 * its derivative is 0). steps: 0..20 (the paper gives no number; 6 is this
 * library's default in its bindings). The inverse is exp(-v). */

/* disp = exp(v) - x (ndim planes, voxel units). trajectory (nullable):
 * steps * ndim * nv floats receiving u_0 .. u_{steps-1}, the inputs of the
 * squarings, which al_exp_field_adjoint needs. Without a trajectory and with
 * steps > 0 the call needs a workspace of al_exp_field_workspace_bytes(g). */
al_status al_exp_field(const al_grid *g, int32_t steps, const float *velocity, float *disp,
                       float *trajectory, void *workspace, size_t workspace_bytes,
                       al_stream stream);
size_t al_exp_field_workspace_bytes(const al_grid *g);

/* Adjoint of al_exp_field: grad_velocity = (d disp / d v)^T grad_disp, from
 * its trajectory. The transposed interpolation of each squaring is a scatter;
 * it is summed in 64-bit fixed point with integer atomics (scaled per
 * squaring from the largest |gradient|), so the result is deterministic.
 * Workspace: al_exp_field_adjoint_workspace_bytes(g) (12 * ndim bytes per
 * voxel). */
al_status al_exp_field_adjoint(const al_grid *g, int32_t steps, const float *trajectory,
                               const float *grad_disp, float *grad_velocity, void *workspace,
                               size_t workspace_bytes, al_stream stream);
size_t al_exp_field_adjoint_workspace_bytes(const al_grid *g);

/* J = S(M o f, F) + lambda R_diff(u_steps) with f = exp(v), v the B-spline
 * field of ctrl, and dJ/dc (grad_ctrl nullable): A1, the exponential, A2,
 * A3 and A4 on u_steps, then A5, the exponential's adjoint and A6, through
 * the step kernels. value_dev: {J, S, R, n_mask}. The workspace keeps the
 * trajectory (steps + 5 fields of ndim planes and 3 scalar volumes):
 * al_objective_diffeo_workspace_bytes(pr, steps). */
al_status al_objective_grad_diffeo(const al_problem *pr, int32_t steps, const float *fixed,
                                   const float *moving, const float *ctrl, double *value_dev,
                                   float *grad_ctrl, void *workspace, size_t workspace_bytes,
                                   al_stream stream);
size_t al_objective_diffeo_workspace_bytes(const al_problem *pr, int32_t steps);

/* ---- Batches of independent problems ---------------------------------------
 * Many registration pairs of uneven sizes optimised together (the paper
 * registers one pair at a time; this is a throughput service of the
 * library): every iteration of every problem -- the fused objective and
 * gradient of its MSE objective and its Adam step -- runs in ONE persistent
 * kernel launch whose blocks take work items from a device queue. A batch
 * holds problems of one spacing in {4, 6, 8} with the MSE similarity, 2D and
 * 3D mixed (AL_ERR_UNSUPPORTED otherwise). Each problem's coefficients follow
 * the same arithmetic as al_objective_grad + al_adam_step, bit for bit. */
typedef struct al_batch al_batch; /* opaque host-side plan */

/* Plan a batch of `count` problems (host only, allocates host memory only;
 * free it with al_batch_destroy). */
al_status al_batch_create(const al_problem *problems, int32_t count, al_batch **out);
void al_batch_destroy(al_batch *batch);
/* Device workspace of the batch: queue counters, descriptors, work items and
 * every problem's partial sums. */
size_t al_batch_workspace_bytes(const al_batch *batch);
/* Number of work items of one iteration; per_kind (nullable, 3 entries)
 * receives the bricks, Gram tiles and control chunks among them. */
int32_t al_batch_items(const al_batch *batch, int32_t *per_kind);

/* Attach the problems' device arrays (host arrays of `count` device
 * pointers): fixed and moving images, coefficients (updated in place by
 * al_batch_step), Adam moments m and v (zero before the first step), and
 * optional value histories values[i] (nullable array or entries) of rows of
 * 4 doubles {J, S, R, n_mask}. Uploads the descriptors and the work items to
 * the workspace with synchronous copies (not capturable; call it before any
 * capture). The workspace stays bound to the batch until the next bind. */
al_status al_batch_bind(al_batch *batch, const float *const *fixed, const float *const *moving,
                        float *const *ctrl, float *const *adam_m, float *const *adam_v,
                        double *const *values, void *workspace, size_t workspace_bytes);

/* One Adam iteration (Sec. II-A, Optimization) of every problem: J and dJ/dc
 * at the current coefficients, then the Adam step t = `step` (1-based) as
 * al_adam_step takes it. When record >= 0, row `record` of each value
 * history receives {J, S, R, n_mask} before the step. A memset and one
 * kernel launch on `stream`: capturable in a CUDA graph. */
al_status al_batch_step(const al_batch *batch, const al_adam_params *p, int64_t step,
                        int32_t record, al_stream stream);

/* Autotuner: times `iterations` gradient-only iterations (coefficients and
 * moments untouched) of every (brick tile, work-item order) configuration
 * and keeps the fastest. The batch kernel is built for al_batch_tiles()
 * brick tiles of the batch's spacing (tile 0 is al_objective_grad's brick;
 * a tile sets the cells of control lattice a block covers in x and y, hence
 * its threads, its share of shared memory and registers, and the number of
 * work items); the orders are 0 problems as given, 1 largest problem first,
 * 2 round-robin over problems, 3 Gram tiles first. ms (nullable,
 * al_batch_tiles() x 4 entries, tile-major) receives the milliseconds per
 * iteration of each configuration, chosen_tile / chosen_policy (nullable)
 * the one kept. Synchronises the stream and rewrites the bound descriptors;
 * not capturable. Coefficients follow al_objective_grad + al_adam_step bit
 * for bit with tile 0; with another tile the partial sums are grouped by
 * other bricks, so they agree to fp32 rounding. */
al_status al_batch_tune(al_batch *batch, const al_adam_params *p, int32_t iterations,
                        double *ms, int32_t *chosen_tile, int32_t *chosen_policy,
                        al_stream stream);
/* Select a work-item order directly (0..3). */
al_status al_batch_set_policy(al_batch *batch, int32_t policy);
/* Select a brick tile directly (0 .. al_batch_tiles() - 1; 0 by default).
 * After binding it rewrites the bound descriptors with synchronous copies. */
al_status al_batch_set_tile(al_batch *batch, int32_t tile);
/* Number of brick tiles; cells (nullable, 2 per tile) receives each tile's
 * control cells per block in x and y. */
int32_t al_batch_tiles(const al_batch *batch, int32_t *cells);

/* Bounded waits. A control chunk waits, polling a device counter, until
 * every brick and tile of its problem is done; after max_polls polls it
 * gives up, skips its work and records AL_ERR_TIMEOUT. extra_items > 0 makes
 * the chunks wait for items that do not exist (a test of the timeout path:
 * the kernel returns normally). Defaults: 0 and 20,000,000 polls. */
al_status al_batch_set_wait(al_batch *batch, int32_t extra_items, int64_t max_polls);

/* Synchronise `stream`, then read and clear the batch's error word: AL_OK or
 * AL_ERR_TIMEOUT. */
al_status al_batch_status(const al_batch *batch, al_stream stream);

/* ---- Learned initialisation: convolution layers and the network ------------
 * The paper names learning-based registration as planned work (Sec. I and
 * Sec. V) without a network. This library trains a 3D convolutional
 * encoder-decoder that maps a fixed/moving pair to the cubic B-spline
 * coefficients of spacing 8, which the plain optimiser (al_objective_grad +
 * al_adam_step) then refines. The layers below are the dense contractions of
 * that network, on the tensor cores (tcgen05, bf16 x bf16 with fp32
 * accumulation).
 *
 * Layout: channels last, [b][z][y][x][c], bf16 (uint16 storage) unless a
 * call says fp32. Weights are fp32 masters w[co][t][ci], tap
 * t = (dz+1)*9 + (dy+1)*3 + (dx+1) for offsets in {-1, 0, 1}^3; the layer
 * kernels read them as bf16 copies packed by al_conv3d_pack. */
typedef struct {
    int32_t batch;   /* volumes in the batch, >= 1 */
    int32_t cin;     /* input channels: 2, or a multiple of 8 up to 256 */
    int32_t cout;    /* output channels: a multiple of 16 up to 128 (pad with zero weights) */
    int32_t stride;  /* 1 or 2 */
    int64_t size[3]; /* input grid D, H, W (z, y, x), each 1 .. 2^20; batch*D*H*W < 2^31,
                        3*H*W*cin and 3*Ho*Wo*cout < 2^31 */
} al_conv3d;

/* Output grid (D, H, W): (n - 1)/stride + 1 per axis (zero padding 1). */
al_status al_conv3d_output_size(const al_conv3d *cv, int64_t *out_size);

/* Bytes of the packed bf16 weights for the forward pass (dgrad = 0) or the
 * input adjoint (dgrad = 1; needs cin a multiple of 16 up to 128); 0 for an
 * invalid layer. */
size_t al_conv3d_packed_bytes(const al_conv3d *cv, int32_t dgrad);

/* Round the fp32 weights (cout x 27 x cin) to bf16 and lay them out as the
 * layer kernels read them (K slices of 64 in the tensor cores' shared-memory
 * tile layout). Either packed pointer may be NULL (not both). */
al_status al_conv3d_pack(const al_conv3d *cv, const float *weight, void *packed_fwd,
                         void *packed_dgrad, al_stream stream);

/* out[b][o][co] = bias[co] + sum_t sum_ci in[b][stride*o + d_t][ci] w[co][t][ci]
 * (in = 0 outside the grid); relu != 0 applies max(., 0). input bf16
 * (batch x D x H x W x cin); bias fp32 (cout, nullable); output bf16, or fp32
 * when out_f32 != 0 (batch x output grid x cout).
 * workspace (nullable): when the layer has few output tiles (small batches,
 * coarse levels) the sum over K is split into up to 8 partitions run by
 * separate CTAs, whose fp32 partials (al_conv3d_forward_workspace_bytes, 0
 * when the layer is not split) are then added in a fixed order. A NULL or
 * smaller workspace runs the layer unsplit; both are deterministic and agree
 * to fp32 rounding. */
size_t al_conv3d_forward_workspace_bytes(const al_conv3d *cv);
al_status al_conv3d_forward(const al_conv3d *cv, const void *input, const void *packed_fwd,
                            const float *bias, int32_t relu, int32_t out_f32, void *output,
                            void *workspace, size_t workspace_bytes, al_stream stream);

/* Input adjoint of the layer's linear part:
 *   g_in[b][p][ci] = sum_{t, co} g_out[b][(p - d_t)/stride][co] w[co][t][ci]
 * over the output voxels that exist (integer, in range). Then, optionally,
 * g_in += addend[b][p][addend_offset + ci] (bf16, addend_stride channels per
 * voxel; both multiples of 8), and g_in *= (relu_input[b][p][ci] > 0) when
 * relu_input (bf16, cin channels) is given: the derivative of the ReLU
 * that produced this layer's input. grad_output bf16 (cout channels),
 * grad_input bf16 (cin channels, a multiple of 16). */
al_status al_conv3d_backward_data(const al_conv3d *cv, const void *grad_output,
                                  const void *packed_dgrad, const void *relu_input,
                                  const void *addend, int32_t addend_stride,
                                  int32_t addend_offset, void *grad_input, al_stream stream);

/* Weight and bias adjoints:
 *   g_w[co][t][ci] = sum_b sum_o g_out[b][o][co] in[b][stride*o + d_t][ci]
 *   g_b[co]        = sum_b sum_o g_out[b][o][co]
 * fp32, overwritten (grad_bias nullable). The sum over voxels is split over
 * blocks whose partials (the workspace) are added in a fixed order, so the
 * result is deterministic. */
size_t al_conv3d_backward_weight_workspace_bytes(const al_conv3d *cv);
al_status al_conv3d_backward_weight(const al_conv3d *cv, const void *input,
                                    const void *grad_output, float *grad_weight, float *grad_bias,
                                    void *workspace, size_t workspace_bytes, al_stream stream);

/* The network input of `count` pairs made by the method, with the fixed
 * image F = M o (x + B c) of each pair formed on the fly: x[b][v] = (F[b][v],
 * M[b][v]) as two bf16 channels, equal bit for bit to al_warp_ctrl followed
 * by al_initnet_input, without F in device memory. bs: a 3D grid with spacing
 * 4, 6 or 8 (AL_ERR_UNSUPPORTED otherwise); moving: count volumes; ctrl:
 * count lattices of 3 planes (voxel units); x: count x Z x Y x X x 2 bf16.
 * count 1 .. 65535; every array 16-byte aligned. */
al_status al_initnet_pair_input(const al_bspline *bs, int32_t count, const float *moving,
                                const float *ctrl, void *x, al_stream stream);

/* The network's input: x[b][v] = (F[b][v], M[b][v]) as two bf16 channels,
 * from fp32 volumes of `batch` x size[0] x size[1] x size[2] (z, y, x). */
al_status al_initnet_input(int32_t batch, const int64_t *size, const float *fixed,
                           const float *moving, void *x, al_stream stream);

/* cat = [up(e4), e3] on e3's grid n3 (z, y, x): up(e4)[z][y][x] =
 * e4[z/2][y/2][x/2], e4 on the grid (n3 - 1)/2 + 1, c4 + c3 channels (both
 * multiples of 8), bf16. */
al_status al_initnet_upcat(int32_t batch, const int64_t *n3, int32_t c4, int32_t c3,
                           const void *e4, const void *e3, void *cat, al_stream stream);
/* Transpose for the up-sampled channels, times the ReLU factor of e4:
 * grad_e4[v][c] = (e4[v][c] > 0) sum_{fine voxels copied from v} grad_cat[f][c]. */
al_status al_initnet_upcat_adjoint(int32_t batch, const int64_t *n3, int32_t c4, int32_t c3,
                                   const void *grad_cat, const void *e4, void *grad_e4,
                                   al_stream stream);

/* Head -> control coefficients of the spacing-8 lattice of bs (3D):
 * ctrl[b][i][jz][jy][jx] = head[b][clamp(jz-1)][clamp(jy-1)][clamp(jx-1)][i]
 * (control point j sits at voxel 8 (j - 1), where head voxel j - 1 sits;
 * points beyond the grid take the nearest). head fp32 on n3 = (N - 1)/8 + 1
 * per axis with `channels` per voxel (>= 3, a multiple of 4). */
al_status al_initnet_head_to_ctrl(const al_bspline *bs, int32_t batch, const int64_t *n3,
                                  int32_t channels, const float *head, float *ctrl,
                                  al_stream stream);
/* Its transpose: grad_head (bf16, zero beyond channel 2) from grad_ctrl. */
al_status al_initnet_head_adjoint(const al_bspline *bs, int32_t batch, const int64_t *n3,
                                  int32_t channels, const float *grad_ctrl, void *grad_head,
                                  al_stream stream);

/* Training loss of the network: the mean squared difference of two B-spline
 * displacement fields (Sec. III-C),
 *   L = 1/(3 |X| batch) sum_b sum_i sum_x (u_i(x) - u*_i(x))^2, u = B c, u* = B c*,
 * computed exactly on the lattice as e^T (G_z x G_y x G_x) e with e = c - c*
 * and G = B^T B per axis (banded), and dL/dc = 2/(3 |X| batch) (G x G x G) e.
 * ctrl, ctrl_true, grad_ctrl: batch x 3 coefficient planes; loss_dev: one
 * double. Workspace: al_field_loss_workspace_bytes(batch). At most about
 * 8,000 control points per component (AL_ERR_UNSUPPORTED beyond). */
size_t al_field_loss_workspace_bytes(int32_t batch);
al_status al_field_loss(const al_bspline *bs, int32_t batch, const float *ctrl,
                        const float *ctrl_true, double *loss_dev, float *grad_ctrl,
                        void *workspace, size_t workspace_bytes, al_stream stream);

/* Adam (Kingma and Ba; Sec. III-G) on a flat fp32 array of n parameters:
 * m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
 * p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), t = *step + 1
 * read from the device counter, which is then incremented (capturable). */
al_status al_adam_flat(const al_adam_params *p, int64_t n, int64_t *step, float *param,
                       const float *grad, float *m, float *v, al_stream stream);

/* al_adam_flat that also refreshes the packed bf16 weights of up to 8
 * convolution layers, so that a training step needs no al_conv3d_pack between
 * its Adam update and the next forward pass. Layer j (layers[j]) owns
 * param[weight_offset[j] .. + cout*27*cin) as its weight (cout x 27 x cin);
 * the ranges lie inside [0, n) and do not overlap; parameters outside them
 * (biases) take the plain update. packed_fwd[j] and packed_dgrad[j] (either
 * NULL, not both) must hold an al_conv3d_pack result of the same layer: each
 * updated weight is rounded to bf16 and written to its one place in each copy,
 * the zero padding is left as that pack wrote it. The result equals
 * al_adam_flat followed by al_conv3d_pack of every layer, bit for bit.
 * Errors: AL_ERR_INVALID_ARG (pointers, parameters, ranges), the layer checks
 * of al_conv3d_pack, AL_ERR_ALIGN (16-byte alignment of every buffer). */
al_status al_adam_flat_pack(const al_adam_params *p, int64_t n, int64_t *step, float *param,
                            const float *grad, float *m, float *v, int32_t n_layers,
                            const al_conv3d *layers, const int64_t *weight_offset,
                            void *const *packed_fwd, void *const *packed_dgrad, al_stream stream);

/* Training volumes: out[v][z][y][x] = sum_b a_b exp(-|x - mu_b|^2/(2 sigma_b^2))
 * for `count` volumes of size (z, y, x), blob table[v][b] = {mu_x, mu_y,
 * mu_z, sigma, a} (fp32, n_blobs per volume; sigma > 0). Terms of blobs more
 * than 6 sigma from a voxel's 8 x 8 x 32 box (x, y, z) are dropped (each below
 * 1.6e-8 a). */
al_status al_render_blobs(const int64_t *size, int32_t count, int32_t n_blobs, const float *table,
                          float *out, al_stream stream);

/* Synchronise `stream`, then read and clear the current device's kernel
 * error words (the objective's, the LCC kernels' and the convolution
 * layers'): AL_OK, AL_ERR_BOUNDS or AL_ERR_TIMEOUT (AL_ERR_CUDA if the
 * synchronisation itself failed). AL_ERR_TIMEOUT comes from a bounded wait
 * on an asynchronous copy (the TMA slices of the LCC gradient, the weight
 * slices of a convolution layer) or on another block (al_batch_step). */
al_status al_get_device_error(al_stream stream);

/* Test of the LCC gradient's bounded waits (not part of the method). With
 * drop_slice >= 0, the TMA-staged LCC gradient kernel (used when X is a
 * multiple of 4) does not issue the load of slice `drop_slice` of each
 * block's z range. The wait for that slice runs out after about a second,
 * the block records AL_ERR_TIMEOUT, waits for its other loads in flight and
 * returns without writing its outputs. -1 (the default) restores normal
 * staging. Applies to launches issued after the call on the current device;
 * blocking (a copy to device constant memory). AL_ERR_INVALID_ARG if
 * drop_slice < -1. */
al_status al_lcc_set_wait(int32_t drop_slice);

/* Test of the fused objective's bounded waits (not part of the method). With
 * drop_batch >= 0, the 3D brick kernels that stage their inputs by TMA (X a
 * multiple of 4) do not issue copy batch `drop_batch` of each brick (batch b
 * holds the moving-image slices and fixed-image layer that layer b of the
 * brick adds, or the projection's planes of layer b). The wait for it runs
 * out after about a second, the brick records AL_ERR_TIMEOUT, waits
 * (bounded) for its other copies in flight and returns without writing its
 * partial sums; the call's results are then not valid. -1 (the default)
 * restores normal staging. Applies to launches issued after the call on the
 * current device; blocking (a copy to device constant memory).
 * AL_ERR_INVALID_ARG if drop_batch < -1. */
al_status al_fused_set_wait(int32_t drop_batch);

/* Instrumentation (not part of the method). When enabled, every kernel the
 * library launches is bracketed by two CUDA events recorded on the
 * launching stream. al_profile_collect synchronises on the recorded events,
 * adds their elapsed times to per-kernel totals and reports up to
 * max_kernels totals: total_ms[i], launches[i], and the kernel names as
 * newline-separated text in `names` (truncated to names_bytes). Returns the
 * number of distinct kernels seen. Host only; not thread-safe against
 * concurrent launches on other threads while enabled. Launches on a stream
 * that is being captured into a CUDA graph are not timed (nor are their
 * replays). */
al_status al_profile_enable(int32_t on);
int32_t al_profile_collect(char *names, size_t names_bytes, double *total_ms, int64_t *launches,
                           int32_t max_kernels);
al_status al_profile_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* AIRGB_H */
