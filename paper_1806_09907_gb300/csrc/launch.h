// Host-side launchers shared between the translation units of libairgb.
// Each returns cudaSuccess or the launch error; none synchronises.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

namespace airgb {

// ---- A1 / A6: B-spline expansion and its adjoint (unfused) ----------------
cudaError_t launch_displacement(const Grid &g, const Lattice &L, const float *ctrl, float *disp,
                                cudaStream_t s);
size_t displacement_adjoint_ws(const Grid &g, const Lattice &L);
cudaError_t launch_displacement_adjoint(const Grid &g, const Lattice &L, const float *grad_disp,
                                        float *grad_ctrl, void *ws, cudaStream_t s);

// ---- A2 / A5: warp and its adjoint -----------------------------------------
cudaError_t launch_warp(const Grid &g, const float *moving, const float *disp, float *warped,
                        uint8_t *mask, cudaStream_t s);
cudaError_t launch_warp_adjoint(const Grid &g, const float *moving, const float *disp,
                                const uint8_t *mask, const float *grad_warped, float *grad_disp,
                                int accumulate, cudaStream_t s);

// ---- A4: diffusion regulariser on the voxel grid ----------------------------
size_t regulariser_ws(const Grid &g);
cudaError_t launch_regulariser(const Grid &g, const float *disp, double weight, double *value_dev,
                               float *grad_disp, void *ws, cudaStream_t s);

// ---- A3: similarity (unfused) ------------------------------------------------
size_t similarity_ws(const Grid &g, int kind, int window);
cudaError_t launch_similarity(const Grid &g, int kind, int window, double eps, const float *fixed,
                              const float *warped, const uint8_t *mask, double *value_dev,
                              float *grad_warped, void *ws, cudaStream_t s);

// Streaming multiprocessors of the current device (queried once per device;
// 152, a GB300's count, if the query fails). Sizes grids and z chunks only:
// no workspace size depends on it.
int device_sms();

// LCC statistics + exact gradient, shared by the unfused similarity and the
// fused objective: grad_unscaled = dS/dW * |X_m| (nullable; needs `coef`,
// lcc_coef_bytes(g) of scratch), per-block {sum of rho over masked voxels, masked
// voxel count} partials (lcc_num_blocks(g, window) blocks on the current
// device; lcc_max_blocks(g, window) bounds it on any device and sizes the
// partials' workspace).
int lcc_num_blocks(const Grid &g, int window);
int lcc_max_blocks(const Grid &g, int window);
size_t lcc_coef_bytes(const Grid &g);
// w_masked: the warped image is already zero off the mask (else a masked
// copy is made in grad_unscaled, or in coef when grad_unscaled is NULL).
cudaError_t launch_lcc(const Grid &g, int window, double eps, const float *fixed,
                       const float *warped, const uint8_t *mask, bool w_masked,
                       float *grad_unscaled, double *block_partials, float *coef, cudaStream_t s);

// LCC statistics alone, W already masked: per-block partials and the
// coefficient planes (a', b, c) in coef (lcc_coef_bytes(g)).
cudaError_t launch_lcc_stats(const Grid &g, int window, double eps, const float *fixed,
                             const float *warped_masked, const uint8_t *mask,
                             double *block_partials, float *coef, cudaStream_t s);
// dS/dW * |X_m| from the coefficient planes of launch_lcc_stats (W masked).
cudaError_t launch_lcc_grad(const Grid &g, int window, const float *fixed,
                            const float *warped_masked, const uint8_t *mask, const float *coef,
                            float *grad_unscaled, cudaStream_t s);
// Tiled fp32 tensor map of rank 1..5 (dims and box in elements, x first;
// byte strides of dims 1..rank-1), zero fill outside the tensor. False when
// the driver's encoder is unavailable or rejects the layout (base not
// 16-byte aligned, a stride not a multiple of 16 bytes, ...).
bool encode_tmap_f32(CUtensorMap *map, int rank, const uint64_t *dims, const uint64_t *strides,
                     const uint32_t *box, const void *base);
// Distance in floats between the coefficient planes a', b, c.
int64_t lcc_coef_plane(const Grid &g);

// ---- A7: fused objective -----------------------------------------------------
bool fused_supported(const Grid &g, const Lattice &L, int kind, int window);
size_t fused_ws(const Grid &g, const Lattice &L, int kind, int window);
// Offsets of the warped image and its mask in a fused LCC workspace.
void fused_warped_offsets(const Grid &g, const Lattice &L, int window, size_t *w, size_t *m);
cudaError_t launch_fused(const Grid &g, const Lattice &L, int kind, int window, double eps,
                         double lambda, const float *fixed, const float *moving, const float *ctrl,
                         double *value_dev, float *grad_ctrl, void *ws, cudaStream_t s);

// J = S + lambda * R from the unfused pieces: out[0..3] = {J, S, R, n_mask}.
cudaError_t launch_combine(const double *sim_value /*S, n_mask*/, const double *reg_value /*R*/,
                           double lambda, double *out, cudaStream_t s);

// ---- optimisation loop: Adam, pyramid level, coefficient refinement ---------
struct AdamArgs {
    double beta1, beta2;  // bias corrections are formed from these in double
    float lr, eps;
    float h[3];  // voxel units per normalised unit, (N_k - 1)/2, per component
    int nc;      // coefficients per component plane
    int ndim;
};
cudaError_t launch_adam(const AdamArgs &a, int64_t *step, float *ctrl, const float *grad,
                        float *m, float *v, cudaStream_t s);

constexpr int kMaxPyramidFactor = 8;
struct GaussTaps {
    int r;                                     // taps -r..r
    float w[2 * (3 * kMaxPyramidFactor / 2) + 1];  // normalised to unit sum
};
size_t pyramid_ws(const Grid &g, int factor);
cudaError_t launch_pyramid(const Grid &g, int factor, const GaussTaps &t, const float *image,
                           float *level, void *ws, cudaStream_t s);

// nc, nf: coarse / fine lattice sizes (x, y, z); taps checked by the caller.
cudaError_t launch_refine(int ndim, const int *nc, const int *nf, const float *cc, float *cf,
                          cudaStream_t s);

// ---- batches of independent problems: one persistent launch per iteration ---
// Device descriptor of one problem of a batch (MSE, the batch's spacing).
struct BatchProblem {
    Grid g;
    Lattice L;
    const float *F, *M;
    float *c, *m, *v;  // coefficients (updated in place) and Adam moments
    double *values;    // [rows][4] history {J, S, R, n_mask}, or null
    float *bpart;      // brick partials
    double *mpart;     // brick moment partials
    double *rpart;     // Gram tile partials of R
    float *gR;         // lambda-free dR/dc scaled by 2/|X| (as k_gram writes it)
    float h[3];        // Adam: voxel units per normalised unit, (N_k - 1)/2
    float gscale;      // 2/|X|
    double lambda;
    int gbx, gby, gbz, nbricks;  // brick grid
    int gtx, gty, gtz, ngram;    // Gram tiles per axis and their total over components
    int nA;                      // phase-A items: bricks + Gram tiles
    int nchunks;                 // phase-B items: control-point chunks
};

enum { BATCH_BRICK = 0, BATCH_GRAM = 1, BATCH_CTRL = 2 };
struct BatchItem {
    int prob, kind, idx, pad;
};

// Arguments of one batched iteration.
struct BatchStep {
    double beta1, beta2;  // Adam decays (bias corrections formed in double)
    float lr, eps;
    int64_t t;            // 1-based Adam step
    int record;           // row of each problem's value history to write, < 0: none
    int update;           // 1: Adam step, 0: gradient only (timing runs)
    int extra_wait;       // added to the items a control chunk waits for (test hook)
    long long spin_limit; // polls before a waiting chunk gives up (AL_ERR_TIMEOUT)
    int *err;             // error word
};

// The batch kernel is built for batch_tiles() brick tiles per spacing (tile
// 0: the single-problem path's brick). Geometry of a problem in a batch of
// spacing delta with a tile: brick grid, Gram tiles, floats of one brick's
// partials and doubles of its moments.
int batch_tiles();
void batch_tile_cells(int delta, int tile, int *bcx, int *bcy);
void batch_geometry(const Grid &g, const Lattice &L, int tile, int *gb, int *gt, int *npart,
                    int *nmom);
int batch_threads(int delta, int tile);        // 0 if (delta, tile) has no batch kernel
int batch_blocks_per_sm(int delta, int tile);  // resident blocks of the batch kernel per SM
cudaError_t launch_batch(int delta, int tile, int blocks, const BatchProblem *probs,
                         const BatchItem *items, int nitems, int *counters, const BatchStep &st,
                         cudaStream_t s);

// ---- diffeomorphic transformation: exp(v) by scaling and squaring ------------
// traj (nullable): u_0 .. u_{K-1}; tmp: a field buffer, needed when traj is
// NULL and K > 0.
cudaError_t launch_exp(const Grid &g, int K, const float *v, float *u, float *traj, float *tmp,
                       cudaStream_t s);
size_t exp_adjoint_ws(const Grid &g);
cudaError_t launch_exp_adjoint(const Grid &g, int K, const float *traj, const float *gu, float *gv,
                               void *ws, cudaStream_t s);

// ---- learned initialisation: convolution layers and the network's glue ------
// A 3x3x3 convolution layer, zero padding 1: batch nb of D x H x W voxels
// (z, y, x) with cin channels in, cout out, stride 1 or 2. Channels last, bf16.
struct ConvLayer {
    int nb, D, H, W, cin, cout, stride;
};
int conv_out_size(int n, int stride);
int conv_slices(int kreal);
size_t conv_packed_elems(const ConvLayer &l, int dgrad);
void conv_wgrad_plan(const ConvLayer &l, int *mtiles, int *splits, int *kper);
size_t conv_wgrad_ws_bytes(const ConvLayer &l);
cudaError_t launch_conv_pack(const ConvLayer &l, const float *w, void *fwd, void *dgrad,
                             cudaStream_t s);
int conv_fwd_splits(const ConvLayer &l);
size_t conv_fwd_ws_bytes(const ConvLayer &l);
// ws (nullable, conv_fwd_ws_bytes): split-K partials; NULL runs unsplit.
cudaError_t launch_conv_forward(const ConvLayer &l, const void *in, const void *wpk,
                                const float *bias, int relu, int out_f32, void *out, void *ws,
                                cudaStream_t s);
cudaError_t launch_conv_dgrad(const ConvLayer &l, const void *gout, const void *wpk,
                              const void *mask, const void *addend, int add_stride, int add_off,
                              void *gin, cudaStream_t s);
cudaError_t launch_conv_wgrad(const ConvLayer &l, const void *in, const void *gout, float *gw,
                              float *gb, void *ws, cudaStream_t s);
// Kernel error word of the layers (AL_ERR_TIMEOUT after a bounded wait ran
// out), read and optionally cleared; -1 if the copy failed.
int conv_device_error(bool clear);
// Error words of the units with checked-build index checks (AL_ERR_BOUNDS),
// read and optionally cleared; -1 if the copy failed.
int unit_error_basic(bool clear);
int unit_error_fused(bool clear);
int unit_error_conv(bool clear);
int unit_error_lcc(bool clear);
// Test hook of the LCC gradient's bounded waits (al_lcc_set_wait).
cudaError_t lcc_set_drop_slice(int slice);
cudaError_t fused_set_drop_batch(int batch);
// pair (nullable, 3D only): write the bf16 pairs (W, M) there instead of W and m.
cudaError_t launch_warp_ctrl(const Grid &g, const Lattice &L, int count, const float *M,
                             const float *c, float *W, uint8_t *m, void *pair, cudaStream_t s);

// Grids of the network's two coarsest levels: n3 (e3, the head) and n4 (e4),
// (z, y, x); lat = spacing-8 lattice sizes (x, y, z).
struct NetGrid {
    int nb;
    int n3[3], n4[3];
    int lat[3];
};
cudaError_t launch_net_input(int64_t n, const float *F, const float *M, void *x, cudaStream_t s);
cudaError_t launch_upcat(const NetGrid &g, int c4, int c3, const void *e4, const void *e3,
                         void *cat, cudaStream_t s);
cudaError_t launch_upcat_adjoint(const NetGrid &g, int c4, int c3, const void *gcat,
                                 const void *e4, void *ge4, cudaStream_t s);
cudaError_t launch_head_to_ctrl(const NetGrid &g, int ch, const float *h, float *c, cudaStream_t s);
cudaError_t launch_head_adjoint(const NetGrid &g, int ch, const float *gc, void *gh,
                                cudaStream_t s);

struct FieldLossArgs {
    int n[3];      // lattice nx, ny, nz
    int N[3];      // grid X, Y, Z
    int delta;     // spacing
    double gscale; // 2 / (3 |X| nb)
    double lscale; // 1 / (3 |X| nb)
};
size_t field_loss_smem(const FieldLossArgs &a);
cudaError_t launch_field_loss(const FieldLossArgs &a, int nb, const float *c, const float *ct,
                              float *gc, double *part, double *loss, cudaStream_t s);

struct AdamFlatArgs {
    double beta1, beta2;
    float lr, eps;
    int64_t n;
};
cudaError_t launch_adam_flat(const AdamFlatArgs &a, int64_t *step, float *p, const float *g,
                             float *m, float *v, cudaStream_t s);
// *step += 1 (one thread), after the Adam launches that read it.
cudaError_t launch_step_tick(int64_t *step, cudaStream_t s);
// Adam on a network's flat parameters (k_adam_flat's update) that also
// writes the updated weights of up to kMaxPackLayers layers into their packed
// bf16 copies, as launch_conv_pack lays them out; then ticks *step.
constexpr int kMaxPackLayers = 8;
struct PackLayer {
    int64_t off;         // first weight (cout x 27 x cin) in the flat array
    int cin, cout;
    int dmode;           // dgrad copy: 0 none, 1 stride 1, 2 stride 2 (parity classes)
    int cls0[8];         // dmode 2: first packed slice of each parity class
    void *fwd, *dgrad;   // packed copies (bf16; fwd nullable)
};
struct AdamPackArgs {
    AdamFlatArgs adam;
    int nl;
    PackLayer L[kMaxPackLayers];
};
void adam_pack_layer(const ConvLayer &l, int64_t off, void *fwd, void *dgrad, PackLayer *L);
cudaError_t launch_adam_pack(const AdamPackArgs &a, int64_t *step, float *p, const float *g,
                             float *m, float *v, cudaStream_t s);
cudaError_t launch_render_blobs(int D, int H, int W, int count, int nblobs, const float *table,
                                float *out, cudaStream_t s);

}  // namespace airgb
