// A7: fused evaluation of J = S + lambda*R and dJ/dc.
//
// k_fused streams a brick of control cells slice by slice: the B-spline
// expansion (A1), the masked warp (A2), the point-wise similarity terms (A3),
// the warp adjoint (A5) and the transposed expansion (A6) all happen on
// chip; only the brick's partial sums on its (cells+3)^D control points and
// its moment sums leave it. k_ctrl then sums, for every control point, the
// partials of the (at most 2 per axis) bricks that touch it in a fixed
// order, so the result is deterministic without atomics. The regulariser is
// evaluated on the control lattice in Gram form, by extra blocks of the
// first k_fused launch (Gram tiles):
//   R = (1/|X|) sum_i c_i^T (Gz(x)Gy(x)Hx + Gz(x)Hy(x)Gx + Hz(x)Gy(x)Gx) c_i,
// G = B^T B and H = (DB)^T (DB) per axis (B the sampled 1D B-spline matrix,
// D the forward difference), which equals the voxel-grid definition exactly.
//
// LCC needs W in a neighbourhood, so it runs as: k_fused<FWD> writes W, the
// mask and dM~/dy, k_lcc_stats and k_lcc_grad turn W into dS/dW, and
// k_fused<GW> projects dS/dW * dM~/dy onto the control points.
#include <cuda_bf16.h>
#include <string.h>

#include "launch.h"
#include "profile.h"

namespace airgb {

namespace {

enum { MODE_MSE = 0, MODE_NCC = 1, MODE_FWD = 2, MODE_GW = 3 };

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Brick of control cells handled by one CTA: BCX x BCY cells in x/y (one
// thread per voxel column, lanes consecutive in x) and BCZ cell layers in z
// streamed slice by slice. Every axis spans >= 3 cells, so a control point
// is touched by at most two bricks per axis (k_ctrl relies on it).
__host__ __device__ constexpr int brick_bcx(int delta) { return delta <= 4 ? 8 : 4; }
__host__ __device__ constexpr int brick_bcy(int delta) { return delta <= 4 ? 4 : 3; }
__host__ __device__ constexpr int brick_bcz(int ndim) { return ndim == 3 ? 4 : 1; }

// Brick tiles the batch kernel is built for, per spacing: control cells per
// block in x and y, and the resident blocks per SM the kernel is compiled
// for (its register budget). Tile 0 is the single-problem path's brick at
// one block per SM; the others are the batch autotuner's alternatives (every
// axis still spans >= 3 cells):
//   spacing 4: (8, 4, 1), (8, 4, 2), (6, 4, 2)
//   spacing 6: (4, 3, 1), (4, 3, 2), (3, 3, 2)
//   spacing 8: (4, 3, 1), (3, 3, 1), (3, 4, 1)
constexpr int kBatchTiles = 3;
__host__ __device__ constexpr int batch_tile_bcx(int delta, int t)
{
    return delta <= 4 ? (t == 2 ? 6 : 8) : (t == 0 || (t == 1 && delta == 6) ? 4 : 3);
}
__host__ __device__ constexpr int batch_tile_bcy(int delta, int t)
{
    return delta <= 4 ? 4 : (delta == 8 && t == 2 ? 4 : 3);
}
__host__ __device__ constexpr int batch_tile_minb(int delta, int t)
{
    return delta == 8 || t == 0 ? 1 : 2;
}

template <int D, int DELTA, int MODE, int BCX_ = brick_bcx(DELTA), int BCY_ = brick_bcy(DELTA)>
struct FCfg {
    static constexpr int BCX = BCX_, BCY = BCY_, BCZ = brick_bcz(D);
    static constexpr int BX = BCX * DELTA, BY = BCY * DELTA;
    static constexpr int THREADS = BX * BY;
    static constexpr int JX = BCX + 3, JY = BCY + 3, JZ = (D == 3) ? BCZ + 3 : 1;
    static constexpr int CH = (MODE == MODE_NCC) ? 3 * D : (MODE == MODE_FWD ? 0 : D);
    static constexpr int CHS = CH > 0 ? CH : 1;  // storage size
    static constexpr int NMOM = (MODE == MODE_MSE) ? 2 : (MODE == MODE_NCC ? 6 : 0);
    static constexpr int NPART = CH * JZ * JY * JX;  // floats of one brick's partials
    static constexpr int VC = (MODE == MODE_FWD) ? 2 : 1;  // slices whose gathers are in flight together
    // dynamic shared memory of the flush of up to NPL planes (flush_planes):
    // region A, the column partials P[NPL][BY][BX][CHS], later their x
    // contraction; region B, the per-cell sums S1[NPL][BY][BCX][4][CHS], later
    // S2[NPL][BCY][4][JX][CHS]
    static constexpr int NPL = (D == 3) ? 4 : 1;
    static constexpr int nP = (MODE == MODE_FWD) ? 0 : NPL * BY * BX * CHS;
    static constexpr int nX = (MODE == MODE_FWD) ? 0 : NPL * BY * BCX * 4 * CHS;
    // the x contractions of the lattice rows of four planes, per voxel column
    // (plane_rows), after the flush buffers; GW does not expand
    static constexpr int RPL = D * JY * BX;  // floats of one plane's row contractions
    static constexpr int nR = (MODE == MODE_GW) ? 0 : 4 * RPL;
    static constexpr size_t dyn_smem = (size_t)(nP + nX + nR) * sizeof(float);
};

// Shared-memory staging of a 3D brick by TMA (single-problem path, X a
// multiple of 4 so that image rows can be tensor-map rows):
// * the moving image: one box of (BX + 2 HX) x (BY + 2 HY) voxels per slice,
//   from (x0 - HX, y0 - HY), in a ring of NSLOT slices. While layer l (its
//   DELTA output slices from zl = z0 + l DELTA) is computed, slices
//   zl - HZ .. zl + DELTA + HZ - 1 are resident and the DELTA slices the next
//   layer adds are in flight. A sample whose trilinear cell lies inside that
//   window reads its 8 corners from shared memory, any other from global
//   memory (|u| <= HZ voxels keeps every sample inside);
// * the fixed image (MSE, NCC): one box of BX x BY x DELTA voxels per layer,
//   two layers buffered;
// * the control lattice: c's rows (nx floats) are not tensor-map rows, so it
//   is copied through a one-dimensional view: one box per lattice plane of
//   the brick's D x JZ x JY x JX block when the plane's JY rows fit one box of
//   at most 256 floats (the box starts at the plane's first point rounded
//   down to a 16-byte boundary), else one box of 16 floats per row; the
//   boxes are then compacted into the brick's lattice block.
// Copies land on mbarriers with bounded waits: batch b (the first: the
// resident slices of layer 0; then the DELTA new slices and the fixed-image
// layer of layer b) on barrier b % 2, the lattice rows on barrier 2.
// Coordinates outside the volume or the lattice read zeros.
__host__ __device__ constexpr int round128(int b) { return (b + 127) / 128 * 128; }

template <int DELTA, int MODE>
struct TCfg {
    using C = FCfg<3, DELTA, MODE>;
    static constexpr int BX = C::BX, BY = C::BY;
    static constexpr int HX = 4, HY = 4, HZ = 4;  // HX keeps x0 - HX on a 16-byte boundary
    static constexpr int TWX = BX + 2 * HX, TWY = BY + 2 * HY;
    static constexpr int SLOTB = TWX * TWY * 4;
    static constexpr int NRES = DELTA + 2 * HZ;  // slices resident while a layer is computed
    static constexpr int NSLOT = NRES + DELTA;   // + the next layer's new slices
    static constexpr int NF = (MODE == MODE_FWD) ? 0 : 2;
    static constexpr int FSLOTB = BX * BY * DELTA * 4;
    static constexpr int NROW = 3 * C::JZ * C::JY;  // lattice rows
    static constexpr int LBOX = 16;                  // floats per row copy (offset <= 3, JX <= 11)
    static constexpr int NPLN = 3 * C::JZ;           // lattice planes (one box each, <= 1 KB)
    static constexpr int LSTAGE = NROW * 128 > NPLN * 1024 ? NROW * 128 : NPLN * 1024;
    static constexpr int nP1 = (MODE == MODE_FWD) ? 0 : BY * BX * C::CHS;   // one-plane flush
    static constexpr int nX1 = (MODE == MODE_FWD) ? 0 : BY * C::BCX * 4 * C::CHS;
    static constexpr int oRing = 0;
    static constexpr int oF = oRing + NSLOT * SLOTB;
    static constexpr int oU = oF + NF * FSLOTB;  // lattice rows, later the flush buffers
    static constexpr int oR = (nP1 + nX1) * 4;  // row contractions, inside the union
    static constexpr int nU = (LSTAGE > oR + C::nR * 4) ? LSTAGE : oR + C::nR * 4;
    static constexpr int oBar = oU + round128(nU);
    static constexpr int bytes = oBar + 3 * 8;
    static_assert(SLOTB % 128 == 0 && FSLOTB % 128 == 0, "TMA destinations are 128-byte aligned");
    static_assert(C::JX + 3 <= LBOX, "a lattice row copy holds the row");
    static_assert(BX % 4 == 0, "brick origins stay on 16-byte boundaries");
    static_assert(TWX <= 256 && TWY <= 256 && BX <= 256 && BY <= 256, "TMA box limits");
};

// Tensor maps of a brick staged by TMA (addresses of kernel parameters) and
// the lattice copies: lbox floats per box into slots of lslot bytes, one box
// per plane (lplane) or per row.
struct BrickMaps {
    const CUtensorMap *M, *F, *c;
    int lbox, lslot, lplane;
};

// Host choice of the lattice copies of a brick (plane boxes when a plane's
// rows fit one box of at most 256 floats).
template <int DELTA>
void lattice_boxes(const Lattice &L, int *lbox, int *lslot, int *lplane)
{
    using C = FCfg<3, DELTA, MODE_FWD>;
    const int span = (C::JY - 1) * L.nx + C::JX + 3;  // offset <= 3
    if (span <= 256) {
        *lbox = (span + 3) / 4 * 4;
        *lslot = round128(*lbox * 4);
        *lplane = 1;
    } else {
        *lbox = 16;
        *lslot = 128;
        *lplane = 0;
    }
}

constexpr int kFusedTimeout = 6;  // AL_ERR_TIMEOUT

// Test of the bounded waits of the TMA-staged bricks: the copy batch (layer
// index within a brick) that is not issued, so the wait for it runs out;
// -1 = none.
__constant__ int c_fused_drop_batch = -1;

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            int z, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_1d(uint32_t dst, const CUtensorMap *map, int x,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2}], [%3];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// Batch b of a brick's copies (issued by one thread): the moving-image
// slices it adds to the ring and, for MSE/NCC, the fixed-image layer b.
template <int DELTA, int MODE>
__device__ __forceinline__ void brick_issue(const BrickMaps &tm, uint32_t sbase, int b, int x0,
                                            int y0, int z0)
{
    using T = TCfg<DELTA, MODE>;
    if (b == c_fused_drop_batch)
        return;
    const uint32_t bar = sbase + T::oBar + 8 * (b & 1);
    const int r0 = b == 0 ? 0 : T::NRES + (b - 1) * DELTA, r1 = T::NRES + b * DELTA;
    mbar_expect(bar, (uint32_t)((r1 - r0) * T::SLOTB + (T::NF > 0 ? T::FSLOTB : 0)));
    for (int r = r0; r < r1; ++r) {
        const int slot = r % T::NSLOT;
        tma_load_3d(sbase + T::oRing + slot * T::SLOTB, tm.M, x0 - T::HX, y0 - T::HY,
                    z0 - T::HZ + r, bar);
    }
    if constexpr (T::NF > 0)
        tma_load_3d(sbase + T::oF + (b & 1) * T::FSLOTB, tm.F, x0, y0, z0 + b * DELTA, bar);
}

// Staging of the projection pass (GW) by TMA: per layer one box of dS/dW
// (BX x BY x DELTA) and one of the D planes of dM~/dy (a 4D box), two layers
// buffered, on mbarriers 0 and 1 with bounded waits; then the one-plane flush
// buffers.
template <int DELTA>
struct GCfg {
    using C = FCfg<3, DELTA, MODE_GW>;
    static constexpr int FSLOTB = C::BX * C::BY * DELTA * 4;  // one plane of a layer
    static constexpr int LAYERB = 4 * FSLOTB;                  // dS/dW, then 3 planes
    static constexpr int oU = 2 * LAYERB;
    static constexpr int nU = (C::BY * C::BX * C::CHS + C::BY * C::BCX * 4 * C::CHS) * 4;
    static constexpr int oBar = oU + round128(nU);
    static constexpr int bytes = oBar + 2 * 8;
    static_assert(FSLOTB % 128 == 0, "TMA destinations are 128-byte aligned");
};

template <int DELTA>
__device__ __forceinline__ void gw_issue(const BrickMaps &tm, uint32_t sbase, int b, int x0, int y0,
                                         int z0)
{
    using G = GCfg<DELTA>;
    if (b == c_fused_drop_batch)
        return;
    const uint32_t bar = sbase + G::oBar + 8 * (b & 1), dst = sbase + (b & 1) * G::LAYERB;
    mbar_expect(bar, (uint32_t)G::LAYERB);
    tma_load_3d(dst, tm.M, x0, y0, z0 + b * DELTA, bar);  // dS/dW
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst + G::FSLOTB),
        "l"(reinterpret_cast<uint64_t>(tm.F)), "r"(x0), "r"(y0), "r"(z0 + b * DELTA), "r"(0),
        "r"(bar)
        : "memory");
}

// xy contraction of control plane jz for the voxel columns of a brick, in
// two steps that share the x contraction among the DELTA columns of a cell
// row:
// plane_rows (every thread of the block): for each of its items (component
// i, lattice row ly, voxel column tx = the thread's own column),
//   Rw[i][ly][tx] = sum_e wx[e] cb[i][jz][ly][qx + e];
// plane_cols (after a barrier): the thread's column,
//   out[i] = sum_b wy[b] Rw[i][qy + b][tx].
template <int D, int JZ, int JY, int JX, int BX, int THREADS>
__device__ __forceinline__ void plane_rows(const float (&cb)[D][JZ][JY][JX], int jz, int qx,
                                           const float (&wx)[4], float *Rw)
{
    if (jz >= JZ)
        return;
    for (int e = threadIdx.x; e < D * JY * BX; e += THREADS) {
        const int r = e / BX;  // i * JY + ly; e % BX is the thread's column
        const float *row = &cb[0][0][0][0] + ((r / JY) * JZ + jz) * (JY * JX) + (r % JY) * JX + qx;
        float v = wx[0] * row[0];
        v = fmaf(wx[1], row[1], v);
        v = fmaf(wx[2], row[2], v);
        v = fmaf(wx[3], row[3], v);
        Rw[e] = v;
    }
}

template <int D, int JZ, int JY, int BX>
__device__ __forceinline__ void plane_cols(const float *Rw, int jz, int qy, int tx,
                                           const float (&wy)[4], float2 &oxy, float &oz)
{
    float out[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < D; ++i) {
        if (jz < JZ) {
            const float *col = Rw + (i * JY + qy) * BX + tx;
            float acc = wy[0] * col[0];
            acc = fmaf(wy[1], col[BX], acc);
            acc = fmaf(wy[2], col[2 * BX], acc);
            acc = fmaf(wy[3], col[3 * BX], acc);
            out[i] = acc;
        }
    }
    oxy = make_float2(out[0], out[1]);
    oz = out[2];
}

// Planes 0..NPL-1 of the thread's column partials qz -> x contraction -> y
// contraction -> the brick's partial sums of local planes lp0 .. lp0+NPL-1.
// Every thread of the block calls it. Each axis takes two steps: the four
// weighted sums of every cell (the DELTA voxels of the cell times the
// compile-time weights of their phases), then for every control point the
// sum over the (up to four) cells it supports. A holds the column partials,
// later the x contraction; B the per-cell sums of x, later those of y.
template <int D, int DELTA, int MODE, int NPL, int BCX_ = brick_bcx(DELTA),
          int BCY_ = brick_bcy(DELTA)>
__device__ __forceinline__ void flush_planes(int lp0, const float (&qz)[4][FCfg<D, DELTA, MODE>::CHS],
                                             bool colvalid, int tx, int ty, float *A, float *B,
                                             float *dst)
{
    using C = FCfg<D, DELTA, MODE, BCX_, BCY_>;
    constexpr int CHS = C::CHS, BX = C::BX, BY = C::BY, JX = C::JX, JY = C::JY, JZ = C::JZ;
    constexpr int BCX = C::BCX, BCY = C::BCY;
    constexpr WTab<DELTA> kW{};
    const int tid = threadIdx.x;
#pragma unroll
    for (int a = 0; a < NPL; ++a)
#pragma unroll
        for (int k = 0; k < CHS; ++k)
            A[((a * BY + ty) * BX + tx) * CHS + k] = colvalid ? qz[a][k] : 0.0f;
    __syncthreads();
    // x, per cell: S1[(a BY + y) BCX + qx][q][k] = sum_px w[px][q] P[a][y][qx DELTA + px][k]
    for (int e = tid; e < NPL * BY * BCX * CHS; e += C::THREADS) {
        const int k = e % CHS, r = e / CHS;
        const int qx = r % BCX, ay = r / BCX;
        const float *src = A + (ay * BX + qx * DELTA) * CHS + k;
        float sq[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int px = 0; px < DELTA; ++px) {
            const float v = src[px * CHS];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                sq[q] = fmaf(kW.w[px][q], v, sq[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            B[(r * 4 + q) * CHS + k] = sq[q];
    }
    __syncthreads();
    // x, per control point jx: cells jx - 3 .. jx (into A; P is dead)
    for (int e = tid; e < NPL * BY * JX * CHS; e += C::THREADS) {
        const int k = e % CHS, r = e / CHS;
        const int jx = r % JX, ay = r / JX;
        float sum = 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int qx = jx - q;
            if (qx >= 0 && qx < BCX)
                sum += B[((ay * BCX + qx) * 4 + q) * CHS + k];
        }
        A[r * CHS + k] = sum;
    }
    __syncthreads();
    // y, per cell: S2[a BCY + qy][q][jx][k] = sum_py w[py][q] X[a][qy DELTA + py][jx][k]
    for (int e = tid; e < NPL * BCY * JX * CHS; e += C::THREADS) {
        const int k = e % CHS, r = e / CHS;
        const int jx = r % JX, aq = r / JX;
        const int a = aq / BCY, qy = aq - a * BCY;
        const float *src = A + ((a * BY + qy * DELTA) * JX + jx) * CHS + k;
        float sq[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int py = 0; py < DELTA; ++py) {
            const float v = src[py * JX * CHS];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                sq[q] = fmaf(kW.w[py][q], v, sq[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            B[((aq * 4 + q) * JX + jx) * CHS + k] = sq[q];
    }
    __syncthreads();
    // y, per control point jy: cells jy - 3 .. jy
    for (int e = tid; e < NPL * JY * JX * CHS; e += C::THREADS) {
        const int jx = e % JX, r = e / JX;
        const int jy = r % JY, r1 = r / JY;
        const int k = r1 % CHS, a = r1 / CHS;
        float sum = 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int qy = jy - q;
            if (qy >= 0 && qy < BCY)
                sum += B[(((a * BCY + qy) * 4 + q) * JX + jx) * CHS + k];
        }
        dst[(k * JZ + lp0 + a) * JY * JX + jy * JX + jx] = sum;
    }
}

// One brick (bx, by, bz) of one problem: the whole per-voxel work of the
// brick, its partial sums written to bpart / mpart at index `brick`. Every
// thread of a block of FCfg::THREADS threads calls it; it uses the block's
// shared memory (static arrays here and FCfg::dyn_smem of dynamic memory,
// or TCfg::bytes + 128 with TMA). With TMA (3D, MSE/NCC/FWD) the lattice
// block, the moving-image neighbourhood and the fixed image arrive by
// tensor-map copies (TCfg); the arithmetic is the same either way, so both
// give the same bits. Returns false if a copy did not land in time (the
// brick's partials are then not written).
template <int D, int DELTA, int MODE, int BCX_ = brick_bcx(DELTA), int BCY_ = brick_bcy(DELTA),
          bool TMA = false, bool PAIR = false>
__device__ __forceinline__ bool fused_brick(const Grid &g, const Lattice &L,
                                            const float *__restrict__ F,
                                            const float *__restrict__ M,
                                            const float *__restrict__ c,
                                            const float *__restrict__ gw_in,
                                            float *__restrict__ W_out, uint8_t *__restrict__ m_out,
                                            float *__restrict__ G_io, float *__restrict__ bpart,
                                            double *__restrict__ mpart, int bx, int by, int bz,
                                            int brick, BrickMaps tm = BrickMaps{},
                                            int *__restrict__ icnt = nullptr)
{
    // MODE_FWD writes W, the mask and (when G_io is given) dM~/dy as D planes;
    // with PAIR it writes only the bf16 pairs (W, M) of the network input,
    // W_out then pointing at them. MODE_GW reads dS/dW and those planes back
    // (no expansion, no gathers).
    using C = FCfg<D, DELTA, MODE, BCX_, BCY_>;
    using T = TCfg<DELTA, MODE == MODE_GW ? MODE_FWD : MODE>;
    using GS = GCfg<DELTA>;
    static_assert(!TMA || (D == 3 && BCX_ == brick_bcx(DELTA) && BCY_ == brick_bcy(DELTA)),
                  "TMA staging: 3D single-problem bricks");
    constexpr int JX = C::JX, JY = C::JY, JZ = C::JZ, CHS = C::CHS, BX = C::BX;
    constexpr WTab<DELTA> kW{};  // weights of the compile-time z phases
    __shared__ float cb[D][JZ][JY][JX];
    __shared__ float wt[DELTA][4];
    __shared__ double red[(C::NMOM > 0 ? C::NMOM : 1) * ((C::THREADS + 31) / 32)];
    extern __shared__ float dsm[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(dsm);
    if constexpr (TMA)
        sm += (128u - (al_smem_u32(dsm) & 127u)) & 127u;
    const uint32_t sbase = al_smem_u32(sm);
    float *P = TMA ? reinterpret_cast<float *>(sm + (MODE == MODE_GW ? GS::oU : T::oU)) : dsm;
    float *Xc = TMA ? P + (MODE == MODE_GW ? C::BY * BX * CHS : T::nP1) : dsm + C::nP;
    float *Rw = TMA ? reinterpret_cast<float *>(sm + T::oU + T::oR) : dsm + C::nP + C::nX;
    const float *ring = reinterpret_cast<const float *>(sm + T::oRing);
    const float *Fs = reinterpret_cast<const float *>(sm + T::oF);

    const int tid = threadIdx.x;
    const int tx = tid % BX, ty = tid / BX;
    const int cx0 = bx * C::BCX, cy0 = by * C::BCY, cz0 = bz * C::BCZ;
    const int x = cx0 * DELTA + tx, y = cy0 * DELTA + ty, z0 = (D == 3) ? cz0 * DELTA : 0;
    const int x0 = cx0 * DELTA, y0 = cy0 * DELTA;

    if (tid < DELTA * 4)
        wt[tid / 4][tid % 4] = L.w[tid / 4][tid % 4];
    bool ok = true;
    if constexpr (TMA && MODE == MODE_GW) {
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbase + GS::oBar)
                         : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbase + GS::oBar + 8)
                         : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (tid == 0) {
            gw_issue<DELTA>(tm, sbase, 0, x0, y0, z0);
            if (C::BCZ > 1)
                gw_issue<DELTA>(tm, sbase, 1, x0, y0, z0);
        }
    } else if constexpr (TMA) {
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbase + T::oBar + 8 * k)
                             : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (tid == 0) {
            brick_issue<DELTA, MODE>(tm, sbase, 0, x0, y0, z0);
            if (C::BCZ > 1)
                brick_issue<DELTA, MODE>(tm, sbase, 1, x0, y0, z0);
        }
        // lattice boxes (one per plane or one per row), issued by the lanes
        // of warp 1
        const uint32_t lbar = sbase + T::oBar + 16;
        const int nbox = tm.lplane ? D * JZ : D * JZ * JY;
        if (tid >> 5 == 1) {
            const int lane = tid & 31;
            if (lane == 0)
                mbar_expect(lbar, (uint32_t)(nbox * tm.lbox * 4));
            __syncwarp();
            for (int r = lane; r < nbox; r += 32) {
                const int pl = tm.lplane ? r : r / JY, ly = tm.lplane ? 0 : r % JY;
                const int i = pl / JZ, lz = pl % JZ;
                const int row = ((i * L.nz + cz0 + lz) * L.ny + cy0 + ly) * L.nx;
                tma_load_1d(sbase + T::oU + r * tm.lslot, tm.c, (row + cx0) & ~3, lbar);
            }
        }
        ok = al_mbar_wait(lbar, 0);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(&g_unit_error, kFusedTimeout);
                al_mbar_wait(sbase + T::oBar, 0);
                if (C::BCZ > 1)
                    al_mbar_wait(sbase + T::oBar + 8, 0);
                al_mbar_wait(lbar, 0);
            }
            return false;
        }
        const float *boxes = reinterpret_cast<const float *>(sm + T::oU);
        for (int e = tid; e < D * JZ * JY * JX; e += C::THREADS) {
            const int r = e / JX, lx = e - r * JX;  // r = (i JZ + lz) JY + ly
            const int pl = r / JY, ly = r - pl * JY;
            const int i = pl / JZ, lz = pl - i * JZ;
            const int row = ((i * L.nz + cz0 + lz) * L.ny + cy0 + (tm.lplane ? 0 : ly)) * L.nx;
            const int b = tm.lplane ? pl : r;  // the box holding the point
            const int o = ((row + cx0) & 3) + (tm.lplane ? ly * L.nx : 0) + lx;
            (&cb[0][0][0][0])[e] = boxes[b * (tm.lslot / 4) + o];
        }
    } else {
        for (int e = tid; e < D * JZ * JY * JX; e += C::THREADS) {
            const int i = e / (JZ * JY * JX);
            int r = e - i * JZ * JY * JX;
            const int lz = r / (JY * JX);
            r -= lz * JY * JX;
            const int ly = r / JX, lx = r - ly * JX;
            const int jx = cx0 + lx, jy = cy0 + ly, jz = cz0 + lz;
            float v = 0.0f;
            if (jx < L.nx && jy < L.ny && jz < L.nz)
                v = __ldg(c + (((int64_t)i * L.nz + jz) * L.ny + jy) * L.nx + jx);
            cb[i][lz][ly][lx] = v;
        }
    }
    __syncthreads();

    const int qxl = tx / DELTA, px = tx - qxl * DELTA;
    const int qyl = ty / DELTA, py = ty - qyl * DELTA;
    float wx[4], wy[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        wx[e] = wt[px][e];
        wy[e] = wt[py][e];
    }
    const bool colvalid = x < g.X && y < g.Y;
    // sample bounds of axis_cell: y = x + u inside when -x <= u <= n - 1 - x
    const float lox = (float)(-x), hix = (float)(g.X - 1 - x);
    const float loy = (float)(-y), hiy = (float)(g.Y - 1 - y);
    // xy-contracted control values of the four active planes: (x, y) packed
    // for the f32x2 z expansion, z apart (3D)
    float2 cxy2[4];
    float cxyz[4];
    if constexpr (MODE != MODE_GW) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
            plane_rows<D, JZ, JY, JX, BX, C::THREADS>(cb, a, qxl, wx, Rw + a * C::RPL);
        __syncthreads();
#pragma unroll
        for (int a = 0; a < 4; ++a)
            plane_cols<D, JZ, JY, BX>(Rw + a * C::RPL, a, qyl, tx, wy, cxy2[a], cxyz[a]);
    }
    float qz[4][CHS];  // column partial sums of the four active planes
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < CHS; ++k)
            qz[a][k] = 0.0f;
    float mom[C::NMOM > 0 ? C::NMOM : 1];
#pragma unroll
    for (int k = 0; k < (C::NMOM > 0 ? C::NMOM : 1); ++k)
        mom[k] = 0.0f;

    float *const dstp = bpart + (int64_t)brick * C::NPART;
    const int cells_z = (D == 3) ? (g.Z + DELTA - 1) / DELTA : 1;
    const int nlayers = (D == 3) ? min(C::BCZ, cells_z - cz0) : 1;
    constexpr int VC = TMA ? 1 : C::VC;  // slices whose loads are in flight together
    int fail_layer = -1;
    for (int cz = 0; cz < C::BCZ; ++cz) {
        const bool active = cz < nlayers && colvalid;
        const int zl0 = z0 + cz * DELTA;
        const float loz0 = (float)(-zl0), hiz0 = (float)(g.Z - 1 - zl0);  // slice zl0 + pz: - pz
        // GW: the layer's loads are issued before the flush of the previous
        // plane, so they are in flight while the block contracts it
        float gv[MODE == MODE_GW ? DELTA : 1], gr[MODE == MODE_GW ? DELTA : 1][D];
        if constexpr (MODE == MODE_GW && !TMA) {
            if (active) {
                // 32-bit voxel offsets (nv < 2^31), one per slice, shared by
                // the D + 1 planes read
                const int v0 = (min(zl0, g.Z - 1) * g.Y + y) * g.X + x;
                const int sxy = g.X * g.Y;
#pragma unroll
                for (int pz = 0; pz < DELTA; ++pz) {
                    const int v = zl0 + pz < g.Z ? v0 + pz * sxy : v0 + (g.Z - 1 - zl0) * sxy;
                    gv[pz] = __ldg(gw_in + v);
#pragma unroll
                    for (int i = 0; i < D; ++i)
                        gr[pz][i] = __ldg(G_io + i * g.nv + v);
                }
            }
        }
        if (cz > 0) {
            // plane cz - 1 has all its contributions: write it out, roll
            if (MODE != MODE_FWD)
                flush_planes<D, DELTA, MODE, 1, BCX_, BCY_>(cz - 1, qz, colvalid, tx, ty, P, Xc,
                                                            dstp);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
#pragma unroll
                for (int k = 0; k < CHS; ++k)
                    qz[a][k] = qz[a + 1][k];
                cxy2[a] = cxy2[a + 1];
                cxyz[a] = cxyz[a + 1];
            }
#pragma unroll
            for (int k = 0; k < CHS; ++k)
                qz[3][k] = 0.0f;
            // row contractions of plane cz + 3 (into the buffer of plane
            // cz - 1, last read before the previous layer's barrier)
            if (MODE != MODE_GW)
                plane_rows<D, JZ, JY, JX, BX, C::THREADS>(cb, cz + 3, qxl, wx,
                                                          Rw + ((cz + 3) & 3) * C::RPL);
        }
        if constexpr (TMA && MODE == MODE_GW) {
            ok = al_mbar_wait(sbase + GS::oBar + 8 * (cz & 1), (uint32_t)(cz >> 1) & 1u);
            if (__syncthreads_or(!ok)) {
                fail_layer = cz;
                break;
            }
            if (tid == 0 && cz >= 1 && cz + 1 < C::BCZ) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                gw_issue<DELTA>(tm, sbase, cz + 1, x0, y0, z0);
            }
        } else if constexpr (TMA) {
            // this layer's copies; then every thread is past layer cz - 1, so
            // the slots it used take the next layer's copies
            ok = al_mbar_wait(sbase + T::oBar + 8 * (cz & 1), (uint32_t)(cz >> 1) & 1u);
            if (__syncthreads_or(!ok)) {
                fail_layer = cz;
                break;
            }
            if (tid == 0 && cz >= 1 && cz + 1 < C::BCZ) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                brick_issue<DELTA, MODE>(tm, sbase, cz + 1, x0, y0, z0);
            }
        } else if (MODE != MODE_GW && cz > 0) {
            __syncthreads();  // the row contractions of plane cz + 3 are written
        }
        if (MODE != MODE_GW && cz > 0)
            plane_cols<D, JZ, JY, BX>(Rw + ((cz + 3) & 3) * C::RPL, cz + 3, qyl, tx, wy, cxy2[3],
                                      cxyz[3]);
        if (!active)
            continue;
        if constexpr (MODE == MODE_GW) {
            static_assert(C::VC >= 1, "the GW layer loads all DELTA slices at once");
            const float *Gl = reinterpret_cast<const float *>(sm + (cz & 1) * GS::LAYERB) +
                              ty * BX + tx;
#pragma unroll
            for (int pz = 0; pz < DELTA; ++pz) {
                if (zl0 + pz >= g.Z)
                    break;
                if constexpr (TMA) {
                    constexpr int PL = GS::FSLOTB / 4;
                    gv[pz] = Gl[pz * (BX * C::BY)];
#pragma unroll
                    for (int i = 0; i < D; ++i)
                        gr[pz][i] = Gl[(1 + i) * PL + pz * (BX * C::BY)];
                }
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    const float vch = gv[pz] * gr[pz][i];
                    if (D == 3) {
                        const float2 v2 = make_float2(vch, vch);
                        const float2 lo = __ffma2_rn(make_float2(kW.w[pz][0], kW.w[pz][1]), v2,
                                                     make_float2(qz[0][i], qz[1][i]));
                        const float2 hi = __ffma2_rn(make_float2(kW.w[pz][2], kW.w[pz][3]), v2,
                                                     make_float2(qz[2][i], qz[3][i]));
                        qz[0][i] = lo.x;
                        qz[1][i] = lo.y;
                        qz[2][i] = hi.x;
                        qz[3][i] = hi.y;
                    } else {
                        qz[0][i] += vch;
                    }
                }
            }
        } else {
        const float *Fl = Fs + (cz & 1) * (T::FSLOTB / 4) + ty * BX + tx;
#pragma unroll
        for (int p0 = 0; p0 < DELTA; p0 += VC) {
            // issue every load of VC slices, then use them
            // corners paired by z: mc[q] = (slice kz, slice kz + 1) at y x bits q
            float2 mc[VC][4];
            float aux[VC], fx[VC], fy[VC], fz[VC];
            bool inb[VC];
#pragma unroll
            for (int j = 0; j < VC; ++j) {
                const int pz = p0 + j;
                if (pz >= DELTA)
                    break;
                const int z = zl0 + pz;
                float uu[3] = {cxy2[0].x, cxy2[0].y, 0.f};
                if constexpr (D == 3) {
                    // u = sum_a w[pz][a] (x, y, z)[a]: x and y as f32x2 pairs
                    float2 v = __fmul2_rn(make_float2(kW.w[pz][0], kW.w[pz][0]), cxy2[0]);
                    v = __ffma2_rn(make_float2(kW.w[pz][1], kW.w[pz][1]), cxy2[1], v);
                    v = __ffma2_rn(make_float2(kW.w[pz][2], kW.w[pz][2]), cxy2[2], v);
                    v = __ffma2_rn(make_float2(kW.w[pz][3], kW.w[pz][3]), cxy2[3], v);
                    float w = kW.w[pz][0] * cxyz[0];
                    w = fmaf(kW.w[pz][1], cxyz[1], w);
                    w = fmaf(kW.w[pz][2], cxyz[2], w);
                    w = fmaf(kW.w[pz][3], cxyz[3], w);
                    uu[0] = v.x;
                    uu[1] = v.y;
                    uu[2] = w;
                }
                // cells are clamped into the volume even outside the mask, so
                // every load is in bounds; the values outside are not used
                int kx, ky, kz = 0;
                bool in = axis_cell(x, uu[0], lox, hix, g.X, kx, fx[j]);
                in &= axis_cell(y, uu[1], loy, hiy, g.Y, ky, fy[j]);
                if (D == 3)
                    in &= axis_cell(z, uu[2], loz0 - (float)pz, hiz0 - (float)pz, g.Z, kz, fz[j]);
                inb[j] = in && (z < g.Z);
                if (!(al_index_ok(kx, g.X - 1) & al_index_ok(ky, g.Y - 1) &
                      al_index_ok(kz, D == 3 ? g.Z - 1 : 1)))
                    kx = ky = kz = 0;  // checked builds only: the cell left the volume
                bool staged = false;
                if constexpr (TMA) {
                    // the cell and its +1 neighbours inside the staged window
                    const unsigned rx = (unsigned)(kx - (x0 - T::HX));
                    const unsigned ry = (unsigned)(ky - (y0 - T::HY));
                    const unsigned rz = (unsigned)(kz - (zl0 - T::HZ));
                    staged = rx <= (unsigned)(T::TWX - 2) && ry <= (unsigned)(T::TWY - 2) &&
                             rz <= (unsigned)(T::NRES - 2);
                    if (staged) {
                        const int k0 = kz - (z0 - T::HZ);  // ring index of slice kz
                        const int s0 = k0 >= T::NSLOT ? k0 - T::NSLOT : k0;
                        const int s1 = k0 + 1 >= T::NSLOT ? k0 + 1 - T::NSLOT : k0 + 1;
                        const int o = (int)ry * T::TWX + (int)rx;
                        const float *p0s = ring + s0 * (T::SLOTB / 4) + o;
                        const float *p1s = ring + s1 * (T::SLOTB / 4) + o;
                        mc[j][0] = make_float2(p0s[0], p1s[0]);
                        mc[j][1] = make_float2(p0s[1], p1s[1]);
                        mc[j][2] = make_float2(p0s[T::TWX], p1s[T::TWX]);
                        mc[j][3] = make_float2(p0s[T::TWX + 1], p1s[T::TWX + 1]);
                    }
                }
                if (!staged) {
                    const float *mp = M + ((D == 3 ? kz * g.Y : 0) + ky) * g.X + kx;  // nv < 2^31
                    const int sxy = (D == 3) ? g.X * g.Y : 0;
                    mc[j][0] = make_float2(__ldg(mp), D == 3 ? __ldg(mp + sxy) : 0.0f);
                    mc[j][1] = make_float2(__ldg(mp + 1), D == 3 ? __ldg(mp + sxy + 1) : 0.0f);
                    mc[j][2] = make_float2(__ldg(mp + g.X), D == 3 ? __ldg(mp + sxy + g.X) : 0.0f);
                    mc[j][3] = make_float2(__ldg(mp + g.X + 1),
                                           D == 3 ? __ldg(mp + sxy + g.X + 1) : 0.0f);
                }
                aux[j] = 0.0f;
                if constexpr (MODE == MODE_MSE || MODE == MODE_NCC) {
                    if constexpr (TMA) {
                        aux[j] = Fl[pz * (BX * C::BY)];  // zeros beyond the volume (unused)
                    } else if (al_index_ok((min(z, g.Z - 1) * g.Y + y) * g.X + x, g.nv)) {
                        aux[j] = __ldg(F + (min(z, g.Z - 1) * g.Y + y) * g.X + x);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < VC; ++j) {
                const int pz = p0 + j;
                if (pz >= DELTA)
                    break;
                const int z = zl0 + pz;
                if (z >= g.Z)
                    break;
                Interp ip;
                if constexpr (D == 3) {
                    ip = interp8_z2(mc[j], fx[j], fy[j], fz[j]);
                } else {
                    const float c4[4] = {mc[j][0].x, mc[j][1].x, mc[j][2].x, mc[j][3].x};
                    ip = interp4(c4, fx[j], fy[j]);
                }
                const int v = (z * g.Y + y) * g.X + x;
                if (MODE == MODE_FWD) {
                    if constexpr (PAIR) {
                        reinterpret_cast<__nv_bfloat162 *>(W_out)[v] =
                            __floats2bfloat162_rn(inb[j] ? ip.v : 0.0f, __ldg(M + v));
                    } else {
                        W_out[v] = inb[j] ? ip.v : 0.0f;
                        if (m_out)
                            m_out[v] = inb[j] ? 1 : 0;
                        if (G_io) {
                            G_io[v] = inb[j] ? ip.gx : 0.0f;
                            G_io[g.nv + v] = inb[j] ? ip.gy : 0.0f;
                            if (D == 3)
                                G_io[2 * g.nv + v] = inb[j] ? ip.gz : 0.0f;
                        }
                    }
                } else if (inb[j]) {
                    const float gr[3] = {ip.gx, ip.gy, ip.gz};
                    float vch[CHS];
                    if (MODE == MODE_MSE) {
                        const float d = ip.v - aux[j];
                        mom[0] = fmaf(d, d, mom[0]);
                        mom[1] += 1.0f;
#pragma unroll
                        for (int i = 0; i < D; ++i)
                            vch[i] = d * gr[i];
                    } else if (MODE == MODE_NCC) {
                        const float f = aux[j], w = ip.v;
                        mom[0] += 1.0f;
                        mom[1] += f;
                        mom[2] += w;
                        mom[3] = fmaf(f, f, mom[3]);
                        mom[4] = fmaf(w, w, mom[4]);
                        mom[5] = fmaf(f, w, mom[5]);
#pragma unroll
                        for (int i = 0; i < D; ++i) {
                            vch[i] = f * gr[i];
                            vch[D + i] = w * gr[i];
                            vch[2 * D + i] = gr[i];
                        }
                    }
                    if (D == 3) {
                        // qz[a][k] += w[pz][a] vch[k], planes paired (0, 1), (2, 3)
                        const float2 w01 = make_float2(kW.w[pz][0], kW.w[pz][1]);
                        const float2 w23 = make_float2(kW.w[pz][2], kW.w[pz][3]);
#pragma unroll
                        for (int k = 0; k < CHS; ++k) {
                            const float2 v2 = make_float2(vch[k], vch[k]);
                            const float2 lo = __ffma2_rn(w01, v2, make_float2(qz[0][k], qz[1][k]));
                            const float2 hi = __ffma2_rn(w23, v2, make_float2(qz[2][k], qz[3][k]));
                            qz[0][k] = lo.x;
                            qz[1][k] = lo.y;
                            qz[2][k] = hi.x;
                            qz[3][k] = hi.y;
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < CHS; ++k)
                            qz[0][k] += vch[k];
                    }
                }
            }
        }
        }  // MODE != MODE_GW
    }
    if constexpr (TMA) {
        if (fail_layer >= 0) {
            // record the timeout; let the copies in flight land before the
            // block's shared memory goes
            if (tid == 0) {
                atomicExch(&g_unit_error, kFusedTimeout);
                // unconfirmed: batch fail_layer, and batch 1 when layer 0 failed
                const int last = fail_layer == 0 ? min(1, C::BCZ - 1) : fail_layer;
                const uint32_t bars = sbase + (MODE == MODE_GW ? GS::oBar : T::oBar);
                for (int b = fail_layer; b <= last; ++b)
                    al_mbar_wait(bars + 8 * (b & 1), (uint32_t)(b >> 1) & 1u);
            }
            return false;
        }
    }
    if (MODE != MODE_FWD) {
        if constexpr (TMA) {
            // the last four planes one at a time (the staging leaves room for one)
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                flush_planes<D, DELTA, MODE, 1, BCX_, BCY_>(C::BCZ - 1 + a, qz, colvalid, tx, ty,
                                                            P, Xc, dstp);
                if (a < 3) {
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int k = 0; k < CHS; ++k)
                            qz[b][k] = qz[b + 1][k];
                }
            }
        } else {
            // the last four planes (a single plane in 2D), together
            flush_planes<D, DELTA, MODE, C::NPL, BCX_, BCY_>(D == 3 ? C::BCZ - 1 : 0, qz,
                                                             colvalid, tx, ty, P, Xc, dstp);
        }
    }
    if (C::NMOM > 0) {
        double mm[C::NMOM > 0 ? C::NMOM : 1];
        block_reduce_fd<(C::NMOM > 0 ? C::NMOM : 1)>(mom, mm, red);
        if (tid == 0) {
            for (int k = 0; k < C::NMOM; ++k)
                mpart[(int64_t)brick * C::NMOM + k] = mm[k];
            if (MODE == MODE_MSE && icnt)  // the brick's masked voxels, for k_ctrl
                icnt[brick] = (int)mm[1];
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// Gram-form diffusion regulariser on the control lattice.
// Band entries of G = B^T B and H = (DB)^T (DB) along one axis of size N:
//   G[j][j+o] = sum_{x=0}^{N-1} b_j(x) b_{j+o}(x),
//   H[j][j+o] = sum_{x=0}^{N-2} (b_j(x+1)-b_j(x)) (b_{j+o}(x+1)-b_{j+o}(x)),
// b_j(x) = w[x mod delta][j - x/delta] when that index is in 0..3, else 0.
__device__ void band_entry(const Lattice &L, int N, int n, int j, int o, float &G, float &H)
{
    const int j2 = j + o;
    G = 0.0f;
    H = 0.0f;
    if (j < 0 || j >= n || j2 < 0 || j2 >= n)
        return;
    const int delta = L.delta;
    const int lo = max(0, (max(j, j2) - 3) * delta - 1);
    const int hi = min(N, (min(j, j2) + 1) * delta + 1);
    // walk x with its cell q and phase p (no divisions in the loop)
    int q = lo / delta, p = lo - q * delta;
    auto b = [&](int jj, int qq, int pp) {
        const int a = jj - qq;
        return (a >= 0 && a <= 3) ? L.w[pp][a] : 0.0f;
    };
    float bj = b(j, q, p), bj2 = b(j2, q, p);
    for (int x = lo; x < hi; ++x) {
        G = fmaf(bj, bj2, G);
        int qn = q, pn = p + 1;
        if (pn == delta) {
            pn = 0;
            ++qn;
        }
        const float nj = b(j, qn, pn), nj2 = b(j2, qn, pn);
        if (x + 1 < N)
            H = fmaf(nj - bj, nj2 - bj2, H);
        bj = nj;
        bj2 = nj2;
        q = qn;
        p = pn;
    }
}

constexpr int kGramT3 = 8, kGramT2 = 16;

// One tile (tile x, y, z) of component i of dR/dc on the lattice; the
// tile's share of R (before the 1/|X|) goes to *rpart. Every thread of the
// block calls it (any block size up to 1024).
// Shared floats a Gram tile needs (carved from the caller's dynamic memory).
constexpr int kGram3Floats = 14 * 14 * 14 + 2 * 14 * 14 * 8 + 3 * 14 * 8 * 8 + 2 * 3 * 8 * 7;
constexpr int kGram2Floats = 22 * 22 + 2 * 22 * 16 + 2 * 2 * 16 * 7;

__device__ __forceinline__ void gram3_tile(const Grid &g, const Lattice &L,
                                           const float *__restrict__ c, float gscale,
                                           float *__restrict__ gR, int tile_x, int tile_y,
                                           int tile_z, int i, double *rpart, float *sm)
{
    constexpr int T = kGramT3, H3 = T + 6;
    static_assert(kGram3Floats == H3 * H3 * H3 + 2 * H3 * H3 * T + 3 * H3 * T * T + 2 * 3 * T * 7,
                  "Gram tile layout");
    auto cs = reinterpret_cast<float (*)[H3][H3]>(sm);
    auto A = reinterpret_cast<float (*)[H3][T]>(sm + H3 * H3 * H3);
    auto B = reinterpret_cast<float (*)[H3][T]>(sm + H3 * H3 * H3 + H3 * H3 * T);
    float *const g0 = sm + H3 * H3 * H3 + 2 * H3 * H3 * T;
    auto GA = reinterpret_cast<float (*)[T][T]>(g0);
    auto HB = reinterpret_cast<float (*)[T][T]>(g0 + H3 * T * T);
    auto GB = reinterpret_cast<float (*)[T][T]>(g0 + 2 * H3 * T * T);
    auto tG = reinterpret_cast<float (*)[T][7]>(g0 + 3 * H3 * T * T);
    auto tH = reinterpret_cast<float (*)[T][7]>(g0 + 3 * H3 * T * T + 3 * T * 7);
    __shared__ double red[32];
    const int nthr = blockDim.x;
    const int j0[3] = {tile_x * T, tile_y * T, tile_z * T};
    const int nn[3] = {L.nx, L.ny, L.nz};
    const int NN[3] = {g.X, g.Y, g.Z};
    const int tid = threadIdx.x;
    for (int e = tid; e < 3 * T * 7; e += nthr) {
        const int k = e / (T * 7), r = e - k * T * 7, l = r / 7, o = r - l * 7 - 3;
        band_entry(L, NN[k], nn[k], j0[k] + l, o, tG[k][l][o + 3], tH[k][l][o + 3]);
    }
    float rsum = 0.0f;
    {
        __syncthreads();
        for (int e = tid; e < H3 * H3 * H3; e += nthr) {
            const int lz = e / (H3 * H3), r = e - lz * H3 * H3, ly = r / H3, lx = r - ly * H3;
            const int jx = j0[0] + lx - 3, jy = j0[1] + ly - 3, jz = j0[2] + lz - 3;
            float v = 0.0f;
            if (jx >= 0 && jx < L.nx && jy >= 0 && jy < L.ny && jz >= 0 && jz < L.nz)
                v = __ldg(c + (((int64_t)i * L.nz + jz) * L.ny + jy) * L.nx + jx);
            (&cs[0][0][0])[e] = v;
        }
        __syncthreads();
        for (int e = tid; e < H3 * H3 * T; e += nthr) {
            const int lz = e / (H3 * T), r = e - lz * H3 * T, ly = r / T, lx = r - ly * T;
            float a = 0.f, b = 0.f;
#pragma unroll
            for (int o = 0; o < 7; ++o) {
                const float v = cs[lz][ly][lx + o];
                a = fmaf(tH[0][lx][o], v, a);
                b = fmaf(tG[0][lx][o], v, b);
            }
            A[lz][ly][lx] = a;
            B[lz][ly][lx] = b;
        }
        __syncthreads();
        for (int e = tid; e < H3 * T * T; e += nthr) {
            const int lz = e / (T * T), r = e - lz * T * T, ly = r / T, lx = r - ly * T;
            float ga = 0.f, hb = 0.f, gb = 0.f;
#pragma unroll
            for (int o = 0; o < 7; ++o) {
                const float a = A[lz][ly + o][lx], b = B[lz][ly + o][lx];
                ga = fmaf(tG[1][ly][o], a, ga);
                hb = fmaf(tH[1][ly][o], b, hb);
                gb = fmaf(tG[1][ly][o], b, gb);
            }
            GA[lz][ly][lx] = ga;
            HB[lz][ly][lx] = hb;
            GB[lz][ly][lx] = gb;
        }
        __syncthreads();
        for (int e = tid; e < T * T * T; e += nthr) {
            const int lz = e / (T * T), r = e - lz * T * T, ly = r / T, lx = r - ly * T;
            const int jx = j0[0] + lx, jy = j0[1] + ly, jz = j0[2] + lz;
            if (jx >= L.nx || jy >= L.ny || jz >= L.nz)
                continue;
            float s = 0.f;
#pragma unroll
            for (int o = 0; o < 7; ++o) {
                s = fmaf(tG[2][lz][o], GA[lz + o][ly][lx] + HB[lz + o][ly][lx], s);
                s = fmaf(tH[2][lz][o], GB[lz + o][ly][lx], s);
            }
            rsum = fmaf(cs[lz + 3][ly + 3][lx + 3], s, rsum);
            gR[(((int64_t)i * L.nz + jz) * L.ny + jy) * L.nx + jx] = gscale * s;
        }
    }
    double acc[1] = {rsum};
    block_reduce_d<1>(acc, red);
    if (tid == 0)
        *rpart = acc[0];
}

__device__ __forceinline__ void gram2_tile(const Grid &g, const Lattice &L,
                                           const float *__restrict__ c, float gscale,
                                           float *__restrict__ gR, int tile_x, int tile_y, int i,
                                           double *rpart, float *sm)
{
    constexpr int T = kGramT2, H2 = T + 6;
    static_assert(kGram2Floats == H2 * H2 + 2 * H2 * T + 2 * 2 * T * 7, "Gram tile layout");
    auto cs = reinterpret_cast<float (*)[H2]>(sm);
    auto A = reinterpret_cast<float (*)[T]>(sm + H2 * H2);
    auto B = reinterpret_cast<float (*)[T]>(sm + H2 * H2 + H2 * T);
    auto tG = reinterpret_cast<float (*)[T][7]>(sm + H2 * H2 + 2 * H2 * T);
    auto tH = reinterpret_cast<float (*)[T][7]>(sm + H2 * H2 + 2 * H2 * T + 2 * T * 7);
    __shared__ double red[32];
    const int nthr = blockDim.x;
    const int j0[2] = {tile_x * T, tile_y * T};
    const int nn[2] = {L.nx, L.ny};
    const int NN[2] = {g.X, g.Y};
    const int tid = threadIdx.x;
    for (int e = tid; e < 2 * T * 7; e += nthr) {
        const int k = e / (T * 7), r = e - k * T * 7, l = r / 7, o = r - l * 7 - 3;
        band_entry(L, NN[k], nn[k], j0[k] + l, o, tG[k][l][o + 3], tH[k][l][o + 3]);
    }
    float rsum = 0.0f;
    {
        __syncthreads();
        for (int e = tid; e < H2 * H2; e += nthr) {
            const int ly = e / H2, lx = e - ly * H2;
            const int jx = j0[0] + lx - 3, jy = j0[1] + ly - 3;
            float v = 0.0f;
            if (jx >= 0 && jx < L.nx && jy >= 0 && jy < L.ny)
                v = __ldg(c + ((int64_t)i * L.ny + jy) * L.nx + jx);
            cs[ly][lx] = v;
        }
        __syncthreads();
        for (int e = tid; e < H2 * T; e += nthr) {
            const int ly = e / T, lx = e - ly * T;
            float a = 0.f, b = 0.f;
#pragma unroll
            for (int o = 0; o < 7; ++o) {
                const float v = cs[ly][lx + o];
                a = fmaf(tH[0][lx][o], v, a);
                b = fmaf(tG[0][lx][o], v, b);
            }
            A[ly][lx] = a;
            B[ly][lx] = b;
        }
        __syncthreads();
        for (int e = tid; e < T * T; e += nthr) {
            const int ly = e / T, lx = e - ly * T;
            const int jx = j0[0] + lx, jy = j0[1] + ly;
            if (jx >= L.nx || jy >= L.ny)
                continue;
            float s = 0.f;
#pragma unroll
            for (int o = 0; o < 7; ++o) {
                s = fmaf(tG[1][ly][o], A[ly + o][lx], s);
                s = fmaf(tH[1][ly][o], B[ly + o][lx], s);
            }
            rsum = fmaf(cs[ly + 3][lx + 3], s, rsum);
            gR[((int64_t)i * L.ny + jy) * L.nx + jx] = gscale * s;
        }
    }
    double acc[1] = {rsum};
    block_reduce_d<1>(acc, red);
    if (tid == 0)
        *rpart = acc[0];
}

// ---------------------------------------------------------------------------
// Load of data that other blocks of the same launch wrote (CG: through L2,
// bypassing the non-coherent L1) or of data written before the launch.
template <bool CG, typename T>
__device__ __forceinline__ T load_part(const T *p)
{
    if constexpr (CG)
        return __ldcg(p);
    else
        return *p;
}

template <int K, bool CG = false>
__device__ void sum_parts(const double *__restrict__ p, int nb, double (&t)[K], double *red)
{
#pragma unroll
    for (int k = 0; k < K; ++k)
        t[k] = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < K; ++k)
            t[k] += load_part<CG>(p + (int64_t)b * K + k);
    block_reduce_d<K>(t, red);
}

// Sums of two partial arrays (K1 doubles per entry of p1, K2 of p2) in one
// block reduction: t[0 .. K1-1] from p1, t[K1 ..] from p2.
template <int K1, int K2, bool CG = false>
__device__ void sum_parts2(const double *__restrict__ p1, int n1, const double *__restrict__ p2,
                           int n2, double (&t)[K1 + K2], double *red)
{
#pragma unroll
    for (int k = 0; k < K1 + K2; ++k)
        t[k] = 0.0;
    // unrolled so that a thread's loads are in flight together
#pragma unroll 4
    for (int b = threadIdx.x; b < n1; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < K1; ++k)
            t[k] += load_part<CG>(p1 + (int64_t)b * K1 + k);
#pragma unroll 4
    for (int b = threadIdx.x; b < n2; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < K2; ++k)
            t[K1 + k] += load_part<CG>(p2 + (int64_t)b * K2 + k);
    block_reduce_d<K1 + K2>(t, red);
}

// Scalars of the objective from the fixed-order sums of the partials:
// writes {J, S, R, n_mask} to value (when not NULL) and the coefficients of
// the projected channels in dS/dc to the shared array k[3]. Every thread of
// the block takes part; k is valid for all threads on return.
struct Parts {
    const double *mpart, *rpart, *lpart;
    int nbricks, ngram, nlcc;
};

// The scalars of the objective computed by block 0 of a k_fused launch (the
// bricks then start at block 1): the projection pass of LCC runs after the
// statistics, so block 0 forms J and the channel coefficients beside the
// bricks instead of in a launch of its own.
struct ScalBlock {
    int on, mode;
    int64_t nv;
    double lambda, eps;
    Parts P;
    double *value, *ks;
};

template <bool CG = false>
__device__ void objective_scalars(int mode, int64_t nv, double lambda, double eps, const Parts &P,
                                  double *value, double *k, double *red)
{
    // the regulariser's tile shares and the similarity's partials, summed in
    // one block reduction
    double R = 0.0, S = 0.0, n = 0.0;
    if (mode == MODE_NCC) {
        double t[7];
        sum_parts2<1, 6, CG>(P.rpart, P.ngram, P.mpart, P.nbricks, t, red);
        if (threadIdx.x == 0) {
            R = t[0] / (double)nv;
            n = t[1];
            k[0] = k[1] = k[2] = 0.0;
            if (n > 0.0) {
                const double muf = t[2] / n, muw = t[3] / n;
                const double cov = t[6] - n * muf * muw;
                const double vf = t[4] - n * muf * muf;
                const double vw = t[5] - n * muw * muw;
                const double Dd = vf * vw + eps;
                const double sD = sqrt(Dd);
                S = 1.0 - cov / sD;
                const double al = -1.0 / sD, be = cov * vf / (Dd * sD);
                k[0] = al;
                k[1] = be;
                k[2] = -al * muf - be * muw;
            }
        }
    } else {
        double t[3];
        if (mode == MODE_MSE)
            sum_parts2<1, 2, CG>(P.rpart, P.ngram, P.mpart, P.nbricks, t, red);
        else
            sum_parts2<1, 2, CG>(P.rpart, P.ngram, P.lpart, P.nlcc, t, red);
        if (threadIdx.x == 0) {
            R = t[0] / (double)nv;
            n = t[2];
            const double inv_n = n > 0.0 ? 1.0 / n : 0.0;  // the two divisions run side by side
            if (mode == MODE_MSE) {
                S = t[1] * inv_n;
                k[0] = 2.0 * inv_n;
            } else {  // LCC
                S = n > 0.0 ? 1.0 - t[1] * inv_n : 0.0;
                k[0] = inv_n;
            }
        }
    }
    if (threadIdx.x == 0 && value) {
        value[0] = S + lambda * R;
        value[1] = S;
        value[2] = R;
        value[3] = n;
    }
    __syncthreads();
}

// The scalars of the objective, once per evaluation (one block): {J, S, R,
// n_mask} to value (when not NULL) and the channel coefficients to ks[3]
// (when not NULL), for k_ctrl.
__global__ void k_finalize(int mode, int64_t nv, double lambda, double eps, Parts P,
                           double *__restrict__ value, double *__restrict__ ks)
{
    __shared__ double red[7 * 32];  // objective_scalars: up to 7 sums per warp
    __shared__ double k[3];
    objective_scalars(mode, nv, lambda, eps, P, value, k, red);
    if (ks && threadIdx.x < 3)
        ks[threadIdx.x] = k[threadIdx.x];
}

// dJ/dc at control point e: the fixed-order sum of the partials of the (at
// most two per axis) bricks that touch it, the channel combination with the
// scalars k0..k2, plus lambda * dR/dc. CG: the partials were written by other
// blocks of the same launch.
template <int D, int CH, int BCX, int BCY, int BCZ, bool CG>
__device__ __forceinline__ void ctrl_sum(const Lattice &L, int gbx, int gby, int gbz,
                                         const float *__restrict__ bpart,
                                         const float *__restrict__ gR, int64_t e, float (&p)[CH],
                                         float (&gr)[D])
{
    constexpr int JX = BCX + 3, JY = BCY + 3, JZ = (D == 3) ? BCZ + 3 : 1;
    constexpr int NPART = CH * JZ * JY * JX;
    const int64_t total = (int64_t)L.nc;
    const int jx = (int)(e % L.nx);
    const int64_t r = e / L.nx;
    const int jy = (int)(r % L.ny), jz = (int)(r / L.ny);
#pragma unroll
    for (int k = 0; k < CH; ++k)
        p[k] = 0.0f;
    const int bz_hi = (D == 3) ? min(jz / BCZ, gbz - 1) : 0;
    const int bz_lo = (D == 3) ? max(0, jz / BCZ - 1) : 0;
    for (int bz = bz_lo; bz <= bz_hi; ++bz) {
        const int lz = (D == 3) ? jz - bz * BCZ : 0;
        if (lz >= JZ)
            continue;
        for (int by = max(0, jy / BCY - 1); by <= min(jy / BCY, gby - 1); ++by) {
            const int ly = jy - by * BCY;
            if (ly >= JY)
                continue;
            for (int bx = max(0, jx / BCX - 1); bx <= min(jx / BCX, gbx - 1); ++bx) {
                const int lx = jx - bx * BCX;
                if (lx >= JX)
                    continue;
                const int brick = (bz * gby + by) * gbx + bx;
                const float *src = bpart + (int64_t)brick * NPART + (lz * JY + ly) * JX + lx;
#pragma unroll
                for (int k = 0; k < CH; ++k)
                    p[k] += CG ? __ldcg(src + k * (JZ * JY * JX)) : __ldg(src + k * (JZ * JY * JX));
            }
        }
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
        gr[i] = CG ? __ldcg(gR + (int64_t)i * total + e) : __ldg(gR + (int64_t)i * total + e);
}

// ctrl_sum for component i alone: the projected channels of i (i, and for
// NCC D + i and 2D + i) and lambda * dR/dc_i.
template <int D, int CH, int BCX, int BCY, int BCZ>
__device__ __forceinline__ void ctrl_sum1(const Lattice &L, int gbx, int gby, int gbz,
                                          const float *__restrict__ bpart,
                                          const float *__restrict__ gR, int i, int64_t e,
                                          float (&p)[CH / D], float &gr)
{
    constexpr int JX = BCX + 3, JY = BCY + 3, JZ = (D == 3) ? BCZ + 3 : 1;
    constexpr int NPART = CH * JZ * JY * JX, NC = CH / D;
    const int jx = (int)(e % L.nx);
    const int64_t r = e / L.nx;
    const int jy = (int)(r % L.ny), jz = (int)(r / L.ny);
#pragma unroll
    for (int k = 0; k < NC; ++k)
        p[k] = 0.0f;
    const int bz_hi = (D == 3) ? min(jz / BCZ, gbz - 1) : 0;
    const int bz_lo = (D == 3) ? max(0, jz / BCZ - 1) : 0;
    for (int bz = bz_lo; bz <= bz_hi; ++bz) {
        const int lz = (D == 3) ? jz - bz * BCZ : 0;
        if (lz >= JZ)
            continue;
        for (int by = max(0, jy / BCY - 1); by <= min(jy / BCY, gby - 1); ++by) {
            const int ly = jy - by * BCY;
            if (ly >= JY)
                continue;
            for (int bx = max(0, jx / BCX - 1); bx <= min(jx / BCX, gbx - 1); ++bx) {
                const int lx = jx - bx * BCX;
                if (lx >= JX)
                    continue;
                const int brick = (bz * gby + by) * gbx + bx;
                const float *src = bpart + (int64_t)brick * NPART + (lz * JY + ly) * JX + lx;
#pragma unroll
                for (int k = 0; k < NC; ++k)
                    p[k] += __ldg(src + (k * D + i) * (JZ * JY * JX));
            }
        }
    }
    gr = __ldg(gR + (int64_t)i * L.nc + e);
}

template <int D, int CH>
__device__ __forceinline__ void ctrl_combine(const float (&p)[CH], const float (&gr)[D], float k0,
                                             float k1, float k2, float lam, float (&out)[D])
{
#pragma unroll
    for (int i = 0; i < D; ++i) {
        float v;
        if (CH == 3 * D)
            v = fmaf(k0, p[i], fmaf(k1, p[D + i], k2 * p[2 * D + i]));
        else
            v = k0 * p[i];
        out[i] = fmaf(lam, gr[i], v);
    }
}

template <int D, int CH, int BCX, int BCY, int BCZ, bool CG>
__device__ __forceinline__ void ctrl_point(const Lattice &L, int gbx, int gby, int gbz,
                                           const float *__restrict__ bpart,
                                           const float *__restrict__ gR, int64_t e, float k0,
                                           float k1, float k2, float lam, float (&out)[D])
{
    float p[CH], gr[D];
    ctrl_sum<D, CH, BCX, BCY, BCZ, CG>(L, gbx, gby, gbz, bpart, gR, e, p, gr);
    ctrl_combine<D, CH>(p, gr, k0, k1, k2, lam, out);
}

// Per control point and component (one per thread): fixed-order sum of the
// partials of the bricks that touch it, channel combination with the scalars
// ks (k_finalize), plus lambda * dR/dc.
// MSE (sb.on): block 0 forms J and the objective's scalars instead (the
// points start at block 1), and the other blocks take k0 = 2 / n from the
// bricks' integer mask counts (exact integer sums), so no separate launch
// has to finish before them.
template <int D, int CH, int BCX, int BCY, int BCZ>
__global__ void __launch_bounds__(256, 4)
    k_ctrl(Lattice L, int gbx, int gby, int gbz, float lambda, const double *__restrict__ ks,
           const float *__restrict__ bpart, const float *__restrict__ gR,
           float *__restrict__ gc, ScalBlock sb, const int *__restrict__ icnt)
{
    constexpr int NC = CH / D;
    if (sb.on && blockIdx.x == 0) {
        __shared__ double sred[7 * 32];
        __shared__ double sk[3];
        objective_scalars(sb.mode, sb.nv, sb.lambda, sb.eps, sb.P, sb.value, sk, sred);
        return;
    }
    const int64_t total = (int64_t)L.nc;
    const int64_t t = (blockIdx.x - sb.on) * (int64_t)blockDim.x + threadIdx.x;
    const int i = (int)(t / total);
    const int64_t e = t - (int64_t)i * total;
    float p[NC], gr = 0.0f;
    if (i < D)
        ctrl_sum1<D, CH, BCX, BCY, BCZ>(L, gbx, gby, gbz, bpart, gR, i, e, p, gr);
    float k0, k1 = 0.0f, k2 = 0.0f;
    if (sb.on) {
        __shared__ int scnt[8];
        int n = 0;
        for (int b = threadIdx.x; b < sb.P.nbricks; b += blockDim.x)
            n += __ldg(icnt + b);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            n += __shfl_down_sync(0xffffffffu, n, off);
        if ((threadIdx.x & 31) == 0)
            scnt[threadIdx.x >> 5] = n;
        __syncthreads();
        n = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            n += scnt[w];
        k0 = n > 0 ? 2.0f / (float)n : 0.0f;
    } else {
        k0 = (float)ks[0];
        if (NC == 3) {
            k1 = (float)ks[1];
            k2 = (float)ks[2];
        }
    }
    if (i >= D)
        return;
    float v;
    if (NC == 3)
        v = fmaf(k0, p[0], fmaf(k1, p[1 % NC], k2 * p[2 % NC]));
    else
        v = k0 * p[0];
    gc[(int64_t)i * total + e] = fmaf(lambda, gr, v);
}

// ---------------------------------------------------------------------------
struct Layout {
    size_t scal, rpart, gR, bpart, mpart, icnt, Wb, mb, gb, lpart, coef, Gb, total;
    int nbricks, gbx, gby, gbz, ngram, nlcc;
};

Layout make_layout(const Grid &g, const Lattice &L, int kind, int window)
{
    Layout o{};
    const int D = g.ndim;
    const int BCX = brick_bcx(L.delta), BCY = brick_bcy(L.delta), BCZ = brick_bcz(D);
    const int cx = (g.X + L.delta - 1) / L.delta, cy = (g.Y + L.delta - 1) / L.delta;
    const int cz = (D == 3) ? (g.Z + L.delta - 1) / L.delta : 1;
    o.gbx = (cx + BCX - 1) / BCX;
    o.gby = (cy + BCY - 1) / BCY;
    o.gbz = (cz + BCZ - 1) / BCZ;
    o.nbricks = o.gbx * o.gby * o.gbz;
    const int CH = (kind == 1) ? 3 * D : D;
    const int npart = CH * ((D == 3) ? BCZ + 3 : 1) * (BCY + 3) * (BCX + 3);
    if (D == 3)
        o.ngram = 3 * ((L.nx + kGramT3 - 1) / kGramT3) * ((L.ny + kGramT3 - 1) / kGramT3) *
                  ((L.nz + kGramT3 - 1) / kGramT3);  // one block per tile and component
    else
        o.ngram = 2 * ((L.nx + kGramT2 - 1) / kGramT2) * ((L.ny + kGramT2 - 1) / kGramT2);
    o.nlcc = (kind == 2) ? lcc_num_blocks(g, window) : 0;
    size_t off = 0;
    o.scal = off;
    off += 256;
    o.rpart = off;
    off += align256((size_t)o.ngram * 8);
    o.gR = off;
    off += align256((size_t)D * L.nc * 4);
    o.bpart = off;
    off += align256((size_t)o.nbricks * npart * 4);
    o.mpart = off;
    off += align256((size_t)o.nbricks * 6 * 8);
    o.icnt = off;
    off += align256((size_t)o.nbricks * 4);
    if (kind == 2) {
        o.Wb = off;
        off += align256((size_t)g.nv * 4);
        o.mb = off;
        off += align256((size_t)g.nv);
        o.gb = off;
        off += align256((size_t)g.nv * 4);
        o.lpart = off;
        off += align256((size_t)lcc_max_blocks(g, window) * 2 * 8);
        o.coef = off;
        off += lcc_coef_bytes(g);
        o.Gb = off;
        off += align256((size_t)g.nv * D * 4);
    }
    o.total = off;
    return o;
}

// Gram tiles run by the blocks after the bricks of a k_fused launch (none
// when ngram = 0): the regulariser needs only c, so its tiles share the
// launch of the first brick pass instead of a launch of their own. Placed
// after the bricks they fill the last wave; placed first they delayed the
// bricks' streaming loads and measured slower.
struct GramBlocks {
    float *gR;
    double *rpart;
    float gscale;
    int gbx, gby, nbricks;     // brick grid (x, y) and number of bricks
    int gtx, gty, gtz, ngram;  // Gram tiles per axis (gtz = 1 in 2D), total over components
    int *icnt;                 // MSE: each brick's masked voxel count (or NULL)
};


template <int D, int DELTA, int MODE>
__global__ void __launch_bounds__(FCfg<D, DELTA, MODE>::THREADS,
                                  (FCfg<D, DELTA, MODE>::THREADS <= 512 && MODE != MODE_NCC) ? 2
                                                                                            : 1)
    k_fused(Grid g, Lattice L, const float *__restrict__ F, const float *__restrict__ M,
            const float *__restrict__ c, const float *__restrict__ gw_in,
            float *__restrict__ W_out, uint8_t *__restrict__ m_out, float *__restrict__ G_io,
            float *__restrict__ bpart, double *__restrict__ mpart, GramBlocks gb, ScalBlock sb)
{
    if (sb.on && blockIdx.x == 0) {
        __shared__ double sred[7 * 32];
        __shared__ double sk[3];
        objective_scalars(sb.mode, sb.nv, sb.lambda, sb.eps, sb.P, sb.value, sk, sred);
        if (threadIdx.x < 3)
            sb.ks[threadIdx.x] = sk[threadIdx.x];
        return;
    }
    const int b = blockIdx.x - sb.on;
    if (b < gb.nbricks) {
        const int bx = b % gb.gbx, by = (b / gb.gbx) % gb.gby, bz = b / (gb.gbx * gb.gby);
        fused_brick<D, DELTA, MODE>(g, L, F, M, c, gw_in, W_out, m_out, G_io, bpart, mpart, bx,
                                    by, bz, b, BrickMaps{}, gb.icnt);
        return;
    }
    // tile index w = ((component * gtz + tz) * gty + ty) * gtx + tx, its R partial at rpart[w]
    const int w = b - gb.nbricks;
    const int tx = w % gb.gtx, r = w / gb.gtx, ty = r % gb.gty, r2 = r / gb.gty;
    const int tz = r2 % gb.gtz, comp = r2 / gb.gtz;
    extern __shared__ float gtile_sm[];
    if constexpr (D == 3)
        gram3_tile(g, L, c, gb.gscale, gb.gR, tx, ty, tz, comp, gb.rpart + w, gtile_sm);
    else
        gram2_tile(g, L, c, gb.gscale, gb.gR, tx, ty, comp, gb.rpart + w, gtile_sm);
}

// k_fused for 3D bricks staged by TMA (MSE, NCC, FWD; X a multiple of 4).
template <int DELTA, int MODE>
__global__ void __launch_bounds__(FCfg<3, DELTA, MODE>::THREADS,
                                  (FCfg<3, DELTA, MODE>::THREADS <= 512 && MODE != MODE_NCC) ? 2
                                                                                             : 1)
    k_fused_tma(const __grid_constant__ CUtensorMap mapM, const __grid_constant__ CUtensorMap mapF,
                const __grid_constant__ CUtensorMap mapC, int3 lb, Grid g, Lattice L,
                const float *__restrict__ F, const float *__restrict__ M,
                const float *__restrict__ c, float *__restrict__ W_out,
                uint8_t *__restrict__ m_out, float *__restrict__ G_io, float *__restrict__ bpart,
                double *__restrict__ mpart, GramBlocks gb, ScalBlock sb)
{
    if (sb.on && blockIdx.x == 0) {
        __shared__ double sred[7 * 32];
        __shared__ double sk[3];
        objective_scalars(sb.mode, sb.nv, sb.lambda, sb.eps, sb.P, sb.value, sk, sred);
        if (threadIdx.x < 3)
            sb.ks[threadIdx.x] = sk[threadIdx.x];
        return;
    }
    const int b = blockIdx.x - sb.on;
    if (b < gb.nbricks) {
        const int bx = b % gb.gbx, by = (b / gb.gbx) % gb.gby, bz = b / (gb.gbx * gb.gby);
        fused_brick<3, DELTA, MODE, brick_bcx(DELTA), brick_bcy(DELTA), true>(
            g, L, F, M, c, nullptr, W_out, m_out, G_io, bpart, mpart, bx, by, bz, b,
            BrickMaps{&mapM, &mapF, &mapC, lb.x, lb.y, lb.z}, gb.icnt);
        return;
    }
    const int w = b - gb.nbricks;
    const int tx = w % gb.gtx, r = w / gb.gtx, ty = r % gb.gty, r2 = r / gb.gty;
    const int tz = r2 % gb.gtz, comp = r2 / gb.gtz;
    extern __shared__ float gtile_sm[];
    gram3_tile(g, L, c, gb.gscale, gb.gR, tx, ty, tz, comp, gb.rpart + w, gtile_sm);
}

// Tensor maps of the TMA brick path; false when the volume does not allow
// them (rows not on 16-byte boundaries, a box larger than the volume) or an
// encoding fails, and the launch then takes the gathering path.
template <int DELTA, int MODE>
bool brick_tmaps(const Grid &g, const Lattice &L, const float *F, const float *M, const float *c,
                 CUtensorMap *mM, CUtensorMap *mF, CUtensorMap *mC, int *lbox, int *lslot,
                 int *lplane)
{
    using T = TCfg<DELTA, MODE>;
    memset(mM, 0, sizeof(*mM));
    memset(mF, 0, sizeof(*mF));
    memset(mC, 0, sizeof(*mC));
    if (g.ndim != 3 || g.X % 4 != 0 || g.X < T::TWX || g.Y < T::TWY || g.Z < DELTA)
        return false;
    const uint64_t dims[3] = {(uint64_t)g.X, (uint64_t)g.Y, (uint64_t)g.Z};
    const uint64_t strides[2] = {(uint64_t)g.X * 4, (uint64_t)g.X * g.Y * 4};
    const uint32_t boxM[3] = {(uint32_t)T::TWX, (uint32_t)T::TWY, 1u};
    const uint32_t boxF[3] = {(uint32_t)T::BX, (uint32_t)T::BY, (uint32_t)DELTA};
    lattice_boxes<DELTA>(L, lbox, lslot, lplane);
    const uint64_t dimC[1] = {(uint64_t)3 * L.nc};
    const uint32_t boxC[1] = {(uint32_t)*lbox};
    if (!encode_tmap_f32(mM, 3, dims, strides, boxM, M) ||
        !encode_tmap_f32(mC, 1, dimC, nullptr, boxC, c))
        return false;
    if (T::NF > 0 && !encode_tmap_f32(mF, 3, dims, strides, boxF, F))
        return false;
    return true;
}

template <int D, int DELTA, int MODE>
cudaError_t run_fused_kernel(const Grid &g, const Lattice &L, const Layout &lay, char *ws,
                             const float *F, const float *M, const float *c, const float *gw,
                             float *Wo, uint8_t *mo, float *G, bool with_gram, cudaStream_t s,
                             const ScalBlock &sb = ScalBlock{})
{
    using C = FCfg<D, DELTA, MODE>;
    GramBlocks gb{};
    gb.gR = (float *)(ws + lay.gR);
    gb.rpart = (double *)(ws + lay.rpart);
    gb.gscale = (float)(2.0 / (double)g.nv);
    gb.gbx = lay.gbx;
    gb.gby = lay.gby;
    gb.nbricks = lay.nbricks;
    const int T = (D == 3) ? kGramT3 : kGramT2;
    gb.gtx = (L.nx + T - 1) / T;
    gb.gty = (L.ny + T - 1) / T;
    gb.gtz = (D == 3) ? (L.nz + T - 1) / T : 1;
    gb.ngram = with_gram ? lay.ngram : 0;
    gb.icnt = MODE == MODE_MSE ? (int *)(ws + lay.icnt) : nullptr;
    const size_t gsm = (size_t)((D == 3) ? kGram3Floats : kGram2Floats) * sizeof(float);
    const size_t dyn = (with_gram && gsm > C::dyn_smem) ? gsm : C::dyn_smem;
    ProfScope ps(s, MODE == MODE_MSE   ? "k_fused_mse"
                    : MODE == MODE_NCC ? "k_fused_ncc"
                    : MODE == MODE_FWD ? "k_fused_fwd"
                                       : "k_fused_gw");
    if constexpr (D == 3 && MODE == MODE_GW) {
        // dS/dW (3D box) and the D planes of dM~/dy (4D box) per layer
        using GS = GCfg<DELTA>;
        CUtensorMap mW, mG, mC;
        memset(&mW, 0, sizeof(mW));
        memset(&mG, 0, sizeof(mG));
        memset(&mC, 0, sizeof(mC));
        const uint64_t dims[4] = {(uint64_t)g.X, (uint64_t)g.Y, (uint64_t)g.Z, 3};
        const uint64_t strides[3] = {(uint64_t)g.X * 4, (uint64_t)g.X * g.Y * 4,
                                     (uint64_t)g.nv * 4};
        const uint32_t box[4] = {(uint32_t)C::BX, (uint32_t)C::BY, (uint32_t)DELTA, 3u};
        if (g.X % 4 == 0 && g.nv % 4 == 0 && g.X >= C::BX && g.Y >= C::BY && g.Z >= DELTA &&
            encode_tmap_f32(&mW, 3, dims, strides, box, gw) &&
            encode_tmap_f32(&mG, 4, dims, strides, box, G)) {
            const size_t tdyn = (size_t)GS::bytes + 128;
            cudaError_t e = cudaFuncSetAttribute(k_fused_tma<DELTA, MODE>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)tdyn);
            if (e != cudaSuccess)
                return e;
            k_fused_tma<DELTA, MODE><<<sb.on + lay.nbricks, C::THREADS, tdyn, s>>>(
                mW, mG, mC, int3{0, 0, 0}, g, L, F, M, c, Wo, mo, G, (float *)(ws + lay.bpart),
                (double *)(ws + lay.mpart), gb, sb);
            return cudaGetLastError();
        }
    }
    if constexpr (D == 3 && MODE != MODE_GW) {
        CUtensorMap mM, mF, mC;
        int lbox = 0, lslot = 0, lplane = 0;
        if (brick_tmaps<DELTA, MODE>(g, L, F, M, c, &mM, &mF, &mC, &lbox, &lslot, &lplane)) {
            using T = TCfg<DELTA, MODE>;
            const size_t tdyn = (size_t)T::bytes + 128 > gsm ? (size_t)T::bytes + 128 : gsm;
            cudaError_t e = cudaFuncSetAttribute(k_fused_tma<DELTA, MODE>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)tdyn);
            if (e != cudaSuccess)
                return e;
            k_fused_tma<DELTA, MODE><<<sb.on + lay.nbricks + gb.ngram, C::THREADS, tdyn, s>>>(
                mM, mF, mC, int3{lbox, lslot, lplane}, g, L, F, M, c, Wo, mo, G,
                (float *)(ws + lay.bpart), (double *)(ws + lay.mpart), gb, sb);
            return cudaGetLastError();
        }
    }
    if (dyn > 0) {  // static + dynamic may pass 48 KB: always opt in
        const size_t most = gsm > C::dyn_smem ? gsm : C::dyn_smem;
        cudaError_t e = cudaFuncSetAttribute(k_fused<D, DELTA, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)most);
        if (e != cudaSuccess)
            return e;
    }
    k_fused<D, DELTA, MODE><<<sb.on + lay.nbricks + gb.ngram, C::THREADS, dyn, s>>>(
        g, L, F, M, c, gw, Wo, mo, G, (float *)(ws + lay.bpart), (double *)(ws + lay.mpart),
        gb, sb);
    return cudaGetLastError();
}

template <int D, int DELTA>
cudaError_t run_all(const Grid &g, const Lattice &L, int kind, int window, double eps,
                    double lambda, const float *F, const float *M, const float *c, double *value,
                    float *gc, char *ws, cudaStream_t s)
{
    const Layout lay = make_layout(g, L, kind, window);
    double *rpart = (double *)(ws + lay.rpart);
    float *gR = (float *)(ws + lay.gR);
    cudaError_t e;
    int mode;
    if (kind == 0) {
        mode = MODE_MSE;
        e = run_fused_kernel<D, DELTA, MODE_MSE>(g, L, lay, ws, F, M, c, nullptr, nullptr, nullptr,
                                                 nullptr, true, s);
    } else if (kind == 1) {
        mode = MODE_NCC;
        e = run_fused_kernel<D, DELTA, MODE_NCC>(g, L, lay, ws, F, M, c, nullptr, nullptr, nullptr,
                                                 nullptr, true, s);
    } else {
        mode = 2;
        float *Wb = (float *)(ws + lay.Wb), *gb = (float *)(ws + lay.gb);
        uint8_t *mb = (uint8_t *)(ws + lay.mb);
        float *Gb = gc ? (float *)(ws + lay.Gb) : nullptr;
        e = run_fused_kernel<D, DELTA, MODE_FWD>(g, L, lay, ws, F, M, c, nullptr, Wb, mb, Gb, true,
                                                 s);
        if (e != cudaSuccess)
            return e;
        float *coef = (float *)(ws + lay.coef);
        if (!gc) {
            e = launch_lcc(g, window, eps, F, Wb, mb, true, nullptr, (double *)(ws + lay.lpart),
                           coef, s);
        } else {
            // statistics -> coefficient planes -> dS/dW * |X_m| -> projection
            e = launch_lcc_stats(g, window, eps, F, Wb, mb, (double *)(ws + lay.lpart), coef, s);
            if (e != cudaSuccess)
                return e;
            e = launch_lcc_grad(g, window, F, Wb, mb, coef, gb, s);
            if (e != cudaSuccess)
                return e;
            ScalBlock sb{1, 2, g.nv, lambda, eps,
                         Parts{(const double *)(ws + lay.mpart), rpart,
                               (const double *)(ws + lay.lpart), lay.nbricks, lay.ngram, lay.nlcc},
                         value, (double *)(ws + lay.scal)};
            e = run_fused_kernel<D, DELTA, MODE_GW>(g, L, lay, ws, F, M, c, gb, nullptr, nullptr,
                                                    Gb, false, s, sb);
        }
    }
    if (e != cudaSuccess)
        return e;
    Parts parts{(const double *)(ws + lay.mpart), rpart, (const double *)(ws + lay.lpart),
                lay.nbricks, lay.ngram, lay.nlcc};
    double *ks = (double *)(ws + lay.scal);  // channel coefficients for k_ctrl
    // MSE with gradient: block 0 of k_ctrl forms the scalars (selfk)
    const bool selfk = kind == 0 && gc;
    if (!(kind == 2 && gc) && !selfk) {  // LCC: block 0 of the projection pass did it
        ProfScope ps(s, "k_finalize");
        k_finalize<<<1, 256, 0, s>>>(mode, g.nv, lambda, eps, parts, value, gc ? ks : nullptr);
        e = cudaGetLastError();
        if (e != cudaSuccess || !gc)
            return e;
    }
    {
        const int th = 256;
        const ScalBlock sb{selfk ? 1 : 0, mode, g.nv, lambda, eps, parts, value, nullptr};
        const int64_t nb = sb.on + ((int64_t)D * L.nc + th - 1) / th;  // one (component, point) per thread
        const float *bp = (const float *)(ws + lay.bpart);
        const int *icnt = (const int *)(ws + lay.icnt);
        ProfScope ps(s, "k_ctrl");
        constexpr int BCX = brick_bcx(DELTA), BCY = brick_bcy(DELTA), BCZ = brick_bcz(D);
        if (kind == 1)
            k_ctrl<D, 3 * D, BCX, BCY, BCZ><<<(int)nb, th, 0, s>>>(
                L, lay.gbx, lay.gby, lay.gbz, (float)lambda, ks, bp, gR, gc, sb, icnt);
        else
            k_ctrl<D, D, BCX, BCY, BCZ><<<(int)nb, th, 0, s>>>(
                L, lay.gbx, lay.gby, lay.gbz, (float)lambda, ks, bp, gR, gc, sb, icnt);
        e = cudaGetLastError();
    }
    return e;
}

// ---------------------------------------------------------------------------
// Warp of `count` volumes by the B-spline fields of their control lattices
// (A1 + A2 fused, the forward brick with no gradient planes): W[v] =
// M[v] o (x + B c[v]), mask[v] when given. With PAIR, W points at bf16 pairs
// (W[v], M[v]) instead (the network input of the pair F = W). blockIdx.y is
// the volume.
template <int D, int DELTA, bool PAIR>
__global__ void __launch_bounds__(FCfg<D, DELTA, MODE_FWD>::THREADS,
                                  FCfg<D, DELTA, MODE_FWD>::THREADS <= 512 ? 2 : 1)
    k_warp_ctrl(Grid g, Lattice L, int gbx, int gby, const float *__restrict__ M,
                const float *__restrict__ c, float *__restrict__ W, uint8_t *__restrict__ m)
{
    const int b = blockIdx.x;
    const int64_t vol = blockIdx.y;
    const int bx = b % gbx, by = (b / gbx) % gby, bz = b / (gbx * gby);
    fused_brick<D, DELTA, MODE_FWD, brick_bcx(DELTA), brick_bcy(DELTA), false, PAIR>(
        g, L, nullptr, M + vol * g.nv, c + vol * D * L.nc, nullptr, W + vol * g.nv,
        m ? m + vol * g.nv : nullptr, nullptr, nullptr, nullptr, bx, by, bz, b);
}

template <int D, int DELTA, bool PAIR>
cudaError_t warp_ctrl_run(const Grid &g, const Lattice &L, int count, const float *M,
                          const float *c, float *W, uint8_t *m, cudaStream_t s)
{
    using C = FCfg<D, DELTA, MODE_FWD>;
    const Layout lay = make_layout(g, L, 0, 3);
    if (C::dyn_smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_warp_ctrl<D, DELTA, PAIR>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::dyn_smem);
        if (e != cudaSuccess)
            return e;
    }
    ProfScope ps(s, PAIR ? "k_warp_ctrl_pair" : "k_warp_ctrl");
    k_warp_ctrl<D, DELTA, PAIR><<<dim3(lay.nbricks, count), C::THREADS, C::dyn_smem, s>>>(
        g, L, lay.gbx, lay.gby, M, c, W, m);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batches: one persistent launch per iteration over many problems.
//
// The launch's blocks take work items from a device queue (one atomic
// counter) in the order of the item list. Phase A items -- the bricks and
// the Gram tiles of every problem -- come first and wait for nothing; phase B
// items -- chunks of a problem's control points: fixed-order sum of its
// brick partials, dJ/dc and the Adam step -- wait until every phase A item of
// their problem has published its results. Every phase A item is taken
// before any phase B item, by a block that is running, so a wait only ever
// waits for running blocks; it is bounded anyway (BatchStep::spin_limit
// polls, then AL_ERR_TIMEOUT in the error word and the chunk is skipped).
// The per-item arithmetic is that of k_fused (bricks, Gram tiles) and k_ctrl + k_adam, so
// a problem's coefficients follow the single-problem path bit for bit.
template <int DELTA, int T>
struct BCfg {
    static constexpr int BCX = batch_tile_bcx(DELTA, T), BCY = batch_tile_bcy(DELTA, T);
    using C3 = FCfg<3, DELTA, MODE_MSE, BCX, BCY>;
    using C2 = FCfg<2, DELTA, MODE_MSE, BCX, BCY>;
    static constexpr int THREADS = C3::THREADS;
    static constexpr int MINB = batch_tile_minb(DELTA, T);  // resident blocks per SM
    static_assert(C2::THREADS == THREADS, "2D and 3D bricks share the block size");
    static constexpr size_t fsm = C3::dyn_smem > C2::dyn_smem ? C3::dyn_smem : C2::dyn_smem;
    static constexpr size_t gsm = (size_t)kGram3Floats * sizeof(float);  // > the 2D tile
    static constexpr size_t dyn_smem = fsm > gsm ? fsm : gsm;
};

__device__ __forceinline__ int load_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int D, int DELTA, int T>
__device__ __forceinline__ void batch_ctrl_adam(const BatchProblem &P, const BatchStep &st,
                                                int64_t e, float k0, float inv_bc1,
                                                float inv_bc2)
{
    constexpr int BCX = batch_tile_bcx(DELTA, T), BCY = batch_tile_bcy(DELTA, T);
    constexpr int BCZ = brick_bcz(D);
    float gv[D];
    ctrl_point<D, D, BCX, BCY, BCZ, true>(P.L, P.gbx, P.gby, P.gbz, P.bpart, P.gR, e, k0, 0.0f,
                                          0.0f, (float)P.lambda, gv);
    if (!st.update)
        return;
    const float b1 = (float)st.beta1, b2 = (float)st.beta2;
    const float omb1 = (float)(1.0 - st.beta1), omb2 = (float)(1.0 - st.beta2);
    const int64_t nc = P.L.nc;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const int64_t q = i * nc + e;
        const float h = P.h[i];
        const float gn = gv[i] * h;
        const float mm = fmaf(b1, P.m[q], omb1 * gn);
        const float vv = fmaf(b2, P.v[q], omb2 * gn * gn);
        P.m[q] = mm;
        P.v[q] = vv;
        const float den = sqrtf(vv * inv_bc2) + st.eps;
        P.c[q] -= (st.lr * h) * ((mm * inv_bc1) / den);
    }
}

template <int DELTA, int T>
__global__ void __launch_bounds__(BCfg<DELTA, T>::THREADS, BCfg<DELTA, T>::MINB)
    k_batch(const BatchProblem *__restrict__ probs, const BatchItem *__restrict__ items, int nitems,
            int *__restrict__ counters, BatchStep st)
{
    __shared__ int s_item, s_ok;
    __shared__ double red[7 * 32];  // objective_scalars: up to 7 sums per warp
    __shared__ double ks[3];
    __shared__ float s_inv_bc[2];
    if (threadIdx.x == 0) {
        s_inv_bc[0] = adam_inv_bias(st.beta1, (long long)st.t);
        s_inv_bc[1] = adam_inv_bias(st.beta2, (long long)st.t);
    }
    for (;;) {
        __syncthreads();  // the previous item is done with shared memory
        if (threadIdx.x == 0)
            s_item = atomicAdd(counters, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems)
            break;
        const BatchItem w = items[it];
        const BatchProblem &P = probs[w.prob];
        if (w.kind == BATCH_BRICK) {
            const int bx = w.idx % P.gbx, r = w.idx / P.gbx, by = r % P.gby, bz = r / P.gby;
            constexpr int BCX = BCfg<DELTA, T>::BCX, BCY = BCfg<DELTA, T>::BCY;
            if (P.g.ndim == 3)
                fused_brick<3, DELTA, MODE_MSE, BCX, BCY>(P.g, P.L, P.F, P.M, P.c, nullptr, nullptr,
                                                          nullptr, nullptr, P.bpart, P.mpart, bx,
                                                          by, bz, w.idx);
            else
                fused_brick<2, DELTA, MODE_MSE, BCX, BCY>(P.g, P.L, P.F, P.M, P.c, nullptr, nullptr,
                                                          nullptr, nullptr, P.bpart, P.mpart, bx,
                                                          by, bz, w.idx);
        } else if (w.kind == BATCH_GRAM) {
            // tile index = ((component * gtz + tz) * gty + ty) * gtx + tx
            const int tx = w.idx % P.gtx, r = w.idx / P.gtx, ty = r % P.gty, r2 = r / P.gty;
            const int tz = r2 % P.gtz, comp = r2 / P.gtz;
            extern __shared__ float bsm[];
            if (P.g.ndim == 3)
                gram3_tile(P.g, P.L, P.c, P.gscale, P.gR, tx, ty, tz, comp, P.rpart + w.idx, bsm);
            else
                gram2_tile(P.g, P.L, P.c, P.gscale, P.gR, tx, ty, comp, P.rpart + w.idx, bsm);
        }
        if (w.kind != BATCH_CTRL) {
            __syncthreads();  // every write of the item has been issued
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(counters + 1 + w.prob, 1);
            }
            continue;
        }
        // phase B: wait (bounded) for the problem's phase A items
        if (threadIdx.x == 0) {
            const int need = P.nA + st.extra_wait;
            long long polls = 0;
            int ok = 1;
            while (load_acquire(counters + 1 + w.prob) < need) {
                if (++polls > st.spin_limit) {
                    ok = 0;
                    atomicExch(st.err, 6 /* AL_ERR_TIMEOUT */);
                    break;
                }
                __nanosleep(128);
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok)
            continue;
        const Parts parts{P.mpart, P.rpart, nullptr, P.nbricks, P.ngram, 0};
        double *val = (w.idx == 0 && P.values && st.record >= 0) ? P.values + 4 * st.record : nullptr;
        objective_scalars<true>(MODE_MSE, P.g.nv, P.lambda, 0.0, parts, val, ks, red);
        const float k0 = (float)ks[0];
        const int64_t e = (int64_t)w.idx * blockDim.x + threadIdx.x;
        if (e < P.L.nc) {
            if (P.g.ndim == 3)
                batch_ctrl_adam<3, DELTA, T>(P, st, e, k0, s_inv_bc[0], s_inv_bc[1]);
            else
                batch_ctrl_adam<2, DELTA, T>(P, st, e, k0, s_inv_bc[0], s_inv_bc[1]);
        }
    }
}

template <int DELTA, int T>
cudaError_t run_batch(int blocks, const BatchProblem *probs, const BatchItem *items, int nitems,
                      int *counters, const BatchStep &st, cudaStream_t s)
{
    using B = BCfg<DELTA, T>;
    cudaError_t e = cudaFuncSetAttribute(k_batch<DELTA, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)B::dyn_smem);
    if (e != cudaSuccess)
        return e;
    ProfScope ps(s, "k_batch");
    k_batch<DELTA, T><<<blocks, B::THREADS, B::dyn_smem, s>>>(probs, items, nitems, counters, st);
    return cudaGetLastError();
}

template <int DELTA, int T>
int batch_occupancy()
{
    using B = BCfg<DELTA, T>;
    if (cudaFuncSetAttribute(k_batch<DELTA, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)B::dyn_smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<DELTA, T>, B::THREADS,
                                                      B::dyn_smem) != cudaSuccess)
        return 0;
    return n;
}

// (delta, tile) -> f<delta, tile>(args...), or `fail` for an unknown pair.
#define AL_BATCH_DISPATCH(delta, tile, fail, CALL)          \
    switch ((delta) * 16 + (tile)) {                        \
    case 4 * 16 + 0: return CALL(4, 0);                     \
    case 4 * 16 + 1: return CALL(4, 1);                     \
    case 4 * 16 + 2: return CALL(4, 2);                     \
    case 6 * 16 + 0: return CALL(6, 0);                     \
    case 6 * 16 + 1: return CALL(6, 1);                     \
    case 6 * 16 + 2: return CALL(6, 2);                     \
    case 8 * 16 + 0: return CALL(8, 0);                     \
    case 8 * 16 + 1: return CALL(8, 1);                     \
    case 8 * 16 + 2: return CALL(8, 2);                     \
    }                                                       \
    return fail;

}  // namespace

bool fused_supported(const Grid &g, const Lattice &L, int kind, int window)
{
    (void)g;
    (void)kind;
    (void)window;
    return L.delta == 4 || L.delta == 6 || L.delta == 8;
}

size_t fused_ws(const Grid &g, const Lattice &L, int kind, int window)
{
    return make_layout(g, L, kind, window).total;
}

void fused_warped_offsets(const Grid &g, const Lattice &L, int window, size_t *w, size_t *m)
{
    const Layout lay = make_layout(g, L, 2, window);
    *w = lay.Wb;
    *m = lay.mb;
}

cudaError_t launch_fused(const Grid &g, const Lattice &L, int kind, int window, double eps,
                         double lambda, const float *F, const float *M, const float *c,
                         double *value, float *gc, void *ws, cudaStream_t s)
{
    char *w = (char *)ws;
    if (g.ndim == 3) {
        switch (L.delta) {
        case 4: return run_all<3, 4>(g, L, kind, window, eps, lambda, F, M, c, value, gc, w, s);
        case 6: return run_all<3, 6>(g, L, kind, window, eps, lambda, F, M, c, value, gc, w, s);
        case 8: return run_all<3, 8>(g, L, kind, window, eps, lambda, F, M, c, value, gc, w, s);
        }
    } else {
        switch (L.delta) {
        case 4: return run_all<2, 4>(g, L, kind, window, eps, lambda, F, M, c, value, gc, w, s);
        case 6: return run_all<2, 6>(g, L, kind, window, eps, lambda, F, M, c, value, gc, w, s);
        case 8: return run_all<2, 8>(g, L, kind, window, eps, lambda, F, M, c, value, gc, w, s);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_warp_ctrl(const Grid &g, const Lattice &L, int count, const float *M,
                             const float *c, float *W, uint8_t *m, void *pair, cudaStream_t s)
{
    if (pair) {  // the network input: 3D only
        float *P = static_cast<float *>(pair);
        if (g.ndim != 3)
            return cudaErrorInvalidValue;
        switch (L.delta) {
        case 4: return warp_ctrl_run<3, 4, true>(g, L, count, M, c, P, nullptr, s);
        case 6: return warp_ctrl_run<3, 6, true>(g, L, count, M, c, P, nullptr, s);
        case 8: return warp_ctrl_run<3, 8, true>(g, L, count, M, c, P, nullptr, s);
        }
    } else if (g.ndim == 3) {
        switch (L.delta) {
        case 4: return warp_ctrl_run<3, 4, false>(g, L, count, M, c, W, m, s);
        case 6: return warp_ctrl_run<3, 6, false>(g, L, count, M, c, W, m, s);
        case 8: return warp_ctrl_run<3, 8, false>(g, L, count, M, c, W, m, s);
        }
    } else {
        switch (L.delta) {
        case 4: return warp_ctrl_run<2, 4, false>(g, L, count, M, c, W, m, s);
        case 6: return warp_ctrl_run<2, 6, false>(g, L, count, M, c, W, m, s);
        case 8: return warp_ctrl_run<2, 8, false>(g, L, count, M, c, W, m, s);
        }
    }
    return cudaErrorInvalidValue;
}

void batch_geometry(const Grid &g, const Lattice &L, int tile, int *gb, int *gt, int *npart,
                    int *nmom)
{
    const int D = g.ndim;
    const int BCX = batch_tile_bcx(L.delta, tile), BCY = batch_tile_bcy(L.delta, tile);
    const int BCZ = brick_bcz(D);
    const int cx = (g.X + L.delta - 1) / L.delta, cy = (g.Y + L.delta - 1) / L.delta;
    const int cz = (D == 3) ? (g.Z + L.delta - 1) / L.delta : 1;
    gb[0] = (cx + BCX - 1) / BCX;
    gb[1] = (cy + BCY - 1) / BCY;
    gb[2] = (cz + BCZ - 1) / BCZ;
    const int T = (D == 3) ? kGramT3 : kGramT2;
    gt[0] = (L.nx + T - 1) / T;
    gt[1] = (L.ny + T - 1) / T;
    gt[2] = (D == 3) ? (L.nz + T - 1) / T : 1;
    *npart = D * ((D == 3) ? BCZ + 3 : 1) * (BCY + 3) * (BCX + 3);
    *nmom = 2;
}

int batch_tiles() { return kBatchTiles; }

void batch_tile_cells(int delta, int tile, int *bcx, int *bcy)
{
    *bcx = batch_tile_bcx(delta, tile);
    *bcy = batch_tile_bcy(delta, tile);
}

int batch_threads(int delta, int tile)
{
#define AL_THREADS(d, t) BCfg<d, t>::THREADS
    AL_BATCH_DISPATCH(delta, tile, 0, AL_THREADS)
#undef AL_THREADS
}

int batch_blocks_per_sm(int delta, int tile)
{
#define AL_OCC(d, t) batch_occupancy<d, t>()
    AL_BATCH_DISPATCH(delta, tile, 0, AL_OCC)
#undef AL_OCC
}

cudaError_t launch_batch(int delta, int tile, int blocks, const BatchProblem *probs,
                         const BatchItem *items, int nitems, int *counters, const BatchStep &st,
                         cudaStream_t s)
{
#define AL_RUN(d, t) run_batch<d, t>(blocks, probs, items, nitems, counters, st, s)
    AL_BATCH_DISPATCH(delta, tile, cudaErrorInvalidValue, AL_RUN)
#undef AL_RUN
}

AL_UNIT_ERROR_READER(unit_error_fused)

cudaError_t fused_set_drop_batch(int batch)
{
    return cudaMemcpyToSymbol(c_fused_drop_batch, &batch, sizeof(int));
}

}  // namespace airgb
