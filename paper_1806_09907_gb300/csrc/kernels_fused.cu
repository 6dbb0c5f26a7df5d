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
    static constexpr int VC = (MODE == MODE_FWD || MODE == MODE_MSE) ? 2 : 1;  // slices whose loads are in flight
    // dynamic shared memory: up to NPL planes of column partials
    // P[NPL][BY][BX][CHS] and their x contraction X[NPL][BY][JX][CHS]
    static constexpr int NPL = (D == 3) ? 4 : 1;
    static constexpr int nP = (MODE == MODE_FWD) ? 0 : NPL * BY * BX * CHS;
    static constexpr int nX = (MODE == MODE_FWD) ? 0 : NPL * BY * JX * CHS;
    static constexpr size_t dyn_smem = (size_t)(nP + nX) * sizeof(float);
};

// xy contraction of control plane jz for the column (qx + px/DELTA, ...):
// sum_b wy[b] sum_e wx[e] cb[i][jz][qy + b][qx + e].
template <int D, int JZ, int JY, int JX>
__device__ __forceinline__ void plane_xy(const float (&cb)[D][JZ][JY][JX], int jz, int qy, int qx,
                                         const float (&wx)[4], const float (&wy)[4], float (&out)[D])
{
#pragma unroll
    for (int i = 0; i < D; ++i) {
        float acc = 0.0f;
        if (jz < JZ) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                float r = wx[0] * cb[i][jz][qy + b][qx];
                r = fmaf(wx[1], cb[i][jz][qy + b][qx + 1], r);
                r = fmaf(wx[2], cb[i][jz][qy + b][qx + 2], r);
                r = fmaf(wx[3], cb[i][jz][qy + b][qx + 3], r);
                acc = fmaf(wy[b], r, acc);
            }
        }
        out[i] = acc;
    }
}

// Planes 0..NPL-1 of the thread's column partials qz -> x contraction -> y
// contraction -> the brick's partial sums of local planes lp0 .. lp0+NPL-1.
// Every thread of the block calls it. Cell-wise loops with compile-time
// bounds and two accumulators per output.
template <int D, int DELTA, int MODE, int NPL, int BCX_ = brick_bcx(DELTA),
          int BCY_ = brick_bcy(DELTA)>
__device__ __forceinline__ void flush_planes(int lp0, const float (&qz)[4][FCfg<D, DELTA, MODE>::CHS],
                                             bool colvalid, int tx, int ty, float *P, float *Xc,
                                             const float (*wt)[4], float *dst)
{
    using C = FCfg<D, DELTA, MODE, BCX_, BCY_>;
    constexpr int CHS = C::CHS, BX = C::BX, BY = C::BY, JX = C::JX, JY = C::JY, JZ = C::JZ;
    const int tid = threadIdx.x;
#pragma unroll
    for (int a = 0; a < NPL; ++a)
#pragma unroll
        for (int k = 0; k < CHS; ++k)
            P[((a * BY + ty) * BX + tx) * CHS + k] = colvalid ? qz[a][k] : 0.0f;
    __syncthreads();
    for (int e = tid; e < NPL * BY * JX * CHS; e += C::THREADS) {
        const int k = e % CHS, r0 = e / CHS;
        const int jxl = r0 % JX, r1 = r0 / JX;
        const int yy = r1 % BY, a = r1 / BY;
        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
        for (int e4 = 0; e4 < 4; ++e4) {
            const int q = jxl - e4;
            if (q >= 0 && q < C::BCX) {
                const float *src = P + ((a * BY + yy) * BX + q * DELTA) * CHS + k;
#pragma unroll
                for (int px = 0; px < DELTA; ++px) {
                    if (px & 1)
                        s1 = fmaf(wt[px][e4], src[px * CHS], s1);
                    else
                        s0 = fmaf(wt[px][e4], src[px * CHS], s0);
                }
            }
        }
        Xc[((a * BY + yy) * JX + jxl) * CHS + k] = s0 + s1;
    }
    __syncthreads();
    for (int e = tid; e < NPL * JY * JX * CHS; e += C::THREADS) {
        const int jxl = e % JX, r0 = e / JX;
        const int jyl = r0 % JY, r1 = r0 / JY;
        const int k = r1 % CHS, a = r1 / CHS;
        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
        for (int e4 = 0; e4 < 4; ++e4) {
            const int q = jyl - e4;
            if (q >= 0 && q < C::BCY) {
                const float *src = Xc + ((a * BY + q * DELTA) * JX + jxl) * CHS + k;
#pragma unroll
                for (int py = 0; py < DELTA; ++py) {
                    if (py & 1)
                        s1 = fmaf(wt[py][e4], src[py * JX * CHS], s1);
                    else
                        s0 = fmaf(wt[py][e4], src[py * JX * CHS], s0);
                }
            }
        }
        dst[(k * JZ + lp0 + a) * JY * JX + jyl * JX + jxl] = s0 + s1;
    }
}

// One brick (bx, by, bz) of one problem: the whole per-voxel work of the
// brick, its partial sums written to bpart / mpart at index `brick`. Every
// thread of a block of FCfg::THREADS threads calls it; it uses the block's
// shared memory (static arrays here and FCfg::dyn_smem of dynamic memory).
template <int D, int DELTA, int MODE, int BCX_ = brick_bcx(DELTA), int BCY_ = brick_bcy(DELTA)>
__device__ __forceinline__ void fused_brick(const Grid &g, const Lattice &L,
                                            const float *__restrict__ F,
                                            const float *__restrict__ M,
                                            const float *__restrict__ c,
                                            const float *__restrict__ gw_in,
                                            float *__restrict__ W_out, uint8_t *__restrict__ m_out,
                                            float *__restrict__ G_io, float *__restrict__ bpart,
                                            double *__restrict__ mpart, int bx, int by, int bz,
                                            int brick)
{
    // MODE_FWD writes W, the mask and (when G_io is given) dM~/dy as D planes;
    // MODE_GW reads dS/dW and those planes back (no expansion, no gathers).
    using C = FCfg<D, DELTA, MODE, BCX_, BCY_>;
    constexpr int JX = C::JX, JY = C::JY, JZ = C::JZ, CHS = C::CHS, BX = C::BX;
    constexpr WTab<DELTA> kW{};  // weights of the compile-time z phases
    __shared__ float cb[D][JZ][JY][JX];
    __shared__ float wt[DELTA][4];
    __shared__ double red[(C::NMOM > 0 ? C::NMOM : 1) * ((C::THREADS + 31) / 32)];
    extern __shared__ float dsm[];
    float *P = dsm, *Xc = dsm + C::nP;

    const int tid = threadIdx.x;
    const int tx = tid % BX, ty = tid / BX;
    const int cx0 = bx * C::BCX, cy0 = by * C::BCY, cz0 = bz * C::BCZ;
    const int x = cx0 * DELTA + tx, y = cy0 * DELTA + ty, z0 = (D == 3) ? cz0 * DELTA : 0;

    if (tid < DELTA * 4)
        wt[tid / 4][tid % 4] = L.w[tid / 4][tid % 4];
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
    float cxy[4][D];  // xy-contracted control values of the four active planes
#pragma unroll
    for (int a = 0; a < 4; ++a)
        if (MODE != MODE_GW)
            plane_xy<D, JZ, JY, JX>(cb, a, qyl, qxl, wx, wy, cxy[a]);
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
    constexpr int NCOR = (D == 3) ? 8 : 4;
    for (int cz = 0; cz < C::BCZ; ++cz) {
        const bool active = cz < nlayers && colvalid;
        const int zl0 = z0 + cz * DELTA;
        // GW: the layer's loads are issued before the flush of the previous
        // plane, so they are in flight while the block contracts it
        float gv[MODE == MODE_GW ? DELTA : 1], gr[MODE == MODE_GW ? DELTA : 1][D];
        if constexpr (MODE == MODE_GW) {
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
                                                            wt, dstp);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
#pragma unroll
                for (int k = 0; k < CHS; ++k)
                    qz[a][k] = qz[a + 1][k];
#pragma unroll
                for (int i = 0; i < D; ++i)
                    cxy[a][i] = cxy[a + 1][i];
            }
#pragma unroll
            for (int k = 0; k < CHS; ++k)
                qz[3][k] = 0.0f;
            if (MODE != MODE_GW)
                plane_xy<D, JZ, JY, JX>(cb, cz + 3, qyl, qxl, wx, wy, cxy[3]);
        }
        if (!active)
            continue;
        if constexpr (MODE == MODE_GW) {
            static_assert(C::VC >= 1, "the GW layer loads all DELTA slices at once");
#pragma unroll
            for (int pz = 0; pz < DELTA; ++pz) {
                if (zl0 + pz >= g.Z)
                    break;
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    const float vch = gv[pz] * gr[pz][i];
                    if (D == 3) {
#pragma unroll
                        for (int a = 0; a < 4; ++a)
                            qz[a][i] = fmaf(kW.w[pz][a], vch, qz[a][i]);
                    } else {
                        qz[0][i] += vch;
                    }
                }
            }
        } else {
#pragma unroll
        for (int p0 = 0; p0 < DELTA; p0 += C::VC) {
            // issue every load of VC slices, then use them
            float mcor[C::VC][NCOR], aux[C::VC], fx[C::VC], fy[C::VC], fz[C::VC];
            bool inb[C::VC];
#pragma unroll
            for (int j = 0; j < C::VC; ++j) {
                const int pz = p0 + j;
                if (pz >= DELTA)
                    break;
                const int z = zl0 + pz;
                float uu[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    float v = kW.w[pz][0] * cxy[0][i];
                    v = fmaf(kW.w[pz][1], cxy[1][i], v);
                    v = fmaf(kW.w[pz][2], cxy[2][i], v);
                    v = fmaf(kW.w[pz][3], cxy[3][i], v);
                    uu[i] = (D == 3) ? v : cxy[0][i];
                }
                // cells are clamped into the volume even outside the mask, so
                // every load is in bounds; the values outside are not used
                int cx, cy, cz = 0;
                bool in = axis_cell(x, uu[0], g.X, cx, fx[j]);
                in &= axis_cell(y, uu[1], g.Y, cy, fy[j]);
                if (D == 3)
                    in &= axis_cell(z, uu[2], g.Z, cz, fz[j]);
                inb[j] = in && (z < g.Z);
                if (!(al_index_ok(cx, g.X - 1) & al_index_ok(cy, g.Y - 1) &
                      al_index_ok(cz, D == 3 ? g.Z - 1 : 1)))
                    cx = cy = cz = 0;  // checked builds only: the cell left the volume
                const float *mp = M + ((D == 3 ? cz * g.Y : 0) + cy) * g.X + cx;  // nv < 2^31
                mcor[j][0] = __ldg(mp);
                mcor[j][1] = __ldg(mp + 1);
                mcor[j][2] = __ldg(mp + g.X);
                mcor[j][3] = __ldg(mp + g.X + 1);
                if constexpr (D == 3) {
                    const int sxy = g.X * g.Y;
                    mcor[j][4] = __ldg(mp + sxy);
                    mcor[j][5] = __ldg(mp + sxy + 1);
                    mcor[j][6] = __ldg(mp + sxy + g.X);
                    mcor[j][7] = __ldg(mp + sxy + g.X + 1);
                }
                aux[j] = 0.0f;
                if ((MODE == MODE_MSE || MODE == MODE_NCC) &&
                    al_index_ok((min(z, g.Z - 1) * g.Y + y) * g.X + x, g.nv))
                    aux[j] = __ldg(F + (min(z, g.Z - 1) * g.Y + y) * g.X + x);

            }
#pragma unroll
            for (int j = 0; j < C::VC; ++j) {
                const int pz = p0 + j;
                if (pz >= DELTA)
                    break;
                const int z = zl0 + pz;
                if (z >= g.Z)
                    break;
                Interp ip;
                if constexpr (D == 3)
                    ip = interp8(mcor[j], fx[j], fy[j], fz[j]);
                else
                    ip = interp4(mcor[j], fx[j], fy[j]);
                const int v = (z * g.Y + y) * g.X + x;
                if (MODE == MODE_FWD) {
                    W_out[v] = inb[j] ? ip.v : 0.0f;
                    m_out[v] = inb[j] ? 1 : 0;
                    if (G_io) {
                        G_io[v] = inb[j] ? ip.gx : 0.0f;
                        G_io[g.nv + v] = inb[j] ? ip.gy : 0.0f;
                        if (D == 3)
                            G_io[2 * g.nv + v] = inb[j] ? ip.gz : 0.0f;
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
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int k = 0; k < CHS; ++k)
                                qz[a][k] = fmaf(kW.w[pz][a], vch[k], qz[a][k]);
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
    if (MODE != MODE_FWD) {
        // the last four planes (a single plane in 2D), together
        flush_planes<D, DELTA, MODE, C::NPL, BCX_, BCY_>(D == 3 ? C::BCZ - 1 : 0, qz, colvalid,
                                                         tx, ty, P, Xc,
                                             wt, dstp);
    }
    if (C::NMOM > 0) {
        double mm[C::NMOM > 0 ? C::NMOM : 1];
#pragma unroll
        for (int k = 0; k < (C::NMOM > 0 ? C::NMOM : 1); ++k)
            mm[k] = mom[k];
        block_reduce_d<(C::NMOM > 0 ? C::NMOM : 1)>(mm, red);
        if (tid == 0)
            for (int k = 0; k < C::NMOM; ++k)
                mpart[(int64_t)brick * C::NMOM + k] = mm[k];
    }
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

// Scalars of the objective from the fixed-order sums of the partials:
// writes {J, S, R, n_mask} to value (when not NULL) and the coefficients of
// the projected channels in dS/dc to the shared array k[3]. Every thread of
// the block takes part; k is valid for all threads on return.
struct Parts {
    const double *mpart, *rpart, *lpart;
    int nbricks, ngram, nlcc;
};

template <bool CG = false>
__device__ void objective_scalars(int mode, int64_t nv, double lambda, double eps, const Parts &P,
                                  double *value, double *k, double *red)
{
    double r[1];
    sum_parts<1, CG>(P.rpart, P.ngram, r, red);
    const double R = r[0] / (double)nv;
    double S = 0.0, n = 0.0;
    if (mode == MODE_MSE) {
        double t[2];
        sum_parts<2, CG>(P.mpart, P.nbricks, t, red);
        if (threadIdx.x == 0) {
            n = t[1];
            S = n > 0.0 ? t[0] / n : 0.0;
            k[0] = n > 0.0 ? 2.0 / n : 0.0;
        }
    } else if (mode == MODE_NCC) {
        double t[6];
        sum_parts<6, CG>(P.mpart, P.nbricks, t, red);
        if (threadIdx.x == 0) {
            n = t[0];
            k[0] = k[1] = k[2] = 0.0;
            if (n > 0.0) {
                const double muf = t[1] / n, muw = t[2] / n;
                const double cov = t[5] - n * muf * muw;
                const double vf = t[3] - n * muf * muf;
                const double vw = t[4] - n * muw * muw;
                const double Dd = vf * vw + eps;
                const double sD = sqrt(Dd);
                S = 1.0 - cov / sD;
                const double al = -1.0 / sD, be = cov * vf / (Dd * sD);
                k[0] = al;
                k[1] = be;
                k[2] = -al * muf - be * muw;
            }
        }
    } else {  // LCC
        double t[2];
        sum_parts<2, CG>(P.lpart, P.nlcc, t, red);
        if (threadIdx.x == 0) {
            n = t[1];
            S = n > 0.0 ? 1.0 - t[0] / n : 0.0;
            k[0] = n > 0.0 ? 1.0 / n : 0.0;
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

// Value only (no gradient requested).
__global__ void k_finalize(int mode, int64_t nv, double lambda, double eps, Parts P,
                           double *__restrict__ value)
{
    __shared__ double red[6 * 32];
    __shared__ double k[3];
    objective_scalars(mode, nv, lambda, eps, P, value, k, red);
}

// dJ/dc at control point e: the fixed-order sum of the partials of the (at
// most two per axis) bricks that touch it, the channel combination with the
// scalars k0..k2, plus lambda * dR/dc. CG: the partials were written by other
// blocks of the same launch.
template <int D, int CH, int BCX, int BCY, int BCZ, bool CG>
__device__ __forceinline__ void ctrl_point(const Lattice &L, int gbx, int gby, int gbz,
                                           const float *__restrict__ bpart,
                                           const float *__restrict__ gR, int64_t e, float k0,
                                           float k1, float k2, float lam, float (&out)[D])
{
    constexpr int JX = BCX + 3, JY = BCY + 3, JZ = (D == 3) ? BCZ + 3 : 1;
    constexpr int NPART = CH * JZ * JY * JX;
    const int64_t total = (int64_t)L.nc;
    const int jx = (int)(e % L.nx);
    const int64_t r = e / L.nx;
    const int jy = (int)(r % L.ny), jz = (int)(r / L.ny);
    float p[CH];
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
    for (int i = 0; i < D; ++i) {
        float v;
        if (CH == 3 * D)
            v = fmaf(k0, p[i], fmaf(k1, p[D + i], k2 * p[2 * D + i]));
        else
            v = k0 * p[i];
        const float gr = CG ? __ldcg(gR + (int64_t)i * total + e) : __ldg(gR + (int64_t)i * total + e);
        out[i] = fmaf(lam, gr, v);
    }
}

// Per control point: fixed-order sum of the partials of the bricks that
// touch it, channel combination, plus lambda * dR/dc.
// Every block first evaluates the scalars of the objective (the partial
// sums are few), block 0 writes {J, S, R, n_mask}.
template <int D, int CH, int BCX, int BCY, int BCZ>
__global__ void __launch_bounds__(256)
    k_ctrl(Lattice L, int gbx, int gby, int gbz, int mode, int64_t nv, double lambda, double eps,
           Parts P, const float *__restrict__ bpart, const float *__restrict__ gR,
           float *__restrict__ gc, double *__restrict__ value)
{
    __shared__ double red[6 * 8];
    __shared__ double ks[3];
    objective_scalars(mode, nv, lambda, eps, P, blockIdx.x == 0 ? value : nullptr, ks, red);
    const int64_t total = (int64_t)L.nc;
    const float k0 = (float)ks[0];
    float k1 = 0.f, k2 = 0.f;
    if (CH == 3 * D) {
        k1 = (float)ks[1];
        k2 = (float)ks[2];
    }
    const float lam = (float)lambda;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        float v[D];
        ctrl_point<D, CH, BCX, BCY, BCZ, false>(L, gbx, gby, gbz, bpart, gR, e, k0, k1, k2, lam,
                                                v);
#pragma unroll
        for (int i = 0; i < D; ++i)
            gc[(int64_t)i * total + e] = v[i];
    }
}

// ---------------------------------------------------------------------------
struct Layout {
    size_t scal, rpart, gR, bpart, mpart, Wb, mb, gb, lpart, coef, Gb, total;
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
};

template <int D, int DELTA, int MODE>
__global__ void __launch_bounds__(FCfg<D, DELTA, MODE>::THREADS,
                                  (FCfg<D, DELTA, MODE>::THREADS <= 512 && MODE != MODE_NCC) ? 2
                                                                                            : 1)
    k_fused(Grid g, Lattice L, const float *__restrict__ F, const float *__restrict__ M,
            const float *__restrict__ c, const float *__restrict__ gw_in,
            float *__restrict__ W_out, uint8_t *__restrict__ m_out, float *__restrict__ G_io,
            float *__restrict__ bpart, double *__restrict__ mpart, GramBlocks gb)
{
    const int b = blockIdx.x;
    if (b < gb.nbricks) {
        const int bx = b % gb.gbx, by = (b / gb.gbx) % gb.gby, bz = b / (gb.gbx * gb.gby);
        fused_brick<D, DELTA, MODE>(g, L, F, M, c, gw_in, W_out, m_out, G_io, bpart, mpart, bx,
                                    by, bz, b);
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

template <int D, int DELTA, int MODE>
cudaError_t run_fused_kernel(const Grid &g, const Lattice &L, const Layout &lay, char *ws,
                             const float *F, const float *M, const float *c, const float *gw,
                             float *Wo, uint8_t *mo, float *G, bool with_gram, cudaStream_t s)
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
    const size_t gsm = (size_t)((D == 3) ? kGram3Floats : kGram2Floats) * sizeof(float);
    const size_t dyn = (with_gram && gsm > C::dyn_smem) ? gsm : C::dyn_smem;
    ProfScope ps(s, MODE == MODE_MSE   ? "k_fused_mse"
                    : MODE == MODE_NCC ? "k_fused_ncc"
                    : MODE == MODE_FWD ? "k_fused_fwd"
                                       : "k_fused_gw");
    if (dyn > 0) {  // static + dynamic may pass 48 KB: always opt in
        const size_t most = gsm > C::dyn_smem ? gsm : C::dyn_smem;
        cudaError_t e = cudaFuncSetAttribute(k_fused<D, DELTA, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)most);
        if (e != cudaSuccess)
            return e;
    }
    k_fused<D, DELTA, MODE><<<lay.nbricks + gb.ngram, C::THREADS, dyn, s>>>(
        g, L, F, M, c, gw, Wo, mo, G, (float *)(ws + lay.bpart), (double *)(ws + lay.mpart),
        gb);
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
            e = run_fused_kernel<D, DELTA, MODE_GW>(g, L, lay, ws, F, M, c, gb, nullptr, nullptr,
                                                    Gb, false, s);
        }
    }
    if (e != cudaSuccess)
        return e;
    Parts parts{(const double *)(ws + lay.mpart), rpart, (const double *)(ws + lay.lpart),
                lay.nbricks, lay.ngram, lay.nlcc};
    if (!gc) {
        ProfScope ps(s, "k_finalize");
        k_finalize<<<1, 1024, 0, s>>>(mode, g.nv, lambda, eps, parts, value);
        return cudaGetLastError();
    }
    {
        const int th = 256;
        int64_t nb = ((int64_t)L.nc + th - 1) / th;
        if (nb > 2 * device_sms())
            nb = 2 * device_sms();
        const float *bp = (const float *)(ws + lay.bpart);
        ProfScope ps(s, "k_ctrl");
        constexpr int BCX = brick_bcx(DELTA), BCY = brick_bcy(DELTA), BCZ = brick_bcz(D);
        if (kind == 1)
            k_ctrl<D, 3 * D, BCX, BCY, BCZ><<<(int)nb, th, 0, s>>>(
                L, lay.gbx, lay.gby, lay.gbz, mode, g.nv, lambda, eps, parts, bp, gR, gc, value);
        else
            k_ctrl<D, D, BCX, BCY, BCZ><<<(int)nb, th, 0, s>>>(
                L, lay.gbx, lay.gby, lay.gbz, mode, g.nv, lambda, eps, parts, bp, gR, gc, value);
        e = cudaGetLastError();
    }
    return e;
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
    __shared__ double red[6 * 32];
    __shared__ double ks[3];
    __shared__ float s_inv_bc[2];
    if (threadIdx.x == 0) {
        s_inv_bc[0] = (float)(1.0 / (1.0 - pow(st.beta1, (double)st.t)));
        s_inv_bc[1] = (float)(1.0 / (1.0 - pow(st.beta2, (double)st.t)));
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

}  // namespace airgb
