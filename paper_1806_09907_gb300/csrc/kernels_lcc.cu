// LCC (local NCC, Sec. III-B) statistics and exact gradient.
//
// S = 1 - (1/|X_m|) sum_{x in mask} rho(x), rho the correlation of F and W
// in the (2R+1)^D box around x (zero padding, fixed count n). With
// a, b, c = -drho/dS_W, -drho/dS_WW, -drho/dS_FW (zero off the mask),
//   dS/dW(y) * |X_m| = sum_{x: y in box(x)} [a + 2 W(y) b + F(y) c](x)
// on the mask (the box is symmetric, so the sum runs over box(y)).
//
// Numerics. fp32 local sums S_FF - S_F^2/n cancel catastrophically when the
// intensities are large compared with their local spread (CT: -1000 HU with
// 20 HU noise). Every partial sum here is therefore taken relative to the
// value at the centre of its own window, and merging windows converts the
// partial sums to the new centre exactly:
//   sum (v - b)   = sum (v - a) + n (a - b)
//   sum (v - b)^2 = sum (v - a)^2 + 2 (a - b) sum (v - a) + n (a - b)^2
// (and the cross term likewise), so every quantity stays of the size of the
// local spread. The statistics are shift invariant, so the derivatives with
// respect to the shifted sums are the derivatives with respect to the plain
// ones, and the shift re-enters the gradient as
//   a'(x) = a(x) - 2 W(x) b(x) - F(x) c(x),   dS/dW(y) ~ A' + 2 W B + F C.
//
// k_lcc_stats: z-streaming tiles. Per input slice the tile (with an R halo)
// enters a ring of 2R+1 slices in shared memory; the z sums of every column
// are taken directly from the ring (relative to the column's centre value),
// then merged along x and along y with the conversion above. It writes
// (a', b, c) per voxel and per-block {sum rho, count} partials.
// k_lcc_grad: plain box sums of (a', b, c) (three planes; z through a
// register ring of x/y sums) and dS/dW * |X_m| on the mask. When the row
// pitch allows a tensor map (X a multiple of 4), k_lcc_grad_tma stages the
// coefficient slices with TMA tile loads into a ring of shared-memory slots
// instead of register prefetches; both give the same sums in the same order.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "launch.h"
#include "profile.h"

namespace airgb {

namespace {

template <int D, int R>
struct LccA {
    static constexpr int TX = 32, TY = 16;
    static constexpr int RZ = (D == 3) ? R : 0, NR = 2 * RZ + 1, W1 = 2 * R + 1;
    static constexpr int LX = TX + 2 * R, LY = TY + 2 * R;
    static constexpr int NL = LX * LY, NX = LY * TX, NC = TX * TY;
    static constexpr int ZC = (D == 3) ? 64 : 1;  // most output slices per block
    static constexpr double HALO = 0.1;  // a halo slice is only staged (relative cost)
    static constexpr int THREADS = 512;
    static constexpr int KL = (NL + THREADS - 1) / THREADS;  // load elements per thread
    // shared memory: ring of (F, masked W) pairs, z sums (5 planes + 2 of
    // centre values), x-merged sums, mask ring (bytes, at the end)
    static constexpr int oRFW = 0, oZ = oRFW + 2 * NR * NL, oX = oZ + 7 * NL;
    static constexpr int oM = oX + 5 * NX;  // in floats; mask bytes start here
    static constexpr size_t smem = (size_t)oM * 4 + (size_t)NR * NL;
    static_assert(LX % 2 == 0 && NL % 2 == 0 && NX % 2 == 0 && TX % 2 == 0,
                  "column pairs are read as float2");
};

template <int D, int R>
struct LccB {
    static constexpr int TX = 32, TY = 16;  // one thread per core column
    static constexpr int RZ = (D == 3) ? R : 0, NR = 2 * RZ + 1, W1 = 2 * R + 1;
    static constexpr int LX = TX + 2 * R, LY = TY + 2 * R;
    static constexpr int NL = LX * LY, NX = LY * TX, NC = TX * TY;
    static constexpr int ZC = (D == 3) ? 64 : 1;  // most output slices per block
    static constexpr double HALO = 1.0;  // a halo slice takes its x/y box sums too
    static constexpr int THREADS = NC;
    static constexpr int KL = (NL + THREADS - 1) / THREADS;
    // one buffer: the staged slice as planes a', b, c of NL floats, then the
    // x box sums as three planes of NX floats; two buffers alternate by slice
    static constexpr int BUF = 3 * NL + 3 * NX;
    static constexpr size_t smem = (size_t)2 * BUF * sizeof(float);
    static_assert(LX % 2 == 0 && NL % 2 == 0 && NX % 2 == 0, "rows are read as float2");
    static_assert(NX / 2 <= THREADS, "one x pair per thread");
};

// k_lcc_grad_tma: the tile of LccB with its coefficient slices staged by
// one 4D TMA tile load each (x, y, z, plane). A TMA row must start on a
// 16-byte boundary, so the staged row runs from x0 - 4 to x0 + 35 (40
// floats) and column x0 - R sits at XOFF = 4 - R. Out-of-range elements of
// the box arrive as zeros, as the zero padding of the box sums wants.
template <int D, int R>
struct LccT {
    static constexpr int TX = 32, TY = 16;
    static constexpr int RZ = (D == 3) ? R : 0, NR = 2 * RZ + 1, W1 = 2 * R + 1;
    static constexpr int LXT = 40, XOFF = 4 - R, LY = TY + 2 * R;
    static constexpr int NX = LY * TX, NC = TX * TY;
    static constexpr int ZC = (D == 3) ? 64 : 1;  // most output slices per block
    static constexpr double HALO = 1.0;  // a halo slice takes its x/y box sums too
    static constexpr int THREADS = NC;
    static constexpr int NS = 4;                 // slices in flight
    static constexpr int PLANE = LY * LXT;       // floats of one staged plane
    static constexpr uint32_t BOX_BYTES = 3u * PLANE * 4u;
    static constexpr int STAGE = (int)((BOX_BYTES + 127) / 128 * 128);
    static constexpr int oX = NS * STAGE;        // two buffers of x sums, 3 planes of NX
    static constexpr int oBar = oX + 2 * 3 * NX * 4;
    static constexpr size_t smem = (size_t)oBar + NS * 8 + 128;  // + base alignment slack
    static_assert(R >= 1 && R <= 4 && XOFF + TX + 2 * R <= LXT, "staged row covers the halo");
    static_assert(NX / 2 <= THREADS, "one x pair per thread");
};

// Distance in floats between the planes a', b, c of the LCC coefficients.
__host__ __device__ inline int64_t lcc_plane(int nv) { return ((int64_t)nv * 4 + 255) / 256 * 64; }

// Window sums (of F, W, F^2, W^2, FW) relative to a reference (bf, bw).
struct Sums {
    float s1f, s1w, s2f, s2w, sfw;
};

// The sums of a partial window (relative to its centre (af, aw), n points)
// converted to the reference (bf, bw); returned, not accumulated.
__device__ __forceinline__ Sums shifted(float t1f, float t1w, float t2f, float t2w, float tfw,
                                        float af, float aw, float bf, float bw, float n)
{
    const float d = af - bf, e = aw - bw;
    Sums o;
    o.s1f = fmaf(n, d, t1f);
    o.s1w = fmaf(n, e, t1w);
    o.s2f = fmaf(d, fmaf(n, d, 2.0f * t1f), t2f);
    o.s2w = fmaf(e, fmaf(n, e, 2.0f * t1w), t2w);
    o.sfw = fmaf(d, fmaf(n, e, t1w), fmaf(e, t1f, tfw));
    return o;
}

__device__ __forceinline__ void add_to(Sums &S, const Sums &t)
{
    S.s1f += t.s1f;
    S.s1w += t.s1w;
    S.s2f += t.s2f;
    S.s2w += t.s2w;
    S.sfw += t.sfw;
}

// Registers a k_lcc_stats thread carries from slice to slice.
template <int KL>
struct StatsCarry {
    float pf[KL], pw[KL];  // prefetched slice: F, W
    uint8_t pm[KL];        // and the mask
    float rho_sum, cnt;
};

template <int D, int R>
__device__ __forceinline__ void lcc_stats_prefetch(const Grid &g, int zi, int x0, int y0,
                                                   const float *__restrict__ F,
                                                   const float *__restrict__ W,
                                                   const uint8_t *__restrict__ m,
                                                   StatsCarry<LccA<D, R>::KL> &st)
{
    using C = LccA<D, R>;
    const int tid = threadIdx.x;
    const int64_t sY = g.X, sZ = (int64_t)g.X * g.Y;
    const bool zin = zi >= 0 && zi < g.Z;
#pragma unroll
    for (int k = 0; k < C::KL; ++k) {
        const int e = tid + k * C::THREADS;
        st.pf[k] = 0.0f;
        st.pw[k] = 0.0f;
        st.pm[k] = 0;
        if (e < C::NL) {
            const int ly = e / C::LX, lx = e - ly * C::LX;
            const int x = x0 - R + lx, y = y0 - R + ly;
            if (zin && x >= 0 && x < g.X && y >= 0 && y < g.Y) {
                const int64_t v = (int64_t)zi * sZ + (int64_t)y * sY + x;
                st.pm[k] = __ldg(m + v);
                st.pf[k] = __ldg(F + v);
                st.pw[k] = __ldg(W + v);  // masked when staged (no dependent load)
            }
        }
    }
}

// One input slice zi of k_lcc_stats. P is its ring slot (compile time), so
// every ring address below is a constant offset.
template <int D, int R, int P>
__device__ __forceinline__ void lcc_stats_step(const Grid &g, float eps, int zi, int zc0,
                                               int zi_end, int x0, int y0,
                                               const float *__restrict__ F,
                                               const float *__restrict__ W,
                                               const uint8_t *__restrict__ m,
                                               float *__restrict__ coef, float *sm,
                                               StatsCarry<LccA<D, R>::KL> &st)
{
    using C = LccA<D, R>;
    constexpr int NL = C::NL, NX = C::NX, NC = C::NC, LX = C::LX, TX = C::TX, NR = C::NR;
    constexpr int W1 = C::W1, RZ = C::RZ;
    constexpr int OLDEST = (P + 1) % NR, CS = (P + 1 + RZ) % NR;  // slots
    float2 *rFW = reinterpret_cast<float2 *>(sm + C::oRFW);
    float *Zs = sm + C::oZ, *Xs = sm + C::oX;
    uint8_t *rM = reinterpret_cast<uint8_t *>(sm + C::oM);
    const int tid = threadIdx.x;
    const int64_t sY = g.X, sZ = (int64_t)g.X * g.Y;
    const float n1 = (float)NR, n2 = (float)(NR * W1), n3 = (float)(NR * W1 * W1);
    const float inv_n = 1.0f / n3;
#pragma unroll
    for (int k = 0; k < C::KL; ++k) {
        const int e = tid + k * C::THREADS;
        if (e < NL) {
            rFW[P * NL + e] = make_float2(st.pf[k], st.pm[k] ? st.pw[k] : 0.0f);
            rM[P * NL + e] = st.pm[k];
        }
    }
    if (zi + 1 < zi_end)
        lcc_stats_prefetch<D, R>(g, zi + 1, x0, y0, F, W, m, st);  // in flight meanwhile
    __syncthreads();
    const int zc = zi - RZ;
    if (zc >= zc0) {
        // ---- z sums of every column, relative to the column's centre value
        for (int e = tid; e < NL; e += C::THREADS) {
            const float2 a = rFW[CS * NL + e];
            float s1f = 0.f, s1w = 0.f, s2f = 0.f, s2w = 0.f, sfw = 0.f;
#pragma unroll
            for (int t = 0; t < NR; ++t) {
                const float2 q = rFW[((OLDEST + t) % NR) * NL + e];
                const float f = q.x - a.x, w = q.y - a.y;
                s1f += f;
                s1w += w;
                s2f = fmaf(f, f, s2f);
                s2w = fmaf(w, w, s2w);
                sfw = fmaf(f, w, sfw);
            }
            Zs[0 * NL + e] = s1f;
            Zs[1 * NL + e] = s1w;
            Zs[2 * NL + e] = s2f;
            Zs[3 * NL + e] = s2w;
            Zs[4 * NL + e] = sfw;
            Zs[5 * NL + e] = a.x;
            Zs[6 * NL + e] = a.y;
        }
        __syncthreads();
        // ---- merge along x, two neighbouring outputs per thread sharing
        //      W1 - 1 of their columns: outputs (ly, tx) and (ly, tx + 1).
        //      The W1 + 1 columns (read as float2 pairs from every plane) are
        //      shifted once, to the centre of the first output, and summed
        //      into both windows; the second window is then shifted to its
        //      own centre.
        for (int e = tid; e < NX / 2; e += C::THREADS) {
            const int ly = e / (TX / 2), tx = 2 * (e - ly * (TX / 2));
            const int base = ly * LX + tx;
            const float bf0 = Zs[5 * NL + base + R], bw0 = Zs[6 * NL + base + R];
            const float bf1 = Zs[5 * NL + base + R + 1], bw1 = Zs[6 * NL + base + R + 1];
            Sums S0{0.f, 0.f, 0.f, 0.f, 0.f}, S1{0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int d2 = 0; d2 <= W1; d2 += 2) {
                float2 q[7];
#pragma unroll
                for (int k = 0; k < 7; ++k)
                    q[k] = *reinterpret_cast<const float2 *>(Zs + k * NL + base + d2);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int d = d2 + h;
                    const Sums t = h == 0 ? shifted(q[0].x, q[1].x, q[2].x, q[3].x, q[4].x, q[5].x,
                                                    q[6].x, bf0, bw0, n1)
                                          : shifted(q[0].y, q[1].y, q[2].y, q[3].y, q[4].y, q[5].y,
                                                    q[6].y, bf0, bw0, n1);
                    if (d < W1)
                        add_to(S0, t);
                    if (d > 0)
                        add_to(S1, t);
                }
            }
            S1 = shifted(S1.s1f, S1.s1w, S1.s2f, S1.s2w, S1.sfw, bf0, bw0, bf1, bw1, n2);
            const int o = ly * TX + tx;
            *reinterpret_cast<float2 *>(Xs + 0 * NX + o) = make_float2(S0.s1f, S1.s1f);
            *reinterpret_cast<float2 *>(Xs + 1 * NX + o) = make_float2(S0.s1w, S1.s1w);
            *reinterpret_cast<float2 *>(Xs + 2 * NX + o) = make_float2(S0.s2f, S1.s2f);
            *reinterpret_cast<float2 *>(Xs + 3 * NX + o) = make_float2(S0.s2w, S1.s2w);
            *reinterpret_cast<float2 *>(Xs + 4 * NX + o) = make_float2(S0.sfw, S1.sfw);
        }
        __syncthreads();
        // ---- merge along y (two outputs per thread, rows ty and ty + 1)
        //      and evaluate the statistics of the core voxels
        for (int e = tid; e < NC / 2; e += C::THREADS) {
            const int tp = e / TX, tx = e - tp * TX;
            const int ty0 = 2 * tp;
            float bfv[2], bwv[2];
            bool on[2];
            int64_t vv[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ty = ty0 + h, x = x0 + tx, y = y0 + ty;
                const int zcol = (ty + R) * LX + tx + R;
                on[h] = x < g.X && y < g.Y && rM[CS * NL + zcol];
                vv[h] = (int64_t)zc * sZ + (int64_t)y * sY + x;
                bfv[h] = Zs[5 * NL + zcol];
                bwv[h] = Zs[6 * NL + zcol];
            }
            // rows shifted once to the first output's centre, summed into
            // both windows; the second window shifted to its own centre
            Sums S[2] = {{0.f, 0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f, 0.f}};
#pragma unroll
            for (int d = 0; d <= W1; ++d) {
                const int r = (ty0 + d) * TX + tx;
                const int zrow = (ty0 + d) * LX + tx + R;
                const Sums t = shifted(Xs[r], Xs[NX + r], Xs[2 * NX + r], Xs[3 * NX + r],
                                       Xs[4 * NX + r], Zs[5 * NL + zrow], Zs[6 * NL + zrow],
                                       bfv[0], bwv[0], n2);
                if (d < W1)
                    add_to(S[0], t);
                if (d > 0)
                    add_to(S[1], t);
            }
            S[1] = shifted(S[1].s1f, S[1].s1w, S[1].s2f, S[1].s2w, S[1].sfw, bfv[0], bwv[0],
                           bfv[1], bwv[1], n3);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int x = x0 + tx, y = y0 + ty0 + h;
                if (x >= g.X || y >= g.Y)
                    continue;
                float ca = 0.f, cb = 0.f, cc = 0.f;
                if (on[h]) {
                    const Sums &T = S[h];
                    const float cov = fmaf(-T.s1f * T.s1w, inv_n, T.sfw);
                    const float vf = fmaf(-T.s1f * T.s1f, inv_n, T.s2f);
                    const float vw = fmaf(-T.s1w * T.s1w, inv_n, T.s2w);
                    const float Dd = fmaf(vf, vw, eps);
                    const float rs = rsqrtf(Dd);
                    const float rs3 = rs * rs * rs;
                    const float rho = cov * rs;
                    cb = 0.5f * cov * vf * rs3;  // -drho/dS_WW
                    cc = -rs;                    // -drho/dS_FW
                    const float a = (T.s1f * rs - cov * vf * T.s1w * rs3) * inv_n;  // -drho/dS_W
                    ca = a - 2.0f * bwv[h] * cb - bfv[h] * cc;
                    st.rho_sum += rho;
                    st.cnt += 1.0f;
                }
                if (coef) {
                    const int64_t pl = lcc_plane(g.nv);
                    coef[vv[h]] = ca;
                    coef[pl + vv[h]] = cb;
                    coef[2 * pl + vv[h]] = cc;
                }
            }
        }
    }
    __syncthreads();
}

template <int D, int R, int P>
__device__ __forceinline__ void lcc_stats_steps(const Grid &g, float eps, int zb, int zc0,
                                                int zi_end, int x0, int y0,
                                                const float *__restrict__ F,
                                                const float *__restrict__ W,
                                                const uint8_t *__restrict__ m,
                                                float *__restrict__ coef, float *sm,
                                                StatsCarry<LccA<D, R>::KL> &st)
{
    if constexpr (P < LccA<D, R>::NR) {
        if (zb + P < zi_end) {
            lcc_stats_step<D, R, P>(g, eps, zb + P, zc0, zi_end, x0, y0, F, W, m, coef, sm, st);
            lcc_stats_steps<D, R, P + 1>(g, eps, zb, zc0, zi_end, x0, y0, F, W, m, coef, sm, st);
        }
    }
}

// Window statistics of a tile of 32 x 16 columns streamed along z in chunks
// of zc output slices: the ring holds the last 2R+1 input slices (slice zi in
// slot (zi - first) mod (2R+1)).
template <int D, int R>
__global__ void __launch_bounds__(LccA<D, R>::THREADS, 2)
    k_lcc_stats(Grid g, int zc, float eps, const float *__restrict__ F,
                const float *__restrict__ W, const uint8_t *__restrict__ m,
                float *__restrict__ coef, double *__restrict__ part)
{
    using C = LccA<D, R>;
    extern __shared__ float sm[];
    __shared__ double red[2 * C::THREADS / 32];
    const int x0 = blockIdx.x * C::TX, y0 = blockIdx.y * C::TY;
    const int zc0 = blockIdx.z * zc, zc1 = min(zc0 + zc, g.Z);
    StatsCarry<C::KL> st;
    st.rho_sum = 0.0f;
    st.cnt = 0.0f;
    const int zs = zc0 - C::RZ, zi_end = zc1 + C::RZ;
    lcc_stats_prefetch<D, R>(g, zs, x0, y0, F, W, m, st);
    for (int zb = zs; zb < zi_end; zb += C::NR)
        lcc_stats_steps<D, R, 0>(g, eps, zb, zc0, zi_end, x0, y0, F, W, m, coef, sm, st);
    double acc[2] = {st.rho_sum, st.cnt};
    block_reduce_d<2>(acc, red);
    if (threadIdx.x == 0) {
        const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        part[2 * b] = acc[0];
        part[2 * b + 1] = acc[1];
    }
}

// Mask, F and W of the thread's core voxel in the next output slice.
struct CoreVox {
    uint8_t m;
    float f, w;
};

// One slice step of k_lcc_grad. The thread owns core column (tx, ty); P is
// the ring slot of slice zi (compile time, so the ring stays in registers).
// The shared buffers alternate with the parity of zi, so a step needs two
// barriers: after staging, and after the x sums.
template <int D, int R, int P>
__device__ __forceinline__ void lcc_grad_step(const Grid &g, int zi, int zc0, int x0, int y0,
                                              const float *__restrict__ coef,
                                              const float *__restrict__ F,
                                              const float *__restrict__ W,
                                              const uint8_t *__restrict__ m,
                                              float *__restrict__ gout, float *smem,
                                              float (&pa)[LccB<D, R>::KL],
                                              float (&pb)[LccB<D, R>::KL],
                                              float (&pc)[LccB<D, R>::KL],
                                              float3 (&ring)[LccB<D, R>::NR], CoreVox &core,
                                              int zi_end)
{
    using C = LccB<D, R>;
    constexpr int NL = C::NL, NX = C::NX, LX = C::LX, TX = C::TX, NR = C::NR, W1 = C::W1;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int64_t sY = g.X, sZ = (int64_t)g.X * g.Y, pl = lcc_plane(g.nv);
    float *L = smem + (zi & 1) * C::BUF;
    float *X = L + 3 * NL;
    // stage slice zi (prefetched), then start fetching zi + 1
#pragma unroll
    for (int k = 0; k < C::KL; ++k) {
        const int e = tid + k * C::THREADS;
        if (e < NL) {
            L[e] = pa[k];
            L[NL + e] = pb[k];
            L[2 * NL + e] = pc[k];
        }
    }
    if (zi + 1 < zi_end) {
        const int zn = zi + 1;
        const bool zin = zn >= 0 && zn < g.Z;
#pragma unroll
        for (int k = 0; k < C::KL; ++k) {
            const int e = tid + k * C::THREADS;
            pa[k] = pb[k] = pc[k] = 0.0f;
            if (e < NL) {
                const int ly = e / LX, lx = e - ly * LX;
                const int x = x0 - R + lx, y = y0 - R + ly;
                if (zin && x >= 0 && x < g.X && y >= 0 && y < g.Y) {
                    const int64_t v = (int64_t)zn * sZ + (int64_t)y * sY + x;
                    pa[k] = __ldg(coef + v);
                    pb[k] = __ldg(coef + pl + v);
                    pc[k] = __ldg(coef + 2 * pl + v);
                }
            }
        }
    }
    // the core voxel of the output slice zo = zi - RZ (fetched one step ago);
    // start fetching the core voxel of the next output slice
    const int zo = zi - C::RZ;
    const int x = x0 + tx, y = y0 + ty;
    const bool out = zo >= zc0 && x < g.X && y < g.Y;
    const int64_t vo = (int64_t)zo * sZ + (int64_t)y * sY + x;
    const uint8_t mo = core.m;
    const float fo = core.f, wo = core.w;
    if (zo + 1 >= zc0 && zo + 1 < zi_end - C::RZ && x < g.X && y < g.Y) {
        const int64_t vn = vo + sZ;
        core.m = __ldg(m + vn);
        core.f = __ldg(F + vn);
        core.w = __ldg(W + vn);
    }
    __syncthreads();
    // x box sums of every row of the load region, two neighbouring outputs
    // per thread: W1 + 1 taps read as float2 (consecutive threads, consecutive
    // pairs: no bank conflicts)
    if (tid < NX / 2) {
        const int ly = tid / (TX / 2), p2 = 2 * (tid - ly * (TX / 2));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float2 *src = reinterpret_cast<const float2 *>(L + k * NL + ly * LX + p2);
            float v[W1 + 1];
#pragma unroll
            for (int q = 0; q <= R; ++q) {
                const float2 t = src[q];
                v[2 * q] = t.x;
                v[2 * q + 1] = t.y;
            }
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int d = 0; d < W1; ++d) {
                s0 += v[d];
                s1 += v[d + 1];
            }
            *reinterpret_cast<float2 *>(X + k * NX + ly * TX + p2) = make_float2(s0, s1);
        }
    }
    __syncthreads();
    // y box sum of this column: this slice's entry of the z ring
    {
        float a = 0.f, b = 0.f, c = 0.f;
#pragma unroll
        for (int d = 0; d < W1; ++d) {
            const int r = (ty + d) * TX + tx;
            a += X[r];
            b += X[NX + r];
            c += X[2 * NX + r];
        }
        ring[P] = make_float3(a, b, c);
    }
    if (out) {
        float gv = 0.0f;
        if (mo) {
            float A = 0.f, B = 0.f, Cc = 0.f;
#pragma unroll
            for (int t = 0; t < NR; ++t) {
                A += ring[t].x;
                B += ring[t].y;
                Cc += ring[t].z;
            }
            gv = fmaf(2.0f * wo, B, fmaf(fo, Cc, A));
        }
        gout[vo] = gv;
    }
}

template <int D, int R, int P>
__device__ __forceinline__ void lcc_grad_steps(const Grid &g, int zb, int zc0, int x0, int y0,
                                               const float *__restrict__ coef,
                                               const float *__restrict__ F,
                                               const float *__restrict__ W,
                                               const uint8_t *__restrict__ m,
                                               float *__restrict__ gout, float *smem,
                                               float (&pa)[LccB<D, R>::KL],
                                               float (&pb)[LccB<D, R>::KL],
                                               float (&pc)[LccB<D, R>::KL],
                                               float3 (&ring)[LccB<D, R>::NR], CoreVox &core,
                                               int zi_end)
{
    if constexpr (P < LccB<D, R>::NR) {
        if (zb + P < zi_end) {
            lcc_grad_step<D, R, P>(g, zb + P, zc0, x0, y0, coef, F, W, m, gout, smem, pa, pb, pc,
                                   ring, core, zi_end);
            lcc_grad_steps<D, R, P + 1>(g, zb, zc0, x0, y0, coef, F, W, m, gout, smem, pa, pb, pc,
                                        ring, core, zi_end);
        }
    }
}

// dS/dW * |X_m| = A' + 2 W B + F C on the mask, with (A', B, C) the box sums
// of the coefficients (three planes a', b, c). One thread per core column;
// x and y box sums through shared memory, the z box sum from a register ring
// of the last 2R+1 x/y sums (summed directly, no running sums).
template <int D, int R>
__global__ void __launch_bounds__(LccB<D, R>::THREADS, 2)
    k_lcc_grad(Grid g, int zc, const float *__restrict__ F, const float *__restrict__ W,
               const uint8_t *__restrict__ m, const float *__restrict__ coef,
               float *__restrict__ gout)
{
    using C = LccB<D, R>;
    extern __shared__ float smf[];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * C::TX, y0 = blockIdx.y * C::TY;
    const int zc0 = blockIdx.z * zc, zc1 = min(zc0 + zc, g.Z);
    const int64_t sY = g.X, sZ = (int64_t)g.X * g.Y, pl = lcc_plane(g.nv);
    float pa[C::KL], pb[C::KL], pc[C::KL];
    float3 ring[C::NR];
#pragma unroll
    for (int t = 0; t < C::NR; ++t)
        ring[t] = make_float3(0.f, 0.f, 0.f);
    const int zs = zc0 - C::RZ, zi_end = zc1 + C::RZ;
    {
        const bool zin = zs >= 0 && zs < g.Z;
#pragma unroll
        for (int k = 0; k < C::KL; ++k) {
            const int e = tid + k * C::THREADS;
            pa[k] = pb[k] = pc[k] = 0.0f;
            if (e < C::NL) {
                const int ly = e / C::LX, lx = e - ly * C::LX;
                const int x = x0 - R + lx, y = y0 - R + ly;
                if (zin && x >= 0 && x < g.X && y >= 0 && y < g.Y) {
                    const int64_t v = (int64_t)zs * sZ + (int64_t)y * sY + x;
                    pa[k] = __ldg(coef + v);
                    pb[k] = __ldg(coef + pl + v);
                    pc[k] = __ldg(coef + 2 * pl + v);
                }
            }
        }
    }
    CoreVox core{0, 0.f, 0.f};
    {
        const int x = x0 + tid % C::TX, y = y0 + tid / C::TX;
        if (x < g.X && y < g.Y) {  // first output slice is zc0
            const int64_t v = (int64_t)zc0 * sZ + (int64_t)y * sY + x;
            core.m = __ldg(m + v);
            core.f = __ldg(F + v);
            core.w = __ldg(W + v);
        }
    }
    for (int zb = zs; zb < zi_end; zb += C::NR)
        lcc_grad_steps<D, R, 0>(g, zb, zc0, x0, y0, coef, F, W, m, gout, smf, pa, pb, pc, ring,
                                core, zi_end);
}

// ---- TMA-staged variant ----------------------------------------------------
constexpr int kErrTimeout = 6;  // AL_ERR_TIMEOUT

__device__ __forceinline__ uint32_t lsm_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool lbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `bar` with this parity, for about one second of
// %globaltimer at most; false if it did not complete.
__device__ __noinline__ bool lbar_wait(uint32_t bar, uint32_t parity)
{
    if (lbar_try_wait(bar, parity))
        return true;
    uint64_t t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (!lbar_try_wait(bar, parity)) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 1000000000ull)
            return false;
    }
    return true;
}

// Test of the bounded waits of k_lcc_grad_tma: the slice (index within each
// block's z range) whose load is not issued, so the wait for it runs out;
// -1 = none.
__constant__ int c_lcc_drop_slice = -1;

// Issue the TMA load of slice k of the block's z range into ring slot k % NS.
template <int D, int R>
__device__ __forceinline__ void lcc_tma_issue(const CUtensorMap *map, uint32_t sbase, int k,
                                              int x0, int y0, int z)
{
    using C = LccT<D, R>;
    if (k == c_lcc_drop_slice)
        return;
    const int slot = k % C::NS;
    const uint32_t dst = sbase + slot * C::STAGE, bar = sbase + C::oBar + 8 * slot;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(C::BOX_BYTES)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x0 - 4), "r"(y0 - R), "r"(z), "r"(0),
        "r"(bar)
        : "memory");
}

// One slice step of k_lcc_grad_tma (slice k of the block's range, zi its z).
// Returns false when the slice's TMA load did not arrive in time (then every
// thread of the block returns false at the same step).
template <int D, int R, int P>
__device__ __forceinline__ bool lcc_grad_tma_step(const CUtensorMap *map, const Grid &g, int k,
                                                  int zs, int zc0, int x0, int y0, int nslices,
                                                  const float *__restrict__ F,
                                                  const float *__restrict__ W,
                                                  const uint8_t *__restrict__ m,
                                                  float *__restrict__ gout, unsigned char *sm,
                                                  float3 (&ring)[LccT<D, R>::NR], CoreVox &core,
                                                  int &kfail)
{
    using C = LccT<D, R>;
    constexpr int NX = C::NX, TX = C::TX, NR = C::NR, W1 = C::W1, LXT = C::LXT;
    constexpr int PLANE = C::PLANE, OFF = C::XOFF & 1, NF2 = (OFF + W1 + 2) / 2;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int64_t sY = g.X, sZ = (int64_t)g.X * g.Y;
    const int zi = zs + k, slot = k % C::NS;
    const uint32_t sbase = lsm_u32(sm);
    const bool arrived = lbar_wait(sbase + C::oBar + 8 * slot, (uint32_t)(k / C::NS) & 1u);
    const float *L = reinterpret_cast<const float *>(sm + slot * C::STAGE);
    float *X = reinterpret_cast<float *>(sm + C::oX) + (k & 1) * 3 * NX;
    // the core voxel of the output slice zo = zi - RZ (fetched one step ago);
    // start fetching the core voxel of the next output slice
    const int zo = zi - C::RZ;
    const int x = x0 + tx, y = y0 + ty;
    const bool out = zo >= zc0 && x < g.X && y < g.Y;
    const int64_t vo = (int64_t)zo * sZ + (int64_t)y * sY + x;
    const uint8_t mo = core.m;
    const float fo = core.f, wo = core.w;
    if (zo + 1 >= zc0 && zo + 1 < zs + nslices - C::RZ && x < g.X && y < g.Y) {
        const int64_t vn = vo + sZ;
        core.m = __ldg(m + vn);
        core.f = __ldg(F + vn);
        core.w = __ldg(W + vn);
    }
    // x box sums of every row of the staged slice, two neighbouring outputs
    // per thread, taps read as float2 from the even column at or below the
    // first tap
    if (arrived && tid < NX / 2) {
        const int ly = tid / (TX / 2), p2 = 2 * (tid - ly * (TX / 2));
#pragma unroll
        for (int q3 = 0; q3 < 3; ++q3) {
            const float2 *src =
                reinterpret_cast<const float2 *>(L + q3 * PLANE + ly * LXT + p2 + (C::XOFF - OFF));
            float v[2 * NF2];
#pragma unroll
            for (int q = 0; q < NF2; ++q) {
                const float2 t = src[q];
                v[2 * q] = t.x;
                v[2 * q + 1] = t.y;
            }
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int d = 0; d < W1; ++d) {
                s0 += v[OFF + d];
                s1 += v[OFF + d + 1];
            }
            *reinterpret_cast<float2 *>(X + q3 * NX + ly * TX + p2) = make_float2(s0, s1);
        }
    }
    // every thread has read slot `slot`: it may be refilled with slice k + NS
    if (__syncthreads_or(!arrived)) {
        kfail = k;
        return false;
    }
    if (tid == 0 && k + C::NS < nslices) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        lcc_tma_issue<D, R>(map, sbase, k + C::NS, x0, y0, zi + C::NS);
    }
    // y box sum of this column: this slice's entry of the z ring
    {
        float a = 0.f, b = 0.f, c = 0.f;
#pragma unroll
        for (int d = 0; d < W1; ++d) {
            const int r = (ty + d) * TX + tx;
            a += X[r];
            b += X[NX + r];
            c += X[2 * NX + r];
        }
        ring[P] = make_float3(a, b, c);
    }
    if (out) {
        float gv = 0.0f;
        if (mo) {
            float A = 0.f, B = 0.f, Cc = 0.f;
#pragma unroll
            for (int t = 0; t < NR; ++t) {
                A += ring[t].x;
                B += ring[t].y;
                Cc += ring[t].z;
            }
            gv = fmaf(2.0f * wo, B, fmaf(fo, Cc, A));
        }
        gout[vo] = gv;
    }
    return true;
}

template <int D, int R, int P>
__device__ __forceinline__ bool lcc_grad_tma_steps(const CUtensorMap *map, const Grid &g, int kb,
                                                   int zs, int zc0, int x0, int y0, int nslices,
                                                   const float *__restrict__ F,
                                                   const float *__restrict__ W,
                                                   const uint8_t *__restrict__ m,
                                                   float *__restrict__ gout, unsigned char *sm,
                                                   float3 (&ring)[LccT<D, R>::NR], CoreVox &core,
                                                   int &kfail)
{
    if constexpr (P < LccT<D, R>::NR) {
        if (kb + P < nslices) {
            if (!lcc_grad_tma_step<D, R, P>(map, g, kb + P, zs, zc0, x0, y0, nslices, F, W, m,
                                            gout, sm, ring, core, kfail))
                return false;
            return lcc_grad_tma_steps<D, R, P + 1>(map, g, kb, zs, zc0, x0, y0, nslices, F, W, m,
                                                   gout, sm, ring, core, kfail);
        }
    }
    return true;
}

// k_lcc_grad with TMA-staged coefficient slices: the block's z range (its
// chunk and the 2R halo slices) streams through NS shared-memory slots, each
// filled by one tile load of the three planes; thread 0 refills a slot once
// every thread has passed the barrier after its x sums. Every wait is
// bounded: a slice that does not arrive within about a second records
// AL_ERR_TIMEOUT, and thread 0 waits (bounded again) for the loads still in
// flight before the block returns.
template <int D, int R>
__global__ void __launch_bounds__(LccT<D, R>::THREADS, 2)
    k_lcc_grad_tma(const __grid_constant__ CUtensorMap map, Grid g, int zc,
                   const float *__restrict__ F, const float *__restrict__ W,
                   const uint8_t *__restrict__ m, float *__restrict__ gout)
{
    using C = LccT<D, R>;
    extern __shared__ unsigned char lsm_raw[];
    unsigned char *sm = lsm_raw + ((128u - (lsm_u32(lsm_raw) & 127u)) & 127u);
    const uint32_t sbase = lsm_u32(sm);
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * C::TX, y0 = blockIdx.y * C::TY;
    const int zc0 = blockIdx.z * zc, zc1 = min(zc0 + zc, g.Z);
    const int zs = zc0 - C::RZ, nslices = zc1 + C::RZ - zs;
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < C::NS; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbase + C::oBar + 8 * k)
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < C::NS && k < nslices; ++k)
            lcc_tma_issue<D, R>(&map, sbase, k, x0, y0, zs + k);
    float3 ring[C::NR];
#pragma unroll
    for (int t = 0; t < C::NR; ++t)
        ring[t] = make_float3(0.f, 0.f, 0.f);
    CoreVox core{0, 0.f, 0.f};
    {
        const int x = x0 + tid % C::TX, y = y0 + tid / C::TX;
        if (x < g.X && y < g.Y) {  // first output slice is zc0
            const int64_t v = (int64_t)zc0 * ((int64_t)g.X * g.Y) + (int64_t)y * g.X + x;
            core.m = __ldg(m + v);
            core.f = __ldg(F + v);
            core.w = __ldg(W + v);
        }
    }
    int kfail = -1;
    for (int kb = 0; kb < nslices; kb += C::NR) {
        if (lcc_grad_tma_steps<D, R, 0>(&map, g, kb, zs, zc0, x0, y0, nslices, F, W, m, gout, sm,
                                        ring, core, kfail))
            continue;
        // slice kfail timed out: record it, then let the loads issued for
        // slices kfail .. kfail + NS - 1 land before the block's memory goes
        if (tid == 0) {
            atomicExch(&g_unit_error, kErrTimeout);
            for (int k = kfail; k < kfail + C::NS && k < nslices; ++k)
                lbar_wait(sbase + C::oBar + 8 * (k % C::NS), (uint32_t)(k / C::NS) & 1u);
        }
        return;
    }
}

// z chunk (output slices per block) of an LCC kernel. The blocks of a launch
// do equal work and run in waves of 2 x 152 (two resident blocks per SM of
// a 152-SM GB300), so the chunk minimises
//   waves x (chunk + 2 rz x halo),
// halo being the cost of one of the 2 rz halo slices a chunk re-reads
// relative to an output slice; a last wave that is barely filled costs as
// much as a full one. At least 2 slices, at most zc_max. Depends on the grid
// only, so workspace sizes and launches agree.
int lcc_chunk(const Grid &g, int tiles_xy, int zc_max, int rz, double halo)
{
    if (g.ndim != 3)
        return 1;
    const int64_t slots = 2 * 152;
    int best = 2;
    double best_cost = 0.0;
    for (int chunks = 1; chunks <= g.Z; ++chunks) {
        const int zc = (g.Z + chunks - 1) / chunks;
        if (zc > zc_max)
            continue;
        if (zc < 2)
            break;
        const int n = (g.Z + zc - 1) / zc;  // chunks launched with this zc
        const int64_t waves = ((int64_t)tiles_xy * n + slots - 1) / slots;
        const double cost = (double)waves * (zc + 2.0 * rz * halo);
        if (best_cost == 0.0 || cost < best_cost - 1e-9) {
            best_cost = cost;
            best = zc;
        }
    }
    return best;
}

template <int D, int R>
int lcc_stats_chunk(const Grid &g)
{
    using A = LccA<D, R>;
    return lcc_chunk(g, ((g.X + A::TX - 1) / A::TX) * ((g.Y + A::TY - 1) / A::TY), A::ZC, A::RZ,
                     A::HALO);
}

// The driver's tensor-map encoder, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Tensor map of the coefficient planes as a 4D fp32 tensor (X, Y, Z, plane)
// with boxes of 40 x (16 + 2R) x 1 x 3. False when TMA cannot address it:
// the row pitch X * 4 B must be a multiple of 16 B and the base 16-B aligned
// (the encoder checks both); the caller then uses the register-staged kernel.
template <int D, int R>
bool lcc_coef_tmap(CUtensorMap *map, const Grid &g, const float *coef)
{
    using C = LccT<D, R>;
    if (g.X % 4 != 0 || ((uintptr_t)coef & 15u) != 0)
        return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc)
        return false;
    const cuuint64_t dims[4] = {(cuuint64_t)g.X, (cuuint64_t)g.Y, (cuuint64_t)g.Z, 3};
    const cuuint64_t strides[3] = {(cuuint64_t)g.X * 4, (cuuint64_t)g.X * g.Y * 4,
                                   (cuuint64_t)lcc_plane(g.nv) * 4};
    const cuuint32_t box[4] = {(cuuint32_t)C::LXT, (cuuint32_t)C::LY, 1, 3};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(coef), dims, strides,
               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <int D, int R>
cudaError_t lcc_run(const Grid &g, double eps, const float *F, const float *W, const uint8_t *m,
                    float *gout, double *part, float *coef, cudaStream_t s)
{
    using A = LccA<D, R>;
    using B = LccB<D, R>;
    static_assert(A::smem <= 227 * 1024 && B::smem <= 227 * 1024, "LCC tile too large");
    cudaError_t e = cudaFuncSetAttribute(k_lcc_stats<D, R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)A::smem);
    if (e != cudaSuccess)
        return e;
    {
        const int zc = lcc_stats_chunk<D, R>(g);
        dim3 grid((g.X + A::TX - 1) / A::TX, (g.Y + A::TY - 1) / A::TY, (g.Z + zc - 1) / zc);
        ProfScope ps(s, "k_lcc_stats");
        k_lcc_stats<D, R><<<grid, A::THREADS, A::smem, s>>>(g, zc, (float)eps, F, W, m,
                                                            gout ? coef : nullptr, part);
    }
    if ((e = cudaGetLastError()) != cudaSuccess || !gout)
        return e;
    using T = LccT<D, R>;
    static_assert(T::smem <= 227 * 1024 && T::TX == B::TX && T::TY == B::TY && T::ZC == B::ZC &&
                      T::HALO == B::HALO,
                  "both gradient kernels tile alike");
    CUtensorMap map;
    const bool tma = lcc_coef_tmap<D, R>(&map, g, coef);
    e = tma ? cudaFuncSetAttribute(k_lcc_grad_tma<D, R>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::smem)
            : cudaFuncSetAttribute(k_lcc_grad<D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)B::smem);
    if (e != cudaSuccess)
        return e;
    {
        const int tiles = ((g.X + B::TX - 1) / B::TX) * ((g.Y + B::TY - 1) / B::TY);
        const int zc = lcc_chunk(g, tiles, B::ZC, B::RZ, B::HALO);
        dim3 grid((g.X + B::TX - 1) / B::TX, (g.Y + B::TY - 1) / B::TY, (g.Z + zc - 1) / zc);
        ProfScope ps(s, "k_lcc_grad");
        if (tma)
            k_lcc_grad_tma<D, R><<<grid, T::THREADS, T::smem, s>>>(map, g, zc, F, W, m, gout);
        else
            k_lcc_grad<D, R><<<grid, B::THREADS, B::smem, s>>>(g, zc, F, W, m, coef, gout);
    }
    return cudaGetLastError();
}

template <int D, int R>
int lcc_blocks(const Grid &g)
{
    using A = LccA<D, R>;
    const int zc = lcc_stats_chunk<D, R>(g);
    return ((g.X + A::TX - 1) / A::TX) * ((g.Y + A::TY - 1) / A::TY) * ((g.Z + zc - 1) / zc);
}

}  // namespace

int lcc_num_blocks(const Grid &g, int window)
{
    const int R = window / 2;
    if (g.ndim == 3)
        return R == 1 ? lcc_blocks<3, 1>(g) : R == 2 ? lcc_blocks<3, 2>(g) : lcc_blocks<3, 3>(g);
    return R == 1 ? lcc_blocks<2, 1>(g) : R == 2 ? lcc_blocks<2, 2>(g) : lcc_blocks<2, 3>(g);
}

size_t lcc_coef_bytes(const Grid &g) { return (size_t)3 * lcc_plane(g.nv) * sizeof(float); }

AL_UNIT_ERROR_READER(unit_error_lcc)

cudaError_t lcc_set_drop_slice(int slice)
{
    return cudaMemcpyToSymbol(c_lcc_drop_slice, &slice, sizeof(int));
}

cudaError_t launch_lcc(const Grid &g, int window, double eps, const float *F, const float *W,
                       const uint8_t *m, float *gout, double *part, float *coef, cudaStream_t s)
{
    const int R = window / 2;
    if (g.ndim == 3) {
        if (R == 1) return lcc_run<3, 1>(g, eps, F, W, m, gout, part, coef, s);
        if (R == 2) return lcc_run<3, 2>(g, eps, F, W, m, gout, part, coef, s);
        return lcc_run<3, 3>(g, eps, F, W, m, gout, part, coef, s);
    }
    if (R == 1) return lcc_run<2, 1>(g, eps, F, W, m, gout, part, coef, s);
    if (R == 2) return lcc_run<2, 2>(g, eps, F, W, m, gout, part, coef, s);
    return lcc_run<2, 3>(g, eps, F, W, m, gout, part, coef, s);
}

}  // namespace airgb
