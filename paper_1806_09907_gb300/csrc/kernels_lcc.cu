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
// 20 HU noise). The sums are therefore taken relative to a reference value
// (r_F, r_W) that is itself a sample of every window summed relative to it:
// then the sums of squares are at most about n times the window's own spread
// (a window holding its reference cannot be more homogeneous than that), and
// in homogeneous regions they are of the size of the noise. Sums taken
// relative to one reference are converted to another exactly,
//   sum (v - b)   = sum (v - a) + n (a - b)
//   sum (v - b)^2 = sum (v - a)^2 + (a - b) (sum (v - a) + sum (v - b))
// (and the cross term likewise). The statistics are shift invariant, so the
// derivatives with respect to the shifted sums are the derivatives with
// respect to the plain ones, and the shift re-enters the gradient as
//   a'(x) = a(x) - 2 r_W(x) b(x) - r_F(x) c(x),   dS/dW(y) ~ A' + 2 W B + F C.
//
// k_lcc_stats: z-streaming tiles of 32 x 16 output columns. The references
// are shared by runs of outputs, each reference at most R (in z: RZ) from
// every output of its run, hence inside all their windows:
//   z: the output slices of a chunk form groups of 2RZ+1; the z sums of a
//      column are relative to the column's own value at the group's middle
//      slice and slide from one output slice to the next (restarted at each
//      group, so rounding does not build up);
//   x: runs of G neighbouring outputs of a row share the reference of the
//      run's column at offset G/2; the column sums are converted to it;
//   y: runs of G rows share the reference of the run's row at offset G/2.
// It writes (a', b, c) per voxel and per-block {sum rho, count} partials.
// k_lcc_grad: plain box sums of (a', b, c) (three planes; z through a
// register ring of x/y sums) and dS/dW * |X_m| on the mask. When the row
// pitch allows a tensor map (X a multiple of 4), k_lcc_grad_tma stages the
// coefficient slices with TMA tile loads into a ring of shared-memory slots
// instead of register prefetches; both give the same sums in the same order.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <string.h>

#include "launch.h"
#include "profile.h"

namespace airgb {

namespace {

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
// dS/dW * |X_m| = A' + 2 W B + F C on the mask, with (A', B, C) the box sums
// of the coefficient planes (a', b, c). Per staged slice k, between two
// barriers:
// * x runs (threads 0 .. NXT-1): four neighbouring outputs of one row of the
//   slice from 2R + 4 taps (a first sum, then sliding), into Xs[k % 2];
// * every thread, for its output column: the y sum of slice k - 1 from
//   Xs[(k - 1) % 2], then the z sums, sliding through a register ring of the
//   last 2R + 1 x/y sums and recomputed from the ring every 2R + 1 slices so
//   rounding does not build up; an output slice is complete once its last
//   slice has entered.
// After the barrier thread 0 refills the slot.
template <int D, int R>
struct LccT {
    static constexpr int TX = 32, TY = 16;
    static constexpr int RZ = (D == 3) ? R : 0, NR = 2 * RZ + 1, W1 = 2 * R + 1;
    static constexpr int LXT = 40, XOFF = 4 - R, LY = TY + 2 * R;
    static constexpr int ZC = (D == 3) ? 64 : 1;  // most output slices per block
    static constexpr double HALO = 1.0;  // a halo slice takes its x/y box sums too
    static constexpr int GX = 4;                    // outputs per x run
    static constexpr int NXT = LY * (TX / GX);      // x-run threads
    static constexpr int THREADS = TX * TY;         // one output column each
    static constexpr int NS = 4;                    // slices in flight
    static constexpr int PLANE = LY * LXT;          // floats of one staged plane
    static constexpr uint32_t BOX_BYTES = 3u * PLANE * 4u;
    static constexpr int STAGE = (int)((BOX_BYTES + 127) / 128 * 128);
    static constexpr int XS = 3 * LY * TX;          // floats of one x-sum buffer
    static constexpr int oX = NS * STAGE;           // two x-sum buffers
    static constexpr int oBar = oX + 2 * XS * 4;
    static constexpr size_t smem = (size_t)oBar + NS * 8 + 128;  // + base alignment slack
    static_assert(R >= 1 && R <= 4 && XOFF + TX + 2 * R <= LXT, "staged row covers the halo");
    static_assert(GX + 2 * R <= 12, "an x run reads three float4 of a staged row");
    static_assert(NXT <= THREADS, "one x run per thread at most");
};

// Distance in floats between the planes a', b, c of the LCC coefficients.
__host__ __device__ inline int64_t lcc_plane(int nv) { return ((int64_t)nv * 4 + 255) / 256 * 64; }

// ---- bounded waits, TMA helpers ---------------------------------------------
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

// Test of the bounded waits of the LCC kernels: the slice (index within each
// block's z range) whose load is not issued, so the wait for it runs out;
// -1 = none.
__constant__ int c_lcc_drop_slice = -1;

// ---- packed fp32 pairs (the f32x2 arithmetic of sm_100 and later) -----------
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b)  // a - b as one fma: b * -1 + a
{
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Window sums relative to a reference (r_F, r_W), packed by image:
// s1 = (sum f, sum w), s2 = (sum f^2, sum w^2), fw = sum f w, with
// f = F - r_F and w = W - r_W.
struct Mom {
    float2 s1, s2;
    float fw;
};

__device__ __forceinline__ Mom mom_zero()
{
    return Mom{make_float2(0.f, 0.f), make_float2(0.f, 0.f), 0.f};
}

__device__ __forceinline__ void mom_add(Mom &S, const Mom &t)
{
    S.s1 = f2add(S.s1, t.s1);
    S.s2 = f2add(S.s2, t.s2);
    S.fw += t.fw;
}

// S + t - u: the window slides by one input
__device__ __forceinline__ void mom_slide(Mom &S, const Mom &t, const Mom &u)
{
    S.s1 = f2add(S.s1, f2sub(t.s1, u.s1));
    S.s2 = f2add(S.s2, f2sub(t.s2, u.s2));
    S.fw += t.fw - u.fw;
}

// Sums of a partial window of n points relative to a = (a_F, a_W),
// converted to the reference b (exact in real arithmetic):
//   s1' = s1 + n d,  s2' = s2 + d (s1 + s1'),  fw' = fw + d_F s1_W + d_W s1_F'
// with d = a - b.
__device__ __forceinline__ Mom mom_conv(const Mom &t, float2 a, float2 b, float2 n)
{
    const float2 d = f2sub(a, b);
    Mom o;
    o.s1 = f2fma(n, d, t.s1);
    o.s2 = f2fma(d, f2add(t.s1, o.s1), t.s2);
    o.fw = fmaf(d.x, t.s1.y, fmaf(d.y, o.s1.x, t.fw));
    return o;
}

// Tile of k_lcc_stats: TX x TY output columns streamed along z. The input
// region (the tile and its R halo, LX x LY columns) of a slice is staged in
// a ring of NS slots as two planes (F, masked W) of LY rows of LXT floats:
// staged column c holds x = x0 - 4 + c (a TMA row starts on 16 bytes), so
// input column lx sits at c = lx + XOFF. Runs of GX outputs of a row (GY of
// a column) share a reference, at run offset OX (OY). The x-run sums are
// double-buffered: the x runs of slice z and the y runs of slice z - 1 run
// at the same time, on separate warps.
template <int D, int R>
struct LccS {
    static constexpr int TX = 32, TY = 16, THREADS = 512;
    static constexpr int RZ = (D == 3) ? R : 0, NR = 2 * RZ + 1, W1 = 2 * R + 1;
    static constexpr int GX = (R >= 2) ? 4 : 2, OX = GX / 2;
    static constexpr int GY = 2, OY = 1;
    static constexpr int NFX = GX + 2 * R, NFY = GY + 2 * R;  // inputs of a run
    static constexpr int NGX = TX / GX, NGY = TY / GY;
    static constexpr int LX = TX + 2 * R, LY = TY + 2 * R, NL = LX * LY;
    static constexpr int LXT = 40, XOFF = 4 - R;
    static constexpr int P = (D == 3) ? 2 : 0;   // slices loaded ahead of use
    static constexpr int NS = NR + P;            // ring slots
    static constexpr int LXP = LX + 1, XP = TX + 1;  // odd row pitches: conflict-free runs
    static constexpr int KL = (NL + THREADS - 1) / THREADS;  // columns per thread
    static constexpr int NXT = NGX * LY, NYT = TX * NGY;     // x-run and y-run threads
    static constexpr int Y0 = THREADS - NYT;                 // first y-run thread
    static constexpr int ZC = (D == 3) ? 64 : 1;  // most output slices per block
    static constexpr double HALO = 0.1;  // a halo slice is only staged (relative cost)
    static constexpr int BOX = LY * LXT * 4;              // bytes of one plane's TMA box
    static constexpr int PLANE = (BOX + 127) / 128 * 128;  // a tensor copy lands on 128 bytes
    static constexpr int SLOT = 2 * PLANE;
    // shared memory (bytes from a 128-byte aligned base): the ring; z sums of
    // the input columns (Zq = (s1, s2) as float4, Zf = fw); two buffers of
    // x-run sums (Xq, Xf) and of the runs' references (XR); the mbarriers.
    // The columns' references are read from the ring's slot of the z group's
    // middle slice, which stays in the ring for the whole group.
    static constexpr int oRing = 0;
    static constexpr int oZq = oRing + NS * SLOT;
    static constexpr int oZf = oZq + LY * LXP * 16;
    static constexpr int XBUF = (LY * XP * 20 + LY * NGX * 8 + 15) / 16 * 16;
    static constexpr int oX = (oZf + LY * LXP * 4 + 15) / 16 * 16;  // + b * XBUF: Xq, Xf, XR
    static constexpr int oBar = (oX + 2 * XBUF + 7) / 8 * 8;
    static constexpr size_t smem = (size_t)oBar + NS * 8 + 128;  // + base alignment slack
    static_assert(TX % GX == 0 && TY % GY == 0 && (LX % 2) == 0, "tile of runs");
    static_assert(OX <= R && GX - 1 - OX <= R && OY <= R && GY - 1 - OY <= R,
                  "a run's reference lies in all its windows");
    static_assert(R >= 1 && R <= 4 && XOFF + LX <= LXT, "staged row covers the halo");
    static_assert(NXT <= THREADS && NYT <= THREADS && (LY * XP * 20) % 8 == 0,
                  "one run per thread (x runs and y runs on separate threads where they fit)");
    static_assert(PLANE % 128 == 0 && SLOT % 128 == 0 && XBUF % 16 == 0,
                  "TMA destinations on 128 bytes, float4 rows on 16");
};

// Stage slice k (local index; z = its slice) of a block into ring slot s:
// one TMA box per plane, or (unaligned rows) per-thread cp.async with zero
// fill, each thread arriving on the slot's mbarrier when its copies land.
template <int D, int R, bool TMA>
__device__ __forceinline__ void lcc_stage(const CUtensorMap *mapF, const CUtensorMap *mapW,
                                          const Grid &g, const float *__restrict__ F,
                                          const float *__restrict__ Wm, uint32_t sbase, int k,
                                          int s, int x0, int y0, int z)
{
    using C = LccS<D, R>;
    const uint32_t dst = sbase + C::oRing + s * C::SLOT, bar = sbase + C::oBar + 8 * s;
    const bool drop = (k == c_lcc_drop_slice);
    if constexpr (TMA) {
        if (threadIdx.x != 0 || drop)
            return;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((uint32_t)(2 * C::BOX))
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
            "l"(reinterpret_cast<uint64_t>(mapF)), "r"(x0 - 4), "r"(y0 - R), "r"(z), "r"(bar)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst + C::PLANE),
            "l"(reinterpret_cast<uint64_t>(mapW)), "r"(x0 - 4), "r"(y0 - R), "r"(z), "r"(bar)
            : "memory");
    } else {
        if (drop)
            return;
        const bool zin = z >= 0 && z < g.Z;
#pragma unroll
        for (int q = 0; q < C::KL; ++q) {
            const int e = threadIdx.x + q * C::THREADS;
            if (e < C::NL) {
                const int ly = e / C::LX, lx = e - ly * C::LX;
                const int x = x0 - R + lx, y = y0 - R + ly;
                const bool in = zin && x >= 0 && x < g.X && y >= 0 && y < g.Y;
                const int64_t v = in ? ((int64_t)z * g.Y + y) * g.X + x : 0;
                const uint32_t o = (uint32_t)(ly * C::LXT + lx + C::XOFF) * 4u;
                const uint32_t n = in ? 4u : 0u;  // 0: fill with zeros
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst + o),
                             "l"(F + v), "r"(n)
                             : "memory");
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst + C::PLANE + o),
                             "l"(Wm + v), "r"(n)
                             : "memory");
            }
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
    }
}

// Statistics of one output voxel from its window sums S (relative to the
// reference b): adds rho to the thread's partials, returns (a', b, c).
__device__ __forceinline__ float3 lcc_coefs(const Mom &S, float2 b, float inv_n, float eps,
                                            float &rho_sum, float &cnt)
{
    const float2 v2 = f2fma(__fmul2_rn(S.s1, S.s1), make_float2(-inv_n, -inv_n), S.s2);
    const float cov = fmaf(-S.s1.x * S.s1.y, inv_n, S.fw);
    const float vf = fmaxf(v2.x, 0.0f), vw = fmaxf(v2.y, 0.0f);
    const float Dd = fmaf(vf, vw, eps);
    const float rs = rsqrtf(Dd);
    const float rs3 = rs * rs * rs;
    const float cb = 0.5f * cov * vf * rs3;  // -drho/dS_WW
    const float cc = -rs;                    // -drho/dS_FW
    const float a = (S.s1.x * rs - cov * vf * S.s1.y * rs3) * inv_n;  // -drho/dS_W
    rho_sum += cov * rs;
    cnt += 1.0f;
    return make_float3(a - 2.0f * b.y * cb - b.x * cc, cb, cc);
}

// The x runs of one output slice: thread t < NXT takes row ly = t % LY and
// run gx = t / LY (consecutive lanes, consecutive rows), converts the NFX z
// sums of its columns to the reference of the run's column OX (read, like
// the columns' own references, from the ring's slot of the z group's middle
// slice) and writes the GX window sums and the reference to buffer X.
template <int D, int R>
__device__ __forceinline__ void lcc_xruns(int t, const float *ringr, const float4 *Zq,
                                          const float *Zf, unsigned char *X, float2 n1)
{
    using C = LccS<D, R>;
    constexpr int GX = C::GX, W1 = C::W1, LXT = C::LXT, PL = C::PLANE / 4;
    float4 *Xq = reinterpret_cast<float4 *>(X);
    float *Xf = reinterpret_cast<float *>(X + C::LY * C::XP * 16);
    float2 *XR = reinterpret_cast<float2 *>(X + C::LY * C::XP * 20);
    const int ly = t % C::LY, gx = t / C::LY;
    const int rb = ly * C::LXP + GX * gx, sb = ly * LXT + GX * gx + C::XOFF;
    const float2 b = make_float2(ringr[sb + C::OX + R], ringr[PL + sb + C::OX + R]);
    Mom acc = mom_zero(), keep[GX - 1];
#pragma unroll
    for (int k = 0; k < C::NFX; ++k) {
        const float4 t4 = Zq[rb + k];
        const Mom tm{make_float2(t4.x, t4.y), make_float2(t4.z, t4.w), Zf[rb + k]};
        const Mom c = mom_conv(tm, make_float2(ringr[sb + k], ringr[PL + sb + k]), b, n1);
        if (k < GX - 1)
            keep[k] = c;
        if (k < W1)
            mom_add(acc, c);
        else
            mom_slide(acc, c, keep[k - W1]);
        if (k >= W1 - 1) {
            const int o = ly * C::XP + GX * gx + k - (W1 - 1);
            Xq[o] = make_float4(acc.s1.x, acc.s1.y, acc.s2.x, acc.s2.y);
            Xf[o] = acc.fw;
        }
    }
    XR[ly * C::NGX + gx] = b;
}

// The y runs of one output slice: thread t < NYT takes column x = t % TX and
// run hy = t / TX, converts the NFY x-run sums of its rows to the reference
// of the run's row OY and evaluates the statistics of its GY voxels
// (mask bits mk, first voxel index v, the next one v + X).
template <int D, int R>
__device__ __forceinline__ void lcc_yruns(int t, const Grid &g, const unsigned char *X,
                                          unsigned mk, int64_t v, int gxv, int gyv0, float2 n2,
                                          float inv_n, float eps, int64_t pl,
                                          float *__restrict__ coef, float &rho_sum, float &cnt)
{
    using C = LccS<D, R>;
    constexpr int GY = C::GY, W1 = C::W1;
    const float4 *Xq = reinterpret_cast<const float4 *>(X);
    const float *Xf = reinterpret_cast<const float *>(X + C::LY * C::XP * 16);
    const float2 *XR = reinterpret_cast<const float2 *>(X + C::LY * C::XP * 20);
    const int x = t % C::TX, hy = t / C::TX, gx = x / C::GX;
    const float2 b = XR[(GY * hy + C::OY + R) * C::NGX + gx];
    Mom acc = mom_zero(), keep[GY > 1 ? GY - 1 : 1];
#pragma unroll
    for (int k = 0; k < C::NFY; ++k) {
        const int ly = GY * hy + k;
        const float4 t4 = Xq[ly * C::XP + x];
        const Mom tm{make_float2(t4.x, t4.y), make_float2(t4.z, t4.w), Xf[ly * C::XP + x]};
        const Mom c = mom_conv(tm, XR[ly * C::NGX + gx], b, n2);
        if (k < GY - 1)
            keep[k] = c;
        if (k < W1)
            mom_add(acc, c);
        else
            mom_slide(acc, c, keep[k - W1]);
        if (k >= W1 - 1) {
            const int j = k - (W1 - 1);
            if (gxv < g.X && gyv0 + j < g.Y) {
                float3 cf = make_float3(0.f, 0.f, 0.f);
                if ((mk >> j) & 1u)
                    cf = lcc_coefs(acc, b, inv_n, eps, rho_sum, cnt);
                if (coef) {
                    const int64_t vj = v + (int64_t)j * g.X;
                    coef[vj] = cf.x;
                    coef[pl + vj] = cf.y;
                    coef[2 * pl + vj] = cf.z;
                }
            }
        }
    }
}

// Window statistics of a tile of 32 x 16 columns streamed along z in chunks
// of zc output slices (W masked: zero off the mask). Per output slice z:
//   A: z sums of every input column (all threads; restarted at the first
//      slice of each group of NR, else slid by one slice) -> barrier ->
//   B: x runs of slice z (NXT threads) while the y runs and the statistics
//      of slice z - 1 run on the last NYT threads -> barrier,
// and the y runs of the chunk's last slice after the loop. The ring holds
// slices up to z + RZ + P. A slice that does not arrive within about a
// second records AL_ERR_TIMEOUT and ends the block (after the copies in
// flight have landed).
template <int D, int R, bool TMA>
__global__ void __launch_bounds__(LccS<D, R>::THREADS, 2)
    k_lcc_stats(const __grid_constant__ CUtensorMap mapF, const __grid_constant__ CUtensorMap mapW,
                Grid g, int zc, float eps, const float *__restrict__ F,
                const float *__restrict__ Wm, const uint8_t *__restrict__ m,
                float *__restrict__ coef, double *__restrict__ part)
{
    using C = LccS<D, R>;
    constexpr int NS = C::NS, NR = C::NR, RZ = C::RZ, W1 = C::W1, PL = C::PLANE / 4;
    constexpr int LX = C::LX, LXT = C::LXT, LXP = C::LXP, TX = C::TX;
    extern __shared__ unsigned char lsm_raw[];
    unsigned char *sm = lsm_raw + ((128u - (lsm_u32(lsm_raw) & 127u)) & 127u);
    __shared__ double red[2 * C::THREADS / 32];
    const uint32_t sbase = lsm_u32(sm);
    const float *ring = reinterpret_cast<const float *>(sm + C::oRing);
    float4 *Zq = reinterpret_cast<float4 *>(sm + C::oZq);
    float *Zf = reinterpret_cast<float *>(sm + C::oZf);
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * C::TY;
    const int zc0 = blockIdx.z * zc, zc1 = min(zc0 + zc, g.Z);
    const int zs = zc0 - RZ, nsl = zc1 + RZ - zs;  // input slices zs .. zs + nsl - 1
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NS; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sbase + C::oBar + 8 * k),
                         "r"(TMA ? 1 : C::THREADS)
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    for (int k = 0; k < NS && k < nsl; ++k)
        lcc_stage<D, R, TMA>(&mapF, &mapW, g, F, Wm, sbase, k, k, x0, y0, zs + k);
    // the thread's input columns: staged offset and z-sum offset
    int ro[C::KL], pe[C::KL];
#pragma unroll
    for (int q = 0; q < C::KL; ++q) {
        const int e = tid + q * C::THREADS;
        const int ly = e / LX, lx = e - ly * LX;
        ro[q] = e < C::NL ? ly * LXT + lx + C::XOFF : -1;
        pe[q] = ly * LXP + lx;
    }
    Mom zsum[C::KL];
#pragma unroll
    for (int q = 0; q < C::KL; ++q)
        zsum[q] = mom_zero();
    // y-run threads: their column, first row, voxel index and mask bits of
    // the output slice they do next (loaded one slice ahead)
    const int ty = tid - C::Y0;
    const bool ythr = ty >= 0;
    const int yx = ythr ? ty % TX : 0, gxv = x0 + yx, gyv0 = y0 + C::GY * (ythr ? ty / TX : 0);
    const int64_t sxy = (int64_t)g.X * g.Y;
    int64_t yv = ((int64_t)zc0 * g.Y + gyv0) * g.X + gxv;  // voxel of the y thread's slice
    unsigned ymask = 0;
    auto load_mask = [&](int64_t v) {
        unsigned mk = 0;
#pragma unroll
        for (int j = 0; j < C::GY; ++j)
            if (gxv < g.X && gyv0 + j < g.Y && __ldg(m + v + (int64_t)j * g.X))
                mk |= 1u << j;
        return mk;
    };
    if (ythr)
        ymask = load_mask(yv);
    const float2 n1 = make_float2((float)NR, (float)NR);
    const float2 n2 = make_float2((float)(NR * W1), (float)(NR * W1));
    const float inv_n = 1.0f / (float)(NR * W1 * W1);
    const int64_t pl = lcc_plane(g.nv);
    float rho_sum = 0.0f, cnt = 0.0f;
    int kfail = -1, iss = min(NS, nsl);  // first unconfirmed slice on failure, slices issued
    int snew = 2 * RZ % NS, sold = NS - 1, sref = 0;  // ring slots: slice z + RZ, z - RZ - 1, ref
    int nz = zc1 - zc0;
    for (int i = 0; i < nz; ++i) {
        // ---- A: the window's slices (all of them first, then the new one)
        bool ok = true;
        {
            const int k0 = i == 0 ? 0 : 2 * RZ + i;
            int sk = i == 0 ? 0 : snew;
            for (int k = k0; k <= 2 * RZ + i; ++k, sk = sk + 1 == NS ? 0 : sk + 1) {
                const uint32_t bar = sbase + C::oBar + 8 * sk, par = (uint32_t)(k / NS) & 1u;
                if (!lbar_try_wait(bar, par))
                    ok &= lbar_wait(bar, par);
            }
        }
        const bool restart = i % NR == 0;
        if (restart)
            sref = snew;  // reference slice of the group: its middle slice z + RZ
        const float *Fn = ring + snew * (C::SLOT / 4), *Fo = ring + sold * (C::SLOT / 4);
        const float *Fr = ring + sref * (C::SLOT / 4);
#pragma unroll
        for (int q = 0; q < C::KL; ++q) {
            if (ro[q] < 0)
                continue;
            Mom &S = zsum[q];
            const float2 r = make_float2(Fr[ro[q]], Fr[PL + ro[q]]);
            if (restart) {
                S = mom_zero();
                int st = sold;  // slices z - RZ .. z + RZ follow slice z - RZ - 1
#pragma unroll
                for (int tt = 0; tt < NR; ++tt) {
                    st = st + 1 == NS ? 0 : st + 1;
                    const float *Ft = ring + st * (C::SLOT / 4);
                    const float2 d = f2sub(make_float2(Ft[ro[q]], Ft[PL + ro[q]]), r);
                    S.s1 = f2add(S.s1, d);
                    S.s2 = f2fma(d, d, S.s2);
                    S.fw = fmaf(d.x, d.y, S.fw);
                }
            } else {
                const float2 fn = f2sub(make_float2(Fn[ro[q]], Fn[PL + ro[q]]), r);
                const float2 fo = f2sub(make_float2(Fo[ro[q]], Fo[PL + ro[q]]), r);
                const float2 dd = f2sub(fn, fo), ss = f2add(fn, fo);
                S.s1 = f2add(S.s1, dd);
                S.s2 = f2fma(dd, ss, S.s2);
                S.fw = fmaf(fn.x, fn.y, fmaf(-fo.x, fo.y, S.fw));
            }
            Zq[pe[q]] = make_float4(S.s1.x, S.s1.y, S.s2.x, S.s2.y);
            Zf[pe[q]] = S.fw;
        }
        if (__syncthreads_or(!ok)) {
            kfail = i == 0 ? 0 : 2 * RZ + i;
            break;
        }
        // the slot of slice z - RZ - 1 (local i - 1) is free: refill it
        if (i > 0 && i - 1 + NS < nsl) {
            if (TMA && tid == 0)  // the slot was read through the generic proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            lcc_stage<D, R, TMA>(&mapF, &mapW, g, F, Wm, sbase, i - 1 + NS, sold, x0, y0,
                                 zs + i - 1 + NS);
            iss = i + NS;
        }
        // ---- B: x runs of slice z, y runs of slice z - 1
        unsigned char *Xb = sm + C::oX + (i & 1) * C::XBUF;
        if (tid < C::NXT)
            lcc_xruns<D, R>(tid, Fr, Zq, Zf, Xb, n1);
        if (ythr && i > 0) {
            lcc_yruns<D, R>(ty, g, sm + C::oX + ((i - 1) & 1) * C::XBUF, ymask, yv, gxv, gyv0,
                            n2, inv_n, eps, pl, coef, rho_sum, cnt);
            yv += sxy;
            if (i < nz)
                ymask = load_mask(yv);
        }
        __syncthreads();
        snew = snew + 1 == NS ? 0 : snew + 1;
        sold = sold + 1 == NS ? 0 : sold + 1;
    }
    if (kfail >= 0) {
        // a slice timed out: record it and let the copies in flight land
        // before the block's shared memory goes
        if (TMA) {
            if (tid == 0) {
                atomicExch(&g_unit_error, kErrTimeout);
                for (int k = kfail; k < iss; ++k)
                    lbar_wait(sbase + C::oBar + 8 * (k % NS), (uint32_t)(k / NS) & 1u);
            }
        } else {
            if (tid == 0)
                atomicExch(&g_unit_error, kErrTimeout);
            asm volatile("cp.async.wait_all;" ::: "memory");
        }
        return;
    }
    // ---- the y runs of the chunk's last slice
    if (ythr && nz > 0)
        lcc_yruns<D, R>(ty, g, sm + C::oX + ((nz - 1) & 1) * C::XBUF, ymask, yv, gxv, gyv0, n2,
                        inv_n, eps, pl, coef, rho_sum, cnt);
    float accf[2] = {rho_sum, cnt};
    double acc[2];
    block_reduce_fd<2>(accf, acc, red);
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

// x runs of one staged row (k_lcc_grad_tma): run t covers outputs
// x0 + 4r .. x0 + 4r + 3 of row ly, from staged columns 4r .. 4r + 11.
template <int D, int R>
__device__ __forceinline__ void lcc_grad_xrun(const float *L, float *Xb, int t)
{
    using C = LccT<D, R>;
    constexpr int RUNS = C::TX / C::GX, J0 = 4 - R;
    const int ly = t / RUNS, r = t - ly * RUNS;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const float4 *src =
            reinterpret_cast<const float4 *>(L + f * C::PLANE + ly * C::LXT + 4 * r);
        float v[12];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float4 t4 = src[q];
            v[4 * q] = t4.x;
            v[4 * q + 1] = t4.y;
            v[4 * q + 2] = t4.z;
            v[4 * q + 3] = t4.w;
        }
        float o[4];
        float s = v[J0];
#pragma unroll
        for (int d = 1; d <= 2 * R; ++d)
            s += v[J0 + d];
        o[0] = s;
#pragma unroll
        for (int i = 1; i < 4; ++i) {
            s = (s - v[J0 + i - 1]) + v[J0 + i + 2 * R];
            o[i] = s;
        }
        *reinterpret_cast<float4 *>(Xb + (f * C::LY + ly) * C::TX + 4 * r) =
            make_float4(o[0], o[1], o[2], o[3]);
    }
}

// Per-thread state of the y/z phase: the output column (tx, ty), the ring of
// the last NR x/y sums, the running z sums and the core voxel (mask, F, W)
// of the next output slice.
template <int D, int R>
struct GradYZ {
    float3 ring[LccT<D, R>::NR];
    float3 zs;
    CoreVox core;
};

// Slice step k of k_lcc_grad_tma; P = k % NR at compile time (the block's
// steps run in groups of NR), so the ring stays in registers. Returns false
// when slice k did not arrive in time (every thread returns false at the same
// step).
template <int D, int R, int P>
__device__ __forceinline__ bool lcc_grad_tma_step(const CUtensorMap *map, const Grid &g, int k,
                                                  int zs, int zc1, int x0, int y0, int nslices,
                                                  const float *__restrict__ F,
                                                  const float *__restrict__ W,
                                                  const uint8_t *__restrict__ m,
                                                  float *__restrict__ gout, unsigned char *sm,
                                                  GradYZ<D, R> &st, int &kfail)
{
    using C = LccT<D, R>;
    constexpr int TX = C::TX, LY = C::LY, NR = C::NR;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const uint32_t sbase = lsm_u32(sm);
    float *Xs = reinterpret_cast<float *>(sm + C::oX);
    bool ok = true;
    // x runs of slice k
    if (k < nslices && tid < C::NXT) {
        const int slot = k % C::NS;
        const uint32_t bar = sbase + C::oBar + 8 * slot, par = (uint32_t)(k / C::NS) & 1u;
        ok = lbar_try_wait(bar, par) || lbar_wait(bar, par);
        if (ok)
            lcc_grad_xrun<D, R>(reinterpret_cast<const float *>(sm + slot * C::STAGE),
                                Xs + (k & 1) * C::XS, tid);
    }
    // y sum of slice k - 1 for this thread's output column, its z sums
    if (k >= 1) {
        const int kk = k - 1;
        constexpr int IDX = (P + NR - 1) % NR;  // ring slot of slice kk
        const float *Xb = Xs + (kk & 1) * C::XS + ty * TX + tx;
        float a = 0.f, b = 0.f, c = 0.f;
#pragma unroll
        for (int d = 0; d < 2 * R + 1; ++d) {
            a += Xb[d * TX];
            b += Xb[(LY + d) * TX];
            c += Xb[(2 * LY + d) * TX];
        }
        const float3 old = st.ring[IDX];
        st.ring[IDX] = make_float3(a, b, c);
        if (IDX == NR - 1) {
            // the ring holds slices kk - NR + 1 .. kk: recompute the sums
            float3 s = st.ring[0];
#pragma unroll
            for (int q = 1; q < NR; ++q) {
                s.x += st.ring[q].x;
                s.y += st.ring[q].y;
                s.z += st.ring[q].z;
            }
            st.zs = s;
        } else {
            st.zs = make_float3((st.zs.x - old.x) + a, (st.zs.y - old.y) + b,
                                (st.zs.z - old.z) + c);
        }
        if (kk >= 2 * C::RZ) {  // output slice zs + kk - RZ is complete
            const int zo = zs + kk - C::RZ, x = x0 + tx, y = y0 + ty;
            if (x < g.X && y < g.Y) {
                const int64_t sZ = (int64_t)g.X * g.Y;
                const int64_t vo = (int64_t)zo * sZ + (int64_t)y * g.X + x;
                const CoreVox cv = st.core;
                if (zo + 1 < zc1) {
                    st.core.m = __ldg(m + vo + sZ);
                    st.core.f = __ldg(F + vo + sZ);
                    st.core.w = __ldg(W + vo + sZ);
                }
                gout[vo] = cv.m ? fmaf(2.0f * cv.w, st.zs.y, fmaf(cv.f, st.zs.z, st.zs.x)) : 0.0f;
            }
        }
    }
    // every thread is done with slot k % NS and with x buffer (k - 1) % 2
    if (__syncthreads_or(!ok)) {
        kfail = k;
        return false;
    }
    if (tid == 0 && k + C::NS < nslices) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        lcc_tma_issue<D, R>(map, sbase, k + C::NS, x0, y0, zs + k + C::NS);
    }
    return true;
}

template <int D, int R, int P>
__device__ __forceinline__ bool lcc_grad_tma_steps(const CUtensorMap *map, const Grid &g, int kb,
                                                   int zs, int zc1, int x0, int y0, int nslices,
                                                   const float *__restrict__ F,
                                                   const float *__restrict__ W,
                                                   const uint8_t *__restrict__ m,
                                                   float *__restrict__ gout, unsigned char *sm,
                                                   GradYZ<D, R> &st, int &kfail)
{
    if constexpr (P < LccT<D, R>::NR) {
        if (kb + P <= nslices) {
            if (!lcc_grad_tma_step<D, R, P>(map, g, kb + P, zs, zc1, x0, y0, nslices, F, W, m,
                                            gout, sm, st, kfail))
                return false;
            return lcc_grad_tma_steps<D, R, P + 1>(map, g, kb, zs, zc1, x0, y0, nslices, F, W, m,
                                                   gout, sm, st, kfail);
        }
    }
    return true;
}

// k_lcc_grad with TMA-staged coefficient slices (tile and phases: LccT).
// Every wait is bounded: a slice that does not arrive within about a second
// records AL_ERR_TIMEOUT, and thread 0 waits (bounded again) for the loads
// still in flight before the block returns.
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
    GradYZ<D, R> st;
#pragma unroll
    for (int q = 0; q < C::NR; ++q)
        st.ring[q] = make_float3(0.f, 0.f, 0.f);
    st.zs = make_float3(0.f, 0.f, 0.f);
    st.core = CoreVox{0, 0.f, 0.f};
    {
        const int x = x0 + tid % C::TX, y = y0 + tid / C::TX;
        if (x < g.X && y < g.Y) {  // first output slice is zc0
            const int64_t v = (int64_t)zc0 * ((int64_t)g.X * g.Y) + (int64_t)y * g.X + x;
            st.core.m = __ldg(m + v);
            st.core.f = __ldg(F + v);
            st.core.w = __ldg(W + v);
        }
    }
    int kfail = -1;
    for (int kb = 0; kb <= nslices; kb += C::NR) {
        if (lcc_grad_tma_steps<D, R, 0>(&map, g, kb, zs, zc1, x0, y0, nslices, F, W, m, gout, sm,
                                        st, kfail))
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
// do equal work and run in waves of 2 x sms (two resident blocks per SM), so
// the chunk minimises
//   waves x (chunk + 2 rz x halo),
// halo being the cost of one of the 2 rz halo slices a chunk re-reads
// relative to an output slice; a last wave that is barely filled costs as
// much as a full one. At least 2 slices, at most zc_max. Workspaces are
// sized for the smallest chunk (lcc_max_blocks), so a workspace sized on one
// device serves a device with any SM count.
int lcc_chunk(const Grid &g, int tiles_xy, int zc_max, int rz, double halo, int sms)
{
    if (g.ndim != 3)
        return 1;
    const int64_t slots = 2 * (int64_t)sms;
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
    using A = LccS<D, R>;
    return lcc_chunk(g, ((g.X + A::TX - 1) / A::TX) * ((g.Y + A::TY - 1) / A::TY), A::ZC, A::RZ,
                     A::HALO, device_sms());
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

// Tensor map of a volume as a 3D fp32 tensor (X, Y, Z) with boxes of the
// statistics tile's staged slice (LXT x LY x 1). False when TMA cannot
// address it (row pitch X * 4 B not a multiple of 16 B, or an unaligned
// base); the caller then stages by cp.async.
template <int D, int R>
bool lcc_vol_tmap(CUtensorMap *map, const Grid &g, const float *p)
{
    using C = LccS<D, R>;
    if (g.X % 4 != 0 || ((uintptr_t)p & 15u) != 0)
        return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc)
        return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.X, (cuuint64_t)g.Y, (cuuint64_t)g.Z};
    const cuuint64_t strides[2] = {(cuuint64_t)g.X * 4, (cuuint64_t)g.X * g.Y * 4};
    const cuuint32_t box[3] = {(cuuint32_t)C::LXT, (cuuint32_t)C::LY, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(p), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// Wm = W where the mask is set, else 0.
__global__ void k_mask_w(int64_t nv, const float *__restrict__ W, const uint8_t *__restrict__ m,
                         float *__restrict__ Wm)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x)
        Wm[v] = __ldg(m + v) ? __ldg(W + v) : 0.0f;
}

template <int D, int R, bool TMA>
cudaError_t lcc_stats_launch(const Grid &g, double eps, const CUtensorMap &mF,
                             const CUtensorMap &mW, const float *F, const float *Wm,
                             const uint8_t *m, float *coef, double *part, cudaStream_t s)
{
    using A = LccS<D, R>;
    cudaError_t e = cudaFuncSetAttribute(k_lcc_stats<D, R, TMA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)A::smem);
    if (e != cudaSuccess)
        return e;
    const int zc = lcc_stats_chunk<D, R>(g);
    dim3 grid((g.X + A::TX - 1) / A::TX, (g.Y + A::TY - 1) / A::TY, (g.Z + zc - 1) / zc);
    ProfScope ps(s, "k_lcc_stats");
    k_lcc_stats<D, R, TMA><<<grid, A::THREADS, A::smem, s>>>(mF, mW, g, zc, (float)eps, F, Wm, m,
                                                             coef, part);
    return cudaGetLastError();
}

template <int D, int R>
cudaError_t lcc_grad_run(const Grid &g, const float *F, const float *W, const uint8_t *m,
                         float *gout, float *coef, cudaStream_t s);

template <int D, int R>
cudaError_t lcc_run(const Grid &g, double eps, const float *F, const float *W, const uint8_t *m,
                    bool w_masked, float *gout, double *part, float *coef, cudaStream_t s)
{
    using A = LccS<D, R>;
    using B = LccB<D, R>;
    static_assert(A::smem <= 113 * 1024, "two statistics tiles per SM");
    static_assert(B::smem <= 227 * 1024, "LCC tile too large");
    cudaError_t e;
    const float *Wm = W;
    if (!w_masked) {
        // the statistics read W masked; a scratch copy goes where the
        // gradient (or, value only, the unused coefficients) will be written
        float *scratch = gout ? gout : coef;
        const int th = 256;
        int64_t nb = ((int64_t)g.nv + th - 1) / th;
        if (nb > 8 * (int64_t)device_sms())
            nb = 8 * (int64_t)device_sms();
        ProfScope ps(s, "k_mask_w");
        k_mask_w<<<(int)nb, th, 0, s>>>(g.nv, W, m, scratch);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        Wm = scratch;
    }
    CUtensorMap mF, mW;
    memset(&mF, 0, sizeof(mF));
    memset(&mW, 0, sizeof(mW));
    const bool tma_s = lcc_vol_tmap<D, R>(&mF, g, F) && lcc_vol_tmap<D, R>(&mW, g, Wm);
    e = tma_s ? lcc_stats_launch<D, R, true>(g, eps, mF, mW, F, Wm, m, gout ? coef : nullptr, part, s)
              : lcc_stats_launch<D, R, false>(g, eps, mF, mW, F, Wm, m, gout ? coef : nullptr, part,
                                               s);
    if (e != cudaSuccess || !gout)
        return e;
    return lcc_grad_run<D, R>(g, F, W, m, gout, coef, s);
}

// dS/dW * |X_m| from the coefficient planes (k_lcc_grad_tma, or k_lcc_grad
// when the row pitch cannot be a tensor-map stride).
template <int D, int R>
cudaError_t lcc_grad_run(const Grid &g, const float *F, const float *W, const uint8_t *m,
                         float *gout, float *coef, cudaStream_t s)
{
    using B = LccB<D, R>;
    cudaError_t e;
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
        const int zc = lcc_chunk(g, tiles, B::ZC, B::RZ, B::HALO, device_sms());
        dim3 grid((g.X + B::TX - 1) / B::TX, (g.Y + B::TY - 1) / B::TY, (g.Z + zc - 1) / zc);
        ProfScope ps(s, "k_lcc_grad");
        if (tma)
            k_lcc_grad_tma<D, R><<<grid, T::THREADS, T::smem, s>>>(map, g, zc, F, W, m, gout);
        else
            k_lcc_grad<D, R><<<grid, B::THREADS, B::smem, s>>>(g, zc, F, W, m, coef, gout);
    }
    return cudaGetLastError();
}

// Blocks of k_lcc_stats on the current device (chunk from its SM count), or
// (most = true) the most any device launches: chunks of 2 slices.
template <int D, int R>
int lcc_blocks(const Grid &g, bool most)
{
    using A = LccS<D, R>;
    const int zc = most ? (g.ndim == 3 ? 2 : 1) : lcc_stats_chunk<D, R>(g);
    return ((g.X + A::TX - 1) / A::TX) * ((g.Y + A::TY - 1) / A::TY) * ((g.Z + zc - 1) / zc);
}

int lcc_blocks_any(const Grid &g, int window, bool most)
{
    const int R = window / 2;
    if (g.ndim == 3)
        return R == 1   ? lcc_blocks<3, 1>(g, most)
               : R == 2 ? lcc_blocks<3, 2>(g, most)
                        : lcc_blocks<3, 3>(g, most);
    return R == 1 ? lcc_blocks<2, 1>(g, most)
           : R == 2 ? lcc_blocks<2, 2>(g, most)
                    : lcc_blocks<2, 3>(g, most);
}

}  // namespace

int lcc_num_blocks(const Grid &g, int window) { return lcc_blocks_any(g, window, false); }

int lcc_max_blocks(const Grid &g, int window) { return lcc_blocks_any(g, window, true); }

size_t lcc_coef_bytes(const Grid &g) { return (size_t)3 * lcc_plane(g.nv) * sizeof(float); }

AL_UNIT_ERROR_READER(unit_error_lcc)

cudaError_t lcc_set_drop_slice(int slice)
{
    return cudaMemcpyToSymbol(c_lcc_drop_slice, &slice, sizeof(int));
}

bool encode_tmap_f32(CUtensorMap *map, int rank, const uint64_t *dims, const uint64_t *strides,
                     const uint32_t *box, const void *base)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc || rank < 1 || rank > 5 || ((uintptr_t)base & 15u) != 0)
        return false;
    cuuint64_t d[5], st[4];
    cuuint32_t bx[5], es[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        bx[i] = box[i];
        es[i] = 1;
        if (i + 1 < rank)
            st[i] = strides[i];
    }
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void *>(base), d,
               st, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

int64_t lcc_coef_plane(const Grid &g) { return lcc_plane(g.nv); }

namespace {
template <int D, int R>
cudaError_t lcc_stats_only(const Grid &g, double eps, const float *F, const float *Wm,
                           const uint8_t *m, double *part, float *coef, cudaStream_t s)
{
    CUtensorMap mF, mW;
    memset(&mF, 0, sizeof(mF));
    memset(&mW, 0, sizeof(mW));
    const bool tma = lcc_vol_tmap<D, R>(&mF, g, F) && lcc_vol_tmap<D, R>(&mW, g, Wm);
    return tma ? lcc_stats_launch<D, R, true>(g, eps, mF, mW, F, Wm, m, coef, part, s)
               : lcc_stats_launch<D, R, false>(g, eps, mF, mW, F, Wm, m, coef, part, s);
}
}  // namespace

cudaError_t launch_lcc_stats(const Grid &g, int window, double eps, const float *F,
                             const float *Wm, const uint8_t *m, double *part, float *coef,
                             cudaStream_t s)
{
    const int R = window / 2;
    if (g.ndim == 3) {
        if (R == 1) return lcc_stats_only<3, 1>(g, eps, F, Wm, m, part, coef, s);
        if (R == 2) return lcc_stats_only<3, 2>(g, eps, F, Wm, m, part, coef, s);
        return lcc_stats_only<3, 3>(g, eps, F, Wm, m, part, coef, s);
    }
    if (R == 1) return lcc_stats_only<2, 1>(g, eps, F, Wm, m, part, coef, s);
    if (R == 2) return lcc_stats_only<2, 2>(g, eps, F, Wm, m, part, coef, s);
    return lcc_stats_only<2, 3>(g, eps, F, Wm, m, part, coef, s);
}

cudaError_t launch_lcc_grad(const Grid &g, int window, const float *F, const float *W,
                            const uint8_t *m, const float *coef, float *gout, cudaStream_t s)
{
    const int R = window / 2;
    float *cf = const_cast<float *>(coef);
    if (g.ndim == 3) {
        if (R == 1) return lcc_grad_run<3, 1>(g, F, W, m, gout, cf, s);
        if (R == 2) return lcc_grad_run<3, 2>(g, F, W, m, gout, cf, s);
        return lcc_grad_run<3, 3>(g, F, W, m, gout, cf, s);
    }
    if (R == 1) return lcc_grad_run<2, 1>(g, F, W, m, gout, cf, s);
    if (R == 2) return lcc_grad_run<2, 2>(g, F, W, m, gout, cf, s);
    return lcc_grad_run<2, 3>(g, F, W, m, gout, cf, s);
}

cudaError_t launch_lcc(const Grid &g, int window, double eps, const float *F, const float *W,
                       const uint8_t *m, bool w_masked, float *gout, double *part, float *coef,
                       cudaStream_t s)
{
    const int R = window / 2;
    if (g.ndim == 3) {
        if (R == 1) return lcc_run<3, 1>(g, eps, F, W, m, w_masked, gout, part, coef, s);
        if (R == 2) return lcc_run<3, 2>(g, eps, F, W, m, w_masked, gout, part, coef, s);
        return lcc_run<3, 3>(g, eps, F, W, m, w_masked, gout, part, coef, s);
    }
    if (R == 1) return lcc_run<2, 1>(g, eps, F, W, m, w_masked, gout, part, coef, s);
    if (R == 2) return lcc_run<2, 2>(g, eps, F, W, m, w_masked, gout, part, coef, s);
    return lcc_run<2, 3>(g, eps, F, W, m, w_masked, gout, part, coef, s);
}

}  // namespace airgb
