// A3 similarity kernels: MSE and NCC over the mask (two-phase, fixed-order
// FP64 reductions) and the LCC local-correlation tile kernel shared with
// the fused objective.
#include "launch.h"
#include "profile.h"

namespace airgb {

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocksMax = 152 * 8;

int red_blocks(int64_t nv)
{
    int64_t b = (nv + kRedThreads * 4 - 1) / (kRedThreads * 4);
    return (int)(b < 1 ? 1 : (b > kRedBlocksMax ? kRedBlocksMax : b));
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// ---------------------------------------------------------------- MSE ------
__global__ void __launch_bounds__(kRedThreads)
    k_mse_partials(int64_t nv, const float *__restrict__ F, const float *__restrict__ W,
                   const uint8_t *__restrict__ m, double *__restrict__ part)
{
    __shared__ double red[2 * kRedThreads / 32];
    float s = 0.0f, c = 0.0f;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (__ldg(m + v)) {
            const float d = __ldg(W + v) - __ldg(F + v);
            s = fmaf(d, d, s);
            c += 1.0f;
        }
    }
    double acc[2] = {s, c};
    block_reduce_d<2>(acc, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = acc[0];
        part[2 * blockIdx.x + 1] = acc[1];
    }
}

// Sums K partials per block in fixed order; thread 0 then runs `fin`.
template <int K>
__device__ void sum_block_partials(const double *__restrict__ part, int nblocks, double (&tot)[K],
                                   double *red)
{
#pragma unroll
    for (int k = 0; k < K; ++k)
        tot[k] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < K; ++k)
            tot[k] += part[(int64_t)b * K + k];
    block_reduce_d<K>(tot, red);
}

__global__ void k_mse_finalize(const double *__restrict__ part, int nblocks,
                               double *__restrict__ value, double *__restrict__ scal)
{
    __shared__ double red[2 * 32];
    double t[2];
    sum_block_partials<2>(part, nblocks, t, red);
    if (threadIdx.x == 0) {
        const double n = t[1];
        value[0] = n > 0.0 ? t[0] / n : 0.0;
        value[1] = n;
        scal[0] = n > 0.0 ? 2.0 / n : 0.0;
    }
}

__global__ void k_mse_grad(int64_t nv, const float *__restrict__ F, const float *__restrict__ W,
                           const uint8_t *__restrict__ m, const double *__restrict__ scal,
                           float *__restrict__ g)
{
    const float k = (float)scal[0];
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x)
        g[v] = __ldg(m + v) ? k * (__ldg(W + v) - __ldg(F + v)) : 0.0f;
}

// ---------------------------------------------------------------- NCC ------
__global__ void __launch_bounds__(kRedThreads)
    k_ncc_sums(int64_t nv, const float *__restrict__ F, const float *__restrict__ W,
               const uint8_t *__restrict__ m, double *__restrict__ part)
{
    __shared__ double red[3 * kRedThreads / 32];
    float sf = 0.0f, sw = 0.0f, c = 0.0f;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x)
        if (__ldg(m + v)) {
            sf += __ldg(F + v);
            sw += __ldg(W + v);
            c += 1.0f;
        }
    double acc[3] = {sf, sw, c};
    block_reduce_d<3>(acc, red);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k)
            part[3 * blockIdx.x + k] = acc[k];
}

__global__ void k_ncc_means(const double *__restrict__ part, int nblocks, double *__restrict__ scal)
{
    __shared__ double red[3 * 32];
    double t[3];
    sum_block_partials<3>(part, nblocks, t, red);
    if (threadIdx.x == 0) {
        const double n = t[2];
        scal[0] = n > 0.0 ? t[0] / n : 0.0;  // mu_F
        scal[1] = n > 0.0 ? t[1] / n : 0.0;  // mu_W
        scal[2] = n;
    }
}

__global__ void __launch_bounds__(kRedThreads)
    k_ncc_central(int64_t nv, const float *__restrict__ F, const float *__restrict__ W,
                  const uint8_t *__restrict__ m, const double *__restrict__ scal,
                  double *__restrict__ part)
{
    __shared__ double red[3 * kRedThreads / 32];
    const float muf = (float)scal[0], muw = (float)scal[1];
    float cov = 0.0f, vf = 0.0f, vw = 0.0f;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x)
        if (__ldg(m + v)) {
            const float a = __ldg(F + v) - muf, b = __ldg(W + v) - muw;
            cov = fmaf(a, b, cov);
            vf = fmaf(a, a, vf);
            vw = fmaf(b, b, vw);
        }
    double acc[3] = {cov, vf, vw};
    block_reduce_d<3>(acc, red);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k)
            part[3 * blockIdx.x + k] = acc[k];
}

// scal: {muF, muW, n} in; writes {.., .., .., kF, kW} with
// dS/dW = kF*(F - muF) + kW*(W - muW) on the mask.
__global__ void k_ncc_finalize(const double *__restrict__ part, int nblocks, double eps,
                               double *__restrict__ scal, double *__restrict__ value)
{
    __shared__ double red[3 * 32];
    double t[3];
    sum_block_partials<3>(part, nblocks, t, red);
    if (threadIdx.x == 0) {
        const double n = scal[2];
        const double cov = t[0], vf = t[1], vw = t[2];
        const double D = vf * vw + eps;
        if (n > 0.0 && D > 0.0) {
            const double sD = sqrt(D);
            value[0] = 1.0 - cov / sD;
            scal[3] = -1.0 / sD;
            scal[4] = cov * vf / (D * sD);
        } else {
            value[0] = n > 0.0 ? 1.0 : 0.0;
            scal[3] = 0.0;
            scal[4] = 0.0;
        }
        value[1] = n;
    }
}

__global__ void k_ncc_grad(int64_t nv, const float *__restrict__ F, const float *__restrict__ W,
                           const uint8_t *__restrict__ m, const double *__restrict__ scal,
                           float *__restrict__ g)
{
    const float muf = (float)scal[0], muw = (float)scal[1];
    const float kf = (float)scal[3], kw = (float)scal[4];
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x)
        g[v] = __ldg(m + v) ? fmaf(kf, __ldg(F + v) - muf, kw * (__ldg(W + v) - muw)) : 0.0f;
}

// ---------------------------------------------------------------- LCC ------
// Local correlation in a (2R+1)^D box (zero padding, fixed count n), with
// the exact gradient
//   dS/dW(y) = [A(y) + 2 W(y) B(y) + F(y) C(y)] / |X_m|  on the mask,
// A, B, C the box sums of the per-voxel partials of -rho with respect to
// the local sums S_W, S_WW, S_FW (zero off the mask).
//
// Tiling: a CTA owns a TX x TY column of the grid and a chunk of z slices
// and streams through z. Per input slice it loads F and W with a 2R halo
// in x and y, forms the five products, box-sums them in x and y and keeps
// the last 2R+1 slices in a ring; the z box-sum of the ring gives the local
// sums of the middle slice on the core plus an R halo, hence the partials
// there; their x/y box sums enter a second ring whose z sum gives A, B, C
// on the core R slices later. All sums are direct (fixed order).
//
// Every value is shifted by a per-CTA constant s (F at the centre of the
// CTA's region) before it is squared: local covariances are invariant under
// a common shift when padded and masked-off voxels take the value -s (they
// are 0 unshifted), and the shift removes the cancellation of large
// intensities (CT: -1000 HU) in S_FF - S_F^2/n at fp32.
template <int D, int R>
struct LccCfg {
    static constexpr int TX = 32;
    static constexpr int TY = (R <= 3) ? 16 : 8;
    static constexpr int RZ = (D == 3) ? R : 0;
    static constexpr int NR = 2 * RZ + 1;
    static constexpr int LX = TX + 4 * R, LY = TY + 4 * R;
    static constexpr int SX = TX + 2 * R, SY = TY + 2 * R;
    static constexpr int ZC = (D == 3) ? 32 : 1;  // core slices per CTA
    static constexpr int THREADS = 512;
    // shared memory layout (floats)
    static constexpr int oFs = 0, oWs = oFs + LY * LX, oXB = oWs + LY * LX;
    static constexpr int oP = oXB + 5 * LY * SX;
    static constexpr int oQc = oP + NR * 5 * SY * SX;
    static constexpr int oXQ = oQc + 3 * SY * SX;
    static constexpr int oQ2 = oXQ + 3 * SY * TX;
    static constexpr int total = oQ2 + NR * 3 * TY * TX;
    static constexpr size_t smem_bytes = (size_t)total * 4;
};

template <int D, int R>
__global__ void __launch_bounds__(LccCfg<D, R>::THREADS)
    k_lcc_tiles(Grid g, float eps, const float *__restrict__ F, const float *__restrict__ W,
                const uint8_t *__restrict__ m, float *__restrict__ gout,
                double *__restrict__ part)
{
    using C = LccCfg<D, R>;
    extern __shared__ float sm[];
    float *Fs = sm + C::oFs, *Ws = sm + C::oWs, *XB = sm + C::oXB, *P = sm + C::oP;
    float *Qc = sm + C::oQc, *XQ = sm + C::oXQ, *Q2 = sm + C::oQ2;
    __shared__ double red[2 * C::THREADS / 32];

    const int x0 = blockIdx.x * C::TX, y0 = blockIdx.y * C::TY;
    const int zc0 = blockIdx.z * C::ZC, zc1 = min(zc0 + C::ZC, g.Z);
    const int W_ = 2 * R + 1;
    const float n = (D == 3) ? (float)(W_ * W_ * W_) : (float)(W_ * W_);
    const float inv_n = 1.0f / n;
    const int64_t sY = g.X, sZ = (int64_t)g.X * g.Y;
    const float s = __ldg(F + (int64_t)min((zc0 + zc1) / 2, g.Z - 1) * sZ +
                          (int64_t)min(y0 + C::TY / 2, g.Y - 1) * sY + min(x0 + C::TX / 2, g.X - 1));
    float rho_sum = 0.0f, cnt = 0.0f;

    const int zi_begin = zc0 - 2 * C::RZ, zi_end = zc1 + 2 * C::RZ;  // input slices [begin, end)
    for (int zi = zi_begin; zi < zi_end; ++zi) {
        // ---- load shifted F, W of slice zi over the load region
        const bool zin = zi >= 0 && zi < g.Z;
        for (int e = threadIdx.x; e < C::LY * C::LX; e += C::THREADS) {
            const int ly = e / C::LX, lx = e - ly * C::LX;
            const int x = x0 - 2 * R + lx, y = y0 - 2 * R + ly;
            float f = -s, w = -s;
            if (zin && x >= 0 && x < g.X && y >= 0 && y < g.Y) {
                const int64_t v = (int64_t)zi * sZ + (int64_t)y * sY + x;
                f = __ldg(F + v) - s;
                w = (__ldg(m + v) ? __ldg(W + v) : 0.0f) - s;
            }
            Fs[e] = f;
            Ws[e] = w;
        }
        __syncthreads();
        // ---- x box sums of the five products, all load rows, stats columns
        for (int e = threadIdx.x; e < C::LY * C::SX; e += C::THREADS) {
            const int ly = e / C::SX, sx = e - ly * C::SX;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
            for (int d = 0; d < 2 * R + 1; ++d) {
                const float f = Fs[ly * C::LX + sx + d], w = Ws[ly * C::LX + sx + d];
                a0 += f;
                a1 += w;
                a2 = fmaf(f, f, a2);
                a3 = fmaf(w, w, a3);
                a4 = fmaf(f, w, a4);
            }
            XB[(0 * C::LY + ly) * C::SX + sx] = a0;
            XB[(1 * C::LY + ly) * C::SX + sx] = a1;
            XB[(2 * C::LY + ly) * C::SX + sx] = a2;
            XB[(3 * C::LY + ly) * C::SX + sx] = a3;
            XB[(4 * C::LY + ly) * C::SX + sx] = a4;
        }
        __syncthreads();
        // ---- y box sums into the ring slot of slice zi
        const int slot_in = ((zi % C::NR) + C::NR) % C::NR;
        for (int e = threadIdx.x; e < 5 * C::SY * C::SX; e += C::THREADS) {
            const int q = e / (C::SY * C::SX), r = e - q * C::SY * C::SX;
            const int sy = r / C::SX, sx = r - sy * C::SX;
            float a = 0.f;
#pragma unroll
            for (int d = 0; d < 2 * R + 1; ++d)
                a += XB[(q * C::LY + sy + d) * C::SX + sx];
            P[((slot_in * 5 + q) * C::SY + sy) * C::SX + sx] = a;
        }
        __syncthreads();
        // ---- statistics and partials of slice zs = zi - RZ (core + R halo)
        const int zs = zi - C::RZ;
        if (zs >= zc0 - C::RZ) {
            const bool zsin = zs >= 0 && zs < g.Z;
            for (int e = threadIdx.x; e < C::SY * C::SX; e += C::THREADS) {
                const int sy = e / C::SX, sx = e - sy * C::SX;
                const int x = x0 - R + sx, y = y0 - R + sy;
                float ca = 0.f, cb = 0.f, cc = 0.f;
                if (zsin && x >= 0 && x < g.X && y >= 0 && y < g.Y &&
                    __ldg(m + (int64_t)zs * sZ + (int64_t)y * sY + x)) {
                    float S[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int t = 0; t < C::NR; ++t) {
                        const int slot = (((zs - C::RZ + t) % C::NR) + C::NR) % C::NR;
#pragma unroll
                        for (int q = 0; q < 5; ++q)
                            S[q] += P[((slot * 5 + q) * C::SY + sy) * C::SX + sx];
                    }
                    const float SF = S[0], SW = S[1], SFF = S[2], SWW = S[3], SFW = S[4];
                    const float cov = SFW - SF * SW * inv_n;
                    const float vf = SFF - SF * SF * inv_n;
                    const float vw = SWW - SW * SW * inv_n;
                    const float Dd = fmaf(vf, vw, eps);
                    const float rs = rsqrtf(Dd);
                    const float rho = cov * rs;
                    const float rs3 = rs * rs * rs;
                    // coefficients of -rho (S = 1 - mean rho)
                    cb = 0.5f * cov * vf * rs3;                   // -d rho / d S_WW
                    cc = -rs;                                     // -d rho / d S_FW
                    ca = (SF * rs - cov * vf * SW * rs3) * inv_n;  // -d rho / d S_W
                    if (sx >= R && sx < R + C::TX && sy >= R && sy < R + C::TY && zs >= zc0 &&
                        zs < zc1) {
                        rho_sum += rho;
                        cnt += 1.0f;
                    }
                }
                Qc[(0 * C::SY + sy) * C::SX + sx] = ca;
                Qc[(1 * C::SY + sy) * C::SX + sx] = cb;
                Qc[(2 * C::SY + sy) * C::SX + sx] = cc;
            }
            __syncthreads();
            if (gout) {
                // x box of the partials onto the core columns
                for (int e = threadIdx.x; e < 3 * C::SY * C::TX; e += C::THREADS) {
                    const int q = e / (C::SY * C::TX), r = e - q * C::SY * C::TX;
                    const int sy = r / C::TX, tx = r - sy * C::TX;
                    float a = 0.f;
#pragma unroll
                    for (int d = 0; d < 2 * R + 1; ++d)
                        a += Qc[(q * C::SY + sy) * C::SX + tx + d];
                    XQ[(q * C::SY + sy) * C::TX + tx] = a;
                }
                __syncthreads();
                const int slot_s = ((zs % C::NR) + C::NR) % C::NR;
                for (int e = threadIdx.x; e < 3 * C::TY * C::TX; e += C::THREADS) {
                    const int q = e / (C::TY * C::TX), r = e - q * C::TY * C::TX;
                    const int ty = r / C::TX, tx = r - ty * C::TX;
                    float a = 0.f;
#pragma unroll
                    for (int d = 0; d < 2 * R + 1; ++d)
                        a += XQ[(q * C::SY + ty + d) * C::TX + tx];
                    Q2[((slot_s * 3 + q) * C::TY + ty) * C::TX + tx] = a;
                }
                __syncthreads();
                // ---- gradient on the core of slice zo = zs - RZ
                const int zo = zs - C::RZ;
                if (zo >= zc0 && zo < zc1) {
                    for (int e = threadIdx.x; e < C::TY * C::TX; e += C::THREADS) {
                        const int ty = e / C::TX, tx = e - ty * C::TX;
                        const int x = x0 + tx, y = y0 + ty;
                        if (x >= g.X || y >= g.Y)
                            continue;
                        const int64_t v = (int64_t)zo * sZ + (int64_t)y * sY + x;
                        float gv = 0.0f;
                        if (__ldg(m + v)) {
                            float A = 0.f, B = 0.f, Cc = 0.f;
#pragma unroll
                            for (int t = 0; t < C::NR; ++t) {
                                const int slot = (((zo - C::RZ + t) % C::NR) + C::NR) % C::NR;
                                A += Q2[((slot * 3 + 0) * C::TY + ty) * C::TX + tx];
                                B += Q2[((slot * 3 + 1) * C::TY + ty) * C::TX + tx];
                                Cc += Q2[((slot * 3 + 2) * C::TY + ty) * C::TX + tx];
                            }
                            const float wv = __ldg(W + v) - s, fv = __ldg(F + v) - s;
                            gv = fmaf(2.0f * wv, B, fmaf(fv, Cc, A));
                        }
                        gout[v] = gv;
                    }
                }
            }
        }
        __syncthreads();
    }
    double acc[2] = {rho_sum, cnt};
    block_reduce_d<2>(acc, red);
    if (threadIdx.x == 0) {
        const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        part[2 * b] = acc[0];
        part[2 * b + 1] = acc[1];
    }
}

template <int D, int R>
cudaError_t lcc_launch_t(const Grid &g, double eps, const float *F, const float *W,
                         const uint8_t *m, float *gout, double *part, cudaStream_t s)
{
    using C = LccCfg<D, R>;
    static_assert(C::smem_bytes <= 227 * 1024, "LCC tile too large");
    cudaError_t e = cudaFuncSetAttribute(k_lcc_tiles<D, R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::smem_bytes);
    if (e != cudaSuccess)
        return e;
    dim3 grid((g.X + C::TX - 1) / C::TX, (g.Y + C::TY - 1) / C::TY,
              (g.Z + C::ZC - 1) / C::ZC);
    ProfScope ps(s, "k_lcc_tiles");
    k_lcc_tiles<D, R><<<grid, C::THREADS, C::smem_bytes, s>>>(g, (float)eps, F, W, m, gout, part);
    return cudaGetLastError();
}

template <int D, int R>
int lcc_blocks_t(const Grid &g)
{
    using C = LccCfg<D, R>;
    return ((g.X + C::TX - 1) / C::TX) * ((g.Y + C::TY - 1) / C::TY) * ((g.Z + C::ZC - 1) / C::ZC);
}

__global__ void k_lcc_finalize(const double *__restrict__ part, int nblocks,
                               double *__restrict__ value, double *__restrict__ scal)
{
    __shared__ double red[2 * 32];
    double t[2];
    sum_block_partials<2>(part, nblocks, t, red);
    if (threadIdx.x == 0) {
        const double n = t[1];
        value[0] = n > 0.0 ? 1.0 - t[0] / n : 0.0;
        value[1] = n;
        scal[0] = n > 0.0 ? 1.0 / n : 0.0;
    }
}

__global__ void k_scale(int64_t nv, const double *__restrict__ scal, float *__restrict__ g)
{
    const float k = (float)scal[0];
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x)
        g[v] *= k;
}

}  // namespace

int lcc_num_blocks(const Grid &g, int window)
{
    const int R = window / 2;
    if (g.ndim == 3)
        return R == 1 ? lcc_blocks_t<3, 1>(g) : R == 2 ? lcc_blocks_t<3, 2>(g) : lcc_blocks_t<3, 3>(g);
    return R == 1 ? lcc_blocks_t<2, 1>(g) : R == 2 ? lcc_blocks_t<2, 2>(g) : lcc_blocks_t<2, 3>(g);
}

cudaError_t launch_lcc_tiles(const Grid &g, int window, double eps, const float *fixed,
                             const float *warped, const uint8_t *mask, float *grad_unscaled,
                             double *block_partials, cudaStream_t s)
{
    const int R = window / 2;
    if (g.ndim == 3) {
        if (R == 1) return lcc_launch_t<3, 1>(g, eps, fixed, warped, mask, grad_unscaled, block_partials, s);
        if (R == 2) return lcc_launch_t<3, 2>(g, eps, fixed, warped, mask, grad_unscaled, block_partials, s);
        return lcc_launch_t<3, 3>(g, eps, fixed, warped, mask, grad_unscaled, block_partials, s);
    }
    if (R == 1) return lcc_launch_t<2, 1>(g, eps, fixed, warped, mask, grad_unscaled, block_partials, s);
    if (R == 2) return lcc_launch_t<2, 2>(g, eps, fixed, warped, mask, grad_unscaled, block_partials, s);
    return lcc_launch_t<2, 3>(g, eps, fixed, warped, mask, grad_unscaled, block_partials, s);
}

size_t similarity_ws(const Grid &g, int kind, int window)
{
    const size_t scal = 256;
    if (kind == 2)
        return scal + align256((size_t)lcc_num_blocks(g, window) * 2 * sizeof(double));
    return scal + align256((size_t)red_blocks(g.nv) * 3 * sizeof(double));
}

cudaError_t launch_similarity(const Grid &g, int kind, int window, double eps, const float *F,
                              const float *W, const uint8_t *m, double *value, float *grad,
                              void *ws, cudaStream_t s)
{
    double *scal = (double *)ws;
    double *part = (double *)((char *)ws + 256);
    const int nb = red_blocks(g.nv);
    const int th = kRedThreads;
    if (kind == 0) {
        k_mse_partials<<<nb, th, 0, s>>>(g.nv, F, W, m, part);
        k_mse_finalize<<<1, 1024, 0, s>>>(part, nb, value, scal);
        if (grad)
            k_mse_grad<<<nb, th, 0, s>>>(g.nv, F, W, m, scal, grad);
    } else if (kind == 1) {
        k_ncc_sums<<<nb, th, 0, s>>>(g.nv, F, W, m, part);
        k_ncc_means<<<1, 1024, 0, s>>>(part, nb, scal);
        k_ncc_central<<<nb, th, 0, s>>>(g.nv, F, W, m, scal, part);
        k_ncc_finalize<<<1, 1024, 0, s>>>(part, nb, eps, scal, value);
        if (grad)
            k_ncc_grad<<<nb, th, 0, s>>>(g.nv, F, W, m, scal, grad);
    } else {
        const int lb = lcc_num_blocks(g, window);
        cudaError_t e = launch_lcc_tiles(g, window, eps, F, W, m, grad, part, s);
        if (e != cudaSuccess)
            return e;
        k_lcc_finalize<<<1, 1024, 0, s>>>(part, lb, value, scal);
        if (grad)
            k_scale<<<nb, th, 0, s>>>(g.nv, scal, grad);
    }
    return cudaGetLastError();
}

}  // namespace airgb
