// A3 similarity kernels: MSE and NCC over the mask (two-phase, fixed-order
// FP64 reductions) and the LCC local-correlation tile kernel shared with
// the fused objective.
#include "launch.h"
#include "profile.h"

namespace airgb {

namespace {

constexpr int kRedThreads = 256;
// At most 8 blocks per SM of a 152-SM GB300: the count sizes the partials'
// workspace, so it is a constant, not the current device's SM count.
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

size_t similarity_ws(const Grid &g, int kind, int window)
{
    const size_t scal = 256;
    if (kind == 2)
        return scal + align256((size_t)lcc_max_blocks(g, window) * 2 * sizeof(double)) +
               lcc_coef_bytes(g);
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
        float *coef = (float *)((char *)part +
                                align256((size_t)lcc_max_blocks(g, window) * 2 * sizeof(double)));
        cudaError_t e = launch_lcc(g, window, eps, F, W, m, false, grad, part, coef, s);
        if (e != cudaSuccess)
            return e;
        k_lcc_finalize<<<1, 1024, 0, s>>>(part, lb, value, scal);
        if (grad)
            k_scale<<<nb, th, 0, s>>>(g.nv, scal, grad);
    }
    return cudaGetLastError();
}

}  // namespace airgb
