// The optimisation loop around the objective: Adam on the control points
// (Sec. II-A, Optimization; Sec. III-G), one level of the Gaussian image
// pyramid and the dyadic refinement of the B-spline coefficients between
// levels (multi-resolution strategy of Sec. IV-A).
//
// All three are light: Adam streams 7 floats per coefficient (0.19 M
// coefficients at 256x256x160, spacing 6), the pyramid reads an image once per
// axis pass, the refinement gathers at most 27 coarse coefficients per fine
// one. They are plain elementwise / gather kernels sized to the data; what
// matters is that the whole loop stays on the device (no host round trip per
// iteration) so that a level's iterations can be captured in a CUDA graph.
#include "launch.h"
#include "profile.h"

namespace airgb {

namespace {

constexpr int kOptThreads = 256;

int blocks_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : b);
}

// ---- Adam ------------------------------------------------------------------
// m, v are the moments of the gradient in normalised units (the image spans
// [-1, 1] per axis, Sec. III-C); ctrl and grad stay in voxel units, so with
// h = (N_k - 1)/2 voxels per normalised unit:
//   g~ = h g, m <- b1 m + (1 - b1) g~, v <- b2 v + (1 - b2) g~^2,
//   c <- c - h lr (m / bc1) / (sqrt(v / bc2) + eps),  bc = 1 - b^t.
// t = *step + 1 is read from the device counter; k_adam_tick stores it
// afterwards, so a captured graph replays successive steps.
__global__ void __launch_bounds__(kOptThreads)
    k_adam(AdamArgs a, const int64_t *__restrict__ step, float *__restrict__ ctrl,
           const float *__restrict__ grad, float *__restrict__ m, float *__restrict__ v)
{
    __shared__ float s_inv_bc[2];
    if (threadIdx.x == 0) {
        const long long t = (long long)*step + 1;
        s_inv_bc[0] = adam_inv_bias(a.beta1, t);
        s_inv_bc[1] = adam_inv_bias(a.beta2, t);
    }
    __syncthreads();
    const float inv_bc1 = s_inv_bc[0], inv_bc2 = s_inv_bc[1];
    const float b1 = (float)a.beta1, b2 = (float)a.beta2;
    const float omb1 = (float)(1.0 - a.beta1), omb2 = (float)(1.0 - a.beta2);
    const int64_t n = (int64_t)a.ndim * a.nc;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / a.nc);
        const float h = a.h[i];
        const float gn = grad[e] * h;
        const float mm = fmaf(b1, m[e], omb1 * gn);
        const float vv = fmaf(b2, v[e], omb2 * gn * gn);
        m[e] = mm;
        v[e] = vv;
        const float den = sqrtf(vv * inv_bc2) + a.eps;
        ctrl[e] -= (a.lr * h) * ((mm * inv_bc1) / den);
    }
}

__global__ void k_adam_tick(int64_t *step)
{
    if (threadIdx.x == 0 && blockIdx.x == 0)
        *step += 1;
}

// ---- pyramid ---------------------------------------------------------------
// One separable pass: smooth along `axis` with the taps w[0..2r] (indices
// clamped to the grid) and keep every factor-th point from 0. The input is
// in[Z][Y][X]; the output has the same sizes except along `axis`.
__global__ void __launch_bounds__(kOptThreads)
    k_pyramid_axis(const float *__restrict__ in, float *__restrict__ out, int X, int Y, int Z,
                   int OX, int OY, int OZ, int axis, int factor, GaussTaps t)
{
    const int64_t n = (int64_t)OX * OY * OZ;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ox = (int)(e % OX);
        const int oy = (int)((e / OX) % OY);
        const int oz = (int)(e / ((int64_t)OX * OY));
        // the input line through the output point along `axis`
        int64_t base;
        int centre, len, stride;
        if (axis == 0) {
            base = ((int64_t)oz * Y + oy) * X, centre = ox * factor, len = X, stride = 1;
        } else if (axis == 1) {
            base = (int64_t)oz * Y * X + ox, centre = oy * factor, len = Y, stride = X;
        } else {
            base = (int64_t)oy * X + ox, centre = oz * factor, len = Z, stride = X * Y;
        }
        float s = 0.0f;
        for (int k = -t.r; k <= t.r; ++k) {
            const int p = min(max(centre + k, 0), len - 1);
            s = fmaf(t.w[k + t.r], __ldg(in + base + (int64_t)p * stride), s);
        }
        out[e] = s;
    }
}

// ---- refinement ------------------------------------------------------------
// Fine coefficient i from the coarse lattice by the two-scale relation of the
// cubic B-spline: with q = i - 1, j = floor(q/2) + 1, an even q takes
// (1, 6, 1)/8 of coarse j-1, j, j+1 and an odd q takes (1, 1)/2 of j, j+1,
// per axis; the tensor product is multiplied by 2 (coarse voxel units are
// twice the fine ones). The host checks that every tap lies in the coarse
// lattice.
struct Taps1 {
    int j0, n;
    float w[3];
};

__device__ __forceinline__ Taps1 refine_taps(int i)
{
    const int q = i - 1;          // >= -1
    const int j = (q + 2) / 2;    // floor(q/2) + 1
    Taps1 t;
    if ((q & 1) == 0) {
        t.j0 = j - 1, t.n = 3;
        t.w[0] = 0.125f, t.w[1] = 0.75f, t.w[2] = 0.125f;
    } else {
        t.j0 = j, t.n = 2;
        t.w[0] = 0.5f, t.w[1] = 0.5f, t.w[2] = 0.0f;
    }
    return t;
}

__global__ void __launch_bounds__(kOptThreads)
    k_refine(const float *__restrict__ cc, float *__restrict__ cf, int ndim, int cx, int cy,
             int cz, int fx, int fy, int fz)
{
    const int64_t nff = (int64_t)fx * fy * fz, ncc = (int64_t)cx * cy * cz;
    const int64_t n = ndim * nff;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int comp = (int)(e / nff);
        const int64_t r = e - comp * nff;
        const int ix = (int)(r % fx), iy = (int)((r / fx) % fy), iz = (int)(r / ((int64_t)fx * fy));
        const Taps1 tx = refine_taps(ix), ty = refine_taps(iy);
        Taps1 tz;
        if (ndim == 3) {
            tz = refine_taps(iz);
        } else {
            tz.j0 = 0, tz.n = 1, tz.w[0] = 1.0f, tz.w[1] = tz.w[2] = 0.0f;
        }
        const float *src = cc + comp * ncc;
        float s = 0.0f;
        for (int a = 0; a < tz.n; ++a) {
            const int jz = tz.j0 + a;
            for (int b = 0; b < ty.n; ++b) {
                const int jy = ty.j0 + b;
                float sy = 0.0f;
                for (int k = 0; k < tx.n; ++k) {
                    const int jx = tx.j0 + k;
                    sy = fmaf(tx.w[k], __ldg(src + ((int64_t)jz * cy + jy) * cx + jx), sy);
                }
                s = fmaf(tz.w[a] * ty.w[b], sy, s);
            }
        }
        cf[e] = 2.0f * s;
    }
}

}  // namespace

cudaError_t launch_adam(const AdamArgs &a, int64_t *step, float *ctrl, const float *grad,
                        float *m, float *v, cudaStream_t s)
{
    const int64_t n = (int64_t)a.ndim * a.nc;
    const int blocks = blocks_for(n, kOptThreads);
    {
        ProfScope ps(s, "k_adam");
        k_adam<<<blocks, kOptThreads, 0, s>>>(a, step, ctrl, grad, m, v);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    k_adam_tick<<<1, 32, 0, s>>>(step);
    return cudaGetLastError();
}

size_t pyramid_ws(const Grid &g, int factor)
{
    if (factor == 1)
        return 0;
    const int64_t OX = (g.X - 1) / factor + 1, OY = (g.Y - 1) / factor + 1;
    const size_t a = (size_t)OX * g.Y * g.Z * 4, b = (size_t)OX * OY * g.Z * 4;
    return (a + 255) / 256 * 256 + (b + 255) / 256 * 256;
}

cudaError_t launch_pyramid(const Grid &g, int factor, const GaussTaps &t, const float *image,
                           float *level, void *ws, cudaStream_t s)
{
    if (factor == 1)
        return cudaMemcpyAsync(level, image, (size_t)g.nv * 4, cudaMemcpyDeviceToDevice, s);
    const int OX = (g.X - 1) / factor + 1, OY = (g.Y - 1) / factor + 1;
    const int OZ = g.ndim == 3 ? (g.Z - 1) / factor + 1 : 1;
    const size_t a = ((size_t)OX * g.Y * g.Z * 4 + 255) / 256 * 256;
    float *t1 = (float *)ws;
    float *t2 = (float *)((char *)ws + a);
    ProfScope ps(s, "k_pyramid_axis");
    k_pyramid_axis<<<blocks_for((int64_t)OX * g.Y * g.Z, kOptThreads), kOptThreads, 0, s>>>(
        image, t1, g.X, g.Y, g.Z, OX, g.Y, g.Z, 0, factor, t);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    float *yout = g.ndim == 3 ? t2 : level;
    k_pyramid_axis<<<blocks_for((int64_t)OX * OY * g.Z, kOptThreads), kOptThreads, 0, s>>>(
        t1, yout, OX, g.Y, g.Z, OX, OY, g.Z, 1, factor, t);
    if ((e = cudaGetLastError()) != cudaSuccess || g.ndim == 2)
        return e;
    k_pyramid_axis<<<blocks_for((int64_t)OX * OY * OZ, kOptThreads), kOptThreads, 0, s>>>(
        t2, level, OX, OY, g.Z, OX, OY, OZ, 2, factor, t);
    return cudaGetLastError();
}

cudaError_t launch_refine(int ndim, const int *nc, const int *nf, const float *cc, float *cf,
                          cudaStream_t s)
{
    const int64_t n = (int64_t)ndim * nf[0] * nf[1] * nf[2];
    ProfScope ps(s, "k_refine");
    k_refine<<<blocks_for(n, kOptThreads), kOptThreads, 0, s>>>(cc, cf, ndim, nc[0], nc[1], nc[2],
                                                                 nf[0], nf[1], nf[2]);
    return cudaGetLastError();
}

}  // namespace airgb
