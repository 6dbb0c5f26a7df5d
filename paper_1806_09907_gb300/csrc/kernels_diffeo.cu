// Diffeomorphic B-spline transformation (Sec. III-D): f = exp(v) of the
// stationary velocity field v by scaling and squaring,
//   u_0 = v / 2^K,  u_{k+1}(x) = u_k(x) + u~_k(x + u_k(x)),  f = x + u_K,
// and the adjoint of that map. u~_k is the linear interpolant of u_k at the
// sample position clamped to the grid (a field has no mask); along a clamped
// axis the interpolant is constant, so its derivative there is 0.
//
// The adjoint of one squaring is, with p(x) = x + u_k(x),
//   g_k(y) = g_{k+1}(y) + (du~_k/dp at p(y))^T g_{k+1}(y)
//            + sum_x w_y(p(x)) g_{k+1}(x).
// The first two terms are local. The last is the transpose of the
// interpolation, a scatter from every sample to the corners of its cell.
// It is accumulated in 64-bit fixed point with integer atomics: integer
// addition is associative, so the result does not depend on the order in
// which the atomics land (deterministic, unlike float atomics). The scale
// 2^s is chosen per step from the largest |g| (an exact max reduction) so
// that a node can take 2^20 contributions of the largest size without
// overflow; the fixed point then resolves 2^-42 of that size, far below fp32
// rounding of the contributions themselves.
#include "launch.h"
#include "profile.h"

namespace airgb {

namespace {

constexpr int kDiffeoThreads = 256;

int blocks_for(int64_t n)
{
    int64_t b = (n + kDiffeoThreads - 1) / kDiffeoThreads;
    return (int)(b < 1 ? 1 : b);
}

// Cell and offset of the position x + u along an axis of n points, clamped
// into [0, n - 1]; returns whether the position was inside (a non-finite u
// counts as outside, at 0). The integer part of u is split off first, so x +
// u is not rounded in fp32.
__device__ __forceinline__ bool field_axis(int x, float u, int n, int &cell, float &f)
{
    const float fl = floorf(u);
    if (!(fabsf(fl) < 1.0e9f)) {  // non-finite or far outside
        const bool hi = u > 0.0f;   // NaN -> low face
        cell = hi ? n - 2 : 0;
        f = hi ? 1.0f : 0.0f;
        return false;
    }
    const int iy = x + (int)fl;
    const float fr = u - fl;
    if (iy < 0) {
        cell = 0;
        f = 0.0f;
        return false;
    }
    if (iy > n - 1 || (iy == n - 1 && fr > 0.0f)) {
        cell = n - 2;
        f = 1.0f;
        return false;
    }
    cell = min(iy, n - 2);
    f = fr + (float)(iy - cell);
    return true;
}

struct FieldSample {
    int cell[3];
    float f[3];
    bool in[3];
};

// (the field read is u * sc; sc is a power of two, so the product is exact)
template <int D>
__device__ __forceinline__ FieldSample field_sample(const Grid &g, int x, int y, int z,
                                                    const float *__restrict__ u, int64_t v,
                                                    float sc = 1.0f)
{
    FieldSample s;
    s.in[0] = field_axis(x, __ldg(u + v) * sc, g.X, s.cell[0], s.f[0]);
    s.in[1] = field_axis(y, __ldg(u + g.nv + v) * sc, g.Y, s.cell[1], s.f[1]);
    if (D == 3) {
        s.in[2] = field_axis(z, __ldg(u + 2 * (int64_t)g.nv + v) * sc, g.Z, s.cell[2], s.f[2]);
    } else {
        s.cell[2] = 0;
        s.f[2] = 0.0f;
        s.in[2] = false;
    }
    return s;
}

__global__ void __launch_bounds__(kDiffeoThreads)
    k_scale(const float *__restrict__ in, float *__restrict__ out, float s, int64_t n)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = in[e] * s;
}

// One squaring: out = u + u~(x + u), the field read as u * sc (sc = 2^-K on
// the first squaring, which then reads v itself and also writes u_0 = v sc
// to u0 when given; otherwise 1). Scaling by a power of two is exact, so
// this equals scaling v in a pass of its own first.
template <int D, bool SCALED>
__global__ void __launch_bounds__(kDiffeoThreads, 8)
    k_compose(Grid g, const float *__restrict__ u, float *__restrict__ out, float scale,
              float *__restrict__ u0)
{
    const float sc = SCALED ? scale : 1.0f;  // a compile-time 1 on every squaring but the first
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(v % g.X), y = (int)((v / g.X) % g.Y), z = (int)(v / ((int64_t)g.X * g.Y));
        const FieldSample s = field_sample<D>(g, x, y, z, u, v, sc);
        const int64_t base = ((int64_t)s.cell[2] * g.Y + s.cell[1]) * g.X + s.cell[0];
        const int64_t sx = 1, sy = g.X, sz = (int64_t)g.X * g.Y;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const float *p = u + (int64_t)i * g.nv + base;
            float r;
            if (D == 3) {
                const float c00 = (1.0f - s.f[0]) * (__ldg(p) * sc) + s.f[0] * (__ldg(p + sx) * sc);
                const float c10 =
                    (1.0f - s.f[0]) * (__ldg(p + sy) * sc) + s.f[0] * (__ldg(p + sy + sx) * sc);
                const float c01 =
                    (1.0f - s.f[0]) * (__ldg(p + sz) * sc) + s.f[0] * (__ldg(p + sz + sx) * sc);
                const float c11 = (1.0f - s.f[0]) * (__ldg(p + sz + sy) * sc) +
                                  s.f[0] * (__ldg(p + sz + sy + sx) * sc);
                const float c0 = (1.0f - s.f[1]) * c00 + s.f[1] * c10;
                const float c1 = (1.0f - s.f[1]) * c01 + s.f[1] * c11;
                r = (1.0f - s.f[2]) * c0 + s.f[2] * c1;
            } else {
                const float c0 = (1.0f - s.f[0]) * (__ldg(p) * sc) + s.f[0] * (__ldg(p + sx) * sc);
                const float c1 =
                    (1.0f - s.f[0]) * (__ldg(p + sy) * sc) + s.f[0] * (__ldg(p + sy + sx) * sc);
                r = (1.0f - s.f[1]) * c0 + s.f[1] * c1;
            }
            if constexpr (SCALED) {
                const float own = __ldg(u + (int64_t)i * g.nv + v) * sc;
                if (u0)
                    u0[(int64_t)i * g.nv + v] = own;
                out[(int64_t)i * g.nv + v] = own + r;
            } else {
                out[(int64_t)i * g.nv + v] = __ldg(u + (int64_t)i * g.nv + v) + r;
            }
        }
    }
}

// Largest |g| over n floats, as the bits of a non-negative float (ordered
// like unsigned integers), by atomicMax: exact and order-independent.
__global__ void __launch_bounds__(kDiffeoThreads)
    k_absmax(const float *__restrict__ gin, int64_t n, unsigned int *__restrict__ out)
{
    float m = 0.0f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float a = fabsf(gin[e]);
        m = a > m ? a : m;  // a NaN never wins
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, __float_as_uint(m));
}

// 2^s for the fixed-point scatter: |w g| < 2^e, so every contribution stays
// below 2^(s + e) = 2^42 and 2^20 of them below 2^62.
__device__ __forceinline__ float fixed_scale(unsigned int maxbits)
{
    int e = 0;
    frexpf(__uint_as_float(maxbits), &e);
    const int s = min(42 - e, 100);
    return ldexpf(1.0f, s);
}

// Local terms of one squaring's adjoint into h, the scatter into acc.
// Consecutive lanes take consecutive voxels (all lanes run the same number of
// iterations, so the warp shuffles see every lane). The scatter to the +x
// corners of a sample is usually the scatter to the -x corners of the next
// lane's sample (a smooth displacement keeps neighbours in neighbouring
// cells): that lane adds it to its own contribution, as 64-bit integers, and
// one atomic serves both. Integer addition is exact, so the result does not
// change.
template <int D>
__global__ void __launch_bounds__(kDiffeoThreads)
    k_compose_adjoint(Grid g, const float *__restrict__ u, const float *__restrict__ gin,
                      float *__restrict__ h, unsigned long long *__restrict__ acc,
                      const unsigned int *__restrict__ maxbits)
{
    const float S = fixed_scale(*maxbits);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v0 = blockIdx.x * (int64_t)blockDim.x; v0 < g.nv; v0 += stride) {
        const int64_t v = v0 + threadIdx.x;
        const bool valid = v < g.nv;
        const int64_t vv = valid ? v : 0;
        const int x = (int)(vv % g.X), y = (int)((vv / g.X) % g.Y),
                  z = (int)(vv / ((int64_t)g.X * g.Y));
        const FieldSample s = field_sample<D>(g, x, y, z, u, vv);
        const int base = (s.cell[2] * g.Y + s.cell[1]) * g.X + s.cell[0];  // nv < 2^31
        const int sy = g.X, sz = g.X * g.Y;
        float gv[D], loc[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            gv[i] = valid ? __ldg(gin + (int64_t)i * g.nv + vv) : 0.0f;
            loc[i] = gv[i];
        }
        // derivative of the interpolant of each component at the sample
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const float *p = u + (int64_t)i * g.nv + base;
            float d0, d1, d2 = 0.0f;
            if (D == 3) {
                const float a000 = __ldg(p), a001 = __ldg(p + 1), a010 = __ldg(p + sy),
                            a011 = __ldg(p + sy + 1), a100 = __ldg(p + sz),
                            a101 = __ldg(p + sz + 1), a110 = __ldg(p + sz + sy),
                            a111 = __ldg(p + sz + sy + 1);
                const float fx = s.f[0], fy = s.f[1], fz = s.f[2];
                d0 = (1.0f - fz) * ((1.0f - fy) * (a001 - a000) + fy * (a011 - a010)) +
                     fz * ((1.0f - fy) * (a101 - a100) + fy * (a111 - a110));
                d1 = (1.0f - fz) * ((1.0f - fx) * (a010 - a000) + fx * (a011 - a001)) +
                     fz * ((1.0f - fx) * (a110 - a100) + fx * (a111 - a101));
                d2 = (1.0f - fy) * ((1.0f - fx) * (a100 - a000) + fx * (a101 - a001)) +
                     fy * ((1.0f - fx) * (a110 - a010) + fx * (a111 - a011));
            } else {
                const float a00 = __ldg(p), a01 = __ldg(p + 1), a10 = __ldg(p + sy),
                            a11 = __ldg(p + sy + 1);
                d0 = (1.0f - s.f[1]) * (a01 - a00) + s.f[1] * (a11 - a10);
                d1 = (1.0f - s.f[0]) * (a10 - a00) + s.f[0] * (a11 - a01);
            }
            if (s.in[0])
                loc[0] = fmaf(d0, gv[i], loc[0]);
            if (s.in[1])
                loc[1] = fmaf(d1, gv[i], loc[1]);
            if (D == 3 && s.in[2])
                loc[D - 1] = fmaf(d2, gv[i], loc[D - 1]);
        }
        if (valid) {
#pragma unroll
            for (int i = 0; i < D; ++i)
                h[(int64_t)i * g.nv + vv] = loc[i];
        }
        // transposed interpolation: the sample's weights onto the corners,
        // the -x and +x corner of each (y, z) corner pair together
#pragma unroll
        for (int cz = 0; cz < (D == 3 ? 2 : 1); ++cz)
#pragma unroll
            for (int cy = 0; cy < 2; ++cy) {
                const float wyz = (cy ? s.f[1] : 1.0f - s.f[1]) *
                                  (D == 3 ? (cz ? s.f[2] : 1.0f - s.f[2]) : 1.0f);
                const float w0 = (1.0f - s.f[0]) * wyz, w1 = s.f[0] * wyz;
                const int n0 = valid ? base + cz * sz + cy * sy : -2, n1 = valid ? n0 + 1 : -4;
                // the previous lane's +x node is this lane's -x node: take its value;
                // the next lane's -x node is this lane's +x node: give this value
                const int prev_n1 = __shfl_up_sync(FULL, n1, 1);
                const int next_n0 = __shfl_down_sync(FULL, n0, 1);
                const bool take = lane > 0 && prev_n1 == n0;
                const bool give = lane < 31 && next_n0 == n1;
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    long long q0 = valid ? __float2ll_rn(w0 * gv[i] * S) : 0ll;
                    const long long q1 = valid ? __float2ll_rn(w1 * gv[i] * S) : 0ll;
                    const long long qp = __shfl_up_sync(FULL, q1, 1);
                    if (take)
                        q0 += qp;
                    if (q0 != 0)
                        atomicAdd(acc + (int64_t)i * g.nv + n0, (unsigned long long)q0);
                    if (!give && q1 != 0)
                        atomicAdd(acc + (int64_t)i * g.nv + n1, (unsigned long long)q1);
                }
            }
    }
}

// h += acc / 2^s; acc back to zero for the next step. With maxnext, also the
// largest |h| (the next step's input) into *maxnext, as k_absmax does, so that
// step needs no pass of its own for it.
// With dest (the last step), (h + acc / 2^s) * dsc goes to dest instead, for
// every entry (the exponential's final 2^-K).
__global__ void __launch_bounds__(kDiffeoThreads)
    k_compose_finish(float *__restrict__ h, unsigned long long *__restrict__ acc, int64_t n,
                     const unsigned int *__restrict__ maxbits, unsigned int *__restrict__ maxnext,
                     float *__restrict__ dest, float dsc)
{
    const float inv = 1.0f / fixed_scale(*maxbits);  // a power of two: exact
    float m = 0.0f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const long long q = (long long)acc[e];
        float hv;
        if (dest) {
            hv = h[e];
            if (q != 0) {
                hv = hv + __ll2float_rn(q) * inv;
                acc[e] = 0ull;
            }
            dest[e] = hv * dsc;
            continue;
        }
        if (q != 0) {
            hv = h[e] + __ll2float_rn(q) * inv;
            h[e] = hv;
            acc[e] = 0ull;
        } else if (maxnext) {
            hv = h[e];
        } else {
            continue;
        }
        const float a = fabsf(hv);
        m = a > m ? a : m;  // a NaN never wins
    }
    if (!maxnext)
        return;
    // one atomic per block (the grid is a few blocks per SM)
    __shared__ float wm[kDiffeoThreads / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0)
        wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kDiffeoThreads / 32; ++w)
            m = fmaxf(m, wm[w]);
        atomicMax(maxnext, __float_as_uint(m));
    }
}

template <int D>
cudaError_t exp_run(const Grid &g, int K, const float *v, float *u, float *traj, float *tmp,
                    cudaStream_t s)
{
    const int64_t n = (int64_t)D * g.nv;
    const float sc = ldexpf(1.0f, -K);
    // u_0 -> traj[0] (or tmp); each squaring writes the next buffer
    ProfScope ps(s, "k_exp");
    if (K == 0) {
        k_scale<<<blocks_for(n), kDiffeoThreads, 0, s>>>(v, u, sc, n);
        return cudaGetLastError();
    }
    // the first squaring reads v scaled by 2^-K (and stores u_0 = v 2^-K in
    // the trajectory); each squaring writes the next buffer. If v overlaps a
    // buffer the squarings write, u_0 is formed in a pass of its own first.
    auto overlaps = [&](const float *b, int64_t cnt) {
        return b && v < b + cnt && b < v + n;
    };
    const float *cur = v;
    float scale0 = sc;
    cudaError_t e = cudaSuccess;
    if (overlaps(u, n) || overlaps(tmp, n) || overlaps(traj, (int64_t)K * n)) {
        float *u0 = traj ? traj : ((K - 1) % 2 == 0 ? tmp : u);
        if (K == 1 && !traj)
            u0 = tmp;
        k_scale<<<blocks_for(n), kDiffeoThreads, 0, s>>>(v, u0, sc, n);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        cur = u0;
        scale0 = 1.0f;
    }
    for (int k = 0; k < K && e == cudaSuccess; ++k) {
        float *nxt;
        if (k == K - 1)
            nxt = u;
        else if (traj)
            nxt = traj + (int64_t)(k + 1) * n;
        else
            nxt = ((K - 1 - k) % 2 == 0) ? u : tmp;
        if (k == 0 && scale0 != 1.0f)
            k_compose<D, true><<<blocks_for(g.nv), kDiffeoThreads, 0, s>>>(g, cur, nxt, scale0,
                                                                          traj);
        else
            k_compose<D, false><<<blocks_for(g.nv), kDiffeoThreads, 0, s>>>(g, cur, nxt, 1.0f,
                                                                           nullptr);
        e = cudaGetLastError();
        cur = nxt;
    }
    return e;
}

template <int D>
cudaError_t exp_adjoint_run(const Grid &g, int K, const float *traj, const float *gu, float *gv,
                            char *ws, cudaStream_t s)
{
    const int64_t n = (int64_t)D * g.nv;
    unsigned long long *acc = (unsigned long long *)ws;
    float *b0 = (float *)(ws + ((size_t)n * 8 + 255) / 256 * 256);
    float *b1 = b0 + ((size_t)n * 4 + 255) / 256 * 64;
    unsigned int *mx = (unsigned int *)(b1 + ((size_t)n * 4 + 255) / 256 * 64);
    ProfScope ps(s, "k_exp_adjoint");
    cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)n * 8, s);
    const float *gin = gu;
    float *out = b0;
    // mx[0], mx[1]: the largest |g| of a step's input; the first from a pass of
    // its own, the others from the previous step's finish
    if (e == cudaSuccess && K > 0) {
        e = cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned int), s);
        if (e == cudaSuccess) {
            k_absmax<<<blocks_for(n) < 4 * device_sms() ? blocks_for(n) : 4 * device_sms(),
                       kDiffeoThreads, 0, s>>>(gin, n, mx);
            e = cudaGetLastError();
        }
    }
    for (int k = K - 1, j = 0; k >= 0 && e == cudaSuccess; --k, j ^= 1) {
        const float *u = traj + (int64_t)k * n;
        unsigned int *mcur = mx + j, *mnext = k > 0 ? mx + (j ^ 1) : nullptr;
        k_compose_adjoint<D><<<blocks_for(g.nv), kDiffeoThreads, 0, s>>>(g, u, gin, out, acc, mcur);
        if (mnext && (e = cudaMemsetAsync(mnext, 0, sizeof(unsigned int), s)) != cudaSuccess)
            break;
        // the last step writes (its result) * 2^-K to gv directly
        const int fb = blocks_for(n) < 4 * device_sms() ? blocks_for(n) : 4 * device_sms();
        k_compose_finish<<<fb, kDiffeoThreads, 0, s>>>(out, acc, n, mcur, mnext,
                                                       k == 0 ? gv : nullptr, ldexpf(1.0f, -K));
        e = cudaGetLastError();
        gin = out;
        out = (out == b0) ? b1 : b0;
    }
    if (K > 0)
        return e;
    if (e != cudaSuccess)
        return e;
    k_scale<<<blocks_for(n), kDiffeoThreads, 0, s>>>(gin, gv, ldexpf(1.0f, -K), n);
    return cudaGetLastError();
}

}  // namespace

size_t exp_adjoint_ws(const Grid &g)
{
    const size_t n = (size_t)g.ndim * g.nv;
    return (n * 8 + 255) / 256 * 256 + 2 * ((n * 4 + 255) / 256 * 256) + 256;
}

cudaError_t launch_exp(const Grid &g, int K, const float *v, float *u, float *traj, float *tmp,
                       cudaStream_t s)
{
    return g.ndim == 3 ? exp_run<3>(g, K, v, u, traj, tmp, s) : exp_run<2>(g, K, v, u, traj, tmp, s);
}

cudaError_t launch_exp_adjoint(const Grid &g, int K, const float *traj, const float *gu, float *gv,
                               void *ws, cudaStream_t s)
{
    return g.ndim == 3 ? exp_adjoint_run<3>(g, K, traj, gu, gv, (char *)ws, s)
                       : exp_adjoint_run<2>(g, K, traj, gu, gv, (char *)ws, s);
}

}  // namespace airgb
