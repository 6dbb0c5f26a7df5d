// Shared device-side descriptors and helpers of libairgb (CUDA, sm_103a).
// Nothing here is shared with the FP64 oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#ifndef AL_CHECK
#define AL_CHECK 0
#endif

namespace airgb {

constexpr int kMaxDelta = 32;

// Kernel error word of this translation unit (every .cu file that includes
// this header has its own). A checked build (AL_CHECK=1) records
// AL_ERR_BOUNDS (5) here when an index leaves its range and the access is
// skipped; al_get_device_error reads and clears the words of every unit.
static __device__ int g_unit_error = 0;

// True when 0 <= i < n; in a checked build a false result is recorded.
// Unchecked builds compile it to `true`.
__device__ __forceinline__ bool al_index_ok(int64_t i, int64_t n)
{
#if AL_CHECK
    if (i < 0 || i >= n) {
        atomicExch(&g_unit_error, 5);
        return false;
    }
#else
    (void)i;
    (void)n;
#endif
    return true;
}

// Host reader of this unit's error word (read, then clear when asked);
// -1 if a copy failed. Instantiated once per unit that checks indices.
#define AL_UNIT_ERROR_READER(fn)                                                  \
    int fn(bool clear)                                                            \
    {                                                                             \
        int h = 0;                                                                \
        if (cudaMemcpyFromSymbol(&h, g_unit_error, sizeof(int)) != cudaSuccess)  \
            return -1;                                                            \
        if (h != 0 && clear) {                                                    \
            const int zero = 0;                                                   \
            if (cudaMemcpyToSymbol(g_unit_error, &zero, sizeof(int)) != cudaSuccess) \
                return -1;                                                        \
        }                                                                         \
        return h;                                                                 \
    }

// Image grid. 2D grids have Z = 1. nv = X*Y*Z < 2^31 (checked on the host).
struct Grid {
    int ndim;
    int X, Y, Z;
    int nv;
};

// Control lattice of the cubic B-spline transformation (Sec. III-C):
// point j at voxel coordinate (j - 1)*delta, n = (N - 1)/delta + 4 points
// per active axis; w[p][a] is the weight of control index q + a for a voxel
// at x = q*delta + p, i.e. k_B1D(p/delta + 1 - a).
struct Lattice {
    int delta;
    int nx, ny, nz;
    int nc;  // nx*ny*nz
    float w[kMaxDelta][4];
};

// Compile-time cubic B-spline weights for phase p of spacing DELTA
// (t = p/DELTA): (1-t)^3/6, (3t^3 - 6t^2 + 4)/6, (-3t^3 + 3t^2 + 3t + 1)/6,
// t^3/6, evaluated in double and rounded once.
template <int DELTA>
__host__ __device__ constexpr float bsw(int p, int a)
{
    return (float)(a == 0   ? (1.0 - (double)p / DELTA) * (1.0 - (double)p / DELTA) *
                                (1.0 - (double)p / DELTA) / 6.0
                   : a == 1 ? (3.0 * ((double)p / DELTA) * ((double)p / DELTA) * ((double)p / DELTA) -
                               6.0 * ((double)p / DELTA) * ((double)p / DELTA) + 4.0) /
                                  6.0
                   : a == 2 ? (-3.0 * ((double)p / DELTA) * ((double)p / DELTA) * ((double)p / DELTA) +
                               3.0 * ((double)p / DELTA) * ((double)p / DELTA) +
                               3.0 * ((double)p / DELTA) + 1.0) /
                                  6.0
                            : ((double)p / DELTA) * ((double)p / DELTA) * ((double)p / DELTA) / 6.0);
}

// The weights of every phase of DELTA as a constexpr table.
template <int DELTA>
struct WTab {
    float w[DELTA][4];
    __host__ __device__ constexpr WTab() : w{}
    {
        for (int p = 0; p < DELTA; ++p)
            for (int a = 0; a < 4; ++a)
                w[p][a] = bsw<DELTA>(p, a);
    }
};

// Same weights at run time, in double (used by the Gram-form regulariser).
__host__ __device__ inline double bsw_d(int p, int a, int delta)
{
    const double t = (double)p / (double)delta;
    switch (a) {
    case 0: return (1.0 - t) * (1.0 - t) * (1.0 - t) / 6.0;
    case 1: return (3.0 * t * t * t - 6.0 * t * t + 4.0) / 6.0;
    case 2: return (-3.0 * t * t * t + 3.0 * t * t + 3.0 * t + 1.0) / 6.0;
    default: return t * t * t / 6.0;
    }
}

// Sample position of a voxel displaced by u along one axis of size n:
// y = x + u split exactly as integer part + fraction, so no rounding happens
// in forming y (x + u in fp32 would lose bits for large x). Sets `inside` to
// false when y < 0, y > n - 1 or u is not finite. On return (inside) `cell` is
// the floor cell clamped to [0, n-2] and `f` in [0, 1] the offset in it.
struct AxisSample {
    int cell;
    float f;
};

__device__ __forceinline__ bool axis_sample(int x, float u, int n, AxisSample &s)
{
    const float fl = floorf(u);
    if (!(fabsf(fl) < 1.0e9f))  // not finite, or absurdly far outside
        return false;
    const int iy = x + (int)fl;
    const float f = u - fl;  // exact for u >= 0; correctly rounded otherwise
    if (iy < 0 || iy > n - 1 || (iy == n - 1 && f > 0.0f))
        return false;
    if (iy == n - 1) {  // on the last face: clamp the cell, weight 1 on the last voxel
        s.cell = n - 2;
        s.f = 1.0f;
    } else {
        s.cell = iy;
        s.f = f;
    }
    return true;
}

// Branch-free form of axis_sample for kernels that load the cell whatever
// the mask: cell is always in [0, n-2] (so the loads stay in bounds) and,
// when the sample is inside, equals axis_sample's cell with f its offset
// (f = 1 on the last face). Returns whether the sample is inside; f is
// meaningful only then. lo = -x and hi = n - 1 - x (exact floats, n < 2^22):
// y = x + u lies in [0, n-1] exactly when lo <= u <= hi, which is false for
// NaN and infinities too.
//
// floor(u) comes from one round-toward-minus-infinity add of 1.5 * 2^23:
// for |u| < 2^22 the sum lies in [2^23, 2^24], where floats are the
// integers, so it is exactly floor(u) + 1.5 * 2^23 and its low mantissa bits
// hold floor(u) as an integer. Every inside sample has |u| < 2^22; for the
// others the cell is clamped into range whatever the bits hold.
__device__ __forceinline__ bool axis_cell(int x, float u, float lo, float hi, int n, int &cell,
                                          float &f)
{
    constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23, bit pattern 0x4B400000
    const float t = __fadd_rd(u, kMagic);
    const int iy = (int)((unsigned)x + (unsigned)__float_as_int(t) - 0x4B400000u);
    const float fr = u - (t - kMagic);
    const int c = min(max(iy, 0), n - 2);
    cell = c;
    f = iy > c ? fr + 1.0f : fr;  // the last face: weight 1 on the last voxel
    return u >= lo && u <= hi;
}

// Linear interpolation value and gradient in a 3D cell: corners m[z][y][x].
struct Interp {
    float v, gx, gy, gz;
};

__device__ __forceinline__ Interp trilinear(const float *__restrict__ M, int X, int Y, int Z,
                                            const AxisSample &sx, const AxisSample &sy,
                                            const AxisSample &sz)
{
    int64_t base = ((int64_t)sz.cell * Y + sy.cell) * X + sx.cell;
    const int64_t sY = X, sZ = (int64_t)X * Y;
    if (!(al_index_ok(sx.cell, X - 1) & al_index_ok(sy.cell, Y - 1) & al_index_ok(sz.cell, Z - 1)))
        base = 0;  // checked builds only: the cell left the volume
    const float m000 = __ldg(M + base), m001 = __ldg(M + base + 1);
    const float m010 = __ldg(M + base + sY), m011 = __ldg(M + base + sY + 1);
    const float m100 = __ldg(M + base + sZ), m101 = __ldg(M + base + sZ + 1);
    const float m110 = __ldg(M + base + sZ + sY), m111 = __ldg(M + base + sZ + sY + 1);
    const float fx = sx.f, fy = sy.f, fz = sz.f;
    const float gx_ = 1.0f - fx, gy_ = 1.0f - fy, gz_ = 1.0f - fz;
    // along x; (1-f) m0 + f m1 is exact at f = 0 and f = 1, so samples on
    // grid points (including the clamped last face) return the voxel value
    const float d00 = m001 - m000, d01 = m011 - m010, d10 = m101 - m100, d11 = m111 - m110;
    const float a00 = fmaf(fx, m001, gx_ * m000), a01 = fmaf(fx, m011, gx_ * m010);
    const float a10 = fmaf(fx, m101, gx_ * m100), a11 = fmaf(fx, m111, gx_ * m110);
    // along y
    const float e0 = a01 - a00, e1 = a11 - a10;
    const float b0 = fmaf(fy, a01, gy_ * a00), b1 = fmaf(fy, a11, gy_ * a10);
    Interp r;
    r.v = fmaf(fz, b1, gz_ * b0);
    r.gz = b1 - b0;
    r.gy = fmaf(fz, e1 - e0, e0);
    const float gx0 = fmaf(fy, d01 - d00, d00), gx1 = fmaf(fy, d11 - d10, d10);
    r.gx = fmaf(fz, gx1 - gx0, gx0);
    return r;
}

__device__ __forceinline__ Interp bilinear(const float *__restrict__ M, int X, int Y,
                                           const AxisSample &sx, const AxisSample &sy)
{
    int64_t base = (int64_t)sy.cell * X + sx.cell;
    if (!(al_index_ok(sx.cell, X - 1) & al_index_ok(sy.cell, Y - 1)))
        base = 0;  // checked builds only: the cell left the image
    const float m00 = __ldg(M + base), m01 = __ldg(M + base + 1);
    const float m10 = __ldg(M + base + X), m11 = __ldg(M + base + X + 1);
    const float fx = sx.f, fy = sy.f;
    const float gx_ = 1.0f - fx;
    const float d0 = m01 - m00, d1 = m11 - m10;
    const float a0 = fmaf(fx, m01, gx_ * m00), a1 = fmaf(fx, m11, gx_ * m10);
    Interp r;
    r.v = fmaf(fy, a1, (1.0f - fy) * a0);
    r.gy = a1 - a0;
    r.gx = fmaf(fy, d1 - d0, d0);
    r.gz = 0.0f;
    return r;
}

// Interpolation from corner values already loaded: c[0..7] = m000, m001,
// m010, m011, m100, m101, m110, m111 (z, y, x bits), same arithmetic as
// trilinear() / bilinear().
__device__ __forceinline__ Interp interp8(const float (&c)[8], float fx, float fy, float fz)
{
    const float gx_ = 1.0f - fx, gy_ = 1.0f - fy, gz_ = 1.0f - fz;
    const float d00 = c[1] - c[0], d01 = c[3] - c[2], d10 = c[5] - c[4], d11 = c[7] - c[6];
    const float a00 = fmaf(fx, c[1], gx_ * c[0]), a01 = fmaf(fx, c[3], gx_ * c[2]);
    const float a10 = fmaf(fx, c[5], gx_ * c[4]), a11 = fmaf(fx, c[7], gx_ * c[6]);
    const float e0 = a01 - a00, e1 = a11 - a10;
    const float b0 = fmaf(fy, a01, gy_ * a00), b1 = fmaf(fy, a11, gy_ * a10);
    Interp r;
    r.v = fmaf(fz, b1, gz_ * b0);
    r.gz = b1 - b0;
    r.gy = fmaf(fz, e1 - e0, e0);
    const float gx0 = fmaf(fy, d01 - d00, d00), gx1 = fmaf(fy, d11 - d10, d10);
    r.gx = fmaf(fz, gx1 - gx0, gx0);
    return r;
}

// interp8 on corners paired by z: c2[q] = (c[q], c[q + 4]) for q = y x bits.
// The pairs go through packed f32x2 operations (each lane one correctly
// rounded operation), so the result equals interp8's bit for bit.
__device__ __forceinline__ Interp interp8_z2(const float2 (&c2)[4], float fx, float fy, float fz)
{
    const float gx_ = 1.0f - fx, gy_ = 1.0f - fy, gz_ = 1.0f - fz;
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 fx2 = make_float2(fx, fx), gx2 = make_float2(gx_, gx_);
    const float2 fy2 = make_float2(fy, fy), gy2 = make_float2(gy_, gy_);
    const float2 dlo = __ffma2_rn(c2[0], m1, c2[1]);  // (d00, d10)
    const float2 dhi = __ffma2_rn(c2[2], m1, c2[3]);  // (d01, d11)
    const float2 alo = __ffma2_rn(fx2, c2[1], __fmul2_rn(gx2, c2[0]));  // (a00, a10)
    const float2 ahi = __ffma2_rn(fx2, c2[3], __fmul2_rn(gx2, c2[2]));  // (a01, a11)
    const float2 e = __ffma2_rn(alo, m1, ahi);                          // (e0, e1)
    const float2 b = __ffma2_rn(fy2, ahi, __fmul2_rn(gy2, alo));        // (b0, b1)
    const float2 gxp = __ffma2_rn(fy2, __ffma2_rn(dlo, m1, dhi), dlo);  // (gx0, gx1)
    Interp r;
    r.v = fmaf(fz, b.y, gz_ * b.x);
    r.gz = b.y - b.x;
    r.gy = fmaf(fz, e.y - e.x, e.x);
    r.gx = fmaf(fz, gxp.y - gxp.x, gxp.x);
    return r;
}

__device__ __forceinline__ Interp interp4(const float (&c)[4], float fx, float fy)
{
    const float gx_ = 1.0f - fx;
    const float d0 = c[1] - c[0], d1 = c[3] - c[2];
    const float a0 = fmaf(fx, c[1], gx_ * c[0]), a1 = fmaf(fx, c[3], gx_ * c[2]);
    Interp r;
    r.v = fmaf(fy, a1, (1.0f - fy) * a0);
    r.gy = a1 - a0;
    r.gx = fmaf(fy, d1 - d0, d0);
    r.gz = 0.0f;
    return r;
}

// Shared-memory address of a generic pointer into shared memory.
__device__ __forceinline__ uint32_t al_smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// One test of an mbarrier phase (parity); true once it has completed.
__device__ __forceinline__ bool al_mbar_try_wait(uint32_t bar, uint32_t parity)
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

// Wait for an mbarrier phase for about one second of %globaltimer at most;
// false if it did not complete (the caller records AL_ERR_TIMEOUT).
__device__ __noinline__ inline bool al_mbar_wait_slow(uint32_t bar, uint32_t parity)
{
    uint64_t t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (!al_mbar_try_wait(bar, parity)) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 1000000000ull)
            return false;
    }
    return true;
}

__device__ __forceinline__ bool al_mbar_wait(uint32_t bar, uint32_t parity)
{
    return al_mbar_try_wait(bar, parity) || al_mbar_wait_slow(bar, parity);
}

// Deterministic block reduction of K doubles per thread (fixed tree):
// shuffles within each warp, then warp 0 reduces the warps' sums the same
// way (FP64 latency is long on this part, so no serial chain over the
// warps). `scratch` holds at least K * (blockDim.x / 32) doubles (blockDim.x
// <= 1024). Result valid in thread 0 (written back into v).
template <int K>
__device__ __forceinline__ void block_reduce_d(double (&v)[K], double *scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    }
    __syncthreads();  // scratch may still be in use by a previous call
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k)
            scratch[k * nwarp + warp] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = lane < nwarp ? scratch[k * nwarp + lane] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                t += __shfl_down_sync(0xffffffffu, t, off);
            v[k] = t;
        }
    }
}

// Block sum of K fp32 values per thread into doubles (valid in thread 0):
// an fp32 shuffle tree within each warp (32 values of a few dozen terms each
// keep their relative error near 1e-7), then warp 0 adds the warps' sums in
// FP64 with a second tree. FP64 issues slowly on this part; this takes
// 5 K FP64 adds per block instead of 5 K per warp. `scratch` holds at least
// K * (blockDim.x / 32) doubles.
template <int K>
__device__ __forceinline__ void block_reduce_fd(float (&v)[K], double (&out)[K], double *scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    }
    __syncthreads();  // scratch may still be in use by a previous call
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k)
            scratch[k * nwarp + warp] = (double)v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k)
        out[k] = 0.0;
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = lane < nwarp ? scratch[k * nwarp + lane] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                t += __shfl_down_sync(0xffffffffu, t, off);
            out[k] = t;
        }
    }
}

// Adam's bias-correction factor 1 / (1 - beta^t) at step t >= 1 (Kingma and
// Ba), as float. beta^t is formed in FP64 by binary exponentiation (at most
// 2 log2 t products) instead of a library pow: FP64 issues slowly on this
// part, and one pow per block took most of a small Adam launch. The products'
// FP64 roundings lie far below the final fp32 rounding.
__device__ __forceinline__ float adam_inv_bias(double beta, long long t)
{
    double r = 1.0, b = beta;
    for (; t > 0; t >>= 1) {
        if (t & 1)
            r *= b;
        b *= b;
    }
    return (float)(1.0 / (1.0 - r));
}

// One Adam update of a flat parameter (Kingma and Ba): m <- b1 m + o1 g,
// v <- b2 v + o2 g^2 (o = 1 - b), returns p - lr (m ib1) / (sqrt(v ib2) + eps)
// with ib = 1 / (1 - b^t); m and v are updated in place.
__device__ __forceinline__ float adam_flat_update(float p, float g, float &m, float &v, float b1,
                                                  float o1, float b2, float o2, float lr,
                                                  float eps, float ib1, float ib2)
{
    m = fmaf(b1, m, o1 * g);
    v = fmaf(b2, v, o2 * g * g);
    return p - lr * ((m * ib1) / (sqrtf(v * ib2) + eps));
}

}  // namespace airgb
