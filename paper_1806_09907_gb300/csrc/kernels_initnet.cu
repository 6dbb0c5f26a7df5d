// Learned initialisation: the light kernels around the convolution layers.
//
//  * k_net_input     F, M (fp32 volumes) -> the 2-channel bf16 input x
//  * k_upcat         [up(e4), e3]: nearest 2x up-sampling of the coarsest
//                    level, cropped to e3's grid, concatenated before e3
//  * k_upcat_adjoint its transpose for the up-sampled channels, times the
//                    ReLU factor of e4
//  * k_head_to_ctrl  the head's output voxel j - 1 (clamped) gives control
//                    point j of the spacing-8 lattice (point j sits at voxel
//                    8 (j - 1), where output voxel j - 1 of the head sits)
//  * k_head_adjoint  its transpose, a gather over the points each voxel feeds
//  * k_field_loss    L = (1/(3|X| nb)) sum_b sum_i e_i^T (G_z x G_y x G_x) e_i,
//                    e = c - c*, and dL/dc = (2/(3|X| nb)) (G x G x G) e.
//                    G = B^T B is the Gram matrix of the sampled 1D cubic
//                    B-spline basis (Sec. III-C), banded with 7 diagonals,
//                    so the loss is exactly the mean squared difference of
//                    the two displacement fields, computed on the lattice.
//  * k_adam_flat     Adam (Sec. III-G) on a flat fp32 parameter array
//  * k_render_blobs  training volumes: sums of isotropic Gaussian blobs (per-axis
//                    factors, terms beyond 6 sigma dropped: synthetic data)
//
// All are memory- or latency-bound elementwise/gather kernels sized to the
// data; none needs scratch beyond what its caller passes.
#include <cuda_bf16.h>
#include <stdint.h>

#include "launch.h"
#include "profile.h"

namespace airgb {

namespace {

constexpr int kT = 256;

int blocks(int64_t n)
{
    int64_t b = (n + kT - 1) / kT;
    if (b > 64 * (int64_t)device_sms())  // grid-stride loops beyond this
        b = 64 * (int64_t)device_sms();
    return (int)(b < 1 ? 1 : b);
}

__global__ void k_net_input(const float *__restrict__ F, const float *__restrict__ M, int64_t n,
                            __nv_bfloat162 *__restrict__ x)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = __floats2bfloat162_rn(__ldg(F + i), __ldg(M + i));
}

// One thread per 8-channel group of an output voxel of cat.
__global__ void k_upcat(NetGrid g, int c4, int c3, const uint4 *__restrict__ e4,
                        const uint4 *__restrict__ e3, uint4 *__restrict__ cat)
{
    const int g4 = c4 / 8, g3 = c3 / 8, gc = g4 + g3;
    const int64_t total = (int64_t)g.nb * g.n3[0] * g.n3[1] * g.n3[2] * gc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(i % gc);
        int64_t v = i / gc;  // voxel of e3's grid
        if (q >= g4) {
            cat[i] = __ldg(e3 + v * g3 + (q - g4));
            continue;
        }
        const int x = (int)(v % g.n3[2]);
        v /= g.n3[2];
        const int y = (int)(v % g.n3[1]);
        v /= g.n3[1];
        const int z = (int)(v % g.n3[0]);
        const int b = (int)(v / g.n3[0]);
        const int64_t src = (((int64_t)b * g.n4[0] + z / 2) * g.n4[1] + y / 2) * g.n4[2] + x / 2;
        cat[i] = __ldg(e4 + src * g4 + q);
    }
}

// g_e4[v][c] = (e4[v][c] > 0) * sum over the up to 8 fine voxels copied
// from v of g_cat[fine][c], c < c4, summed in a fixed order.
__global__ void k_upcat_adjoint(NetGrid g, int c4, int c3, const __nv_bfloat16 *__restrict__ gcat,
                                const __nv_bfloat16 *__restrict__ e4,
                                __nv_bfloat16 *__restrict__ ge4)
{
    const int cc = c4 + c3;
    const int64_t total = (int64_t)g.nb * g.n4[0] * g.n4[1] * g.n4[2] * c4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % c4);
        int64_t v = i / c4;
        const int x = (int)(v % g.n4[2]);
        v /= g.n4[2];
        const int y = (int)(v % g.n4[1]);
        v /= g.n4[1];
        const int z = (int)(v % g.n4[0]);
        const int b = (int)(v / g.n4[0]);
        float acc = 0.0f;
        for (int dz = 0; dz < 2; ++dz) {
            const int fz = 2 * z + dz;
            if (fz >= g.n3[0])
                continue;
            for (int dy = 0; dy < 2; ++dy) {
                const int fy = 2 * y + dy;
                if (fy >= g.n3[1])
                    continue;
                for (int dx = 0; dx < 2; ++dx) {
                    const int fx = 2 * x + dx;
                    if (fx >= g.n3[2])
                        continue;
                    const int64_t f = (((int64_t)b * g.n3[0] + fz) * g.n3[1] + fy) * g.n3[2] + fx;
                    acc += __bfloat162float(gcat[f * cc + c]);
                }
            }
        }
        ge4[i] = __float2bfloat16_rn(__bfloat162float(e4[i]) > 0.0f ? acc : 0.0f);
    }
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__global__ void k_head_to_ctrl(NetGrid g, int ch, const float *__restrict__ h,
                               float *__restrict__ c)
{
    const int nx = g.lat[0], ny = g.lat[1], nz = g.lat[2];
    const int64_t per = (int64_t)nx * ny * nz;
    const int64_t total = (int64_t)g.nb * 3 * per;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i;
        const int jx = (int)(r % nx);
        r /= nx;
        const int jy = (int)(r % ny);
        r /= ny;
        const int jz = (int)(r % nz);
        r /= nz;
        const int comp = (int)(r % 3);
        const int b = (int)(r / 3);
        const int hx = clampi(jx - 1, 0, g.n3[2] - 1), hy = clampi(jy - 1, 0, g.n3[1] - 1),
                  hz = clampi(jz - 1, 0, g.n3[0] - 1);
        const int64_t v = (((int64_t)b * g.n3[0] + hz) * g.n3[1] + hy) * g.n3[2] + hx;
        c[i] = h[v * ch + comp];
    }
}

// Lattice indices j whose clamp(j - 1) is output voxel o along one axis of
// n3 outputs and n lattice points: [lo, hi].
__device__ __forceinline__ void feeds(int o, int n3, int n, int &lo, int &hi)
{
    lo = o == 0 ? 0 : o + 1;
    hi = o == n3 - 1 ? n - 1 : o + 1;
}

__global__ void k_head_adjoint(NetGrid g, int ch, const float *__restrict__ gc,
                               __nv_bfloat16 *__restrict__ gh)
{
    const int nx = g.lat[0], ny = g.lat[1], nz = g.lat[2];
    const int64_t total = (int64_t)g.nb * g.n3[0] * g.n3[1] * g.n3[2] * ch;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int comp = (int)(i % ch);
        int64_t v = i / ch;
        float acc = 0.0f;
        if (comp < 3) {
            const int x = (int)(v % g.n3[2]);
            v /= g.n3[2];
            const int y = (int)(v % g.n3[1]);
            v /= g.n3[1];
            const int z = (int)(v % g.n3[0]);
            const int b = (int)(v / g.n3[0]);
            int zl, zh, yl, yh, xl, xh;
            feeds(z, g.n3[0], nz, zl, zh);
            feeds(y, g.n3[1], ny, yl, yh);
            feeds(x, g.n3[2], nx, xl, xh);
            const float *base = gc + ((int64_t)b * 3 + comp) * nx * ny * nz;
            for (int jz = zl; jz <= zh; ++jz)
                for (int jy = yl; jy <= yh; ++jy)
                    for (int jx = xl; jx <= xh; ++jx)
                        acc += base[((int64_t)jz * ny + jy) * nx + jx];
        }
        gh[i] = __float2bfloat16_rn(acc);
    }
}

// Cubic B-spline kernel k_B1D (Sec. III-C) at r (in units of the spacing).
__device__ __forceinline__ float kb3(float r)
{
    const float a = fabsf(r);
    if (a < 1.0f)
        return 2.0f / 3.0f - a * a + 0.5f * a * a * a;
    if (a < 2.0f) {
        const float t = 2.0f - a;
        return t * t * t * (1.0f / 6.0f);
    }
    return 0.0f;
}

// One block per (pair, component). Shared: the three banded Gram matrices
// (n x 7 each; fp32 sums of at most 4 delta terms), two float planes of the
// lattice, reduction scratch. With one block per SM at most (a batch of 16
// has 48 blocks), 1024 threads give each SM enough warps to cover the
// shared-memory latency of the three banded passes.
constexpr int kFieldT = 1024;

__global__ void __launch_bounds__(kFieldT) k_field_loss(FieldLossArgs a, const float *__restrict__ c,
                                                   const float *__restrict__ ct,
                                                   float *__restrict__ gc, double *__restrict__ part)
{
    extern __shared__ double fsm[];
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const int np = nx * ny * nz;
    double *red = fsm;  // kFieldT doubles
    float *Gs = reinterpret_cast<float *>(fsm + kFieldT);
    float *G[3] = {Gs, Gs + 7 * nx, Gs + 7 * (nx + ny)};
    float *b0 = Gs + 7 * (nx + ny + nz);
    float *b1 = b0 + np;
    const int nn[3] = {nx, ny, nz};
    // Gram entries G[j][d + 3] = sum_x k((x - 8 (j-1))/8) k((x - 8 (j+d-1))/8).
    for (int e = threadIdx.x; e < 7 * (nx + ny + nz); e += blockDim.x) {
        int ax = 0, r = e;
        while (r >= 7 * nn[ax]) {
            r -= 7 * nn[ax];
            ++ax;
        }
        const int j = r / 7, d = r % 7 - 3, j2 = j + d;
        float acc = 0.0f;
        if (j2 >= 0 && j2 < nn[ax]) {
            const int D = a.delta, N = a.N[ax];
            const float inv = 1.0f / (float)D;
            const int p1 = D * (j - 1), p2 = D * (j2 - 1);
            const int lo = max(0, max(p1, p2) - 2 * D), hi = min(N - 1, min(p1, p2) + 2 * D);
            for (int x = lo; x <= hi; ++x)
                acc += kb3((float)(x - p1) * inv) * kb3((float)(x - p2) * inv);
        }
        G[ax][r] = acc;
    }
    const int64_t off = (int64_t)blockIdx.x * np;
    for (int p = threadIdx.x; p < np; p += blockDim.x)
        b0[p] = c[off + p] - ct[off + p];
    __syncthreads();
    // x pass: b1 = (I x I x G_x) b0
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const int x = p % nx;
        float acc = 0.0f;
        for (int d = -3; d <= 3; ++d)
            if (x + d >= 0 && x + d < nx)
                acc += G[0][x * 7 + d + 3] * b0[p + d];
        b1[p] = acc;
    }
    __syncthreads();
    // y pass: b0 = (I x G_y x I) b1
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const int y = (p / nx) % ny;
        float acc = 0.0f;
        for (int d = -3; d <= 3; ++d)
            if (y + d >= 0 && y + d < ny)
                acc += G[1][y * 7 + d + 3] * b1[p + d * nx];
        b0[p] = acc;
    }
    __syncthreads();
    // z pass and the quadratic form
    double dot = 0.0;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const int z = p / (nx * ny);
        float acc = 0.0f;
        for (int d = -3; d <= 3; ++d)
            if (z + d >= 0 && z + d < nz)
                acc += G[2][z * 7 + d + 3] * b0[p + d * nx * ny];
        const float e = c[off + p] - ct[off + p];
        dot += (double)e * (double)acc;
        gc[off + p] = (float)(a.gscale * acc);
    }
    red[threadIdx.x] = dot;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        part[blockIdx.x] = red[0];
}

__global__ void k_field_loss_finish(const double *__restrict__ part, int n, double scale,
                                    double *__restrict__ loss)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i)
            s += part[i];
        *loss = s * scale;
    }
}

__global__ void k_adam_flat(AdamFlatArgs a, const int64_t *__restrict__ step,
                            float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v)
{
    __shared__ float s_ib[2];
    if (threadIdx.x == 0) {
        const long long t = (long long)*step + 1;
        s_ib[0] = adam_inv_bias(a.beta1, t);
        s_ib[1] = adam_inv_bias(a.beta2, t);
    }
    __syncthreads();
    const float b1 = (float)a.beta1, b2 = (float)a.beta2;
    const float o1 = (float)(1.0 - a.beta1), o2 = (float)(1.0 - a.beta2);
    const float ib1 = s_ib[0], ib2 = s_ib[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float mm = m[i], vv = v[i];
        p[i] = adam_flat_update(p[i], g[i], mm, vv, b1, o1, b2, o2, a.lr, a.eps, ib1, ib2);
        m[i] = mm;
        v[i] = vv;
    }
}

__global__ void k_tick(int64_t *step)
{
    if (threadIdx.x == 0 && blockIdx.x == 0)
        *step += 1;
}

// out[v][z][y][x] = sum_b a_b exp(-|x - mu_b|^2 / (2 sigma_b^2)) for the
// blob table of volume v ([blob][mu_x, mu_y, mu_z, sigma, a]). A block owns
// an 8 x 8 x 32 box (x, y, z) and first keeps the blobs that come within 6
// sigma of it (warp 0, in table order): a dropped term is below
// a exp(-18) < 1.6e-8 a everywhere in the box. A Gaussian separates into
// per-axis factors,
//   a exp(-|p - mu|^2 / (2 sigma^2)) = ex(x) ey(y) (a ez(z)),
// so each kept blob takes 48 exponentials per box (8 + 8 + 32). A thread
// owns 8 voxels of one (x, y) column: per blob one product ex ey, two
// 16-byte shared-memory reads of the 8 z factors and 4 packed f32x2 FMAs.
constexpr int kBrick = 8;                        // x and y extent of a box
constexpr int kBrickZ = 32;                      // z extent: 4 groups of 8 slices
constexpr int kFac = 2 * kBrick + kBrickZ;       // factors per kept blob

__global__ void __launch_bounds__(256) k_render_blobs(int D, int H, int W, int nblobs,
                                                      const float *__restrict__ table,
                                                      float *__restrict__ out)
{
    extern __shared__ float4 fac4[];  // kept blob k: ex[8], ey[8], a ez[32]
    float *fac = reinterpret_cast<float *>(fac4);
    __shared__ int keep[1024];        // kept blob indices, in table order (n_blobs <= 1024)
    __shared__ int nkeep;
    const int vol = blockIdx.y;
    const int bx = (W + kBrick - 1) / kBrick, by = (H + kBrick - 1) / kBrick;
    const int brick = blockIdx.x;
    const int x0 = (brick % bx) * kBrick, y0 = ((brick / bx) % by) * kBrick,
              z0 = (brick / (bx * by)) * kBrickZ;
    const float *tv = table + (int64_t)vol * nblobs * 5;
    if (threadIdx.x < 32) {
        int base = 0;
        for (int b0 = 0; b0 < nblobs; b0 += 32) {
            const int b = b0 + threadIdx.x;
            bool in = false;
            if (b < nblobs) {
                const float *e = tv + (int64_t)b * 5;
                const float mx = e[0], my = e[1], mz = e[2], sg = e[3];
                // distance from the centre to the box
                const float dx = fmaxf(fmaxf((float)x0 - mx, mx - (float)(x0 + kBrick - 1)), 0.0f);
                const float dy = fmaxf(fmaxf((float)y0 - my, my - (float)(y0 + kBrick - 1)), 0.0f);
                const float dz =
                    fmaxf(fmaxf((float)z0 - mz, mz - (float)(z0 + kBrickZ - 1)), 0.0f);
                in = dx * dx + dy * dy + dz * dz <= 36.0f * sg * sg;
            }
            const unsigned m = __ballot_sync(0xffffffffu, in);
            if (in)
                keep[base + __popc(m & ((1u << threadIdx.x) - 1u))] = b;
            base += __popc(m);
        }
        if (threadIdx.x == 0)
            nkeep = base;
    }
    __syncthreads();
    const int n = nkeep;
    // the per-axis factors of the kept blobs at the box's coordinates
    for (int t = threadIdx.x; t < n * kFac; t += blockDim.x) {
        const int k = t / kFac, r = t - k * kFac;
        const int axis = r < kBrick ? 0 : r < 2 * kBrick ? 1 : 2;
        const int o = r - axis * kBrick;
        const float *e = tv + (int64_t)keep[k] * 5;
        const float c = (float)((axis == 0 ? x0 : axis == 1 ? y0 : z0) + o) - e[axis];
        const float v = expf(-0.5f * c * c / (e[3] * e[3]));
        fac[t] = axis == 2 ? e[4] * v : v;
    }
    __syncthreads();
    // thread: column (lx, ly), slices 8 zg .. 8 zg + 7 of the box; the 8
    // sums as 4 pairs, each blob's 8 FMAs as 4 packed f32x2 FMAs (the same
    // rounding per lane)
    const int t = threadIdx.x, lx = t & 7, ly = (t >> 3) & 7, zg = t >> 6;
    float2 acc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        acc[i] = make_float2(0.0f, 0.0f);
    for (int k = 0; k < n; ++k) {
        const float *f = fac + kFac * k;
        const float pxy = f[lx] * f[kBrick + ly];
        const float2 p2 = make_float2(pxy, pxy);
        const float4 za = fac4[(kFac * k + 2 * kBrick + 8 * zg) / 4];
        const float4 zb = fac4[(kFac * k + 2 * kBrick + 8 * zg) / 4 + 1];
        acc[0] = __ffma2_rn(p2, make_float2(za.x, za.y), acc[0]);
        acc[1] = __ffma2_rn(p2, make_float2(za.z, za.w), acc[1]);
        acc[2] = __ffma2_rn(p2, make_float2(zb.x, zb.y), acc[2]);
        acc[3] = __ffma2_rn(p2, make_float2(zb.z, zb.w), acc[3]);
    }
    const int64_t nv = (int64_t)D * H * W;
    const int x = x0 + lx, y = y0 + ly;
    if (x < W && y < H) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int z = z0 + 8 * zg + i;
            if (z < D)
                out[(int64_t)vol * nv + ((int64_t)z * H + y) * W + x] =
                    (i & 1) ? acc[i >> 1].y : acc[i >> 1].x;
        }
    }
}

}  // namespace

cudaError_t launch_net_input(int64_t n, const float *F, const float *M, void *x, cudaStream_t s)
{
    ProfScope ps(s, "k_net_input");
    k_net_input<<<blocks(n), kT, 0, s>>>(F, M, n, static_cast<__nv_bfloat162 *>(x));
    return cudaGetLastError();
}

cudaError_t launch_upcat(const NetGrid &g, int c4, int c3, const void *e4, const void *e3,
                         void *cat, cudaStream_t s)
{
    ProfScope ps(s, "k_upcat");
    const int64_t n = (int64_t)g.nb * g.n3[0] * g.n3[1] * g.n3[2] * ((c4 + c3) / 8);
    k_upcat<<<blocks(n), kT, 0, s>>>(g, c4, c3, static_cast<const uint4 *>(e4),
                                     static_cast<const uint4 *>(e3), static_cast<uint4 *>(cat));
    return cudaGetLastError();
}

cudaError_t launch_upcat_adjoint(const NetGrid &g, int c4, int c3, const void *gcat,
                                 const void *e4, void *ge4, cudaStream_t s)
{
    ProfScope ps(s, "k_upcat_adjoint");
    const int64_t n = (int64_t)g.nb * g.n4[0] * g.n4[1] * g.n4[2] * c4;
    k_upcat_adjoint<<<blocks(n), kT, 0, s>>>(g, c4, c3, static_cast<const __nv_bfloat16 *>(gcat),
                                             static_cast<const __nv_bfloat16 *>(e4),
                                             static_cast<__nv_bfloat16 *>(ge4));
    return cudaGetLastError();
}

cudaError_t launch_head_to_ctrl(const NetGrid &g, int ch, const float *h, float *c, cudaStream_t s)
{
    ProfScope ps(s, "k_head_to_ctrl");
    const int64_t n = (int64_t)g.nb * 3 * g.lat[0] * g.lat[1] * g.lat[2];
    k_head_to_ctrl<<<blocks(n), kT, 0, s>>>(g, ch, h, c);
    return cudaGetLastError();
}

cudaError_t launch_head_adjoint(const NetGrid &g, int ch, const float *gc, void *gh,
                                cudaStream_t s)
{
    ProfScope ps(s, "k_head_adjoint");
    const int64_t n = (int64_t)g.nb * g.n3[0] * g.n3[1] * g.n3[2] * ch;
    k_head_adjoint<<<blocks(n), kT, 0, s>>>(g, ch, gc, static_cast<__nv_bfloat16 *>(gh));
    return cudaGetLastError();
}

size_t field_loss_smem(const FieldLossArgs &a)
{
    const int np = a.n[0] * a.n[1] * a.n[2];
    return sizeof(double) * kFieldT + sizeof(float) * 7 * (a.n[0] + a.n[1] + a.n[2]) +
           sizeof(float) * 2 * np;
}

cudaError_t launch_field_loss(const FieldLossArgs &a, int nb, const float *c, const float *ct,
                              float *gc, double *part, double *loss, cudaStream_t s)
{
    const size_t sm = field_loss_smem(a);
    cudaError_t e = cudaFuncSetAttribute(k_field_loss, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess)
        return e;
    {
        ProfScope ps(s, "k_field_loss");
        k_field_loss<<<nb * 3, kFieldT, sm, s>>>(a, c, ct, gc, part);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    ProfScope ps(s, "k_field_loss_finish");
    k_field_loss_finish<<<1, 32, 0, s>>>(part, nb * 3, a.lscale, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam_flat(const AdamFlatArgs &a, int64_t *step, float *p, const float *g,
                             float *m, float *v, cudaStream_t s)
{
    {
        ProfScope ps(s, "k_adam_flat");
        k_adam_flat<<<blocks(a.n), kT, 0, s>>>(a, step, p, g, m, v);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    return launch_step_tick(step, s);
}

cudaError_t launch_step_tick(int64_t *step, cudaStream_t s)
{
    ProfScope ps(s, "k_tick");
    k_tick<<<1, 32, 0, s>>>(step);
    return cudaGetLastError();
}

cudaError_t launch_render_blobs(int D, int H, int W, int count, int nblobs, const float *table,
                                float *out, cudaStream_t s)
{
    ProfScope ps(s, "k_render_blobs");
    const int bricks = ((W + kBrick - 1) / kBrick) * ((H + kBrick - 1) / kBrick) *
                       ((D + kBrickZ - 1) / kBrickZ);
    dim3 grid(bricks, count);
    // up to 192 KB (1024 blobs), beside the 4 KB keep list
    const size_t smem = sizeof(float) * kFac * (size_t)nblobs;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(
            k_render_blobs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    k_render_blobs<<<grid, 256, smem, s>>>(D, H, W, nblobs, table, out);
    return cudaGetLastError();
}

}  // namespace airgb
