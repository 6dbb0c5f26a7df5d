// Step kernels of the unfused path: A1 B-spline expansion, A6 its adjoint,
// A2 warp, A5 warp adjoint, A4 diffusion regulariser (voxel form).
#include "launch.h"

namespace airgb {

namespace {

constexpr int kDispTX = 128;  // x extent of a displacement tile (threads)
constexpr int kDispTY = 8;    // rows per tile
constexpr int kDispMaxJX = kDispTX + 5;  // control columns a tile can touch (delta >= 1)
constexpr int kDispMaxJY = kDispTY + 5;

// A1: u_i(x) = sum_j c_{i,j} prod_k w. One CTA = one z slice, 8 rows, 128
// columns. Separable: z-contraction of the touched control block into smem,
// then y-contraction per row, then 4 x-taps per voxel.
template <int D>
__global__ void __launch_bounds__(kDispTX) k_displacement(Grid g, Lattice L,
                                                          const float *__restrict__ c,
                                                          float *__restrict__ u)
{
    __shared__ float tz[D][kDispMaxJY][kDispMaxJX];
    __shared__ float ty[D][kDispTY][kDispMaxJX];
    const int x0 = blockIdx.x * kDispTX, y0 = blockIdx.y * kDispTY, z = blockIdx.z;
    const int delta = L.delta;
    const int jx0 = x0 / delta, jy0 = y0 / delta;
    const int xl = min(x0 + kDispTX, g.X) - 1, yl = min(y0 + kDispTY, g.Y) - 1;
    const int njx = xl / delta + 4 - jx0, njy = yl / delta + 4 - jy0;
    const int qz = z / delta, pz = z - qz * delta;
    // z contraction
    for (int e = threadIdx.x; e < D * njy * njx; e += blockDim.x) {
        const int i = e / (njy * njx), r = e - i * njy * njx;
        const int jyl = r / njx, jxl = r - jyl * njx;
        const int jy = jy0 + jyl, jx = jx0 + jxl;
        float acc = 0.0f;
        if (D == 3) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
                acc = fmaf(L.w[pz][a],
                           __ldg(c + (((int64_t)i * L.nz + qz + a) * L.ny + jy) * L.nx + jx), acc);
        } else {
            acc = __ldg(c + ((int64_t)i * L.ny + jy) * L.nx + jx);
        }
        tz[i][jyl][jxl] = acc;
    }
    __syncthreads();
    // y contraction
    for (int e = threadIdx.x; e < D * kDispTY * njx; e += blockDim.x) {
        const int i = e / (kDispTY * njx), r = e - i * kDispTY * njx;
        const int yr = r / njx, jxl = r - yr * njx;
        const int y = min(y0 + yr, g.Y - 1);
        const int qy = y / delta, py = y - qy * delta;
        float acc = 0.0f;
#pragma unroll
        for (int b = 0; b < 4; ++b)
            acc = fmaf(L.w[py][b], tz[i][qy - jy0 + b][jxl], acc);
        ty[i][yr][jxl] = acc;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= g.X)
        return;
    const int qx = x / delta, px = x - qx * delta;
    const float w0 = L.w[px][0], w1 = L.w[px][1], w2 = L.w[px][2], w3 = L.w[px][3];
    const int jxl = qx - jx0;
    for (int yr = 0; yr < kDispTY && y0 + yr < g.Y; ++yr) {
        const int64_t v = ((int64_t)z * g.Y + y0 + yr) * g.X + x;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            float acc = w0 * ty[i][yr][jxl];
            acc = fmaf(w1, ty[i][yr][jxl + 1], acc);
            acc = fmaf(w2, ty[i][yr][jxl + 2], acc);
            acc = fmaf(w3, ty[i][yr][jxl + 3], acc);
            u[(int64_t)i * g.nv + v] = acc;
        }
    }
}

// A6, one axis of the separable transpose: out[.., j, ..] = sum over the
// 4*delta inputs t of axis `axis` in j's support of w(t, j) * in[.., t, ..].
// Each output is a gather in fixed order (ascending t). Shapes are given
// as (outer, len_in, inner) -> (outer, len_out, inner).
__global__ void k_bspline_transpose_axis(const float *__restrict__ in, float *__restrict__ out,
                                         int64_t outer, int len_in, int len_out, int64_t inner,
                                         Lattice L)
{
    const int64_t total = outer * len_out * inner;
    const int delta = L.delta;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = e / ((int64_t)len_out * inner);
        const int64_t r = e - o * len_out * inner;
        const int j = (int)(r / inner);
        const int64_t k = r - (int64_t)j * inner;
        const int t0 = max(0, (j - 3) * delta), t1 = min(len_in, (j + 1) * delta);
        const float *src = in + (o * len_in) * inner + k;
        float acc = 0.0f;
        for (int t = t0; t < t1; ++t) {
            const int q = t / delta, p = t - q * delta;
            acc = fmaf(L.w[p][j - q], __ldg(src + (int64_t)t * inner), acc);
        }
        out[e] = acc;
    }
}

// A2: backward warp with mask.
template <int D>
__global__ void k_warp(Grid g, const float *__restrict__ M, const float *__restrict__ u,
                       float *__restrict__ W, uint8_t *__restrict__ mask)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(v % g.X);
        const int64_t r = v / g.X;
        const int y = (int)(r % g.Y), z = (int)(r / g.Y);
        AxisSample sx, sy, sz;
        bool in = axis_sample(x, __ldg(u + v), g.X, sx);
        in &= axis_sample(y, __ldg(u + g.nv + v), g.Y, sy);
        if (D == 3)
            in &= axis_sample(z, __ldg(u + 2 * (int64_t)g.nv + v), g.Z, sz);
        float w = 0.0f;
        if (in)
            w = (D == 3) ? trilinear(M, g.X, g.Y, g.Z, sx, sy, sz).v : bilinear(M, g.X, g.Y, sx, sy).v;
        W[v] = w;
        mask[v] = in ? 1 : 0;
    }
}

// A5: grad_disp[k] = mask * grad_warped * dM~/dy_k (+ grad_disp if accumulate).
template <int D>
__global__ void k_warp_adjoint(Grid g, const float *__restrict__ M, const float *__restrict__ u,
                               const uint8_t *__restrict__ mask, const float *__restrict__ gw,
                               float *__restrict__ gu, int accumulate)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        float gx = 0.0f, gy = 0.0f, gz = 0.0f;
        const float gwv = __ldg(gw + v);
        if (__ldg(mask + v) && gwv != 0.0f) {
            const int x = (int)(v % g.X);
            const int64_t r = v / g.X;
            const int y = (int)(r % g.Y), z = (int)(r / g.Y);
            AxisSample sx, sy, sz;
            bool in = axis_sample(x, __ldg(u + v), g.X, sx);
            in &= axis_sample(y, __ldg(u + g.nv + v), g.Y, sy);
            if (D == 3)
                in &= axis_sample(z, __ldg(u + 2 * (int64_t)g.nv + v), g.Z, sz);
            if (in) {
                const Interp ip =
                    (D == 3) ? trilinear(M, g.X, g.Y, g.Z, sx, sy, sz) : bilinear(M, g.X, g.Y, sx, sy);
                gx = gwv * ip.gx;
                gy = gwv * ip.gy;
                gz = gwv * ip.gz;
            }
        }
        if (accumulate) {
            gu[v] += gx;
            gu[g.nv + v] += gy;
            if (D == 3)
                gu[2 * (int64_t)g.nv + v] += gz;
        } else {
            gu[v] = gx;
            gu[g.nv + v] = gy;
            if (D == 3)
                gu[2 * (int64_t)g.nv + v] = gz;
        }
    }
}

// A4: R = (1/|X|) sum_i sum_k sum_{x_k < N_k-1} (u_i(x+e_k) - u_i(x))^2 and
// grad = weight * dR/du. One thread per voxel; per-block FP64 partial sums.
template <int D>
__global__ void __launch_bounds__(256) k_regulariser(Grid g, const float *__restrict__ u,
                                                     float gscale, float *__restrict__ gu,
                                                     double *__restrict__ partials)
{
    __shared__ double red[8];
    double acc[1] = {0.0};
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v < g.nv) {
        const int x = (int)(v % g.X);
        const int64_t r = v / g.X;
        const int y = (int)(r % g.Y), z = (int)(r / g.Y);
        const int64_t st[3] = {1, g.X, (int64_t)g.X * g.Y};
        const int pos[3] = {x, y, z};
        const int n[3] = {g.X, g.Y, g.Z};
        float sum = 0.0f;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const float *ui = u + (int64_t)i * g.nv;
            const float c = __ldg(ui + v);
            float lap = 0.0f;  // sum_k (u(x) - u(x-e_k)) - (u(x+e_k) - u(x))
#pragma unroll
            for (int k = 0; k < D; ++k) {
                if (pos[k] + 1 < n[k]) {
                    const float d = __ldg(ui + v + st[k]) - c;
                    sum = fmaf(d, d, sum);
                    lap -= d;
                }
                if (pos[k] > 0)
                    lap += c - __ldg(ui + v - st[k]);
            }
            if (gu)
                gu[(int64_t)i * g.nv + v] = gscale * lap;
        }
        acc[0] = sum;
    }
    block_reduce_d<1>(acc, red);
    if (threadIdx.x == 0)
        partials[blockIdx.x] = acc[0];
}

// Fixed-order sum of `count` partials (one block), scaled, into out[0].
__global__ void k_sum_partials(const double *__restrict__ partials, int count, double scale,
                               double *__restrict__ out)
{
    __shared__ double red[32];
    double acc[1] = {0.0};
    for (int i = threadIdx.x; i < count; i += blockDim.x)
        acc[0] += partials[i];
    block_reduce_d<1>(acc, red);
    if (threadIdx.x == 0)
        out[0] = acc[0] * scale;
}

__global__ void k_combine(const double *__restrict__ sim, const double *__restrict__ reg,
                          double lambda, double *__restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double S = sim[0], n = sim[1], R = reg[0];
        out[0] = S + lambda * R;
        out[1] = S;
        out[2] = R;
        out[3] = n;
    }
}

int elementwise_grid(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    const int64_t most = 64 * (int64_t)device_sms();  // grid-stride loops beyond this
    return (int)(b < most ? (b < 1 ? 1 : b) : most);
}

}  // namespace

cudaError_t launch_displacement(const Grid &g, const Lattice &L, const float *ctrl, float *disp,
                                cudaStream_t s)
{
    dim3 grid((g.X + kDispTX - 1) / kDispTX, (g.Y + kDispTY - 1) / kDispTY, g.Z);
    if (g.ndim == 3)
        k_displacement<3><<<grid, kDispTX, 0, s>>>(g, L, ctrl, disp);
    else
        k_displacement<2><<<grid, kDispTX, 0, s>>>(g, L, ctrl, disp);
    return cudaGetLastError();
}

size_t displacement_adjoint_ws(const Grid &g, const Lattice &L)
{
    // t1: ndim x Z x Y x nx, t2: ndim x Z x ny x nx
    size_t t1 = (size_t)g.ndim * g.Z * g.Y * L.nx;
    size_t t2 = (size_t)g.ndim * g.Z * L.ny * L.nx;
    return ((t1 * 4 + 255) / 256) * 256 + ((t2 * 4 + 255) / 256) * 256;
}

cudaError_t launch_displacement_adjoint(const Grid &g, const Lattice &L, const float *grad_disp,
                                        float *grad_ctrl, void *ws, cudaStream_t s)
{
    const int D = g.ndim;
    float *t1 = (float *)ws;
    size_t t1n = (size_t)D * g.Z * g.Y * L.nx;
    float *t2 = (float *)((char *)ws + ((t1n * 4 + 255) / 256) * 256);
    const int th = 256;
    // x: (D*Z*Y, X, 1) -> (D*Z*Y, nx, 1)
    int64_t n1 = (int64_t)D * g.Z * g.Y * L.nx;
    k_bspline_transpose_axis<<<elementwise_grid(n1, th), th, 0, s>>>(
        grad_disp, t1, (int64_t)D * g.Z * g.Y, g.X, L.nx, 1, L);
    // y: (D*Z, Y, nx) -> (D*Z, ny, nx); in 2D this is the result
    float *ydst = (D == 3) ? t2 : grad_ctrl;
    int64_t n2 = (int64_t)D * g.Z * L.ny * L.nx;
    k_bspline_transpose_axis<<<elementwise_grid(n2, th), th, 0, s>>>(
        t1, ydst, (int64_t)D * g.Z, g.Y, L.ny, L.nx, L);
    if (D == 3) {
        // z: (D, Z, ny*nx) -> (D, nz, ny*nx)
        int64_t n3 = (int64_t)D * L.nz * L.ny * L.nx;
        k_bspline_transpose_axis<<<elementwise_grid(n3, th), th, 0, s>>>(
            t2, grad_ctrl, D, g.Z, L.nz, (int64_t)L.ny * L.nx, L);
    }
    return cudaGetLastError();
}

cudaError_t launch_warp(const Grid &g, const float *moving, const float *disp, float *warped,
                        uint8_t *mask, cudaStream_t s)
{
    const int th = 256;
    if (g.ndim == 3)
        k_warp<3><<<elementwise_grid(g.nv, th), th, 0, s>>>(g, moving, disp, warped, mask);
    else
        k_warp<2><<<elementwise_grid(g.nv, th), th, 0, s>>>(g, moving, disp, warped, mask);
    return cudaGetLastError();
}

cudaError_t launch_warp_adjoint(const Grid &g, const float *moving, const float *disp,
                                const uint8_t *mask, const float *grad_warped, float *grad_disp,
                                int accumulate, cudaStream_t s)
{
    const int th = 256;
    if (g.ndim == 3)
        k_warp_adjoint<3><<<elementwise_grid(g.nv, th), th, 0, s>>>(g, moving, disp, mask,
                                                                     grad_warped, grad_disp,
                                                                     accumulate);
    else
        k_warp_adjoint<2><<<elementwise_grid(g.nv, th), th, 0, s>>>(g, moving, disp, mask,
                                                                     grad_warped, grad_disp,
                                                                     accumulate);
    return cudaGetLastError();
}

size_t regulariser_ws(const Grid &g)
{
    size_t blocks = ((size_t)g.nv + 255) / 256;
    return blocks * sizeof(double);
}

cudaError_t launch_regulariser(const Grid &g, const float *disp, double weight, double *value_dev,
                               float *grad_disp, void *ws, cudaStream_t s)
{
    const int th = 256;
    const int blocks = (int)((g.nv + th - 1) / th);
    double *partials = (double *)ws;
    const float gscale = (float)(2.0 * weight / (double)g.nv);
    if (g.ndim == 3)
        k_regulariser<3><<<blocks, th, 0, s>>>(g, disp, gscale, grad_disp, partials);
    else
        k_regulariser<2><<<blocks, th, 0, s>>>(g, disp, gscale, grad_disp, partials);
    k_sum_partials<<<1, 1024, 0, s>>>(partials, blocks, 1.0 / (double)g.nv, value_dev);
    return cudaGetLastError();
}

cudaError_t launch_combine(const double *sim_value, const double *reg_value, double lambda,
                           double *out, cudaStream_t s)
{
    k_combine<<<1, 32, 0, s>>>(sim_value, reg_value, lambda, out);
    return cudaGetLastError();
}

AL_UNIT_ERROR_READER(unit_error_basic)

}  // namespace airgb
