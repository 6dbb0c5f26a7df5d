/*
 * FP64 CPU oracle for the layers of the learned initialisation: a 3D
 * convolutional encoder-decoder that maps a fixed/moving image pair to
 * cubic B-spline control coefficients, which the plain optimiser then
 * refines. The paper names learning-based registration as planned work
 * (Sec. I and Sec. V) but gives no network; the layers here are the plain
 * textbook definitions of a 3x3x3 convolution and its two adjoints.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it. It shares no code with the
 * CUDA path.
 *
 * Layout (channels last): a batch of nb volumes of D x H x W voxels with C
 * channels is element [b][z][y][x][c] at ((b*D + z)*H + y)*W*C + x*C + c.
 * Weights are w[co][t][ci] with tap t = (dz+1)*9 + (dy+1)*3 + (dx+1) for the
 * offsets dz, dy, dx in {-1, 0, 1}.
 *
 * The layer (cross-correlation, zero padding 1, stride s in {1, 2}):
 *   out[b][o][co] = bias[co] + sum_t sum_ci in[b][s*o + d_t][ci] * w[co][t][ci]
 * where in = 0 outside the grid and the output has (N - 1)/s + 1 voxels per
 * axis of N input voxels. With relu != 0 the result is max(out, 0).
 */
#include <stdint.h>
#include <string.h>

#define ALREF_OK 0
#define ALREF_ERR_ARG 1

static int64_t out_size(int64_t n, int stride) { return (n - 1) / stride + 1; }

static int check_args(int nb, const int64_t *dims, int cin, int cout, int stride)
{
    if (nb < 1 || cin < 1 || cout < 1 || (stride != 1 && stride != 2))
        return ALREF_ERR_ARG;
    for (int k = 0; k < 3; ++k)
        if (dims[k] < 1)
            return ALREF_ERR_ARG;
    return ALREF_OK;
}

/* Forward layer, the definition above summed term by term. dims = input
 * D, H, W. */
int alref_conv3d(int nb, const int64_t *dims, int cin, int cout, int stride, const double *in,
                 const double *w, const double *bias, int relu, double *out)
{
    if (check_args(nb, dims, cin, cout, stride) != ALREF_OK)
        return ALREF_ERR_ARG;
    const int64_t D = dims[0], H = dims[1], W = dims[2];
    const int64_t Do = out_size(D, stride), Ho = out_size(H, stride), Wo = out_size(W, stride);
    for (int b = 0; b < nb; ++b)
        for (int64_t oz = 0; oz < Do; ++oz)
            for (int64_t oy = 0; oy < Ho; ++oy)
                for (int64_t ox = 0; ox < Wo; ++ox)
                    for (int co = 0; co < cout; ++co) {
                        double acc = bias ? bias[co] : 0.0;
                        for (int t = 0; t < 27; ++t) {
                            const int64_t z = stride * oz + (t / 9 - 1);
                            const int64_t y = stride * oy + ((t / 3) % 3 - 1);
                            const int64_t x = stride * ox + (t % 3 - 1);
                            if (z < 0 || z >= D || y < 0 || y >= H || x < 0 || x >= W)
                                continue;
                            const double *src = in + (((b * D + z) * H + y) * W + x) * cin;
                            const double *wr = w + ((int64_t)co * 27 + t) * cin;
                            for (int ci = 0; ci < cin; ++ci)
                                acc += src[ci] * wr[ci];
                        }
                        if (relu && acc < 0.0)
                            acc = 0.0;
                        out[(((b * Do + oz) * Ho + oy) * Wo + ox) * cout + co] = acc;
                    }
    return ALREF_OK;
}

/* Adjoint with respect to the input (the transpose of the linear part of the
 * layer): every output term in[b][s*o + d_t][ci] * w[co][t][ci] sends
 * g_out[b][o][co] * w[co][t][ci] back to the input voxel it read. The result
 * overwrites g_in (input-sized). No ReLU factor is applied here. */
int alref_conv3d_dgrad(int nb, const int64_t *dims, int cin, int cout, int stride,
                       const double *g_out, const double *w, double *g_in)
{
    if (check_args(nb, dims, cin, cout, stride) != ALREF_OK)
        return ALREF_ERR_ARG;
    const int64_t D = dims[0], H = dims[1], W = dims[2];
    const int64_t Do = out_size(D, stride), Ho = out_size(H, stride), Wo = out_size(W, stride);
    memset(g_in, 0, sizeof(double) * (size_t)(nb * D * H * W * cin));
    for (int b = 0; b < nb; ++b)
        for (int64_t oz = 0; oz < Do; ++oz)
            for (int64_t oy = 0; oy < Ho; ++oy)
                for (int64_t ox = 0; ox < Wo; ++ox)
                    for (int co = 0; co < cout; ++co) {
                        const double g = g_out[(((b * Do + oz) * Ho + oy) * Wo + ox) * cout + co];
                        for (int t = 0; t < 27; ++t) {
                            const int64_t z = stride * oz + (t / 9 - 1);
                            const int64_t y = stride * oy + ((t / 3) % 3 - 1);
                            const int64_t x = stride * ox + (t % 3 - 1);
                            if (z < 0 || z >= D || y < 0 || y >= H || x < 0 || x >= W)
                                continue;
                            double *dst = g_in + (((b * D + z) * H + y) * W + x) * cin;
                            const double *wr = w + ((int64_t)co * 27 + t) * cin;
                            for (int ci = 0; ci < cin; ++ci)
                                dst[ci] += g * wr[ci];
                        }
                    }
    return ALREF_OK;
}

/* Adjoint with respect to the weights and the bias:
 *   g_w[co][t][ci] = sum_b sum_o g_out[b][o][co] * in[b][s*o + d_t][ci]
 *   g_b[co]        = sum_b sum_o g_out[b][o][co]
 * Both overwrite their outputs; g_b may be NULL. */
int alref_conv3d_wgrad(int nb, const int64_t *dims, int cin, int cout, int stride,
                       const double *in, const double *g_out, double *g_w, double *g_b)
{
    if (check_args(nb, dims, cin, cout, stride) != ALREF_OK)
        return ALREF_ERR_ARG;
    const int64_t D = dims[0], H = dims[1], W = dims[2];
    const int64_t Do = out_size(D, stride), Ho = out_size(H, stride), Wo = out_size(W, stride);
    memset(g_w, 0, sizeof(double) * (size_t)cout * 27 * cin);
    if (g_b)
        memset(g_b, 0, sizeof(double) * (size_t)cout);
    for (int b = 0; b < nb; ++b)
        for (int64_t oz = 0; oz < Do; ++oz)
            for (int64_t oy = 0; oy < Ho; ++oy)
                for (int64_t ox = 0; ox < Wo; ++ox)
                    for (int co = 0; co < cout; ++co) {
                        const double g = g_out[(((b * Do + oz) * Ho + oy) * Wo + ox) * cout + co];
                        if (g_b)
                            g_b[co] += g;
                        for (int t = 0; t < 27; ++t) {
                            const int64_t z = stride * oz + (t / 9 - 1);
                            const int64_t y = stride * oy + ((t / 3) % 3 - 1);
                            const int64_t x = stride * ox + (t % 3 - 1);
                            if (z < 0 || z >= D || y < 0 || y >= H || x < 0 || x >= W)
                                continue;
                            const double *src = in + (((b * D + z) * H + y) * W + x) * cin;
                            double *gw = g_w + ((int64_t)co * 27 + t) * cin;
                            for (int ci = 0; ci < cin; ++ci)
                                gw[ci] += g * src[ci];
                        }
                    }
    return ALREF_OK;
}
