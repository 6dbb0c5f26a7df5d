/*
 * FP64 CPU oracle for the regularised B-spline registration objective of
 * AIRLab (arXiv 1806.09907) and its gradient with respect to the control
 * points.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA library is checked against. Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it. It shares no code with
 * the CUDA path: no headers, helpers, tables or constants.
 *
 * Every routine computes in double precision, from double inputs (the
 * Python wrapper widens the fp32 arrays the GPU path consumes, which is
 * exact). Each routine states the passage of the paper it follows and the
 * reading taken where the paper is silent.
 *
 * Conventions (readings of the paper, stated once):
 *  - Grid: d in {2,3}; sizes N = (X, Y, Z), Z = 1 in 2D; voxel spacing 1;
 *    linear index (z*Y + y)*X + x, x fastest.
 *  - Vector fields are component planes: u[i][z][y][x], i < d, voxel units.
 *  - Control lattice (Sec. III-C, the B-spline kernel; placement is not
 *    given in the paper): spacing delta (integer); per active axis
 *    n_k = floor((N_k - 1)/delta) + 4 control points, point j at voxel
 *    coordinate p_j = (j - 1)*delta. In 2D n_z = 1. Coefficients are planes
 *    c[i][jz][jy][jx], voxel units.
 *  - The kernel argument is scaled by delta: k(x_j, x) = prod_k
 *    k_B1D((x_k - p_{j,k})/delta) (the spacing defines the kernel's extent,
 *    Sec. III-C).
 *  - Warp (Sec. III-C, Image Warping): y = x + u(x); a point is outside if
 *    any y_k < 0 or y_k > N_k - 1 (the strict test of the masking snippet,
 *    mapped from [-1,1] to voxel units with -1 -> 0 and +1 -> N_k - 1).
 *    A non-finite y_k counts as outside. Linear interpolation uses the floor
 *    cell clamped to [0, N_k - 2].
 *
 * "Parity pins": each routine is pinned by tests against closed forms,
 * invariants, library routines on special cases and central differences;
 * none is unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ALREF_OK 0
#define ALREF_ERR_ARG 1

/* ------------------------------------------------------------------------ */
/* The cubic B-spline kernel k_B1D of Sec. III-C (B-spline item):           */
/*   2/3 - |r|^2 + |r|^3/2   for 0 <= |r| < 1                               */
/*   (2 - |r|)^3 / 6         for 1 <= |r| < 2                               */
/*   0                       for 2 <= |r|                                   */
/* ------------------------------------------------------------------------ */
double alref_kernel_b3(double r)
{
    double a = fabs(r);
    if (a < 1.0)
        return 2.0 / 3.0 - a * a + a * a * a / 2.0;
    if (a < 2.0) {
        double t = 2.0 - a;
        return t * t * t / 6.0;
    }
    return 0.0;
}

/* Control-lattice size per axis (reading: n = floor((N-1)/delta) + 4). */
int alref_lattice_size(int ndim, const int64_t *N, int delta, int64_t *n)
{
    if ((ndim != 2 && ndim != 3) || delta < 1)
        return ALREF_ERR_ARG;
    for (int k = 0; k < 3; ++k) {
        if (k < ndim) {
            if (N[k] < 2)
                return ALREF_ERR_ARG;
            n[k] = (N[k] - 1) / delta + 4;
        } else {
            if (N[k] != 1)
                return ALREF_ERR_ARG;
            n[k] = 1;
        }
    }
    return ALREF_OK;
}

static int64_t nvox(const int64_t *N) { return N[0] * N[1] * N[2]; }

/* Kernel weight of control index j for voxel coordinate xk along an axis.
 * For an inactive axis (2D, z) the single plane has weight 1. */
static double axis_weight(int active, int64_t xk, int64_t j, int delta)
{
    if (!active)
        return 1.0;
    double pj = (double)(j - 1) * (double)delta;
    return alref_kernel_b3(((double)xk - pj) / (double)delta);
}

/* Range of control indices that can have a non-zero weight at xk: the kernel
 * vanishes for |r| >= 2, i.e. outside j in (xk/delta - 1, xk/delta + 3).
 * A generous window is used; the weight itself decides. */
static void axis_range(int active, int64_t xk, int delta, int64_t nk, int64_t *j0, int64_t *j1)
{
    if (!active) {
        *j0 = 0;
        *j1 = 0;
        return;
    }
    int64_t q = xk / delta;
    int64_t a = q - 1, b = q + 4;
    if (a < 0)
        a = 0;
    if (b > nk - 1)
        b = nk - 1;
    *j0 = a;
    *j1 = b;
}

/* ------------------------------------------------------------------------ */
/* Eq. (kernel_basis) with the B-spline basis: u_i(x) = sum_j c_{i,j} k(x_j,x). */
/* The sum runs over every control point whose kernel can be non-zero.      */
/* ------------------------------------------------------------------------ */
int alref_displacement(int ndim, const int64_t *N, int delta, const double *ctrl, double *disp)
{
    int64_t n[3];
    if (alref_lattice_size(ndim, N, delta, n))
        return ALREF_ERR_ARG;
    const int64_t X = N[0], Y = N[1], Z = N[2];
    const int64_t nc = n[0] * n[1] * n[2], nv = nvox(N);
    for (int64_t z = 0; z < Z; ++z)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t x = 0; x < X; ++x) {
                int64_t jx0, jx1, jy0, jy1, jz0, jz1;
                axis_range(1, x, delta, n[0], &jx0, &jx1);
                axis_range(1, y, delta, n[1], &jy0, &jy1);
                axis_range(ndim == 3, z, delta, n[2], &jz0, &jz1);
                /* the kernel is a tensor product: k = kx(jx) * ky(jy) * kz(jz) */
                double kx[8], ky[8], kz[8];
                for (int64_t j = jx0; j <= jx1; ++j)
                    kx[j - jx0] = axis_weight(1, x, j, delta);
                for (int64_t j = jy0; j <= jy1; ++j)
                    ky[j - jy0] = axis_weight(1, y, j, delta);
                for (int64_t j = jz0; j <= jz1; ++j)
                    kz[j - jz0] = axis_weight(ndim == 3, z, j, delta);
                for (int i = 0; i < ndim; ++i) {
                    double acc = 0.0;
                    for (int64_t jz = jz0; jz <= jz1; ++jz)
                        for (int64_t jy = jy0; jy <= jy1; ++jy)
                            for (int64_t jx = jx0; jx <= jx1; ++jx) {
                                double k = kx[jx - jx0] * ky[jy - jy0] * kz[jz - jz0];
                                acc += ctrl[i * nc + (jz * n[1] + jy) * n[0] + jx] * k;
                            }
                    disp[i * nv + (z * Y + y) * X + x] = acc;
                }
            }
    return ALREF_OK;
}

/* Transpose of the expansion above (the adjoint of the up-sampling by
 * transposed convolution, Sec. III-C): g_c[i,j] = sum_x k(x_j,x) g_u[i](x). */
int alref_displacement_adjoint(int ndim, const int64_t *N, int delta, const double *g_disp,
                               double *g_ctrl)
{
    int64_t n[3];
    if (alref_lattice_size(ndim, N, delta, n))
        return ALREF_ERR_ARG;
    const int64_t X = N[0], Y = N[1], Z = N[2];
    const int64_t nc = n[0] * n[1] * n[2], nv = nvox(N);
    for (int64_t i = 0; i < ndim * nc; ++i)
        g_ctrl[i] = 0.0;
    for (int64_t z = 0; z < Z; ++z)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t x = 0; x < X; ++x) {
                int64_t jx0, jx1, jy0, jy1, jz0, jz1;
                axis_range(1, x, delta, n[0], &jx0, &jx1);
                axis_range(1, y, delta, n[1], &jy0, &jy1);
                axis_range(ndim == 3, z, delta, n[2], &jz0, &jz1);
                double kx[8], ky[8], kz[8];
                for (int64_t j = jx0; j <= jx1; ++j)
                    kx[j - jx0] = axis_weight(1, x, j, delta);
                for (int64_t j = jy0; j <= jy1; ++j)
                    ky[j - jy0] = axis_weight(1, y, j, delta);
                for (int64_t j = jz0; j <= jz1; ++j)
                    kz[j - jz0] = axis_weight(ndim == 3, z, j, delta);
                for (int64_t jz = jz0; jz <= jz1; ++jz)
                    for (int64_t jy = jy0; jy <= jy1; ++jy)
                        for (int64_t jx = jx0; jx <= jx1; ++jx) {
                            double k = kx[jx - jx0] * ky[jy - jy0] * kz[jz - jz0];
                            if (k == 0.0)
                                continue;
                            for (int i = 0; i < ndim; ++i)
                                g_ctrl[i * nc + (jz * n[1] + jy) * n[0] + jx] +=
                                    k * g_disp[i * nv + (z * Y + y) * X + x];
                        }
            }
    return ALREF_OK;
}

/* ------------------------------------------------------------------------ */
/* Backward warp with the out-of-domain mask and linear interpolation       */
/* (Sec. III-C, Image Warping). Also returns the derivative of the          */
/* interpolant with respect to the sample position, needed by the exact     */
/* gradient (Sec. III-A): zero where the point is outside.                   */
/*   warped[v] = m(v) * M~(y(v)), mask[v] = m(v), grad_y[k][v] = dM~/dy_k.   */
/* grad_y may be NULL.                                                       */
/* ------------------------------------------------------------------------ */
int alref_warp(int ndim, const int64_t *N, const double *moving, const double *disp,
               double *warped, uint8_t *mask, double *grad_y)
{
    if ((ndim != 2 && ndim != 3) || N[0] < 2 || N[1] < 2 || (ndim == 3 && N[2] < 2) ||
        (ndim == 2 && N[2] != 1))
        return ALREF_ERR_ARG;
    const int64_t X = N[0], Y = N[1], Z = N[2], nv = nvox(N);
    for (int64_t z = 0; z < Z; ++z)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t x = 0; x < X; ++x) {
                const int64_t v = (z * Y + y) * X + x;
                double p[3] = {(double)x, (double)y, (double)z};
                int inside = 1;
                for (int k = 0; k < ndim; ++k) {
                    p[k] += disp[k * nv + v];
                    /* outside iff p > N-1 or p < 0; NaN fails both tests below */
                    if (!(p[k] >= 0.0 && p[k] <= (double)(N[k] - 1)))
                        inside = 0;
                }
                mask[v] = (uint8_t)inside;
                if (!inside) {
                    warped[v] = 0.0;
                    if (grad_y)
                        for (int k = 0; k < ndim; ++k)
                            grad_y[k * nv + v] = 0.0;
                    continue;
                }
                int64_t c[3] = {0, 0, 0};
                double f[3] = {0.0, 0.0, 0.0};
                for (int k = 0; k < ndim; ++k) {
                    int64_t i0 = (int64_t)floor(p[k]);
                    if (i0 > N[k] - 2)
                        i0 = N[k] - 2;
                    if (i0 < 0)
                        i0 = 0;
                    c[k] = i0;
                    f[k] = p[k] - (double)i0;
                }
                double val = 0.0, g[3] = {0.0, 0.0, 0.0};
                const int ncorner = ndim == 3 ? 8 : 4;
                for (int corner = 0; corner < ncorner; ++corner) {
                    int b[3] = {corner & 1, (corner >> 1) & 1, (corner >> 2) & 1};
                    double wk[3], dk[3];
                    for (int k = 0; k < 3; ++k) {
                        if (k < ndim) {
                            wk[k] = b[k] ? f[k] : 1.0 - f[k];
                            dk[k] = b[k] ? 1.0 : -1.0;
                        } else {
                            wk[k] = 1.0;
                            dk[k] = 0.0;
                        }
                    }
                    int64_t zz = c[2] + (ndim == 3 ? b[2] : 0);
                    double m = moving[(zz * Y + (c[1] + b[1])) * X + (c[0] + b[0])];
                    val += wk[0] * wk[1] * wk[2] * m;
                    g[0] += dk[0] * wk[1] * wk[2] * m;
                    g[1] += wk[0] * dk[1] * wk[2] * m;
                    g[2] += wk[0] * wk[1] * dk[2] * m;
                }
                warped[v] = val;
                if (grad_y)
                    for (int k = 0; k < ndim; ++k)
                        grad_y[k * nv + v] = g[k];
            }
    return ALREF_OK;
}

/* ------------------------------------------------------------------------ */
/* Similarity measures (Sec. III-B). Each returns S and dS/dW per voxel.     */
/* g_w may be NULL (value only).                                             */
/* ------------------------------------------------------------------------ */

/* Eq. (mse): mean of squared differences, taken over the points inside the
 * mask (reading: the mask of the warping snippet drops outside points, so
 * the mean runs over |X_m|). */
int alref_mse(const int64_t *N, const double *fixed, const double *warped, const uint8_t *mask,
              double *S, double *g_w)
{
    const int64_t nv = nvox(N);
    double cnt = 0.0, sum = 0.0;
    for (int64_t v = 0; v < nv; ++v)
        if (mask[v]) {
            double d = warped[v] - fixed[v];
            sum += d * d;
            cnt += 1.0;
        }
    *S = cnt > 0.0 ? sum / cnt : 0.0;
    if (g_w)
        for (int64_t v = 0; v < nv; ++v)
            g_w[v] = (mask[v] && cnt > 0.0) ? 2.0 * (warped[v] - fixed[v]) / cnt : 0.0;
    return ALREF_OK;
}

/* NCC (Sec. III-B). The printed formula is garbled; reading: the Pearson
 * correlation over the masked points,
 *   rho = sum (F-muF)(W-muW) / sqrt(sum (F-muF)^2 * sum (W-muW)^2 + eps),
 * and S = 1 - rho (zero for identical images). */
int alref_ncc(const int64_t *N, const double *fixed, const double *warped, const uint8_t *mask,
              double eps, double *S, double *g_w)
{
    const int64_t nv = nvox(N);
    double cnt = 0.0, sf = 0.0, sw = 0.0;
    for (int64_t v = 0; v < nv; ++v)
        if (mask[v]) {
            cnt += 1.0;
            sf += fixed[v];
            sw += warped[v];
        }
    if (cnt == 0.0) {
        *S = 0.0;
        if (g_w)
            for (int64_t v = 0; v < nv; ++v)
                g_w[v] = 0.0;
        return ALREF_OK;
    }
    double muf = sf / cnt, muw = sw / cnt;
    double cov = 0.0, vf = 0.0, vw = 0.0;
    for (int64_t v = 0; v < nv; ++v)
        if (mask[v]) {
            double a = fixed[v] - muf, b = warped[v] - muw;
            cov += a * b;
            vf += a * a;
            vw += b * b;
        }
    double D = vf * vw + eps;
    double rho = cov / sqrt(D);
    *S = 1.0 - rho;
    if (g_w)
        for (int64_t v = 0; v < nv; ++v) {
            if (!mask[v]) {
                g_w[v] = 0.0;
                continue;
            }
            /* d rho / d W(v): the mean terms drop out because the centred
             * values sum to zero over the mask. */
            double drho = (fixed[v] - muf) / sqrt(D) - cov * vf * (warped[v] - muw) / (D * sqrt(D));
            g_w[v] = -drho;
        }
    return ALREF_OK;
}

/* LCC (Sec. III-B): NCC with mean and variance taken in a local window.
 * Readings: a centred box window of odd width w (w^d voxels), zero padding
 * outside the grid, n = w^d constant (plain convolution with a box of ones);
 * W is zero where the mask is off (it enters the sums as zero);
 *   cov = S_FW - S_F S_W / n, var_F = S_FF - S_F^2/n, var_W likewise,
 *   rho(x) = cov / sqrt(var_F var_W + eps),
 *   S = 1 - (1/|X_m|) sum_{x in mask} rho(x).
 * The gradient is exact (Sec. III-B: no approximation): with
 *   a(x) = dS/dS_W(x), b(x) = dS/dS_WW(x), c(x) = dS/dS_FW(x) (zero off mask),
 *   dS/dW(y) = sum_{x: y in window(x)} [a(x) + 2 W(y) b(x) + F(y) c(x)],
 * and the window is symmetric, so the sum runs over the window of y. */
static double box_sum(int ndim, const int64_t *N, const double *f, int64_t x, int64_t y, int64_t z,
                      int r)
{
    const int64_t X = N[0], Y = N[1], Z = N[2];
    double s = 0.0;
    int rz = ndim == 3 ? r : 0;
    for (int64_t dz = -rz; dz <= rz; ++dz)
        for (int64_t dy = -r; dy <= r; ++dy)
            for (int64_t dx = -r; dx <= r; ++dx) {
                int64_t xx = x + dx, yy = y + dy, zz = z + dz;
                if (xx < 0 || xx >= X || yy < 0 || yy >= Y || zz < 0 || zz >= Z)
                    continue; /* zero padding */
                s += f[(zz * Y + yy) * X + xx];
            }
    return s;
}

int alref_lcc(int ndim, const int64_t *N, const double *fixed, const double *warped,
              const uint8_t *mask, int window, double eps, double *S, double *g_w)
{
    if (window < 1 || (window % 2) == 0 || (ndim != 2 && ndim != 3))
        return ALREF_ERR_ARG;
    const int64_t X = N[0], Y = N[1], Z = N[2], nv = nvox(N);
    const int r = window / 2;
    const double n = ndim == 3 ? (double)window * window * window : (double)window * window;
    double *w = (double *)malloc(sizeof(double) * nv);
    double *ff = (double *)malloc(sizeof(double) * nv);
    double *ww = (double *)malloc(sizeof(double) * nv);
    double *fw = (double *)malloc(sizeof(double) * nv);
    double *ca = (double *)malloc(sizeof(double) * nv);
    double *cb = (double *)malloc(sizeof(double) * nv);
    double *cc = (double *)malloc(sizeof(double) * nv);
    if (!w || !ff || !ww || !fw || !ca || !cb || !cc) {
        free(w), free(ff), free(ww), free(fw), free(ca), free(cb), free(cc);
        return ALREF_ERR_ARG;
    }
    double cnt = 0.0;
    for (int64_t v = 0; v < nv; ++v) {
        w[v] = mask[v] ? warped[v] : 0.0;
        ff[v] = fixed[v] * fixed[v];
        ww[v] = w[v] * w[v];
        fw[v] = fixed[v] * w[v];
        if (mask[v])
            cnt += 1.0;
    }
    double rho_sum = 0.0;
    for (int64_t z = 0; z < Z; ++z)
        for (int64_t y = 0; y < Y; ++y)
            for (int64_t x = 0; x < X; ++x) {
                const int64_t v = (z * Y + y) * X + x;
                ca[v] = cb[v] = cc[v] = 0.0;
                if (!mask[v])
                    continue;
                double SF = box_sum(ndim, N, fixed, x, y, z, r);
                double SW = box_sum(ndim, N, w, x, y, z, r);
                double SFF = box_sum(ndim, N, ff, x, y, z, r);
                double SWW = box_sum(ndim, N, ww, x, y, z, r);
                double SFW = box_sum(ndim, N, fw, x, y, z, r);
                double cov = SFW - SF * SW / n;
                double vf = SFF - SF * SF / n;
                double vw = SWW - SW * SW / n;
                double D = vf * vw + eps;
                double sD = sqrt(D);
                double rho = cov / sD;
                rho_sum += rho;
                /* partial derivatives of rho with respect to the three local
                 * sums that depend on W */
                double d_sfw = 1.0 / sD;
                double d_sww = -cov * vf / (2.0 * D * sD);
                double d_sw = -SF / (n * sD) + cov * vf * SW / (n * D * sD);
                /* S = 1 - rho_sum / cnt */
                ca[v] = -d_sw / cnt;
                cb[v] = -d_sww / cnt;
                cc[v] = -d_sfw / cnt;
            }
    *S = cnt > 0.0 ? 1.0 - rho_sum / cnt : 0.0;
    if (g_w) {
        for (int64_t z = 0; z < Z; ++z)
            for (int64_t y = 0; y < Y; ++y)
                for (int64_t x = 0; x < X; ++x) {
                    const int64_t v = (z * Y + y) * X + x;
                    if (!mask[v] || cnt == 0.0) {
                        g_w[v] = 0.0;
                        continue;
                    }
                    double A = box_sum(ndim, N, ca, x, y, z, r);
                    double B = box_sum(ndim, N, cb, x, y, z, r);
                    double C = box_sum(ndim, N, cc, x, y, z, r);
                    g_w[v] = A + 2.0 * w[v] * B + fixed[v] * C;
                }
    }
    free(w), free(ff), free(ww), free(fw), free(ca), free(cb), free(cc);
    return ALREF_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. (diffusion_regularizer): R = (1/|X|) sum_x sum_i ||grad u_i(x)||^2.  */
/* Reading: forward differences with unit spacing; the difference that      */
/* would leave the grid is dropped (Neumann). g_disp = dR/du, may be NULL.   */
/* ------------------------------------------------------------------------ */
int alref_diffusion(int ndim, const int64_t *N, const double *disp, double *R, double *g_disp)
{
    const int64_t X = N[0], Y = N[1], Z = N[2], nv = nvox(N);
    const int64_t stride[3] = {1, X, X * Y};
    double sum = 0.0;
    if (g_disp)
        for (int64_t v = 0; v < ndim * nv; ++v)
            g_disp[v] = 0.0;
    for (int i = 0; i < ndim; ++i) {
        const double *u = disp + i * nv;
        for (int64_t z = 0; z < Z; ++z)
            for (int64_t y = 0; y < Y; ++y)
                for (int64_t x = 0; x < X; ++x) {
                    const int64_t v = (z * Y + y) * X + x;
                    const int64_t pos[3] = {x, y, z};
                    for (int k = 0; k < ndim; ++k) {
                        if (pos[k] + 1 >= N[k])
                            continue;
                        double d = u[v + stride[k]] - u[v];
                        sum += d * d;
                        if (g_disp) {
                            g_disp[i * nv + v + stride[k]] += 2.0 * d / (double)nv;
                            g_disp[i * nv + v] -= 2.0 * d / (double)nv;
                        }
                    }
                }
    }
    *R = sum / (double)nv;
    return ALREF_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. (objective) for one control-point vector, with its exact gradient    */
/* by the chain rule (Sec. III-A):                                           */
/*   u = B c; (W, m) = warp(M, u); S = S(W, F); R = R_diff(u); J = S + lam R */
/*   g_u = m * dS/dW * dM~/dy + lam * dR/du;  dJ/dc = B^T g_u               */
/* kind: 0 = MSE, 1 = NCC, 2 = LCC. out = {J, S, R, |X_m|}. g_ctrl NULL =    */
/* value only.                                                               */
/* ------------------------------------------------------------------------ */
int alref_objective_grad_ex(int ndim, const int64_t *N, int delta, int kind, int window,
                            double eps, double lambda, const double *fixed, const double *moving,
                            const double *ctrl, double *out, double *g_ctrl, double *u_out,
                            double *gw_out);

int alref_objective_grad(int ndim, const int64_t *N, int delta, int kind, int window, double eps,
                         double lambda, const double *fixed, const double *moving,
                         const double *ctrl, double *out, double *g_ctrl)
{
    return alref_objective_grad_ex(ndim, N, delta, kind, window, eps, lambda, fixed, moving, ctrl,
                                   out, g_ctrl, NULL, NULL);
}

/* Same, also returning the displacement u (ndim planes) and dS/dW per voxel
 * when u_out / gw_out are not NULL (test diagnostics). */
int alref_objective_grad_ex(int ndim, const int64_t *N, int delta, int kind, int window,
                            double eps, double lambda, const double *fixed, const double *moving,
                            const double *ctrl, double *out, double *g_ctrl, double *u_out,
                            double *gw_out)
{
    int64_t n[3];
    if (alref_lattice_size(ndim, N, delta, n))
        return ALREF_ERR_ARG;
    const int64_t nv = nvox(N);
    double *u = (double *)malloc(sizeof(double) * ndim * nv);
    double *w = (double *)malloc(sizeof(double) * nv);
    double *gy = (double *)malloc(sizeof(double) * ndim * nv);
    double *gw = (double *)malloc(sizeof(double) * nv);
    double *gu = (double *)malloc(sizeof(double) * ndim * nv);
    uint8_t *m = (uint8_t *)malloc(nv);
    int st = ALREF_ERR_ARG;
    if (!u || !w || !gy || !gw || !gu || !m)
        goto done;
    if ((st = alref_displacement(ndim, N, delta, ctrl, u)))
        goto done;
    if ((st = alref_warp(ndim, N, moving, u, w, m, gy)))
        goto done;
    double S = 0.0, R = 0.0;
    if (kind == 0)
        st = alref_mse(N, fixed, w, m, &S, gw);
    else if (kind == 1)
        st = alref_ncc(N, fixed, w, m, eps, &S, gw);
    else if (kind == 2)
        st = alref_lcc(ndim, N, fixed, w, m, window, eps, &S, gw);
    else
        st = ALREF_ERR_ARG;
    if (st)
        goto done;
    if ((st = alref_diffusion(ndim, N, u, &R, gu)))
        goto done;
    double cnt = 0.0;
    for (int64_t v = 0; v < nv; ++v)
        cnt += m[v];
    out[0] = S + lambda * R;
    out[1] = S;
    out[2] = R;
    out[3] = cnt;
    if (u_out)
        memcpy(u_out, u, sizeof(double) * ndim * nv);
    if (gw_out)
        memcpy(gw_out, gw, sizeof(double) * nv);
    if (g_ctrl) {
        for (int i = 0; i < ndim; ++i)
            for (int64_t v = 0; v < nv; ++v)
                gu[i * nv + v] = (m[v] ? gw[v] * gy[i * nv + v] : 0.0) + lambda * gu[i * nv + v];
        st = alref_displacement_adjoint(ndim, N, delta, gu, g_ctrl);
    }
done:
    free(u), free(w), free(gy), free(gw), free(gu), free(m);
    return st;
}

/* ======================================================================== */
/* The optimisation loop around the objective: Adam on the control points,  */
/* the Gaussian image pyramid of a multi-resolution registration and the    */
/* dyadic refinement of the B-spline coefficients between its levels.       */
/* ======================================================================== */

/* One Adam step (Sec. II-A, Optimization, and Sec. III-G name Adam; the
 * update is the one Kingma and Ba define) on the control coefficients.
 * Reading: the step size lr is in the paper's normalised coordinates
 * (Sec. III-C, Image Warping: the image spans [-1, 1] per axis), so Adam runs
 * on c~_k = c_k * 2/(N_k - 1); ctrl and grad are in voxel units and m, v hold
 * the moments of the normalised gradient dJ/dc~_k = dJ/dc_k * (N_k - 1)/2.
 * With t = step (>= 1):
 *   m <- beta1 m + (1 - beta1) g~,  v <- beta2 v + (1 - beta2) g~^2
 *   c~ <- c~ - lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)
 */
int alref_adam_step(int ndim, const int64_t *N, int delta, double lr, double beta1, double beta2,
                    double eps, int64_t step, double *ctrl, const double *grad, double *m,
                    double *v)
{
    int64_t n[3];
    if (alref_lattice_size(ndim, N, delta, n) || step < 1)
        return ALREF_ERR_ARG;
    const int64_t nc = n[0] * n[1] * n[2];
    const double bc1 = 1.0 - pow(beta1, (double)step);
    const double bc2 = 1.0 - pow(beta2, (double)step);
    for (int i = 0; i < ndim; ++i) {
        const double to_norm = 2.0 / (double)(N[i] - 1); /* voxel -> normalised */
        for (int64_t j = 0; j < nc; ++j) {
            const int64_t e = i * nc + j;
            const double g = grad[e] / to_norm; /* dJ/dc~ */
            m[e] = beta1 * m[e] + (1.0 - beta1) * g;
            v[e] = beta2 * v[e] + (1.0 - beta2) * g * g;
            const double mhat = m[e] / bc1, vhat = v[e] / bc2;
            double cn = ctrl[e] * to_norm;
            cn -= lr * mhat / (sqrt(vhat) + eps);
            ctrl[e] = cn / to_norm;
        }
    }
    return ALREF_OK;
}

/* Output size of a pyramid level along one axis: the points 0, f, 2f, ...
 * of the finer grid. */
static int64_t level_size(int64_t Nk, int factor) { return (Nk - 1) / factor + 1; }

/* One level of the Gaussian image pyramid used by the multi-resolution
 * strategy of Sec. IV-A (FFD item); the paper gives no filter, so the
 * reading is: factor f = 1 is the image itself; for f >= 2 the image is
 * smoothed by a Gaussian of sigma = f/2 voxels, truncated to the taps with
 * |t| <= 3 sigma and normalised to unit sum, with indices clamped to the
 * grid, and sampled at every f-th voxel starting at voxel 0 on each active
 * axis. Computed as the full d-dimensional sum of the product kernel at
 * every output point. out: level_size per active axis. */
int alref_pyramid_level(int ndim, const int64_t *N, const double *image, int factor, double *out)
{
    if ((ndim != 2 && ndim != 3) || factor < 1 || factor > 8)
        return ALREF_ERR_ARG;
    int64_t M[3];
    for (int k = 0; k < 3; ++k) {
        if (k < ndim ? N[k] < 2 : N[k] != 1)
            return ALREF_ERR_ARG;
        M[k] = k < ndim ? level_size(N[k], factor) : 1;
    }
    if (factor == 1) {
        memcpy(out, image, sizeof(double) * nvox(N));
        return ALREF_OK;
    }
    const double sigma = factor / 2.0;
    const int r = (int)floor(3.0 * sigma);
    double w[64];
    double wsum = 0.0;
    for (int t = -r; t <= r; ++t) {
        w[t + r] = exp(-(double)(t * t) / (2.0 * sigma * sigma));
        wsum += w[t + r];
    }
    for (int t = -r; t <= r; ++t)
        w[t + r] /= wsum;
    const int rz = ndim == 3 ? r : 0;
    for (int64_t oz = 0; oz < M[2]; ++oz)
        for (int64_t oy = 0; oy < M[1]; ++oy)
            for (int64_t ox = 0; ox < M[0]; ++ox) {
                double s = 0.0;
                for (int tz = -rz; tz <= rz; ++tz) {
                    int64_t z = oz * factor + tz;
                    z = z < 0 ? 0 : (z > N[2] - 1 ? N[2] - 1 : z);
                    const double wz = ndim == 3 ? w[tz + r] : 1.0;
                    for (int ty = -r; ty <= r; ++ty) {
                        int64_t y = oy * factor + ty;
                        y = y < 0 ? 0 : (y > N[1] - 1 ? N[1] - 1 : y);
                        for (int tx = -r; tx <= r; ++tx) {
                            int64_t x = ox * factor + tx;
                            x = x < 0 ? 0 : (x > N[0] - 1 ? N[0] - 1 : x);
                            s += wz * w[ty + r] * w[tx + r] * image[(z * N[1] + y) * N[0] + x];
                        }
                    }
                }
                out[(oz * M[1] + oy) * M[0] + ox] = s;
            }
    return ALREF_OK;
}

/* Two-scale coefficient of the cubic B-spline: beta3(x) =
 * sum_o h(o) beta3(2x - o) with h = (1, 4, 6, 4, 1)/8 for o = -2..2. */
static double two_scale(int64_t o)
{
    switch (o) {
    case -2: case 2: return 1.0 / 8.0;
    case -1: case 1: return 4.0 / 8.0;
    case 0: return 6.0 / 8.0;
    default: return 0.0;
    }
}

/* Coefficients on the finer level of the pyramid from those of the coarser
 * one, such that the fine displacement equals the coarse one exactly
 * (Sec. IV-A, multi-resolution; the transfer is a reading). The coarse grid
 * is the fine grid sampled at every second voxel, both lattices have the same
 * spacing delta in their own voxels, so a coarse basis function is a fine
 * one dilated by 2 and, by the two-scale relation, a sum of five fine basis
 * functions: fine point i sits at (i - 1) delta fine voxels and coarse point
 * j at 2 (j - 1) delta, hence
 *   c_fine[i] = 2 * sum_j prod_k h((i_k - 1) - 2 (j_k - 1)) c_coarse[j]
 * (the factor 2 converts coarse voxel units to fine ones). Every fine
 * coefficient is the full sum over the coarse lattice. */
int alref_bspline_refine(int ndim, const int64_t *Nc, const int64_t *Nf, int delta,
                         const double *c_coarse, double *c_fine)
{
    int64_t nc[3], nf[3];
    if (alref_lattice_size(ndim, Nc, delta, nc) || alref_lattice_size(ndim, Nf, delta, nf))
        return ALREF_ERR_ARG;
    for (int k = 0; k < ndim; ++k)
        if (level_size(Nf[k], 2) != Nc[k])
            return ALREF_ERR_ARG;
    const int64_t ncc = nc[0] * nc[1] * nc[2], nff = nf[0] * nf[1] * nf[2];
    for (int i = 0; i < ndim; ++i)
        for (int64_t fz = 0; fz < nf[2]; ++fz)
            for (int64_t fy = 0; fy < nf[1]; ++fy)
                for (int64_t fx = 0; fx < nf[0]; ++fx) {
                    double s = 0.0;
                    for (int64_t jz = 0; jz < nc[2]; ++jz) {
                        const double hz = ndim == 3 ? two_scale((fz - 1) - 2 * (jz - 1)) : 1.0;
                        if (hz == 0.0)
                            continue;
                        for (int64_t jy = 0; jy < nc[1]; ++jy) {
                            const double hy = two_scale((fy - 1) - 2 * (jy - 1));
                            if (hy == 0.0)
                                continue;
                            for (int64_t jx = 0; jx < nc[0]; ++jx)
                                s += hz * hy * two_scale((fx - 1) - 2 * (jx - 1)) *
                                     c_coarse[i * ncc + (jz * nc[1] + jy) * nc[0] + jx];
                        }
                    }
                    c_fine[i * nff + (fz * nf[1] + fy) * nf[0] + fx] = 2.0 * s;
                }
    return ALREF_OK;
}

/* ======================================================================== */
/* Diffeomorphic B-spline transformation (Sec. III-D): f = exp(v) of the     */
/* stationary velocity field v = sum_j c_j k(x_j, x), by scaling and         */
/* squaring (the method of the works the section cites; the number of        */
/* squarings K is a reading, the paper gives none):                          */
/*   u_0 = v / 2^K,  u_{k+1}(x) = u_k(x) + u~_k(x + u_k(x)),  f = x + u_K.   */
/* u~_k is the linear interpolant of u_k at a position clamped to the grid   */
/* [0, N-1] per axis (a field has no mask; reading); the floor cell is       */
/* clamped to [0, N-2].                                                      */
/* ======================================================================== */

/* Cell and offset of the clamped position p along an axis of n points, and
 * whether p was inside [0, n-1] (outside, the interpolant is constant along
 * that axis, so its derivative there is 0). */
static int field_cell(double p, int64_t n, int64_t *cell, double *f)
{
    int inside = 1;
    if (!(p >= 0.0)) { /* also NaN */
        p = 0.0;
        inside = 0;
    } else if (p > (double)(n - 1)) {
        p = (double)(n - 1);
        inside = 0;
    }
    int64_t c = (int64_t)floor(p);
    if (c > n - 2)
        c = n - 2;
    *cell = c;
    *f = p - (double)c;
    return inside;
}

/* Linear interpolation of the ndim component planes of u at position p
 * (x, y[, z]): value out[i]; derivative d[i][a] = d out[i] / d p_a (zero
 * along clamped axes). Corner weights are products of (1 - f) and f. */
static void field_sample(int ndim, const int64_t *N, const double *u, const double *p,
                         double *out, double d[3][3], int64_t cell[3], double frac[3], int in[3])
{
    const int64_t nv = nvox(N);
    for (int a = 0; a < 3; ++a) {
        if (a < ndim) {
            in[a] = field_cell(p[a], N[a], &cell[a], &frac[a]);
        } else {
            cell[a] = 0;
            frac[a] = 0.0;
            in[a] = 0;
        }
    }
    for (int i = 0; i < ndim; ++i) {
        out[i] = 0.0;
        for (int a = 0; a < 3; ++a)
            d[i][a] = 0.0;
        const int nz = ndim == 3 ? 2 : 1;
        for (int cz = 0; cz < nz; ++cz)
            for (int cy = 0; cy < 2; ++cy)
                for (int cx = 0; cx < 2; ++cx) {
                    const double wx = cx ? frac[0] : 1.0 - frac[0];
                    const double wy = cy ? frac[1] : 1.0 - frac[1];
                    const double wz = ndim == 3 ? (cz ? frac[2] : 1.0 - frac[2]) : 1.0;
                    const int64_t v = ((cell[2] + cz) * N[1] + cell[1] + cy) * N[0] + cell[0] + cx;
                    const double val = u[i * nv + v];
                    out[i] += wx * wy * wz * val;
                    /* derivative of each weight factor: d(1-f)/dp = -1, df/dp = +1 */
                    d[i][0] += (cx ? 1.0 : -1.0) * wy * wz * val;
                    d[i][1] += (cy ? 1.0 : -1.0) * wx * wz * val;
                    if (ndim == 3)
                        d[i][2] += (cz ? 1.0 : -1.0) * wx * wy * val;
                }
        for (int a = 0; a < ndim; ++a)
            if (!in[a])
                d[i][a] = 0.0;
    }
}

/* f = exp(v): u_out = u_K (ndim planes). traj (nullable) receives u_0 ..
 * u_{K-1}, the inputs of the K squarings, K * ndim * nv doubles. */
int alref_exp_field(int ndim, const int64_t *N, int K, const double *v, double *u_out,
                    double *traj)
{
    if ((ndim != 2 && ndim != 3) || K < 0 || K > 30)
        return ALREF_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (a < ndim ? N[a] < 2 : N[a] != 1)
            return ALREF_ERR_ARG;
    const int64_t nv = nvox(N);
    double *cur = (double *)malloc(sizeof(double) * ndim * nv);
    double *nxt = (double *)malloc(sizeof(double) * ndim * nv);
    if (!cur || !nxt) {
        free(cur), free(nxt);
        return ALREF_ERR_ARG;
    }
    const double s = ldexp(1.0, -K);
    for (int64_t e = 0; e < ndim * nv; ++e)
        cur[e] = v[e] * s;
    for (int k = 0; k < K; ++k) {
        if (traj)
            memcpy(traj + (int64_t)k * ndim * nv, cur, sizeof(double) * ndim * nv);
        for (int64_t z = 0; z < N[2]; ++z)
            for (int64_t y = 0; y < N[1]; ++y)
                for (int64_t x = 0; x < N[0]; ++x) {
                    const int64_t vox = (z * N[1] + y) * N[0] + x;
                    double p[3] = {(double)x, (double)y, (double)z}, out[3], d[3][3], fr[3];
                    int64_t cell[3];
                    int in[3];
                    for (int a = 0; a < ndim; ++a)
                        p[a] += cur[a * nv + vox];
                    field_sample(ndim, N, cur, p, out, d, cell, fr, in);
                    for (int i = 0; i < ndim; ++i)
                        nxt[i * nv + vox] = cur[i * nv + vox] + out[i];
                }
        double *t = cur;
        cur = nxt;
        nxt = t;
    }
    memcpy(u_out, cur, sizeof(double) * ndim * nv);
    free(cur), free(nxt);
    return ALREF_OK;
}

/* Adjoint of alref_exp_field: g_v = (d u_K / d v)^T g_u, from the
 * trajectory u_0 .. u_{K-1}. Per squaring, with p(x) = x + u_k(x):
 *   g_k(y) = g_{k+1}(y) + (d u~_k / d p at p(y))^T g_{k+1}(y)
 *            + sum_x w_y(p(x)) g_{k+1}(x),
 * the last sum the transpose of the interpolation (w_y the weight of node y);
 * then g_v = g_0 / 2^K. */
int alref_exp_field_adjoint(int ndim, const int64_t *N, int K, const double *traj,
                            const double *g_u, double *g_v)
{
    if ((ndim != 2 && ndim != 3) || K < 0 || K > 30)
        return ALREF_ERR_ARG;
    const int64_t nv = nvox(N);
    double *g = (double *)malloc(sizeof(double) * ndim * nv);
    double *h = (double *)malloc(sizeof(double) * ndim * nv);
    if (!g || !h) {
        free(g), free(h);
        return ALREF_ERR_ARG;
    }
    memcpy(g, g_u, sizeof(double) * ndim * nv);
    for (int k = K - 1; k >= 0; --k) {
        const double *u = traj + (int64_t)k * ndim * nv;
        memcpy(h, g, sizeof(double) * ndim * nv);
        for (int64_t z = 0; z < N[2]; ++z)
            for (int64_t y = 0; y < N[1]; ++y)
                for (int64_t x = 0; x < N[0]; ++x) {
                    const int64_t vox = (z * N[1] + y) * N[0] + x;
                    double p[3] = {(double)x, (double)y, (double)z}, out[3], d[3][3], fr[3];
                    int64_t cell[3];
                    int in[3];
                    for (int a = 0; a < ndim; ++a)
                        p[a] += u[a * nv + vox];
                    field_sample(ndim, N, u, p, out, d, cell, fr, in);
                    /* position term: u_k(x) moves the sample point */
                    for (int a = 0; a < ndim; ++a)
                        for (int i = 0; i < ndim; ++i)
                            h[a * nv + vox] += d[i][a] * g[i * nv + vox];
                    /* sampled-field term: scatter to the corners */
                    const int nz = ndim == 3 ? 2 : 1;
                    for (int cz = 0; cz < nz; ++cz)
                        for (int cy = 0; cy < 2; ++cy)
                            for (int cx = 0; cx < 2; ++cx) {
                                const double wx = cx ? fr[0] : 1.0 - fr[0];
                                const double wy = cy ? fr[1] : 1.0 - fr[1];
                                const double wz = ndim == 3 ? (cz ? fr[2] : 1.0 - fr[2]) : 1.0;
                                const int64_t node =
                                    ((cell[2] + cz) * N[1] + cell[1] + cy) * N[0] + cell[0] + cx;
                                for (int i = 0; i < ndim; ++i)
                                    h[i * nv + node] += wx * wy * wz * g[i * nv + vox];
                            }
                }
        double *t = g;
        g = h;
        h = t;
    }
    const double s = ldexp(1.0, -K);
    for (int64_t e = 0; e < ndim * nv; ++e)
        g_v[e] = g[e] * s;
    free(g), free(h);
    return ALREF_OK;
}

/* J = S(M o (x + u_K), F) + lambda R_diff(u_K) for the diffeomorphic
 * B-spline model, u_K = exp(v) - x with v the B-spline field of c, and
 * dJ/dc by the chain rule: A5 + A4 on u_K, the exponential's adjoint, A6. */
int alref_objective_grad_diffeo(int ndim, const int64_t *N, int delta, int K, int kind,
                                int window, double eps, double lambda, const double *fixed,
                                const double *moving, const double *ctrl, double *out,
                                double *g_ctrl)
{
    int64_t n[3];
    if (alref_lattice_size(ndim, N, delta, n) || K < 0 || K > 30)
        return ALREF_ERR_ARG;
    const int64_t nv = nvox(N);
    double *v = (double *)malloc(sizeof(double) * ndim * nv);
    double *u = (double *)malloc(sizeof(double) * ndim * nv);
    double *traj = (double *)malloc(sizeof(double) * (K > 0 ? K : 1) * ndim * nv);
    double *w = (double *)malloc(sizeof(double) * nv);
    double *gy = (double *)malloc(sizeof(double) * ndim * nv);
    double *gw = (double *)malloc(sizeof(double) * nv);
    double *gu = (double *)malloc(sizeof(double) * ndim * nv);
    double *gv = (double *)malloc(sizeof(double) * ndim * nv);
    uint8_t *m = (uint8_t *)malloc(nv);
    int st = ALREF_ERR_ARG;
    if (!v || !u || !traj || !w || !gy || !gw || !gu || !gv || !m)
        goto done;
    if ((st = alref_displacement(ndim, N, delta, ctrl, v)))
        goto done;
    if ((st = alref_exp_field(ndim, N, K, v, u, traj)))
        goto done;
    if ((st = alref_warp(ndim, N, moving, u, w, m, gy)))
        goto done;
    double S = 0.0, R = 0.0;
    if (kind == 0)
        st = alref_mse(N, fixed, w, m, &S, gw);
    else if (kind == 1)
        st = alref_ncc(N, fixed, w, m, eps, &S, gw);
    else if (kind == 2)
        st = alref_lcc(ndim, N, fixed, w, m, window, eps, &S, gw);
    else
        st = ALREF_ERR_ARG;
    if (st)
        goto done;
    if ((st = alref_diffusion(ndim, N, u, &R, gu)))
        goto done;
    double cnt = 0.0;
    for (int64_t e = 0; e < nv; ++e)
        cnt += m[e];
    out[0] = S + lambda * R;
    out[1] = S;
    out[2] = R;
    out[3] = cnt;
    if (g_ctrl) {
        for (int i = 0; i < ndim; ++i)
            for (int64_t e = 0; e < nv; ++e)
                gu[i * nv + e] = (m[e] ? gw[e] * gy[i * nv + e] : 0.0) + lambda * gu[i * nv + e];
        if ((st = alref_exp_field_adjoint(ndim, N, K, traj, gu, gv)))
            goto done;
        st = alref_displacement_adjoint(ndim, N, delta, gv, g_ctrl);
    }
done:
    free(v), free(u), free(traj), free(w), free(gy), free(gw), free(gu), free(gv), free(m);
    return st;
}
