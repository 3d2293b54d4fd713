/*
 * flr_oracle.c -- plain FP64 CPU oracle of Fast Local Regression (FLR),
 * arXiv 2410.11625 ("Fast Local Neural Regression for Low-Cost, Path Traced
 * Lambertian Global Illumination").
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this library.  The GPU library shares no code, header,
 * table or helper with it, and neither side includes or links the other.
 *
 * Everything is double precision, written for a reader who checks it against the
 * paper, with no blocking, fusion or reordering beyond what the paper states.
 *
 * Data layout: every image is planar, channel-major, row-major: plane c, row y,
 * column x lives at [(c * H + y) * W + x].  Inputs are float32 (what the GPU path
 * reads); all arithmetic is done after widening to double.
 *
 * Definition followed (Sec. 3.1, Eqs. matX/matY/argmin/closed_form; Sec. 3.2 box
 * window; Appendix moment decomposition):
 *   - X_k is the N x (Q+1) matrix of the guides inside the square window T_k of
 *     radius r around pixel k, first column all ones (Eq. matX); Y_k the N x 3
 *     radiance matrix (Eq. matY).  Windows are clipped to the image, so N = n_k
 *     counts in-image pixels only.
 *   - Box-filtering the per-pixel outer products x x^T and x y^T (x with its
 *     leading 1) yields exactly X_k^T X_k and X_k^T Y_k (Sec. 3.2).
 *   - Appendix: X^T X = [[n, u_X], [u_X^T, S]], mu_X = u_X / n,
 *     W = S/n - mu_X^T mu_X; the top row of X^T Y is n mu_Y.
 *   - Regulariser (the reading this build takes of "ridge eps"): the Appendix's
 *     W-hat with its multiplicative term set to zero, i.e. M = W + eps I, and no
 *     second additive term on the normalised matrix.  Without that second term the
 *     Appendix's correlation normalisation cancels out, and the model is the
 *     centred ridge  a_k = M^{-1} D,  D = X^T Y / n - mu_X^T mu_Y (guide rows),
 *     b_k = mu_Y - a_k^T mu_X   (the bias is not penalised).
 *   - Optional coefficient averaging over a clipped window of radius rc (rc = 0
 *     switches it off, which is what Sec. 3.2 does), then the model is applied
 *     to the centre pixel's guide vector z_i (Sec. 3.1, I_k = x_k A_k).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_Q 16

/* Clipped window [lo, hi] of radius rad around i inside [0, n). */
static void clip_range(int i, int rad, int n, int *lo, int *hi)
{
    *lo = i - rad < 0 ? 0 : i - rad;
    *hi = i + rad > n - 1 ? n - 1 : i + rad;
}

/*
 * Sum of one plane over the clipped square window of radius rad, done as a row
 * pass then a column pass (the box is separable).  Every output is a direct sum of
 * at most 2*rad+1 terms: no running sums, no prefix differences.
 */
static void box_sum_plane(const double *src, double *dst, double *tmp, int H, int W, int rad)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int lo, hi;
            clip_range(x, rad, W, &lo, &hi);
            double s = 0.0;
            for (int xx = lo; xx <= hi; ++xx) s += src[(size_t)y * W + xx];
            tmp[(size_t)y * W + x] = s;
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        int lo, hi;
        clip_range(y, rad, H, &lo, &hi);
        for (int x = 0; x < W; ++x) {
            double s = 0.0;
            for (int yy = lo; yy <= hi; ++yy) s += tmp[(size_t)yy * W + x];
            dst[(size_t)y * W + x] = s;
        }
    }
}

/* Number of in-image pixels of the clipped window of radius rad at (y, x). */
static double window_count(int y, int x, int H, int W, int rad)
{
    int y0, y1, x0, x1;
    clip_range(y, rad, H, &y0, &y1);
    clip_range(x, rad, W, &x0, &x1);
    return (double)(y1 - y0 + 1) * (double)(x1 - x0 + 1);
}

/*
 * Cholesky factorisation M = L L^T of a q x q symmetric matrix (row-major, lower
 * triangle read), then solve M a = d for nrhs right-hand sides stored as d[i*nrhs+c].
 * Returns 0, or -1 if a pivot is not positive (M not positive definite).
 */
static int cholesky_solve(int q, const double *M, const double *d, int nrhs, double *a)
{
    double L[ORACLE_MAX_Q * ORACLE_MAX_Q];
    double z[ORACLE_MAX_Q * 3];
    for (int j = 0; j < q; ++j) {
        double s = M[j * q + j];
        for (int k = 0; k < j; ++k) s -= L[j * q + k] * L[j * q + k];
        if (!(s > 0.0)) return -1;
        L[j * q + j] = sqrt(s);
        for (int i = j + 1; i < q; ++i) {
            double t = M[i * q + j];
            for (int k = 0; k < j; ++k) t -= L[i * q + k] * L[j * q + k];
            L[i * q + j] = t / L[j * q + j];
        }
    }
    for (int c = 0; c < nrhs; ++c) {
        for (int i = 0; i < q; ++i) { /* L z = d */
            double t = d[i * nrhs + c];
            for (int k = 0; k < i; ++k) t -= L[i * q + k] * z[k * nrhs + c];
            z[i * nrhs + c] = t / L[i * q + i];
        }
        for (int i = q - 1; i >= 0; --i) { /* L^T a = z */
            double t = z[i * nrhs + c];
            for (int k = i + 1; k < q; ++k) t -= L[k * q + i] * a[k * nrhs + c];
            a[i * nrhs + c] = t / L[i * q + i];
        }
    }
    return 0;
}

/* Index of the pair (i <= j) of the (q+1)x(q+1) upper triangle, row by row. */
static int tri_index(int q1, int i, int j)
{
    return i * q1 - (i * (i - 1)) / 2 + (j - i);
}

/*
 * FLR forward pass (Sec. 3.1-3.2, Appendix; see file header).
 *
 *   q          number of guide channels Q (0..16); the ones column is implicit
 *   guide      [q][H][W] float32, the guides X the model is fitted on
 *   map_guide  [q][H][W] float32 the model is applied to, or NULL for guide
 *   radiance   [3][H][W] float32, the noisy signal Y
 *   r          window radius (>= 0); the window is (2r+1)^2 clipped to the image
 *   rc         coefficient-averaging radius (>= 0; 0 = none)
 *   eps        ridge regulariser added to the centred covariance (>= 0)
 *   out        [3][H][W] double, the result I
 *   coef       NULL, or [(q+1)*3][H][W] double: per-pixel A_k before averaging,
 *              plane (i*3 + c) holds row i, column c of A_k; row 0 is the bias b_k
 *
 * Returns 0; -1 for bad arguments; -2 for out of memory; -3 when a window's
 * regularised covariance is not positive definite (only possible with eps = 0).
 */
int flr_oracle_forward(int q, int H, int W, const float *guide, const float *map_guide,
                       const float *radiance, int r, int rc, double eps, double *out,
                       double *coef)
{
    if (q < 0 || q > ORACLE_MAX_Q || H <= 0 || W <= 0 || r < 0 || rc < 0 || !(eps >= 0.0))
        return -1;
    if ((q > 0 && !guide) || !radiance || !out) return -1;
    if (!map_guide) map_guide = guide;

    const int q1 = q + 1;
    const int nxx = q1 * (q1 + 1) / 2; /* upper triangle of X^T X, ones column included */
    const int nxy = q1 * 3;            /* X^T Y */
    const int ncoef = q1 * 3;
    const size_t P = (size_t)H * W;

    double *xx = malloc(sizeof(double) * P * nxx);
    double *xy = malloc(sizeof(double) * P * nxy);
    double *cf = malloc(sizeof(double) * P * ncoef);
    double *plane = malloc(sizeof(double) * P);
    double *tmp = malloc(sizeof(double) * P);
    int status = 0;
    if (!xx || !xy || !cf || !plane || !tmp) { status = -2; goto done; }

    /* Step 1 (Sec. 3.2): per-pixel outer products x x^T and x y^T, x = (1, X_1..X_Q). */
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < P; ++p) {
        double x[ORACLE_MAX_Q + 1], y[3];
        x[0] = 1.0;
        for (int i = 0; i < q; ++i) x[i + 1] = (double)guide[(size_t)i * P + p];
        for (int c = 0; c < 3; ++c) y[c] = (double)radiance[(size_t)c * P + p];
        for (int i = 0; i < q1; ++i)
            for (int j = i; j < q1; ++j) xx[(size_t)tri_index(q1, i, j) * P + p] = x[i] * x[j];
        for (int i = 0; i < q1; ++i)
            for (int c = 0; c < 3; ++c) xy[(size_t)(i * 3 + c) * P + p] = x[i] * y[c];
    }

    /* Step 2 (Sec. 3.2): box-filter every moment plane -> X_k^T X_k and X_k^T Y_k. */
    for (int m = 0; m < nxx; ++m) {
        memcpy(plane, xx + (size_t)m * P, sizeof(double) * P);
        box_sum_plane(plane, xx + (size_t)m * P, tmp, H, W, r);
    }
    for (int m = 0; m < nxy; ++m) {
        memcpy(plane, xy + (size_t)m * P, sizeof(double) * P);
        box_sum_plane(plane, xy + (size_t)m * P, tmp, H, W, r);
    }

    /* Step 3 (Appendix + closed form): per-pixel centred, regularised solve.  A pixel
     * whose matrix is not positive definite sets `failed`; the pass then reports -3. */
    int failed = 0;
#pragma omp parallel for schedule(static) reduction(| : failed)
    for (size_t p = 0; p < P; ++p) {
        const double n = xx[(size_t)tri_index(q1, 0, 0) * P + p];
        double mu_x[ORACLE_MAX_Q], mu_y[3];
        double M[ORACLE_MAX_Q * ORACLE_MAX_Q], D[ORACLE_MAX_Q * 3], a[ORACLE_MAX_Q * 3];
        for (int i = 0; i < q; ++i) mu_x[i] = xx[(size_t)tri_index(q1, 0, i + 1) * P + p] / n;
        for (int c = 0; c < 3; ++c) mu_y[c] = xy[(size_t)(0 * 3 + c) * P + p] / n;
        for (int i = 0; i < q; ++i)
            for (int j = 0; j < q; ++j) {
                int lo = i < j ? i : j, hi = i < j ? j : i;
                double S = xx[(size_t)tri_index(q1, lo + 1, hi + 1) * P + p];
                M[i * q + j] = S / n - mu_x[i] * mu_x[j] + (i == j ? eps : 0.0);
            }
        for (int i = 0; i < q; ++i)
            for (int c = 0; c < 3; ++c)
                D[i * 3 + c] = xy[(size_t)((i + 1) * 3 + c) * P + p] / n - mu_x[i] * mu_y[c];
        if (q > 0 && cholesky_solve(q, M, D, 3, a) != 0) { failed = 1; continue; }
        for (int c = 0; c < 3; ++c) {
            double b = mu_y[c];
            for (int i = 0; i < q; ++i) b -= a[i * 3 + c] * mu_x[i];
            cf[(size_t)(0 * 3 + c) * P + p] = b;
            for (int i = 0; i < q; ++i) cf[(size_t)((i + 1) * 3 + c) * P + p] = a[i * 3 + c];
        }
    }
    if (failed) { status = -3; goto done; }
    if (coef) memcpy(coef, cf, sizeof(double) * P * ncoef);

    /* Step 4: mean of the coefficients over the clipped radius-rc window. */
    if (rc > 0) {
        for (int m = 0; m < ncoef; ++m) {
            memcpy(plane, cf + (size_t)m * P, sizeof(double) * P);
            box_sum_plane(plane, cf + (size_t)m * P, tmp, H, W, rc);
#pragma omp parallel for schedule(static)
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x)
                    cf[(size_t)m * P + (size_t)y * W + x] /= window_count(y, x, H, W, rc);
        }
    }

    /* Step 5 (Sec. 3.1): apply the model to the centre pixel, I = (1, z) A. */
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < P; ++p)
        for (int c = 0; c < 3; ++c) {
            double v = cf[(size_t)(0 * 3 + c) * P + p];
            for (int i = 0; i < q; ++i)
                v += cf[(size_t)((i + 1) * 3 + c) * P + p] * (double)map_guide[(size_t)i * P + p];
            out[(size_t)c * P + p] = v;
        }

done:
    free(xx);
    free(xy);
    free(cf);
    free(plane);
    free(tmp);
    return status;
}

/* Number of threads the parallel loops above use (1 without OpenMP). */
int flr_oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the number of threads of the parallel loops (timing only; no arithmetic depends on it:
 * every loop writes disjoint outputs). */
void flr_oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * FLR backward pass in FP64: the gradient of L = <grad_out, I> with respect to the guides,
 * the map guides, the radiance and eps, for the forward pass above.
 *
 * The paper trains through FLR by backpropagation (Sec. 3.2: the window's sigma and the
 * regularisers are learned; Sec. 3.3: FLNR "builds on a differentiable implementation of
 * FLR") but prints no adjoint.  This is the reverse-mode derivative of the forward's steps
 * in reverse order, with g = grad_out:
 *   apply      I_i = Abar_i^T (1, z_i):      G(Abar_i) = (1, z_i) g_i^T,  dz_i = abar_i g_i
 *   average    Abar_i = mean_{k in T'_i} A_k: G(A_k) = sum_{i: k in T'_i} G(Abar_i) / m_i
 *   bias       b = nu - a^T mu:              G(nu) = Gb,  Ga' = Ga - mu Gb^T,  G(mu) = -a Gb
 *   solve      a = M^{-1} D:                 GD = M^{-1} Ga',  GM = -(GD a^T + a GD^T)/2
 *   regulariser M = W + eps I:               G(eps) = trace(GM)
 *   centring   W = S/n - mu mu^T, D = XY/n - mu nu^T:
 *                  GS = GM/n, GXY = GD/n, G(mu) += -2 GM mu - GD nu, G(nu) += -GD^T mu
 *   means      mu = Sx/n, nu = Sy/n:         GSx = G(mu)/n, GSy = G(nu)/n
 *   window sums (S = sum x x^T, XY = sum x y^T over T_k; j in T_k <=> k in T_j):
 *      dx_j = sum_{k in T_j} GSx_k + 2 GS_k x_j + GXY_k y_j
 *      dy_j = sum_{k in T_j} GSy_k + GXY_k^T x_j
 *
 *   grad_out     [3][H][W] double
 *   grad_guide   [q][H][W] double (model-guide gradient; when map_guide is NULL the map
 *                guide is the guide and its gradient is added here as well)
 *   grad_map     [q][H][W] double or NULL (only with a separate map_guide)
 *   grad_rad     [3][H][W] double
 *   grad_eps     double* or NULL
 * Returns 0, or the forward's error codes.
 */
int flr_oracle_backward(int q, int H, int W, const float *guide, const float *map_guide,
                        const float *radiance, int r, int rc, double eps, const double *grad_out,
                        double *grad_guide, double *grad_map, double *grad_rad, double *grad_eps)
{
    if (q < 1 || q > ORACLE_MAX_Q || H <= 0 || W <= 0 || r < 0 || rc < 0 || !(eps >= 0.0))
        return -1;
    if (!guide || !radiance || !grad_out || !grad_guide || !grad_rad) return -1;
    const float *zg = map_guide ? map_guide : guide;
    const int q1 = q + 1;
    const size_t P = (size_t)H * W;
    const int ncoef = q1 * 3;

    /* forward quantities: per-pixel models A_k (before averaging), via the forward pass */
    double *A = malloc(sizeof(double) * P * ncoef);
    double *outf = malloc(sizeof(double) * P * 3);
    double *xx = malloc(sizeof(double) * P * (q1 * (q1 + 1) / 2));
    double *plane = malloc(sizeof(double) * P);
    double *tmp = malloc(sizeof(double) * P);
    double *GA = malloc(sizeof(double) * P * ncoef);      /* G(A_k) after the average */
    double *GS = malloc(sizeof(double) * P * (q * q + 3 * q + q + 3)); /* per-k gradients */
    int status = 0;
    if (!A || !outf || !xx || !plane || !tmp || !GA || !GS) { status = -2; goto done; }
    status = flr_oracle_forward(q, H, W, guide, map_guide, radiance, r, rc, eps, outf, A);
    if (status) goto done;

    /* window sums again (the forward recomputed, Sec. 3.2), for n, mu, nu and M */
    const int nxx = q1 * (q1 + 1) / 2;
    double *xy = malloc(sizeof(double) * P * q1 * 3);
    if (!xy) { status = -2; goto done; }
    for (size_t p = 0; p < P; ++p) {
        double x[ORACLE_MAX_Q + 1], y[3];
        x[0] = 1.0;
        for (int i = 0; i < q; ++i) x[i + 1] = (double)guide[(size_t)i * P + p];
        for (int c = 0; c < 3; ++c) y[c] = (double)radiance[(size_t)c * P + p];
        for (int i = 0; i < q1; ++i)
            for (int j = i; j < q1; ++j) xx[(size_t)tri_index(q1, i, j) * P + p] = x[i] * x[j];
        for (int i = 0; i < q1; ++i)
            for (int c = 0; c < 3; ++c) xy[(size_t)(i * 3 + c) * P + p] = x[i] * y[c];
    }
    for (int m = 0; m < nxx; ++m) {
        memcpy(plane, xx + (size_t)m * P, sizeof(double) * P);
        box_sum_plane(plane, xx + (size_t)m * P, tmp, H, W, r);
    }
    for (int m = 0; m < q1 * 3; ++m) {
        memcpy(plane, xy + (size_t)m * P, sizeof(double) * P);
        box_sum_plane(plane, xy + (size_t)m * P, tmp, H, W, r);
    }

    /* apply: G(Abar_i) = (1, z_i) g_i^T / m_i (divided by m_i ready for the average's
     * adjoint), and the map-guide gradient abar_i g_i */
    double *abar = malloc(sizeof(double) * P * ncoef);
    if (!abar) { free(xy); status = -2; goto done; }
    memcpy(abar, A, sizeof(double) * P * ncoef);
    if (rc > 0) {
        for (int m = 0; m < ncoef; ++m) {
            memcpy(plane, abar + (size_t)m * P, sizeof(double) * P);
            box_sum_plane(plane, abar + (size_t)m * P, tmp, H, W, rc);
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x)
                    abar[(size_t)m * P + (size_t)y * W + x] /= window_count(y, x, H, W, rc);
        }
    }
    double *gz = map_guide ? grad_map : grad_guide; /* may be NULL with a separate map guide */
    memset(grad_guide, 0, sizeof(double) * P * q);
    if (map_guide && grad_map) memset(grad_map, 0, sizeof(double) * P * q);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const size_t p = (size_t)y * W + x;
            const double m_i = rc > 0 ? window_count(y, x, H, W, rc) : 1.0;
            for (int c = 0; c < 3; ++c) {
                const double g = grad_out[(size_t)c * P + p];
                GA[(size_t)(0 * 3 + c) * P + p] = g / m_i;
                for (int i = 0; i < q; ++i) {
                    GA[(size_t)((i + 1) * 3 + c) * P + p] = (double)zg[(size_t)i * P + p] * g / m_i;
                    if (gz) gz[(size_t)i * P + p] += abar[(size_t)((i + 1) * 3 + c) * P + p] * g;
                }
            }
        }
    free(abar);
    /* average: G(A_k) = sum over i with k in T'_i of G(Abar_i) / m_i */
    if (rc > 0) {
        for (int m = 0; m < ncoef; ++m) {
            memcpy(plane, GA + (size_t)m * P, sizeof(double) * P);
            box_sum_plane(plane, GA + (size_t)m * P, tmp, H, W, rc);
        }
    }

    /* per-pixel adjoint of bias, solve, regulariser, centring and means.
     * GS layout per pixel: [q*q] GS (full symmetric), [3q] GXY, [q] GSx, [3] GSy */
    const int ng = q * q + 3 * q + q + 3;
    double geps = 0.0;
    for (size_t p = 0; p < P; ++p) {
        const double n = xx[(size_t)tri_index(q1, 0, 0) * P + p];
        double mu[ORACLE_MAX_Q], nu[3], M[ORACLE_MAX_Q * ORACLE_MAX_Q], a[ORACLE_MAX_Q * 3];
        double Gb[3], Gap[ORACLE_MAX_Q * 3], GD[ORACLE_MAX_Q * 3], GM[ORACLE_MAX_Q * ORACLE_MAX_Q];
        double Gmu[ORACLE_MAX_Q], Gnu[3];
        for (int i = 0; i < q; ++i) mu[i] = xx[(size_t)tri_index(q1, 0, i + 1) * P + p] / n;
        for (int c = 0; c < 3; ++c) nu[c] = xy[(size_t)c * P + p] / n;
        for (int i = 0; i < q; ++i)
            for (int j = 0; j < q; ++j) {
                int lo = i < j ? i : j, hi = i < j ? j : i;
                M[i * q + j] = xx[(size_t)tri_index(q1, lo + 1, hi + 1) * P + p] / n - mu[i] * mu[j] +
                               (i == j ? eps : 0.0);
            }
        for (int i = 0; i < q; ++i)
            for (int c = 0; c < 3; ++c) a[i * 3 + c] = A[(size_t)((i + 1) * 3 + c) * P + p];
        for (int c = 0; c < 3; ++c) Gb[c] = GA[(size_t)c * P + p];
        /* bias b = nu - a^T mu */
        for (int c = 0; c < 3; ++c) Gnu[c] = Gb[c];
        for (int i = 0; i < q; ++i) {
            Gmu[i] = 0.0;
            for (int c = 0; c < 3; ++c) {
                Gap[i * 3 + c] = GA[(size_t)((i + 1) * 3 + c) * P + p] - mu[i] * Gb[c];
                Gmu[i] -= a[i * 3 + c] * Gb[c];
            }
        }
        /* solve a = M^{-1} D: GD = M^{-1} Ga', GM = -(GD a^T + a GD^T) / 2 */
        if (cholesky_solve(q, M, Gap, 3, GD) != 0) { status = -3; break; }
        for (int i = 0; i < q; ++i)
            for (int j = 0; j < q; ++j) {
                double s = 0.0;
                for (int c = 0; c < 3; ++c) s += GD[i * 3 + c] * a[j * 3 + c] + a[i * 3 + c] * GD[j * 3 + c];
                GM[i * q + j] = -0.5 * s;
            }
        for (int i = 0; i < q; ++i) geps += GM[i * q + i];
        /* centring W = S/n - mu mu^T, D = XY/n - mu nu^T */
        for (int i = 0; i < q; ++i) {
            double s = 0.0;
            for (int j = 0; j < q; ++j) s += GM[i * q + j] * mu[j];
            Gmu[i] -= 2.0 * s;
            for (int c = 0; c < 3; ++c) Gmu[i] -= GD[i * 3 + c] * nu[c];
        }
        for (int c = 0; c < 3; ++c)
            for (int i = 0; i < q; ++i) Gnu[c] -= GD[i * 3 + c] * mu[i];
        double *gs = GS + (size_t)p * ng;
        for (int i = 0; i < q * q; ++i) gs[i] = GM[i] / n;
        for (int i = 0; i < 3 * q; ++i) gs[q * q + i] = GD[i] / n;
        for (int i = 0; i < q; ++i) gs[q * q + 3 * q + i] = Gmu[i] / n;
        for (int c = 0; c < 3; ++c) gs[q * q + 4 * q + c] = Gnu[c] / n;
    }
    free(xy);
    if (status) goto done;
    if (grad_eps) *grad_eps = geps;

    /* window sums of the per-k gradients, contracted with the inputs at j */
    for (int m = 0; m < ng; ++m) {
        for (size_t p = 0; p < P; ++p) plane[p] = GS[p * ng + m];
        box_sum_plane(plane, plane, tmp, H, W, r);
        for (size_t p = 0; p < P; ++p) GS[p * ng + m] = plane[p];
    }
    for (size_t p = 0; p < P; ++p) {
        const double *gs = GS + p * ng;
        double x[ORACLE_MAX_Q], y[3];
        for (int i = 0; i < q; ++i) x[i] = (double)guide[(size_t)i * P + p];
        for (int c = 0; c < 3; ++c) y[c] = (double)radiance[(size_t)c * P + p];
        for (int i = 0; i < q; ++i) {
            double d = gs[q * q + 3 * q + i];
            for (int j = 0; j < q; ++j) d += 2.0 * gs[i * q + j] * x[j];
            for (int c = 0; c < 3; ++c) d += gs[q * q + i * 3 + c] * y[c];
            grad_guide[(size_t)i * P + p] += d;
        }
        for (int c = 0; c < 3; ++c) {
            double d = gs[q * q + 4 * q + c];
            for (int i = 0; i < q; ++i) d += gs[q * q + i * 3 + c] * x[i];
            grad_rad[(size_t)c * P + p] = d;
        }
    }

done:
    free(A);
    free(outf);
    free(xx);
    free(plane);
    free(tmp);
    free(GA);
    free(GS);
    return status;
}

/*
 * Fast FLR in FP64 (Sec. 3.2 "Fast Local Regression", and Sec. 3.2.1 for the joint
 * denoising and upsampling): the paper's implementation choice for speed.
 *   1. outer products x x^T, x y^T at every input pixel (x with its leading 1);
 *   2. downsample: sum them over F x F blocks (the strided box filter of the first of the
 *      paper's four kernels), clipped at the image border;
 *   3. blur the block moments with a separable Gaussian of standard deviation sigma_b
 *      block units (sigma / F for a full-resolution sigma), truncated at `taps` blocks and
 *      clipped at the grid border (second kernel); this is the weighted least squares of
 *      Sec. 3.2 with each pixel weighted by the Gaussian weight of its block;
 *   4. per block the centred ridge model, as in flr_oracle_forward (third kernel);
 *   5. bilinear interpolation of the block models to every output pixel and application
 *      to the map guide there (fourth kernel).
 * The output grid is s times finer than the input grid (s = 1: plain fast FLR; s > 1:
 * joint denoising and upsampling, with model guides and radiance given at the input
 * resolution and the map guide at the output resolution).  Block (i, j) has its centre at
 * output coordinate ((i + 1/2) F s - 1/2, (j + 1/2) F s - 1/2); coordinates outside the
 * outermost centres take the edge block's model.
 *
 *   guide      [q][Hi][Wi]  model guides;  radiance [3][Hi][Wi]
 *   map_guide  [q][Ho][Wo] with Ho = Hi s, Wo = Wi s (NULL: the guide itself, s = 1 only)
 *   out        [3][Ho][Wo] double;  coef: NULL or [(q+1)*3][Hb][Wb] block models
 *   appendix   0: the centred ridge of step 4 with eps;  1: the Appendix's regularised
 *              normalised solve with additive term eps (the paper's epsilon) and
 *              multiplicative term eps_mul (the paper's varepsilon), steps as printed:
 *                W^ = S/n + eps_mul diag(mu^T mu) + eps I - (1 - eps_mul) mu^T mu,
 *                sigma^ = sqrt(diag W^),  C^_ij = W^_ij / (sigma^_i sigma^_j),
 *                B^_ic = (X^T Y_ic / n - mu_i muY_c) / sigma^_i,
 *                A^ = (C^ + eps I)^-1 B^,  y = ((x - mu) / sigma^) A^ + muY,
 *              stored as the same block model: a_ic = A^_ic / sigma^_i,
 *              b_c = muY_c - sum_i a_ic mu_i.
 * Returns 0, -1 for bad arguments, -2 out of memory, -3 not positive definite.
 */
int flr_oracle_fast_reg(int q, int Hi, int Wi, const float *guide, const float *radiance,
                        const float *map_guide, int F, int s, double sigma_b, int taps, double eps,
                        int appendix, double eps_mul, double *out, double *coef)
{
    if (q < 1 || q > ORACLE_MAX_Q || Hi <= 0 || Wi <= 0 || F < 1 || s < 1 || taps < 0 ||
        !(sigma_b > 0.0) || !(eps >= 0.0) || !guide || !radiance || !out || appendix < 0 || appendix > 1 ||
        !(eps_mul >= 0.0 && eps_mul <= 1.0))
        return -1;
    if (!map_guide && s != 1) return -1;
    if (!map_guide) map_guide = guide;
    const int Ho = Hi * s, Wo = Wi * s;
    const int Hb = (Hi + F - 1) / F, Wb = (Wi + F - 1) / F;
    const int q1 = q + 1, nxx = q1 * (q1 + 1) / 2, nm = nxx + 3 * q1;
    const size_t Pi = (size_t)Hi * Wi, Pb = (size_t)Hb * Wb, Po = (size_t)Ho * Wo;
    double *blk = calloc(Pb * nm, sizeof(double));
    double *tmpb = malloc(sizeof(double) * Pb * nm);
    double *cf = malloc(sizeof(double) * Pb * q1 * 3);
    double *w = malloc(sizeof(double) * (2 * taps + 1));
    int status = 0;
    if (!blk || !tmpb || !cf || !w) { status = -2; goto done; }

    /* steps 1-2: block sums of the outer products */
    for (int y = 0; y < Hi; ++y)
        for (int x = 0; x < Wi; ++x) {
            const size_t p = (size_t)y * Wi + x;
            double v[ORACLE_MAX_Q + 1], yv[3];
            v[0] = 1.0;
            for (int i = 0; i < q; ++i) v[i + 1] = (double)guide[(size_t)i * Pi + p];
            for (int c = 0; c < 3; ++c) yv[c] = (double)radiance[(size_t)c * Pi + p];
            double *b = blk + ((size_t)(y / F) * Wb + x / F) * nm;
            for (int i = 0; i < q1; ++i)
                for (int j = i; j < q1; ++j) b[tri_index(q1, i, j)] += v[i] * v[j];
            for (int i = 0; i < q1; ++i)
                for (int c = 0; c < 3; ++c) b[nxx + i * 3 + c] += v[i] * yv[c];
        }
    /* step 3: separable Gaussian over the block grid, clipped */
    for (int d = -taps; d <= taps; ++d) w[d + taps] = exp(-(double)d * d / (2.0 * sigma_b * sigma_b));
    for (int by = 0; by < Hb; ++by)
        for (int bx = 0; bx < Wb; ++bx)
            for (int m = 0; m < nm; ++m) {
                double acc = 0.0;
                for (int d = -taps; d <= taps; ++d) {
                    const int xx2 = bx + d;
                    if (xx2 >= 0 && xx2 < Wb) acc += w[d + taps] * blk[((size_t)by * Wb + xx2) * nm + m];
                }
                tmpb[((size_t)by * Wb + bx) * nm + m] = acc;
            }
    for (int by = 0; by < Hb; ++by)
        for (int bx = 0; bx < Wb; ++bx)
            for (int m = 0; m < nm; ++m) {
                double acc = 0.0;
                for (int d = -taps; d <= taps; ++d) {
                    const int yy = by + d;
                    if (yy >= 0 && yy < Hb) acc += w[d + taps] * tmpb[((size_t)yy * Wb + bx) * nm + m];
                }
                blk[((size_t)by * Wb + bx) * nm + m] = acc;
            }
    /* step 4: per-block centred ridge (Appendix), as in flr_oracle_forward, or the
       Appendix's regularised normalised solve */
    for (size_t k = 0; k < Pb && status == 0; ++k) {
        const double *b = blk + k * nm;
        const double n = b[tri_index(q1, 0, 0)];
        double mu[ORACLE_MAX_Q], mu_y[3], M[ORACLE_MAX_Q * ORACLE_MAX_Q], D[ORACLE_MAX_Q * 3], a[ORACLE_MAX_Q * 3];
        for (int i = 0; i < q; ++i) mu[i] = b[tri_index(q1, 0, i + 1)] / n;
        for (int c = 0; c < 3; ++c) mu_y[c] = b[nxx + c] / n;
        if (appendix) {
            double Wh[ORACLE_MAX_Q * ORACLE_MAX_Q], sg[ORACLE_MAX_Q], Bh[ORACLE_MAX_Q * 3], Ah[ORACLE_MAX_Q * 3];
            for (int i = 0; i < q; ++i)
                for (int j = 0; j < q; ++j) {
                    int lo = i < j ? i : j, hi = i < j ? j : i;
                    Wh[i * q + j] = b[tri_index(q1, lo + 1, hi + 1)] / n
                                  + (i == j ? eps_mul * mu[i] * mu[i] + eps : 0.0)
                                  - (1.0 - eps_mul) * mu[i] * mu[j];
                }
            for (int i = 0; i < q; ++i) sg[i] = sqrt(Wh[i * q + i]);
            for (int i = 0; i < q; ++i)
                for (int j = 0; j < q; ++j) M[i * q + j] = Wh[i * q + j] / (sg[i] * sg[j]) + (i == j ? eps : 0.0);
            for (int i = 0; i < q; ++i)
                for (int c = 0; c < 3; ++c) Bh[i * 3 + c] = (b[nxx + (i + 1) * 3 + c] / n - mu[i] * mu_y[c]) / sg[i];
            if (cholesky_solve(q, M, Bh, 3, Ah) != 0) { status = -3; break; }
            for (int c = 0; c < 3; ++c) {
                double bb = mu_y[c];
                for (int i = 0; i < q; ++i) {
                    const double ai = Ah[i * 3 + c] / sg[i];
                    bb -= ai * mu[i];
                    cf[(size_t)((i + 1) * 3 + c) * Pb + k] = ai;
                }
                cf[(size_t)(0 * 3 + c) * Pb + k] = bb;
            }
            continue;
        }
        for (int i = 0; i < q; ++i)
            for (int j = 0; j < q; ++j) {
                int lo = i < j ? i : j, hi = i < j ? j : i;
                M[i * q + j] = b[tri_index(q1, lo + 1, hi + 1)] / n - mu[i] * mu[j] + (i == j ? eps : 0.0);
            }
        for (int i = 0; i < q; ++i)
            for (int c = 0; c < 3; ++c) D[i * 3 + c] = b[nxx + (i + 1) * 3 + c] / n - mu[i] * mu_y[c];
        if (cholesky_solve(q, M, D, 3, a) != 0) { status = -3; break; }
        for (int c = 0; c < 3; ++c) {
            double bb = mu_y[c];
            for (int i = 0; i < q; ++i) bb -= a[i * 3 + c] * mu[i];
            cf[(size_t)(0 * 3 + c) * Pb + k] = bb;
            for (int i = 0; i < q; ++i) cf[(size_t)((i + 1) * 3 + c) * Pb + k] = a[i * 3 + c];
        }
    }
    if (status) goto done;
    if (coef) memcpy(coef, cf, sizeof(double) * Pb * q1 * 3);
    /* step 5: bilinear interpolation of the block models, applied to the map guide */
    for (int yo = 0; yo < Ho; ++yo)
        for (int xo = 0; xo < Wo; ++xo) {
            double u = (yo + 0.5) / ((double)F * s) - 0.5, v = (xo + 0.5) / ((double)F * s) - 0.5;
            if (u < 0) u = 0;
            if (u > Hb - 1) u = Hb - 1;
            if (v < 0) v = 0;
            if (v > Wb - 1) v = Wb - 1;
            int i0 = (int)floor(u), j0 = (int)floor(v);
            if (i0 > Hb - 2) i0 = Hb > 1 ? Hb - 2 : 0;
            if (j0 > Wb - 2) j0 = Wb > 1 ? Wb - 2 : 0;
            const int i1 = Hb > 1 ? i0 + 1 : 0, j1 = Wb > 1 ? j0 + 1 : 0;
            const double fy = u - i0, fx = v - j0;
            const size_t po = (size_t)yo * Wo + xo;
            for (int c = 0; c < 3; ++c) {
                double o = 0.0;
                for (int i = 0; i <= q; ++i) {
                    const double *pl = cf + (size_t)(i * 3 + c) * Pb;
                    const double val = (1 - fy) * ((1 - fx) * pl[(size_t)i0 * Wb + j0] + fx * pl[(size_t)i0 * Wb + j1]) +
                                       fy * ((1 - fx) * pl[(size_t)i1 * Wb + j0] + fx * pl[(size_t)i1 * Wb + j1]);
                    o += val * (i == 0 ? 1.0 : (double)map_guide[(size_t)(i - 1) * Po + po]);
                }
                out[(size_t)c * Po + po] = o;
            }
        }
done:
    free(blk);
    free(tmpb);
    free(cf);
    free(w);
    return status;
}

/* Fast FLR with the centred ridge of step 4 (flr_oracle_fast_reg with appendix = 0). */
int flr_oracle_fast(int q, int Hi, int Wi, const float *guide, const float *radiance,
                    const float *map_guide, int F, int s, double sigma_b, int taps, double eps,
                    double *out, double *coef)
{
    return flr_oracle_fast_reg(q, Hi, Wi, guide, radiance, map_guide, F, s, sigma_b, taps, eps, 0, 0.0, out, coef);
}
