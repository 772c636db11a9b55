/*
 * fbp_oracle.c -- plain FP64 CPU oracle for parallel-beam filtered
 * backprojection (FBP) and its matched forward projector.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  The product (the CUDA
 * library under paper_2505_13955_gb300/) never calls it, and the two share no
 * code, headers, tables or helpers.
 *
 * What it computes.  The paper reconstructs each slice by FBP in two steps,
 * filtering every projection row and then backprojecting the filtered rows
 * and summing over all angles (Sec. IV-B; Sec. V-A(c), stage 2, whose cost is
 * O(N_p * N_x * N_y * N_z)).  For the filter it cites Kak & Slaney,
 * "Principles of Computerized Tomographic Imaging", ch. 3; this file writes
 * out that chapter's discrete sums in the same order:
 *
 *   taps      h[n], |n| <= D-1 (Ram-Lak or Shepp-Logan band-limited kernel)
 *   filter    q_k[j] = tau * sum_{m=0}^{D-1} h[j-m] * p_k[m]   (linear conv.)
 *   backproj  f[r][c] = scale * sum_k Q_k(u_k),
 *             u_k = alpha * (X cos th_k + Y sin th_k) + c_d,
 *             Q_k(u) = (1-w) q~_k[j0] + w q~_k[j0+1], j0 = floor(u), w = u-j0,
 *             q~ = q inside [0, D), 0 outside
 *   forward   (A f)_k[j] = sum_{r,c} f[r][c] * ((1-w)[j==j0] + w[j==j0+1])
 *
 * with th_k = angle_start + k*angle_step, X = (c - (N-1)/2),
 * Y = (r - (N-1)/2), alpha = pixel_size / det_spacing and c_d = det_center.
 * Backprojection with scale 1 is exactly the transpose of the forward
 * projector.  The paper itself prints no formula for either step; where it is
 * silent (filter kind, padding, normalisation, geometry convention, how the
 * detector is interpolated) this file takes the textbook reading listed in
 * the project's design notes.
 *
 * Everything is double precision.  Loops are the definitions, parallelised
 * over independent outputs only (rows of the image, rows of the sinogram), so
 * the result does not depend on the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n_angles;        /* K: number of projection angles                   */
    int n_det;           /* D: detector bins per projection row              */
    int n;               /* N: output slice is N x N                         */
    double angle_start;  /* theta_0 (radians)                                */
    double angle_step;   /* dtheta (radians)                                 */
    double det_center;   /* c_d: bin coordinate of the rotation axis         */
    double det_spacing;  /* tau: bin width, in the same unit as pixel_size   */
    double pixel_size;   /* pixel width                                      */
} oracle_geometry;

enum { ORACLE_RAMLAK = 0, ORACLE_SHEPP_LOGAN = 1 };

static const double ORACLE_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* Filter taps (Kak & Slaney ch. 3: band-limited ramp kernel and its        */
/* Shepp-Logan-windowed variant), sampled at n*tau for |n| <= D-1.          */
/* h[(D-1) + n] holds h(n*tau).                                             */
/* ------------------------------------------------------------------------ */
double oracle_tap(int kind, long n, double tau)
{
    double t2 = tau * tau;
    if (kind == ORACLE_RAMLAK) {
        if (n == 0) return 1.0 / (4.0 * t2);
        if ((n % 2) == 0) return 0.0;
        return -1.0 / (ORACLE_PI * ORACLE_PI * (double)n * (double)n * t2);
    }
    /* Shepp-Logan */
    return -2.0 / (ORACLE_PI * ORACLE_PI * t2 * (4.0 * (double)n * (double)n - 1.0));
}

int oracle_taps(int kind, int D, double tau, double *h)
{
    if (D < 1 || !(tau > 0.0) || !h) return -1;
    if (kind != ORACLE_RAMLAK && kind != ORACLE_SHEPP_LOGAN) return -1;
    for (long n = -(long)(D - 1); n <= (long)(D - 1); ++n)
        h[(D - 1) + n] = oracle_tap(kind, n, tau);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Filtering by the direct linear-convolution sum.  O(K D^2).               */
/* ------------------------------------------------------------------------ */
int oracle_filter_direct(const double *p, int K, int D, int kind, double tau,
                         double *q)
{
    if (!p || !q || K < 0 || D < 1 || !(tau > 0.0)) return -1;
    if (kind != ORACLE_RAMLAK && kind != ORACLE_SHEPP_LOGAN) return -1;
    double *h = (double *)malloc(sizeof(double) * (size_t)(2 * D - 1));
    if (!h) return -2;
    oracle_taps(kind, D, tau, h);
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k) {
        const double *pk = p + (size_t)k * D;
        double *qk = q + (size_t)k * D;
        for (int j = 0; j < D; ++j) {
            double s = 0.0;
            for (int m = 0; m < D; ++m)
                s += h[(D - 1) + (j - m)] * pk[m];
            qk[j] = tau * s;
        }
    }
    free(h);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* A plain iterative radix-2 FFT (Cooley-Tukey, bit-reversed input order).  */
/* sign = -1: forward  X[k] = sum_n x[n] e^{-2 pi i k n / L}                */
/* sign = +1: unnormalised inverse.  L must be a power of two.              */
/* Twiddles are evaluated directly with cos/sin of 2 pi m / L.              */
/* ------------------------------------------------------------------------ */
int oracle_fft(double *re, double *im, int L, int sign)
{
    if (L < 1 || (L & (L - 1)) != 0 || !re || !im) return -1;
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < L; ++i) {
        int bit = L >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int len = 2; len <= L; len <<= 1) {
        int half = len >> 1;
        for (int m = 0; m < half; ++m) {
            double ang = (double)sign * 2.0 * ORACLE_PI * (double)m / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int s = 0; s < L; s += len) {
                int a = s + m, b = s + m + half;
                double tr = re[b] * wr - im[b] * wi;
                double ti = re[b] * wi + im[b] * wr;
                re[b] = re[a] - tr; im[b] = im[a] - ti;
                re[a] += tr;        im[a] += ti;
            }
        }
    }
    return 0;
}

/* Smallest power of two >= 2D-1 (the linear-convolution length). */
int oracle_conv_length(int D)
{
    int L = 1;
    while (L < 2 * D - 1) L <<= 1;
    return L;
}

/* ------------------------------------------------------------------------ */
/* Filtering by FFT: the same linear convolution, computed as a circular    */
/* convolution of length L >= 2D-1 (no wrap-around reaches [0, D)).         */
/* ------------------------------------------------------------------------ */
int oracle_filter_fft(const double *p, int K, int D, int kind, double tau,
                      double *q)
{
    if (!p || !q || K < 0 || D < 1 || !(tau > 0.0)) return -1;
    if (kind != ORACLE_RAMLAK && kind != ORACLE_SHEPP_LOGAN) return -1;
    int L = oracle_conv_length(D);
    double *hr = (double *)calloc((size_t)L, sizeof(double));
    double *hi = (double *)calloc((size_t)L, sizeof(double));
    if (!hr || !hi) { free(hr); free(hi); return -2; }
    /* kernel laid out circularly: index n mod L holds h(n), |n| <= D-1 */
    for (long n = -(long)(D - 1); n <= (long)(D - 1); ++n)
        hr[(n + L) % L] = oracle_tap(kind, n, tau);
    oracle_fft(hr, hi, L, -1);
    int err = 0;
#pragma omp parallel
    {
        double *xr = (double *)malloc(sizeof(double) * (size_t)L);
        double *xi = (double *)malloc(sizeof(double) * (size_t)L);
        if (!xr || !xi) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int k = 0; k < K; ++k) {
                const double *pk = p + (size_t)k * D;
                for (int n = 0; n < L; ++n) { xr[n] = n < D ? pk[n] : 0.0; xi[n] = 0.0; }
                oracle_fft(xr, xi, L, -1);
                for (int n = 0; n < L; ++n) {
                    double a = xr[n] * hr[n] - xi[n] * hi[n];
                    double b = xr[n] * hi[n] + xi[n] * hr[n];
                    xr[n] = a; xi[n] = b;
                }
                oracle_fft(xr, xi, L, +1);
                double *qk = q + (size_t)k * D;
                for (int j = 0; j < D; ++j) qk[j] = tau * xr[j] / (double)L;
            }
        }
        free(xr); free(xi);
    }
    free(hr); free(hi);
    return err;
}

/* Direct sum up to D = 2048, FFT above (the two agree to rounding). */
int oracle_filter(const double *p, int K, int D, int kind, double tau, double *q)
{
    if (D <= 2048) return oracle_filter_direct(p, K, D, kind, tau, q);
    return oracle_filter_fft(p, K, D, kind, tau, q);
}

/* ------------------------------------------------------------------------ */
/* Geometry helpers                                                          */
/* ------------------------------------------------------------------------ */
static int geometry_ok(const oracle_geometry *g)
{
    return g && g->n_angles >= 0 && g->n_det >= 1 && g->n >= 0 &&
           g->det_spacing > 0.0 && g->pixel_size > 0.0;
}

/* detector coordinate of the centre of pixel [r][c] at angle k */
static double pixel_u(const oracle_geometry *g, double ck, double sk, int r, int c)
{
    double X = (double)c - 0.5 * (double)(g->n - 1);
    double Y = (double)r - 0.5 * (double)(g->n - 1);
    double alpha = g->pixel_size / g->det_spacing;
    return alpha * (X * ck + Y * sk) + g->det_center;
}

static double *angle_table(const oracle_geometry *g)
{
    int K = g->n_angles;
    double *t = (double *)malloc(sizeof(double) * (size_t)(2 * (K > 0 ? K : 1)));
    if (!t) return NULL;
    for (int k = 0; k < K; ++k) {
        double th = g->angle_start + (double)k * g->angle_step;
        t[2 * k] = cos(th);
        t[2 * k + 1] = sin(th);
    }
    return t;
}

/* q~[j]: the filtered row inside the detector, zero outside */
static double qt(const double *qk, int D, long j)
{
    return (j >= 0 && j < D) ? qk[j] : 0.0;
}

/* linear interpolation of row qk at detector coordinate u */
static double interp(const double *qk, int D, double u)
{
    double j0 = floor(u);
    double w = u - j0;
    long j = (long)j0;
    return (1.0 - w) * qt(qk, D, j) + w * qt(qk, D, j + 1);
}

/* ------------------------------------------------------------------------ */
/* Pixel-driven backprojection, every pixel of the N x N square.            */
/* f[r][c] = scale * sum_k Q_k(u_k(r, c)).                                  */
/* ------------------------------------------------------------------------ */
int oracle_backproject(const double *q, const oracle_geometry *g, double scale,
                       double *f)
{
    if (!q || !f || !geometry_ok(g)) return -1;
    int K = g->n_angles, D = g->n_det, N = g->n;
    double *cs = angle_table(g);
    if (!cs) return -2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < N; ++r) {
        for (int c = 0; c < N; ++c) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) {
                double u = pixel_u(g, cs[2 * k], cs[2 * k + 1], r, c);
                acc += interp(q + (size_t)k * D, D, u);
            }
            f[(size_t)r * N + c] = scale * acc;
        }
    }
    free(cs);
    return 0;
}

/* The same sum at an explicit list of pixels (for sampled checks at sizes
 * where the full image is too expensive). */
int oracle_backproject_pixels(const double *q, const oracle_geometry *g,
                              double scale, const int *rows, const int *cols,
                              long npix, double *out)
{
    if (!q || !out || !rows || !cols || npix < 0 || !geometry_ok(g)) return -1;
    int K = g->n_angles, D = g->n_det;
    double *cs = angle_table(g);
    if (!cs) return -2;
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < npix; ++i) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) {
            double u = pixel_u(g, cs[2 * k], cs[2 * k + 1], rows[i], cols[i]);
            acc += interp(q + (size_t)k * D, D, u);
        }
        out[i] = scale * acc;
    }
    free(cs);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Matched forward projector: every pixel splats its value onto the two     */
/* bins around its detector coordinate with the interpolation weights.      */
/* Written in scatter form, independently of the gather-form backprojector  */
/* above, so that the adjoint identity between them is a real check.        */
/* ------------------------------------------------------------------------ */
int oracle_forward(const double *f, const oracle_geometry *g, double *p)
{
    if (!f || !p || !geometry_ok(g)) return -1;
    int K = g->n_angles, D = g->n_det, N = g->n;
    double *cs = angle_table(g);
    if (!cs) return -2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k) {
        double *pk = p + (size_t)k * D;
        for (int j = 0; j < D; ++j) pk[j] = 0.0;
        for (int r = 0; r < N; ++r) {
            for (int c = 0; c < N; ++c) {
                double v = f[(size_t)r * N + c];
                double u = pixel_u(g, cs[2 * k], cs[2 * k + 1], r, c);
                double j0 = floor(u);
                double w = u - j0;
                long j = (long)j0;
                if (j >= 0 && j < D) pk[j] += (1.0 - w) * v;
                if (j + 1 >= 0 && j + 1 < D) pk[j + 1] += w * v;
            }
        }
    }
    free(cs);
    return 0;
}

/* Full FBP: filter, then backproject with scale = angle_step. */
int oracle_fbp(const double *p, const oracle_geometry *g, int kind, double *f)
{
    if (!p || !f || !geometry_ok(g)) return -1;
    size_t n = (size_t)g->n_angles * (size_t)g->n_det;
    double *q = (double *)malloc(sizeof(double) * (n ? n : 1));
    if (!q) return -2;
    int rc = oracle_filter(p, g->n_angles, g->n_det, kind, g->det_spacing, q);
    if (rc == 0) rc = oracle_backproject(q, g, g->angle_step, f);
    free(q);
    return rc;
}

/* Thread count the OpenMP runtime will use (for reporting). */
#ifdef _OPENMP
#include <omp.h>
int oracle_num_threads(void) { return omp_get_max_threads(); }
#else
int oracle_num_threads(void) { return 1; }
#endif
