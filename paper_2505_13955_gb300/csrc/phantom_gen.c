/*
 * phantom_gen.c -- seeded synthetic inputs: ellipse phantoms, their exact
 * (analytic) parallel-beam line integrals, and their rasterisation.
 *
 * This is the input generator that both the CUDA path and the FP64 oracle
 * consume.  It holds none of the filtered-backprojection arithmetic: it
 * evaluates the continuous Radon transform of ellipses in closed form
 * (Kak & Slaney ch. 3, the projection of an ellipse), not the discrete
 * projector or backprojector of the library.
 *
 * Ellipse parameters are rows of 6 doubles in unit-disk coordinates
 * (field-of-view radius 1 <-> R pixels):
 *     x0, y0   centre
 *     A, B     semi-axes (A along the direction phi, B across it)
 *     phi      rotation of the A axis from +x (radians)
 *     rho      density added inside the ellipse
 *
 * Pixel [r][c] of an N x N image has its centre at X = c - (N-1)/2,
 * Y = r - (N-1)/2 pixels.  Detector bin j has its centre at
 * s_j = (j - det_center) * det_spacing pixels, and the projection at angle
 * theta integrates along the lines X cos(theta) + Y sin(theta) = s.
 * Line integrals are returned in pixel units (density x pixels).
 */
#include <math.h>
#include <stdlib.h>

/*
 * out[k*D + j] = sum over ellipses of the line integral at (theta_k, s_j),
 *   p = 2 rho A B sqrt(a2 - t^2) / a2   for t^2 <= a2, else 0,
 *   a2 = A^2 cos^2(theta - phi) + B^2 sin^2(theta - phi),
 *   t  = s - (x0 cos theta + y0 sin theta),
 * all lengths in pixels (unit-disk values times R).
 * out_f64 and/or out_f32 may be NULL.
 */
int phantom_sinogram(const double *ell, int n_ell, int K, int D,
                     double angle_start, double angle_step, double det_center,
                     double det_spacing, double R, double *out_f64,
                     float *out_f32)
{
    if (K < 0 || D < 1 || n_ell < 0 || !(det_spacing > 0.0) || !(R > 0.0))
        return -1;
    if (n_ell > 0 && !ell) return -1;
#pragma omp parallel
    {
        double *row = (double *)malloc(sizeof(double) * (size_t)D);
#pragma omp for schedule(dynamic, 4)
        for (int k = 0; k < K; ++k) {
            if (!row) continue;
            double th = angle_start + (double)k * angle_step;
            double ct = cos(th), st = sin(th);
            for (int j = 0; j < D; ++j) row[j] = 0.0;
            for (int e = 0; e < n_ell; ++e) {
                const double *E = ell + 6 * (size_t)e;
                double x0 = E[0] * R, y0 = E[1] * R, A = E[2] * R, B = E[3] * R;
                double phi = E[4], rho = E[5];
                double cd = cos(th - phi), sd = sin(th - phi);
                double a2 = A * A * cd * cd + B * B * sd * sd;
                double a = sqrt(a2);
                double s0 = x0 * ct + y0 * st;
                /* bins whose centre lies within |s - s0| <= a */
                double jlo = ceil((s0 - a) / det_spacing + det_center);
                double jhi = floor((s0 + a) / det_spacing + det_center);
                if (jlo < 0.0) jlo = 0.0;
                if (jhi > (double)(D - 1)) jhi = (double)(D - 1);
                for (long j = (long)jlo; j <= (long)jhi; ++j) {
                    double t = ((double)j - det_center) * det_spacing - s0;
                    double r2 = a2 - t * t;
                    if (r2 > 0.0) row[j] += 2.0 * rho * A * B * sqrt(r2) / a2;
                }
            }
            if (out_f64)
                for (int j = 0; j < D; ++j) out_f64[(size_t)k * D + j] = row[j];
            if (out_f32)
                for (int j = 0; j < D; ++j) out_f32[(size_t)k * D + j] = (float)row[j];
        }
        free(row);
    }
    return 0;
}

/*
 * Rasterise: out[r*N + c] = sum of rho over ellipses containing the
 * centre of pixel [r][c] (ss = 1), or the mean over an ss x ss grid of
 * sub-pixel points (ss > 1).
 */
int phantom_image(const double *ell, int n_ell, int N, double R, int ss,
                  double *out)
{
    if (N < 0 || n_ell < 0 || ss < 1 || !(R > 0.0) || !out) return -1;
    if (n_ell > 0 && !ell) return -1;
#pragma omp parallel for schedule(dynamic, 8)
    for (int r = 0; r < N; ++r) {
        for (int c = 0; c < N; ++c) {
            double acc = 0.0;
            for (int a = 0; a < ss; ++a) {
                for (int b = 0; b < ss; ++b) {
                    double X = (double)c - 0.5 * (double)(N - 1) + ((double)b + 0.5) / ss - 0.5;
                    double Y = (double)r - 0.5 * (double)(N - 1) + ((double)a + 0.5) / ss - 0.5;
                    for (int e = 0; e < n_ell; ++e) {
                        const double *E = ell + 6 * (size_t)e;
                        double dx = X - E[0] * R, dy = Y - E[1] * R;
                        double cp = cos(E[4]), sp = sin(E[4]);
                        double xa = dx * cp + dy * sp;
                        double xb = -dx * sp + dy * cp;
                        double A = E[2] * R, B = E[3] * R;
                        if (xa * xa / (A * A) + xb * xb / (B * B) <= 1.0) acc += E[5];
                    }
                }
            }
            out[(size_t)r * N + c] = acc / (double)(ss * ss);
        }
    }
    return 0;
}

/*
 * Distance in pixels from the centre of pixel [r][c] to the nearest ellipse
 * boundary, estimated by sampling each boundary every `step` pixels of arc
 * (error <= step / 2), for masking edge pixels in accuracy checks.
 * Ellipses whose boundary provably lies farther than the best distance so
 * far are skipped.
 */
int phantom_edge_distance(const double *ell, int n_ell, int N, double R,
                          double step, double *out)
{
    if (N < 0 || n_ell < 0 || !(step > 0.0) || !(R > 0.0) || !out) return -1;
    if (n_ell > 0 && !ell) return -1;
    const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(dynamic, 8)
    for (int r = 0; r < N; ++r) {
        for (int c = 0; c < N; ++c) {
            double X = (double)c - 0.5 * (double)(N - 1);
            double Y = (double)r - 0.5 * (double)(N - 1);
            double best = 1e300;
            for (int e = 0; e < n_ell; ++e) {
                const double *E = ell + 6 * (size_t)e;
                double A = E[2] * R, B = E[3] * R, x0 = E[0] * R, y0 = E[1] * R;
                double big = A > B ? A : B, small = A > B ? B : A;
                double dc = sqrt((X - x0) * (X - x0) + (Y - y0) * (Y - y0));
                if (dc - big > best || small - dc > best) continue;
                double cp = cos(E[4]), sp = sin(E[4]);
                int n_samp = (int)ceil(two_pi * big / step);
                if (n_samp < 16) n_samp = 16;
                for (int i = 0; i < n_samp; ++i) {
                    double t = two_pi * (double)i / (double)n_samp;
                    double px = x0 + A * cos(t) * cp - B * sin(t) * sp;
                    double py = y0 + A * cos(t) * sp + B * sin(t) * cp;
                    double d2 = (px - X) * (px - X) + (py - Y) * (py - Y);
                    if (d2 < best * best) best = sqrt(d2);
                }
            }
            out[(size_t)r * N + c] = best;
        }
    }
    return 0;
}
