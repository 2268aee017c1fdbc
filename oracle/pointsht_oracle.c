/*
 * pointsht_oracle.c -- plain FP64 CPU oracle for the direct, pixel-free
 * spherical-harmonic transform of a weighted point catalog.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * What it computes, in the paper's own order and notation
 * (Baleato Lizancos & White, "Harmonic analysis of discrete tracers of
 * large-scale structure", arXiv:2312.12285):
 *
 *   a_lm = sum_i w_i Y*_lm(theta_i, phi_i)                       (Eq. alm_def)
 *   Y_lm = sqrt((2l+1)/4pi) Pbar_l^m(x) e^{i m phi},  x = cos(theta),
 *          m >= 0                                                  (App. A)
 *   Pbar_0^0 = 1
 *   Pbar_m^m = -sqrt(1-x^2) sqrt(1 - 1/(2m)) Pbar_{m-1}^{m-1}      (App. A)
 *   Pbar_{m+1}^m = sqrt(2m+1) x Pbar_m^m                            (App. A)
 *   Pbar_l^m = sqrt((l-m)/(l+m)) [ (2l-1)/(l-m) x Pbar_{l-1}^m
 *              - sqrt((l-m-1)/(l+m-1)) (l+m-1)/(l-m) Pbar_{l-2}^m ] (App. A)
 *
 * The paper is silent on underflow: Pbar_m^m ~ (1-x^2)^{m/2} leaves the
 * FP64 range for large m near the poles.  Every Pbar here is therefore
 * carried as a mantissa with a separate binary exponent (value = v * 2^e),
 * rescaled by exact powers of two only, and converted to a double with
 * ldexp() at the point of use, so that each value is the correctly rounded
 * FP64 number of the scaled recurrence (tiny values round to 0 or to a
 * subnormal, exactly as plain FP64 would give them, nothing is cut off).
 *
 * Summation over points uses Neumaier-compensated FP64 sums over a fixed
 * partition of the point range (64 contiguous ranges, combined in order), so
 * results are independent of the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288
#define ORACLE_NBLOCKS 64
/* rescaling unit of the mantissa/exponent representation */
#define ORACLE_SCALE_BITS 256

/* Neumaier compensated accumulator. */
typedef struct { double s, c; } nsum;

static inline void nsum_add(nsum* a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static inline double nsum_val(const nsum* a) { return a->s + a->c; }

/* Recurrence coefficients of App. A for one order m, l = m+2..lmax:
 *   c1[l] = sqrt((l-m)/(l+m)) (2l-1)/(l-m)
 *   c2[l] = sqrt((l-m)/(l+m)) sqrt((l-m-1)/(l+m-1)) (l+m-1)/(l-m)
 * so that Pbar_l = c1[l] x Pbar_{l-1} - c2[l] Pbar_{l-2}.                  */
static void pbar_coeffs(int lmax, int m, double* c1, double* c2) {
    for (int l = m + 2; l <= lmax; ++l) {
        double lm = (double)(l - m), lp = (double)(l + m);
        double r = sqrt(lm / lp);
        c1[l] = r * (2.0 * l - 1.0) / lm;
        c2[l] = r * sqrt((lm - 1.0) / (lp - 1.0)) * (lp - 1.0) / lm;
    }
}

/* Sectoral value Pbar_m^m(x) as (v, e), value = v * 2^e, by the App. A
 * recurrence taken from Pbar_0^0 = 1 upward in m.                          */
static void pbar_sectoral(double x, int m, double* v_out, int* e_out) {
    double s = sqrt((1.0 - x) * (1.0 + x)); /* sqrt(1-x^2) */
    double v = 1.0;
    int e = 0;
    for (int k = 1; k <= m; ++k) {
        v *= -s * sqrt(1.0 - 1.0 / (2.0 * k));
        if (v != 0.0 && fabs(v) < 0x1p-256) {
            v *= 0x1p256;
            e -= ORACLE_SCALE_BITS;
        }
    }
    *v_out = v;
    *e_out = e;
}

/* Pbar_l^m(x) for l = m..lmax (App. A), written as mantissa/exponent pairs
 * (value = mant[l-m] * 2^expo[l-m]).  c1/c2 are from pbar_coeffs().        */
static void pbar_column_scaled(double x, int lmax, int m, const double* c1,
                               const double* c2, double* mant, int* expo) {
    double v0;
    int e;
    pbar_sectoral(x, m, &v0, &e);
    mant[0] = v0;
    expo[0] = e;
    if (lmax == m) return;
    double v1 = sqrt(2.0 * m + 1.0) * x * v0; /* Pbar_{m+1}^m */
    mant[1] = v1;
    expo[1] = e;
    double pm2 = v0, pm1 = v1;
    for (int l = m + 2; l <= lmax; ++l) {
        double p = c1[l] * x * pm1 - c2[l] * pm2;
        pm2 = pm1;
        pm1 = p;
        if (e < 0 && fabs(p) > 0x1p256) {
            /* both carried values share the exponent: rescale both exactly */
            pm1 *= 0x1p-256;
            pm2 *= 0x1p-256;
            e += ORACLE_SCALE_BITS;
        }
        mant[l - m] = pm1;
        expo[l - m] = e;
    }
}

/* ---------------------------------------------------------------- API --- */

/* Pbar_l^m(x), l = m..lmax, as mantissa/exponent pairs (for pins that need
 * values below the FP64 range).                                            */
void oracle_pbar_scaled(double x, int lmax, int m, double* mant, int* expo) {
    double* c1 = (double*)calloc((size_t)lmax + 1, sizeof(double));
    double* c2 = (double*)calloc((size_t)lmax + 1, sizeof(double));
    pbar_coeffs(lmax, m, c1, c2);
    pbar_column_scaled(x, lmax, m, c1, c2, mant, expo);
    free(c1);
    free(c2);
}

/* Y_lm(theta, phi) for l = m..lmax at one point (App. A + Eq. for Y_lm),
 * out interleaved (re, im), length 2*(lmax-m+1).                          */
void oracle_ylm(double x, double phi, int lmax, int m, double* out) {
    int len = lmax - m + 1;
    double* mant = (double*)malloc(sizeof(double) * (size_t)len);
    int* expo = (int*)malloc(sizeof(int) * (size_t)len);
    oracle_pbar_scaled(x, lmax, m, mant, expo);
    double c = cos((double)m * phi), s = sin((double)m * phi);
    for (int l = m; l <= lmax; ++l) {
        double lam = sqrt((2.0 * l + 1.0) / (4.0 * ORACLE_PI)) *
                     ldexp(mant[l - m], expo[l - m]);
        out[2 * (l - m)] = lam * c;
        out[2 * (l - m) + 1] = lam * s;
    }
    free(mant);
    free(expo);
}

/* a_lm = sum_i w_i Y*_lm(n_i)  (Eq. alm_def) for the orders listed in mlist.
 * Output: for each listed m (in list order) the column l = m..lmax,
 * interleaved (re, im), packed one column after another.  Returns 0 on
 * success, -1 on a bad argument, -2 on allocation failure.                */
int oracle_alm(int64_t n, const double* x, const double* phi, const double* w,
               int lmax, int nm, const int* mlist, double* out, int nthreads) {
    if (n < 0 || lmax < 0 || nm < 0) return -1;
    for (int k = 0; k < nm; ++k)
        if (mlist[k] < 0 || mlist[k] > lmax) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int64_t off = 0;
    int status = 0;
    for (int k = 0; k < nm; ++k) {
        const int m = mlist[k];
        const int len = lmax - m + 1;
        double* c1 = (double*)calloc((size_t)lmax + 1, sizeof(double));
        double* c2 = (double*)calloc((size_t)lmax + 1, sizeof(double));
        double* norm = (double*)malloc(sizeof(double) * (size_t)len);
        nsum* blk = (nsum*)calloc((size_t)ORACLE_NBLOCKS * 2 * (size_t)len, sizeof(nsum));
        if (!c1 || !c2 || !norm || !blk) {
            free(c1); free(c2); free(norm); free(blk);
            return -2;
        }
        pbar_coeffs(lmax, m, c1, c2);
        for (int l = m; l <= lmax; ++l)
            norm[l - m] = sqrt((2.0 * l + 1.0) / (4.0 * ORACLE_PI));
#pragma omp parallel for schedule(dynamic, 1)
        for (int b = 0; b < ORACLE_NBLOCKS; ++b) {
            int64_t i0 = n * b / ORACLE_NBLOCKS, i1 = n * (b + 1) / ORACLE_NBLOCKS;
            double* mant = (double*)malloc(sizeof(double) * (size_t)len);
            int* expo = (int*)malloc(sizeof(int) * (size_t)len);
            nsum* acc = blk + (size_t)b * 2 * (size_t)len;
            if (!mant || !expo) {
#pragma omp critical
                status = -2;
                free(mant); free(expo);
                continue;
            }
            for (int64_t i = i0; i < i1; ++i) {
                pbar_column_scaled(x[i], lmax, m, c1, c2, mant, expo);
                /* w Y* = w lambda (cos m phi - i sin m phi) */
                double ph = (double)m * phi[i];
                double wc = w[i] * cos(ph), ws = -w[i] * sin(ph);
                for (int q = 0; q < len; ++q) {
                    double lam = norm[q] * ldexp(mant[q], expo[q]);
                    nsum_add(&acc[2 * q], lam * wc);
                    nsum_add(&acc[2 * q + 1], lam * ws);
                }
            }
            free(mant);
            free(expo);
        }
        for (int q = 0; q < len; ++q) {
            nsum re = {0.0, 0.0}, im = {0.0, 0.0};
            for (int b = 0; b < ORACLE_NBLOCKS; ++b) {
                nsum_add(&re, nsum_val(&blk[(size_t)b * 2 * len + 2 * q]));
                nsum_add(&im, nsum_val(&blk[(size_t)b * 2 * len + 2 * q + 1]));
            }
            out[2 * (off + q)] = nsum_val(&re);
            out[2 * (off + q) + 1] = nsum_val(&im);
        }
        off += len;
        free(c1); free(c2); free(norm); free(blk);
        if (status) return status;
    }
    return status;
}

/* Point-evaluation of sum_{l,m>=0} lambda_lm(x_i) Re(g_lm e^{i m phi_i}) for
 * listed points: the adjoint of oracle_alm with respect to w_i, written from
 * the same definition (d a_lm / d w_i = Y*_lm(n_i)).  g is the full packed
 * m-major triangle (index m(2L+1-m)/2 + l), interleaved (re, im).          */
int oracle_adjoint(int64_t n, const double* x, const double* phi, int lmax,
                   const double* g, double* out, int nthreads) {
    if (n < 0 || lmax < 0) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int status = 0;
#pragma omp parallel
    {
        double* c1 = (double*)calloc((size_t)lmax + 1, sizeof(double));
        double* c2 = (double*)calloc((size_t)lmax + 1, sizeof(double));
        double* mant = (double*)malloc(sizeof(double) * ((size_t)lmax + 1));
        int* expo = (int*)malloc(sizeof(int) * ((size_t)lmax + 1));
        if (!c1 || !c2 || !mant || !expo) {
#pragma omp critical
            status = -2;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t i = 0; i < n; ++i) {
                nsum acc = {0.0, 0.0};
                for (int m = 0; m <= lmax; ++m) {
                    pbar_coeffs(lmax, m, c1, c2);
                    pbar_column_scaled(x[i], lmax, m, c1, c2, mant, expo);
                    double ph = (double)m * phi[i];
                    double c = cos(ph), s = sin(ph);
                    int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2;
                    for (int l = m; l <= lmax; ++l) {
                        double lam = sqrt((2.0 * l + 1.0) / (4.0 * ORACLE_PI)) *
                                     ldexp(mant[l - m], expo[l - m]);
                        const double* gl = g + 2 * (base + l);
                        nsum_add(&acc, lam * (gl[0] * c - gl[1] * s));
                    }
                }
                out[i] = nsum_val(&acc);
            }
        }
        free(c1); free(c2); free(mant); free(expo);
    }
    return status;
}

/* ------------------------------------------------ interpolated transform --
 * The paper's interpolation route (App. "Interpolation"): the smooth
 * y_lm = lambda_lm(cos theta) is known exactly (value and derivative, App. A)
 * on a set of sample points only, and each point's y_lm is the cubic Hermite
 * spline through its two neighbouring samples.  Because the spline is linear
 * in the sampled values, the sum over points is done first, per order m:
 *
 *   v^(m)_{j alpha} = sum_r w_r e^{-i m phi_r} c_{j alpha}(r)
 *   a_lm = sum_j [v_j0 y(s_j) + v_j1 h y'(s_j) + v_j2 y(s_{j+1}) + v_j3 h y'(s_{j+1})]
 *
 * with c_0 = (2t+1)(1-t)^2, c_1 = t(1-t)^2, c_2 = t^2(3-2t), c_3 = t^2(t-1).
 *
 * Reading (the paper samples in x = cos theta and treats |x| > 3/4 apart):
 * here the samples are equispaced in theta, s_k = (k + 1/2) h, h = pi/N,
 * k = 0..N-1, and y' is the theta-derivative.  In theta, y_lm is smooth up to
 * and through the poles once it is continued across them as the function on
 * the great circle, y(-theta) = (-1)^m y(theta) (the point (-theta, phi) is
 * (theta, phi + pi)), and likewise at theta = pi; the two outermost intervals
 * use ghost samples at -h/2 and pi + h/2 given by that continuation, so no
 * point needs separate treatment.  The theta-derivative follows from App. A's
 * derivative of Pbar: d/dtheta = -sin(theta) d/dx,
 *   dPbar_l/dtheta = [l x Pbar_l - (l+m) sqrt((l-m)/(l+m)) Pbar_{l-1}] / sin(theta).
 * All arithmetic in FP64; sums over points and samples Neumaier-compensated. */

/* Hermite basis of the interpolation section at parameter t in [0, 1]. */
void oracle_hermite_basis(double t, double* c) {
    c[0] = (2.0 * t + 1.0) * (1.0 - t) * (1.0 - t);
    c[1] = t * (1.0 - t) * (1.0 - t);
    c[2] = t * t * (3.0 - 2.0 * t);
    c[3] = t * t * (t - 1.0);
}

/* Interval of a point: theta = arccos(x), u = theta/h - 1/2, j = floor(u)
 * clamped to [-1, N-1] (left sample j, right sample j+1), t = u - j.       */
static void interp_interval(double x, int ntheta, int* j_out, double* t_out) {
    double xc = x > 1.0 ? 1.0 : (x < -1.0 ? -1.0 : x);
    double h = ORACLE_PI / (double)ntheta;
    double u = acos(xc) / h - 0.5;
    int j = (int)floor(u);
    if (j < -1) j = -1;
    if (j > ntheta - 1) j = ntheta - 1;
    double t = u - (double)j;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    *j_out = j;
    *t_out = t;
}

/* y_lm(s_k) and h dy_lm/dtheta(s_k) for l = m..lmax at every sample k, as
 * [k][l-m] arrays.                                                          */
static void interp_samples(int ntheta, int lmax, int m, const double* c1, const double* c2, double* ys, double* ds,
                           double* mant, int* expo) {
    const int len = lmax - m + 1;
    const double h = ORACLE_PI / (double)ntheta;
    for (int k = 0; k < ntheta; ++k) {
        double th = (k + 0.5) * h;
        double x = cos(th), s = sin(th);
        pbar_column_scaled(x, lmax, m, c1, c2, mant, expo);
        double prev = 0.0; /* Pbar_{l-1}^m */
        for (int l = m; l <= lmax; ++l) {
            double p = ldexp(mant[l - m], expo[l - m]);
            double dp = (double)l * x * p;
            if (l > m) dp -= (double)(l + m) * sqrt((double)(l - m) / (double)(l + m)) * prev;
            dp /= s;
            double nrm = sqrt((2.0 * l + 1.0) / (4.0 * ORACLE_PI));
            ys[(size_t)k * len + (l - m)] = nrm * p;
            ds[(size_t)k * len + (l - m)] = nrm * h * dp;
            prev = p;
        }
    }
}

/* Interpolated a_lm (full packed triangle, interleaved re/im) of one weighted
 * point set with N = ntheta samples in theta.  Returns 0, -1 (bad argument)
 * or -2 (allocation).                                                       */
int oracle_alm_interp(int64_t n, const double* x, const double* phi, const double* w, int lmax, int ntheta,
                      double* out, int nthreads) {
    if (n < 0 || lmax < 0 || ntheta < 2) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int* jr = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    double* cr = (double*)malloc(sizeof(double) * 4 * (size_t)(n > 0 ? n : 1));
    if (!jr || !cr) {
        free(jr); free(cr);
        return -2;
    }
    for (int64_t r = 0; r < n; ++r) {
        double t;
        interp_interval(x[r], ntheta, &jr[r], &t);
        oracle_hermite_basis(t, cr + 4 * r);
    }
    int status = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int m = 0; m <= lmax; ++m) {
        const int len = lmax - m + 1;
        const int nb = ntheta + 1; /* intervals j = -1..N-1 */
        double* c1 = (double*)calloc((size_t)lmax + 1, sizeof(double));
        double* c2 = (double*)calloc((size_t)lmax + 1, sizeof(double));
        double* mant = (double*)malloc(sizeof(double) * (size_t)len);
        int* expo = (int*)malloc(sizeof(int) * (size_t)len);
        double* ys = (double*)malloc(sizeof(double) * (size_t)ntheta * len);
        double* ds = (double*)malloc(sizeof(double) * (size_t)ntheta * len);
        nsum* v = (nsum*)calloc((size_t)nb * 8, sizeof(nsum));  /* [interval][alpha][re, im] */
        nsum* vy = (nsum*)calloc((size_t)ntheta * 2, sizeof(nsum));
        nsum* vd = (nsum*)calloc((size_t)ntheta * 2, sizeof(nsum));
        if (!c1 || !c2 || !mant || !expo || !ys || !ds || !v || !vy || !vd) {
#pragma omp critical
            status = -2;
        } else {
            pbar_coeffs(lmax, m, c1, c2);
            interp_samples(ntheta, lmax, m, c1, c2, ys, ds, mant, expo);
            /* v^(m)_{j alpha}: sum over points, within their interval */
            for (int64_t r = 0; r < n; ++r) {
                double ph = (double)m * phi[r];
                double wc = w[r] * cos(ph), ws = -w[r] * sin(ph);
                nsum* vb = v + (size_t)(jr[r] + 1) * 8;
                for (int a = 0; a < 4; ++a) {
                    nsum_add(&vb[2 * a], cr[4 * r + a] * wc);
                    nsum_add(&vb[2 * a + 1], cr[4 * r + a] * ws);
                }
            }
            /* per sample: left-sample terms of its interval, right-sample terms
             * of the previous one; the ghosts fold onto the end samples */
            const double sg = (m & 1) ? -1.0 : 1.0;
            for (int b = 0; b < nb; ++b) {
                const int j = b - 1;
                for (int ri = 0; ri < 2; ++ri) {
                    double v0 = nsum_val(&v[(size_t)b * 8 + 0 + ri]), v1 = nsum_val(&v[(size_t)b * 8 + 2 + ri]);
                    double v2 = nsum_val(&v[(size_t)b * 8 + 4 + ri]), v3 = nsum_val(&v[(size_t)b * 8 + 6 + ri]);
                    if (j >= 0) {
                        nsum_add(&vy[2 * j + ri], v0);
                        nsum_add(&vd[2 * j + ri], v1);
                    } else {
                        nsum_add(&vy[0 + ri], sg * v0);
                        nsum_add(&vd[0 + ri], -sg * v1);
                    }
                    if (j + 1 <= ntheta - 1) {
                        nsum_add(&vy[2 * (j + 1) + ri], v2);
                        nsum_add(&vd[2 * (j + 1) + ri], v3);
                    } else {
                        nsum_add(&vy[2 * (ntheta - 1) + ri], sg * v2);
                        nsum_add(&vd[2 * (ntheta - 1) + ri], -sg * v3);
                    }
                }
            }
            const int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2;
            for (int q = 0; q < len; ++q) {
                nsum re = {0.0, 0.0}, im = {0.0, 0.0};
                for (int k = 0; k < ntheta; ++k) {
                    double y = ys[(size_t)k * len + q], d = ds[(size_t)k * len + q];
                    nsum_add(&re, nsum_val(&vy[2 * k]) * y);
                    nsum_add(&re, nsum_val(&vd[2 * k]) * d);
                    nsum_add(&im, nsum_val(&vy[2 * k + 1]) * y);
                    nsum_add(&im, nsum_val(&vd[2 * k + 1]) * d);
                }
                out[2 * (base + m + q)] = nsum_val(&re);
                out[2 * (base + m + q) + 1] = nsum_val(&im);
            }
        }
        free(c1); free(c2); free(mant); free(expo); free(ys); free(ds); free(v); free(vy); free(vd);
    }
    free(jr);
    free(cr);
    return status;
}

/* ------------------------------------------------------------------------
 * Mode coupling (Eq. chat) and the Wigner 3j symbol with zero orders
 * (App. "Wigner 3j symbols").
 *
 * For l1 + l2 + l3 = 2g even and the triangle condition met,
 *   (l1 l2 l3; 0 0 0) = (-1)^g sqrt[(2g-2l1)! (2g-2l2)! (2g-2l3)! / (2g+1)!]
 *                       g! / [(g-l1)! (g-l2)! (g-l3)!],
 * zero otherwise: the textbook closed form for zero orders (the paper's
 * recurrence in App. "Wigner 3j symbols" steps along it).  Factorials enter
 * through a long-double table of log n! (lgammal), so each value carries
 * about 1e-14 relative error up to l ~ 1e4.
 *
 *   M_ll' = (2l'+1)/(4 pi) sum_lambda (2 lambda + 1) (l l' lambda; 0 0 0)^2 W_lambda
 * (Eq. chat), lambda over |l - l'| .. min(l + l', lmax_w), summed in
 * increasing lambda with a Neumaier accumulator.
 * ---------------------------------------------------------------------- */
static long double* logfact_table(int nmax) {
    long double* t = (long double*)malloc(sizeof(long double) * (size_t)(nmax + 1));
    if (!t) return NULL;
    for (int n = 0; n <= nmax; ++n) t[n] = lgammal((long double)n + 1.0L);
    return t;
}

static double threej000_lf(const long double* lf, int l1, int l2, int l3) {
    const int L = l1 + l2 + l3;
    if (L & 1) return 0.0;
    if (l3 < abs(l1 - l2) || l3 > l1 + l2) return 0.0;
    const int g = L / 2;
    const long double lg = 0.5L * (lf[2 * g - 2 * l1] + lf[2 * g - 2 * l2] + lf[2 * g - 2 * l3] - lf[2 * g + 1]) +
                           lf[g] - lf[g - l1] - lf[g - l2] - lf[g - l3];
    const double v = (double)expl(lg);
    return (g & 1) ? -v : v;
}

double oracle_threej000(int l1, int l2, int l3) {
    if (l1 < 0 || l2 < 0 || l3 < 0) return 0.0;
    long double* lf = logfact_table(l1 + l2 + l3 + 1);
    if (!lf) return NAN;
    const double v = threej000_lf(lf, l1, l2, l3);
    free(lf);
    return v;
}

/* M[l * (lmax + 1) + l'] for 0 <= l, l' <= lmax from W[0..lmax_w]. */
int oracle_coupling(int lmax, int lmax_w, const double* W, double* M, int nthreads) {
    if (lmax < 0 || lmax_w < 0) return 1;
    long double* lf = logfact_table(2 * lmax + lmax_w + 2);
    if (!lf) return 2;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int l = 0; l <= lmax; ++l) {
        for (int lp = 0; lp <= lmax; ++lp) {
            nsum acc = {0.0, 0.0};
            const int lo = abs(l - lp), hi = (l + lp < lmax_w) ? l + lp : lmax_w;
            for (int lam = lo; lam <= hi; ++lam) {
                const double tj = threej000_lf(lf, l, lp, lam);
                if (tj == 0.0) continue;
                nsum_add(&acc, (2.0 * lam + 1.0) * tj * tj * W[lam]);
            }
            M[(int64_t)l * (lmax + 1) + lp] = (2.0 * lp + 1.0) / (4.0 * ORACLE_PI) * nsum_val(&acc);
        }
    }
    free(lf);
    return 0;
}

/* One row l of M (for sampled checks at large lmax). */
int oracle_coupling_row(int lmax, int lmax_w, const double* W, int l, double* row) {
    if (lmax < 0 || lmax_w < 0 || l < 0 || l > lmax) return 1;
    long double* lf = logfact_table(2 * lmax + lmax_w + 2);
    if (!lf) return 2;
    for (int lp = 0; lp <= lmax; ++lp) {
        nsum acc = {0.0, 0.0};
        const int lo = abs(l - lp), hi = (l + lp < lmax_w) ? l + lp : lmax_w;
        for (int lam = lo; lam <= hi; ++lam) {
            const double tj = threej000_lf(lf, l, lp, lam);
            if (tj == 0.0) continue;
            nsum_add(&acc, (2.0 * lam + 1.0) * tj * tj * W[lam]);
        }
        row[lp] = (2.0 * lp + 1.0) / (4.0 * ORACLE_PI) * nsum_val(&acc);
    }
    free(lf);
    return 0;
}

/* ------------------------------------------------------------------------
 * Point-evaluation synthesis: f(n_i) = sum_{l} sum_{m=-l}^{l} a_lm Y_lm(n_i)
 * of a real field given by its m >= 0 coefficients, with the negative orders
 * written out from a_{l,-m} = (-1)^m conj(a_lm) and
 * Y_{l,-m} = (-1)^m conj(Y_lm) (App. A's Y_lm, Condon-Shortley phase).
 * out_re gets the real part; out_im (optional) the imaginary part, which is
 * zero for a real field up to rounding.
 * ---------------------------------------------------------------------- */
int oracle_synthesis(int64_t n, const double* x, const double* phi, int lmax, const double* a, double* out_re,
                     double* out_im, int nthreads) {
    if (n < 0 || lmax < 0) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int status = 0;
#pragma omp parallel
    {
        double* c1 = (double*)calloc((size_t)lmax + 1, sizeof(double));
        double* c2 = (double*)calloc((size_t)lmax + 1, sizeof(double));
        double* mant = (double*)malloc(sizeof(double) * ((size_t)lmax + 1));
        int* expo = (int*)malloc(sizeof(int) * ((size_t)lmax + 1));
        if (!c1 || !c2 || !mant || !expo) {
#pragma omp critical
            status = -2;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t i = 0; i < n; ++i) {
                nsum re = {0.0, 0.0}, im = {0.0, 0.0};
                for (int m = 0; m <= lmax; ++m) {
                    pbar_coeffs(lmax, m, c1, c2);
                    pbar_column_scaled(x[i], lmax, m, c1, c2, mant, expo);
                    const double c = cos((double)m * phi[i]), s = sin((double)m * phi[i]);
                    const int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2;
                    const double sg = (m & 1) ? -1.0 : 1.0;
                    for (int l = m; l <= lmax; ++l) {
                        const double lam = sqrt((2.0 * l + 1.0) / (4.0 * ORACLE_PI)) * ldexp(mant[l - m], expo[l - m]);
                        const double yr = lam * c, yi = lam * s;       /* Y_lm */
                        const double ar = a[2 * (base + l)], ai = a[2 * (base + l) + 1];
                        nsum_add(&re, ar * yr - ai * yi);               /* a_lm Y_lm */
                        nsum_add(&im, ar * yi + ai * yr);
                        if (m > 0) {                                    /* a_{l,-m} Y_{l,-m} */
                            const double br = sg * ar, bi = -sg * ai;   /* (-1)^m conj(a_lm) */
                            const double zr = sg * yr, zi = -sg * yi;   /* (-1)^m conj(Y_lm) */
                            nsum_add(&re, br * zr - bi * zi);
                            nsum_add(&im, br * zi + bi * zr);
                        }
                    }
                }
                out_re[i] = nsum_val(&re);
                if (out_im) out_im[i] = nsum_val(&im);
            }
        }
        free(c1); free(c2); free(mant); free(expo);
    }
    return status;
}

/* ------------------------------------------------------------------------
 * Spin-weighted harmonics for a spin-2 (shear) field.  The paper names the
 * generalisation (Sec. 4: use _{+-2}Y_lm, computed by recurrence) without
 * printing it; this is the textbook form through Wigner's small d:
 *
 *   _sY_lm(theta, phi) = (-1)^s sqrt((2l+1)/4pi) d^l_{m,-s}(theta) e^{i m phi},
 *
 * (for s = 0 the Y_lm of App. A), so for m >= 0
 *   _{+2}Y*_lm = lambda^(-2)_lm e^{-i m phi},  _{-2}Y*_lm = lambda^(+2)_lm e^{-i m phi},
 *   lambda^(n)_lm(theta) = sqrt((2l+1)/4pi) d^l_{m,n}(theta).
 * Seed at l0 = max(m, |n|) from the top row of d,
 *   d^l_{l,k}(b) = (-1)^(l-k) sqrt((2l)! / ((l+k)! (l-k)!)) cos^(l+k)(b/2) sin^(l-k)(b/2),
 * with d^l_{m,n} = (-1)^(m-n) d^l_{n,m} = d^l_{-n,-m}; then the three-term
 * recurrence of d in l at fixed (m, n), written for lambda:
 *   lambda_{l+1} = (A_l x + B_l) lambda_l - C_l lambda_{l-1},
 *   A_l = sqrt((2l+3)(2l+1)) (l+1) / R_{l+1},
 *   B_l = -sqrt((2l+3)(2l+1)) m n / (l R_{l+1}),
 *   C_l = sqrt((2l+3)/(2l-1)) (l+1) R_l / (l R_{l+1}),
 *   R_l = sqrt((l^2 - m^2)(l^2 - n^2)).
 * Values are carried as mantissa and binary exponent like Pbar above (the
 * seed ~ cos^p(theta/2) sin^q(theta/2) leaves the FP64 range at high m).
 * The seed's logarithm is taken in long double (lgammal, log2l).
 *
 *   _{+-2}a_lm = sum_i w_i (g1 +- i g2)_i _{+-2}Y*_lm(n_i),
 *   E_lm = -(_{2}a_lm + _{-2}a_lm) / 2,   B_lm = i (_{2}a_lm - _{-2}a_lm) / 2,
 * the usual E/B split of a spin-2 field (g1, g2) (as for Q, U).
 * ---------------------------------------------------------------------- */
static void spin_seed(double x, int m, int n, double* v, int* e, int* l0_out) {
    const int an = n < 0 ? -n : n;
    const int l0 = m > an ? m : an;
    int k, sgn = 1;
    if (m >= an) {
        k = n;                        /* d^m_{m,n}: top row */
    } else if (n > 0) {
        k = m;                        /* d^n_{m,n} = (-1)^(m-n) d^n_{n,m} */
        if ((n - m) & 1) sgn = -sgn;
    } else {
        k = -m;                       /* d^l0_{m,-l0} = d^l0_{l0,-m} */
    }
    if ((l0 - k) & 1) sgn = -sgn;
    const int pc = l0 + k, ps = l0 - k;
    const double c2 = 0.5 * (1.0 + x), s2 = 0.5 * (1.0 - x); /* cos^2, sin^2 of theta/2 */
    *l0_out = l0;
    if ((pc > 0 && !(c2 > 0.0)) || (ps > 0 && !(s2 > 0.0))) {
        *v = 0.0;
        *e = 0;
        return;
    }
    long double lg = 0.5L * log2l((2.0L * l0 + 1.0L) / (4.0L * (long double)ORACLE_PI)) +
                     0.5L * (lgammal(2.0L * l0 + 1.0L) - lgammal((long double)(l0 + k) + 1.0L) -
                             lgammal((long double)(l0 - k) + 1.0L)) / logl(2.0L);
    if (pc > 0) lg += 0.5L * pc * log2l((long double)c2);
    if (ps > 0) lg += 0.5L * ps * log2l((long double)s2);
    const long double fl = floorl(lg);
    *v = sgn * (double)exp2l(lg - fl);
    *e = (int)fl;
}

/* lambda^(n)_lm(x) for l = 0..lmax as mantissa/exponent (zero below l0). */
static void spin_column_scaled(double x, int lmax, int m, int n, double* mant, int* expo) {
    for (int l = 0; l <= lmax; ++l) {
        mant[l] = 0.0;
        expo[l] = 0;
    }
    double v;
    int e, l0;
    spin_seed(x, m, n, &v, &e, &l0);
    if (l0 > lmax) return;
    mant[l0] = v;
    expo[l0] = e;
    double pm1 = v, pm2 = 0.0;
    const double mm = (double)m * m, nn = (double)n * n;
    for (int l = l0; l < lmax; ++l) {
        const double dl = (double)l;
        const double r1 = sqrt(((dl + 1) * (dl + 1) - mm) * ((dl + 1) * (dl + 1) - nn));
        const double q = sqrt((2 * dl + 3) * (2 * dl + 1));
        const double A = q * (dl + 1) / r1;
        const double B = (m == 0 || n == 0) ? 0.0 : -q * (double)m * (double)n / (dl * r1);
        const double C = (l == l0) ? 0.0
                                   : sqrt((2 * dl + 3) / (2 * dl - 1)) * (dl + 1) *
                                         sqrt((dl * dl - mm) * (dl * dl - nn)) / (dl * r1);
        double p = (A * x + B) * pm1 - C * pm2;
        pm2 = pm1;
        pm1 = p;
        if (e < 0 && fabs(p) > 0x1p256) {
            pm1 *= 0x1p-256;
            pm2 *= 0x1p-256;
            e += ORACLE_SCALE_BITS;
        }
        mant[l + 1] = pm1;
        expo[l + 1] = e;
    }
}

void oracle_spin_lambda(double x, int lmax, int m, int n, double* out) {
    double* mant = (double*)malloc(sizeof(double) * ((size_t)lmax + 1));
    int* expo = (int*)malloc(sizeof(int) * ((size_t)lmax + 1));
    spin_column_scaled(x, lmax, m, n, mant, expo);
    for (int l = 0; l <= lmax; ++l) out[l] = ldexp(mant[l], expo[l]);
    free(mant);
    free(expo);
}

/* E_lm, B_lm (packed m-major triangle, interleaved re/im) of the spin-2
 * field (g1, g2) carried by weighted points.  One order m per task, points
 * summed in order with Neumaier accumulators: independent of threads. */
int oracle_alm_spin2(int64_t np, const double* x, const double* phi, const double* w, const double* g1,
                     const double* g2, int lmax, double* E, double* B, int nthreads) {
    if (np < 0 || lmax < 0) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int status = 0;
#pragma omp parallel
    {
        const size_t L1 = (size_t)lmax + 1;
        double* mp = (double*)malloc(sizeof(double) * L1);
        double* mq = (double*)malloc(sizeof(double) * L1);
        int* ep = (int*)malloc(sizeof(int) * L1);
        int* eq = (int*)malloc(sizeof(int) * L1);
        nsum* acc = (nsum*)malloc(sizeof(nsum) * 4 * L1);
        if (!mp || !mq || !ep || !eq || !acc) {
#pragma omp critical
            status = -2;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int m = 0; m <= lmax; ++m) {
                memset(acc, 0, sizeof(nsum) * 4 * L1);
                for (int64_t i = 0; i < np; ++i) {
                    spin_column_scaled(x[i], lmax, m, -2, mp, ep); /* _{+2}Y* */
                    spin_column_scaled(x[i], lmax, m, +2, mq, eq); /* _{-2}Y* */
                    const double c = cos((double)m * phi[i]), s = -sin((double)m * phi[i]); /* e^{-i m phi} */
                    const double pr = w[i] * (g1[i] * c - g2[i] * s), pi_ = w[i] * (g1[i] * s + g2[i] * c);
                    const double qr = w[i] * (g1[i] * c + g2[i] * s), qi = w[i] * (g1[i] * s * 1.0 - g2[i] * c);
                    for (int l = m > 2 ? m : 2; l <= lmax; ++l) {
                        const double lp = ldexp(mp[l], ep[l]), lq = ldexp(mq[l], eq[l]);
                        nsum_add(&acc[4 * l + 0], pr * lp);
                        nsum_add(&acc[4 * l + 1], pi_ * lp);
                        nsum_add(&acc[4 * l + 2], qr * lq);
                        nsum_add(&acc[4 * l + 3], qi * lq);
                    }
                }
                const int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2;
                for (int l = m; l <= lmax; ++l) {
                    double ar = 0, ai = 0, br = 0, bi = 0;
                    if (l >= 2) {
                        ar = nsum_val(&acc[4 * l]);
                        ai = nsum_val(&acc[4 * l + 1]);
                        br = nsum_val(&acc[4 * l + 2]);
                        bi = nsum_val(&acc[4 * l + 3]);
                    }
                    E[2 * (base + l)] = -0.5 * (ar + br);
                    E[2 * (base + l) + 1] = -0.5 * (ai + bi);
                    B[2 * (base + l)] = -0.5 * (ai - bi);
                    B[2 * (base + l) + 1] = 0.5 * (ar - br);
                }
            }
        }
        free(mp); free(mq); free(ep); free(eq); free(acc);
    }
    return status;
}

/* The same E/B transform for a list of orders only, summed over a fixed
 * partition of the points (64 contiguous ranges, Neumaier sums combined in
 * order): for sampled columns of large catalogs.  E/B out: [nm][lmax+1]
 * interleaved re/im, zero for l < max(m, 2). */
int oracle_alm_spin2_cols(int64_t np, const double* x, const double* phi, const double* w, const double* g1,
                          const double* g2, int lmax, int nm, const int* mlist, double* E, double* B, int nthreads) {
    if (np < 0 || lmax < 0 || nm < 0) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const size_t L1 = (size_t)lmax + 1;
    for (int t = 0; t < nm; ++t) {
        const int m = mlist[t];
        if (m < 0 || m > lmax) return -3;
        nsum* part = (nsum*)calloc((size_t)ORACLE_NBLOCKS * 4 * L1, sizeof(nsum));
        if (!part) return -2;
        int status = 0;
#pragma omp parallel
        {
            double* mp = (double*)malloc(sizeof(double) * L1);
            double* mq = (double*)malloc(sizeof(double) * L1);
            int* ep = (int*)malloc(sizeof(int) * L1);
            int* eq = (int*)malloc(sizeof(int) * L1);
            if (!mp || !mq || !ep || !eq) {
#pragma omp critical
                status = -2;
            } else {
#pragma omp for schedule(dynamic, 1)
                for (int blk = 0; blk < ORACLE_NBLOCKS; ++blk) {
                    const int64_t i0 = np * blk / ORACLE_NBLOCKS, i1 = np * (blk + 1) / ORACLE_NBLOCKS;
                    nsum* acc = part + (size_t)blk * 4 * L1;
                    for (int64_t i = i0; i < i1; ++i) {
                        spin_column_scaled(x[i], lmax, m, -2, mp, ep);
                        spin_column_scaled(x[i], lmax, m, +2, mq, eq);
                        const double c = cos((double)m * phi[i]), s = -sin((double)m * phi[i]);
                        const double pr = w[i] * (g1[i] * c - g2[i] * s), pi_ = w[i] * (g1[i] * s + g2[i] * c);
                        const double qr = w[i] * (g1[i] * c + g2[i] * s), qi = w[i] * (g1[i] * s - g2[i] * c);
                        for (int l = m > 2 ? m : 2; l <= lmax; ++l) {
                            const double lp = ldexp(mp[l], ep[l]), lq = ldexp(mq[l], eq[l]);
                            nsum_add(&acc[4 * l + 0], pr * lp);
                            nsum_add(&acc[4 * l + 1], pi_ * lp);
                            nsum_add(&acc[4 * l + 2], qr * lq);
                            nsum_add(&acc[4 * l + 3], qi * lq);
                        }
                    }
                }
            }
            free(mp); free(mq); free(ep); free(eq);
        }
        if (status) {
            free(part);
            return status;
        }
        for (size_t l = 0; l < L1; ++l) {
            nsum tot[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
            for (int blk = 0; blk < ORACLE_NBLOCKS; ++blk)
                for (int c = 0; c < 4; ++c) nsum_add(&tot[c], nsum_val(&part[((size_t)blk * 4 * L1) + 4 * l + c]));
            const double ar = nsum_val(&tot[0]), ai = nsum_val(&tot[1]), br = nsum_val(&tot[2]), bi = nsum_val(&tot[3]);
            double* e = E + 2 * ((size_t)t * L1 + l);
            double* b = B + 2 * ((size_t)t * L1 + l);
            e[0] = -0.5 * (ar + br);
            e[1] = -0.5 * (ai + bi);
            b[0] = -0.5 * (ai - bi);
            b[1] = 0.5 * (ar - br);
        }
        free(part);
    }
    return 0;
}
