/*
 * pointsht.h -- C ABI of libpointsht: the direct, pixel-free spherical-harmonic
 * transform of weighted point catalogs, its pseudo-C_l and its adjoint, on one
 * GB300 GPU (sm_103a).
 *
 * Method: Baleato Lizancos & White, "Harmonic analysis of discrete tracers of
 * large-scale structure", arXiv:2312.12285.
 *   a_lm = sum_i w_i Y*_lm(theta_i, phi_i)                      (Eq. alm_def)
 *   field = data - alpha * randoms, transformed as one signed-weight sum
 *                                                          (Sec. 2.1, Sec. 2.3)
 *   C_l  = 1/(2l+1) sum_{m=-l..l} |a_lm|^2                      (Eq. pseudoCl)
 *   Y_lm = sqrt((2l+1)/4pi) Pbar_l^m(cos theta) e^{i m phi}     (App. A)
 *
 * Conventions shared by every call
 * --------------------------------
 * - All array arguments are DEVICE pointers owned by the caller unless a
 *   comment says "host".  The library never frees caller memory.  Apart from
 *   pointsht_plan_create (which allocates the plan's coefficient tables) no
 *   call allocates device memory: scratch space is the caller's workspace.
 * - Every call is asynchronous on the caller's CUDA stream `stream`
 *   (a cudaStream_t passed as void*; NULL = legacy default stream) and
 *   returns after enqueueing.  Argument errors are detected on the host and
 *   returned synchronously before anything is enqueued.  Errors found by a
 *   kernel (an input outside its domain, a bounded wait that gave up) are
 *   recorded in the plan and returned by pointsht_plan_check().
 * - Coefficients for m >= 0 only are stored (a_{l,-m} = (-1)^m conj(a_lm) for
 *   real weights, Sec. 2.2).  A set of coefficients for 0 <= m <= l <= lmax is
 *   a packed m-major triangle of M = (lmax+1)(lmax+2)/2 complex128 values
 *   (interleaved re, im), index(l, m) = m*(2*lmax+1-m)/2 + l.  The
 *   Condon-Shortley phase is included (the minus sign of the sectoral
 *   recurrence, App. A).
 * - Outputs are overwritten, never accumulated into.  Results are bitwise
 *   reproducible run to run for the same inputs and tuning (fixed reduction
 *   order, no floating-point atomics).
 * - Point coordinates: x = cos(theta) in [-1, 1], phi in radians (any finite
 *   value; reduced modulo 2pi internally).  Dtype follows the precision:
 *   double for POINTSHT_FP64, float for POINTSHT_FP32 / POINTSHT_MIXED.
 * - pointsht_last_error() returns a thread-local message for the last
 *   non-OK status returned on the calling thread.
 */
#ifndef POINTSHT_H
#define POINTSHT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    POINTSHT_OK = 0,
    POINTSHT_EINVAL = 1,   /* bad argument: null pointer, size, lmax, field index, alignment */
    POINTSHT_ERANGE = 2,   /* an input value outside its domain (|x| > 1, non-finite) */
    POINTSHT_ENOMEM = 3,   /* workspace too small, or plan allocation failed */
    POINTSHT_ECUDA = 4,    /* a CUDA runtime call failed (message has the CUDA error) */
    POINTSHT_EARCH = 5,    /* current device is not a compute-capability 10.3 GPU */
    POINTSHT_ETIMEOUT = 6  /* a bounded wait inside a kernel gave up */
} pointsht_status;

typedef enum {
    POINTSHT_FP64 = 0,  /* FP64 recurrence (App. A) on double inputs */
    POINTSHT_FP32 = 1,  /* FP32 recurrence, FP64-accurate seed and phase, FP64 sums */
    POINTSHT_MIXED = 2  /* FP32 recurrence, per-m contraction on tensor cores (fp16 hi+lo) */
} pointsht_precision;

/* One point catalog contributing to one output field with a coefficient:
 * +1 for data, -alpha for randoms (field n_g - alpha n_r, Sec. 2.1).  The
 * catalogs of one field are transformed together as one signed-weight sum.
 * Catalogs of one field must be different point sets. */
typedef struct {
    const void* x;    /* device, n values of cos(theta) */
    const void* phi;  /* device, n azimuths (radians) */
    const void* w;    /* device, n weights */
    int64_t n;        /* number of points, >= 0 */
    int32_t field;    /* output field index, 0 <= field < nfield */
    int32_t pad_;     /* set to 0 */
    double coeff;     /* coefficient of this catalog in its field */
} pointsht_catalog;

/* One catalog of a spin-2 (shear) field: positions, weights and the two
 * components (g1, g2) of the spin-2 quantity at each point (pointsht_alm_spin2).
 * FP32 device arrays of n values; coeff multiplies w. */
typedef struct {
    const void* x;    /* cos(theta) */
    const void* phi;  /* azimuth (radians) */
    const void* w;    /* weight */
    const void* g1;   /* first component (as Q) */
    const void* g2;   /* second component (as U) */
    int64_t n;
    int32_t field;
    int32_t pad_;     /* set to 0 */
    double coeff;
} pointsht_shear_catalog;

/* Opaque plan: recurrence tables for one lmax on one device.  Creating it
 * allocates and fills device tables (this is the only allocating call). */
typedef struct pointsht_plan_s* pointsht_plan;

/* Library version string, e.g. "1.0.0". */
const char* pointsht_version(void);

/* Message for the last non-OK status returned on this thread. */
const char* pointsht_last_error(void);

/* Create a plan for multipoles 0..lmax (1 <= lmax <= 8192) on the current CUDA
 * device.  Builds, in FP64 on the host, the recurrence tables of the
 * normalised functions lambda_lm = sqrt((2l+1)/4pi) Pbar_l^m (App. A) and
 * copies them to the device.  Returns EARCH on a device that is not sm_103,
 * ENOMEM if an allocation fails.  *out receives the plan (host handle). */
pointsht_status pointsht_plan_create(int32_t lmax, pointsht_plan* out);

/* Release a plan (synchronises its device).  NULL is ignored. */
void pointsht_plan_destroy(pointsht_plan plan);

/* lmax of a plan, or -1 for NULL. */
int32_t pointsht_plan_lmax(pointsht_plan plan);

/* Wait for the plan's device, then read and clear the error flags that
 * kernels recorded since the last check: returns ERANGE if some x was outside
 * [-1, 1] or some input was non-finite, ETIMEOUT if a bounded wait gave up,
 * OK otherwise. */
pointsht_status pointsht_plan_check(pointsht_plan plan);

/* Timing hook: while set, every pointsht_alm (and pointsht_alm_columns) call
 * on this plan records `start` on its stream immediately before launching the
 * analysis kernel(s) and `stop` immediately after, so
 * cudaEventElapsedTime(start, stop) is their device time.  start/stop are cudaEvent_t handles passed as void*
 * (created by the caller); NULL, NULL clears the hook.  The paper has no
 * counterpart; this exists for measurement only. */
pointsht_status pointsht_plan_set_timing_events(pointsht_plan plan, void* start, void* stop);

/* Tuning of the FP32 analysis kernel for this plan (the paper has no
 * counterpart; chosen by the autotuner): variant 0 = library default, or
 * 8 / 12 / 16 = points per lane with scalar FMAs, 116 = 16 points per lane as
 * f32x2 pairs, 108 = four warps sharing each order pair's accumulator (only
 * 116 carries the near-pole form, pointsht_plan_set_pole_threshold);
 * chunk_log2 0 = automatic, else log2 of the points per accumulation chunk
 * (10..22).  Changes the workspace size: query pointsht_workspace_size after
 * setting.  EINVAL for values outside these sets. */
pointsht_status pointsht_plan_set_tuning(pointsht_plan plan, int32_t variant, int32_t chunk_log2);

/* Accuracy near the poles (App. A recurrence, read numerically; the paper
 * does not discuss it).  Near x = +-1 the three-term recurrence in l has a
 * double root and FP32 rounding grows like l^1.5 eps there.  In the FP32
 * analysis (default variant) and the FP32 adjoint / synthesis, a tile (warp)
 * of points that all have x >= pole_x, or all x <= -pole_x, runs the
 * recurrence of orders m < 256 (at higher orders lambda_lm near the poles
 * carries sin^m theta and is negligible) in Reinsch's difference form on |x|
 * (relative error ~1e-6 of
 * the column maximum up to lmax 2048 at any x, instead of up to ~5e-3 at
 * theta ~ 1e-3): one more packed FP32 operation per point and step.  The
 * interpolated route's sample transform uses the same form, for orders
 * m < 64, in warps whose sample positions all have x >= min(pole_x, 0.75).  Default 0.9; a value
 * above 1 turns the form off everywhere.  EINVAL for values below 0.5 or NaN
 * (the form is less accurate than the standard one near x = 0). */
pointsht_status pointsht_plan_set_pole_threshold(pointsht_plan plan, float pole_x);

/* Measurement hook (the paper has no counterpart): while counters is not
 * NULL, every FP32 analysis launch of variant 116 adds to the device
 * array counters[2] (uint64, caller-owned, zeroed by the caller) the number of
 * 16-step recurrence blocks (times the warp's points) whose accumulation was
 * skipped because every point of the warp was still below the FP32 range
 * ([0]) and the number of all such blocks ([1]).  Their ratio is the fraction
 * of nominal (point, m, l) accumulation steps not executed (they contribute
 * exact zeros).  NULL turns it off.  EINVAL if counters is not 8-byte
 * aligned. */
pointsht_status pointsht_plan_set_skip_counters(pointsht_plan plan, void* counters);

/* Kernel of the mixed-precision weight-column contraction
 * (pointsht_alm_columns with POINTSHT_MIXED; the per-m contraction of Eq.
 * alm_def for several weight columns): 0 = warp-level mma.sync (the
 * default, the faster one), 1, 2, 3 = fifth-generation tensor cores
 * (tcgen05.mma, tensor-memory accumulators) with 8 producer warps and 32
 * multipoles per stage, 4 and 64, 2 and 128.  All split both operands into
 * fp16 hi + lo and accumulate in FP32; results agree to FP32 rounding.
 * EINVAL for other values. */
pointsht_status pointsht_plan_set_mixed_kernel(pointsht_plan plan, int32_t which);

/* Test hook of the bounded waits (the paper has no counterpart).  While
 * enabled, the first CTA of each FP32/FP64 analysis launch waits, bounded, on
 * a shared-memory barrier that no copy and no thread ever arrives at; the
 * wait gives up, the CTA records the timeout in the plan's error word and
 * leaves before it takes a work unit or issues a copy (the other CTAs take
 * every unit, so the a_lm are still complete when the launch has more than
 * one CTA).  The next pointsht_plan_check returns POINTSHT_ETIMEOUT.  Never
 * faults or hangs: nothing is left in flight. */
pointsht_status pointsht_plan_set_wait_probe(pointsht_plan plan, int32_t enable);

/* Bytes of device workspace pointsht_alm / pointsht_alm_backward need for
 * this set of catalogs (host array cats[ncat]; only n and field are read).
 * Returns 0 and sets the last error if an argument is invalid. */
size_t pointsht_workspace_size(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat,
                               int32_t nfield, pointsht_precision prec);

/* a_lm of each field f (Eq. alm_def):
 *   alm_out[f] = sum_{catalogs c with field f} coeff_c sum_i w_i Y*_lm(n_i)
 * cats: HOST array of ncat catalog descriptors (device data pointers);
 * nfield >= 1; alm_out: device, nfield*M complex128 (2*nfield*M doubles,
 * 16-byte aligned); workspace: device, >= pointsht_workspace_size() bytes,
 * 256-byte aligned, contents need not be initialised and are clobbered.
 * Every step (point preparation, the per-point recurrences, the sums over
 * points and the final reduction) runs in this library's kernels.
 * lmax limits: FP32 4096 (the recurrence's exponent handling); FP64 the
 * largest lmax whose per-warp accumulator rows fit in the device's shared
 * memory (2970 on a GB300).  A larger plan is refused with EINVAL, whose
 * message names the bound.
 * Errors: EINVAL on bad arguments, ENOMEM if ws_bytes is too small. */
pointsht_status pointsht_alm(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat,
                             int32_t nfield, pointsht_precision prec, double* alm_out,
                             void* workspace, size_t ws_bytes, void* stream);

/* Poisson shot noise of each field (Sec. 2.1, last paragraphs; addition
 * theorem with P_l(1) = 1) as the nfield x nfield matrix used by pointsht_cl:
 *   noise_out[f*nfield + f] = sum_{c in f} coeff_c^2 sum_i w_i^2 / 4pi,
 * off-diagonal entries 0 (catalogs of a field are disjoint point sets and
 * different fields share no catalog).  noise_out: device, nfield*nfield
 * doubles.  workspace: device, >= 256-byte aligned, at least
 * 512*max(ncat,1) bytes (pointsht_workspace_size always suffices). */
pointsht_status pointsht_shot_noise(const pointsht_catalog* cats, int32_t ncat, int32_t nfield,
                                    pointsht_precision prec, double* noise_out, void* workspace,
                                    size_t ws_bytes, void* stream);

/* Linear combination of fields (the FKP field D_b - alpha_b R of a shared
 * random catalog, Sec. 2.1):
 *   alm_out[o] = sum_s coef[o*nsrc + s] alm_src[s]
 *   noise_out = C noise_src C^T, i.e. noise_out[o*nout + p] =
 *       sum_{s,t} coef[o*nsrc+s] coef[p*nsrc+t] noise_src[s*nsrc+t]
 * coef: device, nout*nsrc doubles; noise_src: device nsrc*nsrc (e.g. from
 * pointsht_shot_noise), noise_out: device nout*nout; both NULL to skip. */
pointsht_status pointsht_combine(int32_t lmax, const double* alm_src, int32_t nsrc, const double* coef,
                                 int32_t nout, const double* noise_src, double* alm_out,
                                 double* noise_out, void* stream);

/* Pseudo-C_l (Eq. pseudoCl) of all auto and cross pairs f <= g:
 *   C_l^{fg} = [Re(a_l0^f conj a_l0^g) + 2 sum_{m=1..l} Re(a_lm^f conj a_lm^g)] / (2l+1)
 *              - N^{fg}
 * alm: device nfield*M complex128; noise: device nfield*nfield doubles (the
 * shot-noise matrix to subtract) or NULL for none; cl_out: device,
 * npair*(lmax+1) doubles, pair index of (f, g), f <= g, in row-major upper
 * triangle order p = f*nfield - f*(f-1)/2 + (g - f). */
pointsht_status pointsht_cl(int32_t lmax, const double* alm, int32_t nfield, const double* noise,
                            double* cl_out, void* stream);

/* Vector-Jacobian product of pointsht_cl: given grad_cl (npair*(lmax+1)),
 * writes grad_alm[f] = dL/dRe(a^f) + i dL/dIm(a^f) (nfield*M complex128) and,
 * if grad_noise != NULL, grad_noise[f*nfield+g] = dL/dN^{fg}. */
pointsht_status pointsht_cl_backward(int32_t lmax, const double* alm, int32_t nfield,
                                     const double* grad_cl, double* grad_alm, double* grad_noise,
                                     void* stream);

/* Bandpowers C_b = sum_l theta_b^l C_l with theta_b^l = 1/Delta_l on
 * [edges[b], edges[b+1]) (Sec. 2.1): cl: device nspec*(lmax+1); edges: device
 * nbin+1 int32 increasing in [0, lmax+1] (clamped into that range on the
 * device; an empty bin gives 0); out: device nspec*nbin. */
pointsht_status pointsht_bin(int32_t lmax, const double* cl, int32_t nspec, const int32_t* edges,
                             int32_t nbin, double* out, void* stream);

/* Transpose of pointsht_bin: grad_cl[s][l] = sum_b theta_b^l grad_b[s][b]. */
pointsht_status pointsht_bin_backward(int32_t lmax, const double* grad_b, int32_t nspec,
                                      const int32_t* edges, int32_t nbin, double* grad_cl,
                                      void* stream);

/* Adjoint (vector-Jacobian product) of pointsht_alm with respect to the
 * weights, plus the shot-noise term:
 *   grad_w_c[i] = coeff_c sum_{l, m>=0} lambda_lm(x_i) Re(g^f_lm e^{i m phi_i})
 *                 + 2 coeff_c^2 w_i gnoise_f / 4pi
 * where g^f = grad_alm[f] (dL/dRe a + i dL/dIm a, nfield*M complex128) and
 * gnoise_f = grad_noise[f*nfield + f] (the diagonal of dL/dN, device
 * nfield*nfield doubles as written by pointsht_cl_backward, or NULL for 0).
 * This is a point-evaluation synthesis that reruns the recurrence per point
 * (derived from Eq. alm_def; the paper has no adjoint).  grad_w: HOST array of
 * ncat device pointers, each n_c values of the dtype of w (may alias nothing
 * else).  workspace as for pointsht_alm (pointsht_workspace_size bytes).
 * FP32 (and MIXED, which runs as FP32): the points are prepared and
 * |x|-sorted as for the analysis, each keeping its id, so the total number
 * of points must be below 2^32 - 1 (EINVAL otherwise); lmax <= the FP32
 * path's limit.  FP64: catalog order. */
pointsht_status pointsht_alm_backward(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat,
                                      int32_t nfield, pointsht_precision prec, const double* grad_alm,
                                      const double* grad_noise, void* const* grad_w, void* workspace,
                                      size_t ws_bytes, void* stream);

/* ---- Weight columns on one point set ----------------------------------
 * F weight columns on the same n points (for example per-bin weights on a
 * shared random catalog, systematics or jackknife weights):
 *   alm_out[f] = sum_i w[f*n + i] Y*_lm(n_i),   f = 0..ncol-1   (Eq. alm_def)
 * For one order m this is the contraction a_m[l, f] = sum_i lambda_lm(x_i)
 * W_m[i, f] with W_m[i, f] = w_f,i e^{-i m phi_i}: the recurrence runs once per
 * point for all columns.
 * - POINTSHT_MIXED: lambda_lm from the FP32 recurrence; the contraction runs on
 *   the tensor cores with both operands split into fp16 hi + lo parts
 *   (hi*hi + lo*hi + hi*lo, FP32 accumulation, FP64 sums over chunks).  Each
 *   column is scaled by a power of two so that max|w| lies in [1, 2) (exact,
 *   undone in FP64).  Up to 8 columns share one pass; more columns take
 *   further passes over the prepared points.  lmax <= 4096 (the FP32
 *   recurrence's range, as for POINTSHT_FP32).
 * - POINTSHT_FP32: the same result through pointsht_alm with one catalog and
 *   field per column (the plain FP32 path, for comparison).
 * x, phi: device, n floats; w: device, ncol*n floats (column-major: column f
 * at w + f*n); alm_out: device, ncol*M complex128, 16-byte aligned;
 * workspace: device, >= pointsht_workspace_size_columns() bytes, 256-byte
 * aligned, clobbered.  1 <= ncol <= 64.  Errors as for pointsht_alm;
 * non-finite x, phi, w or |x| > 1 set the ERANGE flag (the point is dropped). */
size_t pointsht_workspace_size_columns(pointsht_plan plan, int64_t n, int32_t ncol, pointsht_precision prec);

pointsht_status pointsht_alm_columns(pointsht_plan plan, const float* x, const float* phi, const float* w,
                                     int64_t n, int32_t ncol, pointsht_precision prec, double* alm_out,
                                     void* workspace, size_t ws_bytes, void* stream);

/* ---- Interpolated transform (the paper's fast route) -------------------
 * a_lm of each field by App. "Interpolation": y_lm = lambda_lm(cos theta) and
 * its theta-derivative are evaluated exactly (App. A) on ntheta samples
 * equispaced in theta, s_k = (k + 1/2) pi/ntheta, and each point takes the
 * cubic Hermite spline of its interval; the sum over points runs first, per
 * order m (binning of w e^{-i m phi} times the 4 spline weights into the
 * intervals), then a transform of the samples (the mixed tensor-core kernel;
 * a sample and its mirror pi - theta share one position, six weight columns)
 * and an FP64 combination.  The theta-derivative is taken in its
 * order-coupled form (lambda at m +- 1), free of the 1/sin(theta)
 * cancellation near the poles.  The samples are in theta, not in x as in the
 * paper: in theta y_lm stays smooth through the poles when continued across
 * them (y(-theta) = (-1)^m y(theta)), so the two outer intervals use ghost
 * samples and no point is treated apart.
 * Several fields: each field is sorted, binned and folded into its own sample
 * table; fields are taken in groups of up to 4 whose 6 x fields weight
 * columns share the transform's passes of up to 8 columns (one sample
 * recurrence per pass instead of one per field).
 * Error: the spline's O(h^4) interpolation error, about 2e-5 relative per
 * value at ntheta = 8 lmax and 1.5e-6 at 16 lmax (h = pi/ntheta), plus the
 * mixed path's rounding; work O(N lmax + ntheta lmax^2) instead of
 * O(N lmax^2).
 * cats as for pointsht_alm with float x, phi, w (POINTSHT_FP32 layout);
 * ntheta even, 2 <= ntheta <= 32768; fewer than 2^31 points per field;
 * alm_out: device, nfield*M complex128; workspace: device, >=
 * pointsht_workspace_size_interp() bytes (per field of a group
 * ~(lmax+1) ntheta x 16 bytes of sample table, plus ~(lmax+1)(ntheta+1) x 32
 * bytes and ~52 bytes per point of the largest field: about 4.3 GB at lmax
 * 2048, ntheta 32768, 1e7 points, one field), 256-byte aligned, clobbered.
 * Errors as for pointsht_alm. */
size_t pointsht_workspace_size_interp(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat,
                                      int32_t nfield, int32_t ntheta);

pointsht_status pointsht_alm_interp(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat,
                                    int32_t nfield, int32_t ntheta, double* alm_out, void* workspace,
                                    size_t ws_bytes, void* stream);

/* Point-evaluation synthesis: out[i] = sum_{l <= lmax, |m| <= l} a_lm Y_lm(theta_i, phi_i)
 * for the real field whose m >= 0 coefficients are `alm` (a_{l,-m} =
 * (-1)^m conj(a_lm), Condon-Shortley phase), i.e.
 * sum_l [a_l0 Y_l0 + 2 sum_{m>0} Re(a_lm Y_lm)].  This is the operation the
 * paper names for releasing or apodising the a_lm as a band-limited function
 * (Sec. "Conclusions"; Eq. alm_def read backwards), and the transpose of the
 * analysis: it runs the adjoint kernels with unit weights.
 * x = cos(theta), phi: device, n values of float (POINTSHT_FP32) or double
 * (POINTSHT_FP64); alm: device, M complex128 (the packed m-major triangle of
 * the plan's lmax); out: device, n values of the input type, overwritten;
 * workspace: >= pointsht_workspace_size_synthesis() bytes, 256-byte aligned,
 * clobbered.  |x| > 1 or non-finite inputs raise ERANGE at the next
 * pointsht_plan_check (those points get the value at x = 0, phi = 0).  FP32:
 * lmax <= the FP32 path's limit and n < 2^32 - 1. */
size_t pointsht_workspace_size_synthesis(pointsht_plan plan, int64_t n, pointsht_precision prec);

pointsht_status pointsht_synthesis(pointsht_plan plan, const void* x, const void* phi, int64_t n,
                                   pointsht_precision prec, const double* alm, void* out, void* workspace,
                                   size_t ws_bytes, void* stream);

/* Spin-2 (shear) transform of weighted point catalogs: the generalisation
 * to fields of non-zero spin that Sec. 4 names (spin-weighted harmonics
 * _{+-2}Y_lm from a recurrence):
 *   _{+-2}a_lm = sum_i coeff w_i (g1 +- i g2)_i _{+-2}Y*_lm(n_i),
 *   E_lm = -(_{2}a_lm + _{-2}a_lm)/2,  B_lm = i (_{2}a_lm - _{-2}a_lm)/2,
 * with _sY_lm = (-1)^s sqrt((2l+1)/4pi) d^l_{m,-s}(theta) e^{i m phi} (Wigner's
 * small d; s = 0 gives the Y_lm of App. A; _{2}Y = sqrt((l-2)!/(l+2)!) eth eth Y
 * with eth the usual spin-raising operator).  E and B are the coefficients of
 * real fields (negative m implicit), zero for l < 2.
 * cats: host array of ncat descriptors (FP32 device arrays); E_out, B_out:
 * device, nfield*M complex128 each (packed m-major triangle, 16-byte
 * aligned), overwritten; workspace: >= pointsht_workspace_size_spin2() bytes
 * (~36 bytes per point + (lmax+1)^2 x 16 bytes + ~M x 32 bytes per chunk of
 * up to 2^20 points), 256-byte aligned.  FP32 recurrence (one recurrence per
 * point serves both spins through d^l_{m,2}(theta) =
 * (-1)^(l+m) d^l_{m,-2}(pi - theta)), FP64 sums over chunks; lmax <= the FP32
 * path's limit.  |x| > 1 or non-finite inputs: ERANGE at the next
 * pointsht_plan_check (those points count with zero weight). */
size_t pointsht_workspace_size_spin2(pointsht_plan plan, const pointsht_shear_catalog* cats, int32_t ncat,
                                     int32_t nfield);

pointsht_status pointsht_alm_spin2(pointsht_plan plan, const pointsht_shear_catalog* cats, int32_t ncat,
                                   int32_t nfield, double* E_out, double* B_out, void* workspace, size_t ws_bytes,
                                   void* stream);

/* ---------------------------------------------------------------------
 * Mode coupling of the masked pseudo-spectrum (Sec. 2.1).
 *
 * The window's spectrum W_l (Eq. wldef) is the pseudo-C_l of the scaled
 * randoms: pointsht_alm on the randoms with coeff = alpha, then pointsht_cl
 * (with their shot noise alpha^2 sum w^2 / 4pi as `noise` when few randoms
 * estimate the window).  The functions below take W_l on the device.
 * All pointers are device pointers unless noted; everything is enqueued on
 * `stream`; only argument errors are returned synchronously.
 * ------------------------------------------------------------------- */

/* Workspace of pointsht_coupling: two FP64 tables of 2 lmax + 1 entries. */
size_t pointsht_workspace_size_coupling(int32_t lmax);

/* M_ll' = (2l'+1)/(4 pi) sum_lambda (2 lambda+1) (l l' lambda; 0 0 0)^2 W_lambda
 * (Eq. chat) for 0 <= l, l' <= lmax, lambda <= min(l + l', lmax_w); W_lambda
 * beyond lmax_w counts as zero.  The 3j symbols with zero orders are those of
 * App. "Wigner 3j symbols", evaluated through their closed form squared.
 * W: lmax_w + 1 doubles; M: (lmax+1)^2 doubles, row-major M[l][l'],
 * overwritten; workspace: >= pointsht_workspace_size_coupling(lmax) bytes,
 * 256-byte aligned, clobbered.  0 <= lmax <= 8192.  FP64 throughout; work
 * ~lmax^2 min(lmax, lmax_w)/6 terms.  Deterministic. */
pointsht_status pointsht_coupling(int32_t lmax, int32_t lmax_w, const double* W, double* M,
                                  void* workspace, size_t ws_bytes, void* stream);

/* Binned coupling (Sec. 2.1, theta_b^l = 1/Delta_l on [edges[b], edges[b+1])):
 * R[b][l'] = sum_l theta_b^l M_ll' (nbin x (lmax+1)) and
 * M_bb' = sum_{l' in b'} R[b][l'] (nbin x nbin), the coupling between binned
 * C^ and a true C_l that is constant on each bin.  edges: nbin + 1 int32
 * (clamped into [0, lmax+1] on the device); 1 <= nbin <= 512. */
pointsht_status pointsht_coupling_binned(int32_t lmax, const double* M, const int32_t* edges, int32_t nbin,
                                         double* R, double* Mbb, void* stream);

/* Workspace of pointsht_decouple: the augmented nbin x 2 nbin matrix. */
size_t pointsht_workspace_size_decouple(int32_t nbin);

/* Mode decoupling (Eq. mode_coupling, Eq. expectation_value): Minv = M_bb'^-1
 * (Gauss-Jordan, partial pivoting, FP64; a singular matrix gives NaN
 * everywhere in Minv and in what is computed from it), and optionally the
 * window matrix Mcal[b][l'] = sum_b' Minv[b][b'] R[b'][l'] (R and Mcal both
 * given or both NULL) and the decoupled bandpowers
 * cl_dec[s][b] = sum_b' Minv[b][b'] cl_binned[s][b'] for nspec spectra
 * (cl_binned and cl_dec both given or both NULL).  workspace: >=
 * pointsht_workspace_size_decouple(nbin) bytes, 256-byte aligned. */
pointsht_status pointsht_decouple(int32_t lmax, int32_t nbin, const double* Mbb, const double* R,
                                  const double* cl_binned, int32_t nspec, double* Minv, double* Mcal,
                                  double* cl_dec, void* workspace, size_t ws_bytes, void* stream);

/* FKP-like normalisation (Sec. 2.1): norm[0] = 1 / [sum_l (2l+1) W_l / 4pi]
 * over l <= lmax_w (it leaves the amplitude of a shot-noise spectrum
 * unchanged), and optionally Mprime = norm R (nbin x (lmax+1)) and
 * cl_norm = norm cl_binned (nspec x nbin); pairs both given or both NULL. */
pointsht_status pointsht_fkp_normalise(int32_t lmax_w, const double* W, int32_t lmax, int32_t nbin,
                                       const double* R, const double* cl_binned, int32_t nspec,
                                       double* norm, double* Mprime, double* cl_norm, void* stream);

/* Size of the fixed scratch array used by pointsht_alm_noalloc (64 MiB). */
#define POINTSHT_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)

/* pointsht_alm for callers that cannot allocate device memory (the paper has
 * no counterpart: this exists for callers such as host frameworks that own
 * every device allocation, or pipelines that forbid allocation once running,
 * and so cannot provide a workspace).  Same arguments and results as
 * pointsht_alm minus the workspace: the scratch is a fixed array of
 * POINTSHT_NOALLOC_SCRATCH_BYTES inside the library's device image, held by
 * every GPU that loads the library until the process exits.  The call itself
 * performs no allocation of any kind.
 * - Limit: returns ENOMEM (nothing enqueued) when pointsht_workspace_size()
 *   for these catalogs exceeds POINTSHT_NOALLOC_SCRATCH_BYTES (roughly lmax
 *   <= 512 with up to ~1e6 points; larger problems need pointsht_alm).
 * - The first call on a device looks up the array's device address on that
 *   device; with CUDA's lazy module loading that lookup is also what loads the
 *   library's device code, and the array with it, onto that device.  Callers
 *   that must not see any allocation once running should make one warm-up
 *   call on each device first (and before any stream capture); later calls
 *   reuse the address and allocate nothing.
 * - All calls share the one array and it keeps the last call's contents;
 *   everything the transform needs to start at zero is cleared by the call.
 *   Calls whose work overlaps on the GPU (different streams, or different host
 *   threads without ordering) race on the array: serialise them. */
pointsht_status pointsht_alm_noalloc(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat,
                                     int32_t nfield, pointsht_precision prec, double* alm_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* POINTSHT_H */
