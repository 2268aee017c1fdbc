// api.cu -- C ABI of libpointsht (declared in include/pointsht.h).
//
// Host side: argument validation, the plan's recurrence tables, the workspace
// layout and the kernel launches.  No call except pointsht_plan_create
// allocates device memory; every kernel is enqueued on the caller's stream.
#include "pointsht.h"

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace psht {
template <typename T>
cudaError_t launch_prep(const PrepParams&, int, cudaStream_t);
template <typename T>
cudaError_t launch_prep_sorted(const SortParams&, cudaStream_t);
cudaError_t launch_analysis(const AnalysisParams&, int, int, int, cudaStream_t, int*);
cudaError_t launch_reduce(const ReduceParams&, cudaStream_t);
int analysis_tile_points(int, int);
cudaError_t launch_cl(int, const double*, int, const double*, double*, cudaStream_t);
cudaError_t launch_cl_backward(int, const double*, int, const double*, double*, double*, cudaStream_t);
cudaError_t launch_bin(int, const double*, int, const int*, int, double*, cudaStream_t);
cudaError_t launch_bin_backward(int, const double*, int, const int*, int, double*, cudaStream_t);
cudaError_t launch_combine(int, const double*, int, const double*, int, const double*, double*, double*,
                           cudaStream_t);
cudaError_t launch_shot_noise(const PrepParams&, int, double*, int, double*, cudaStream_t);
cudaError_t launch_build_gtab(int, int, int, const double*, const double*, const int64_t*, int64_t, int, void*,
                              cudaStream_t);
int adjoint_points_per_warp(int);
cudaError_t launch_adjoint(int, const AdjointParams&, cudaStream_t);
int adjoint_sorted_points_per_cta();
size_t analysis_smem_need(int prec_is_f64, int k32, int lmax);
size_t coupling_smem_bytes(int);
size_t spin2_workspace_bytes(int, const pointsht_shear_catalog*, int, int);
cudaError_t spin2_run(int, const pointsht_shear_catalog*, int, int, void*, unsigned*, int, double*, double*,
                      cudaStream_t);
cudaError_t launch_coupling(int, int, const double*, double*, double*, double*, cudaStream_t);
cudaError_t launch_coupling_binned(int, const double*, const int*, int, double*, double*, cudaStream_t);
size_t decouple_workspace_bytes(int);
cudaError_t launch_decouple(int, int, const double*, const double*, const double*, int, double*, double*, double*,
                            double*, cudaStream_t);
cudaError_t launch_fkp_normalise(int, const double*, int, int, const double*, const double*, int, double*, double*,
                                 double*, cudaStream_t);
cudaError_t launch_adjoint_sorted(const AdjointParams&, const double*, const double*, int, cudaStream_t);
cudaError_t launch_fill_ones(int64_t, int, void*, cudaStream_t);
cudaError_t launch_sort_offsets_f32(const SortParams&, cudaStream_t);
size_t mixed_smem_bytes(int);
int mixed_tile_points();
int mixed_max_columns();
int mixed_geometry_arrays();
int64_t mixed_acc_stride(int);
cudaError_t launch_mixed_prep(const PrepColsParams&, int64_t, cudaStream_t);
cudaError_t launch_mixed(const MixedParams&, int, cudaStream_t);
cudaError_t launch_mixed_tc(const MixedParams&, int, cudaStream_t, int);
int64_t interp_nranges(int64_t);
int64_t interp_range();
cudaError_t launch_interp_sort(const InterpParams&, cudaStream_t);
cudaError_t launch_interp_tables(const InterpParams&, int, cudaStream_t);
cudaError_t launch_interp_combine(int, int64_t, const double*, double*, cudaStream_t);
}  // namespace psht

using namespace psht;

struct pointsht_plan_s {
    int lmax = 0;
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;       // the device's opt-in shared memory per block
    int64_t nmodes = 0;
    int64_t acol = 0;  // colstart[lmax+1]: padded column-table length
    void* blob = nullptr;
    float* alpha_f = nullptr;
    float2* alpha_f2 = nullptr;  // (alpha, alpha) pairs for packed f32x2 arithmetic
    float4* pole_ae = nullptr;   // near-pole tables (a, a, a - 2, a - 2), see build_tables
    float* pole_rho = nullptr;   // odd-chain scale rho_m of the near-pole normalisation
    int pole_mmax = 256;         // ... for orders m < pole_mmax
    float pole_x = 0.9f;         // tiles (warps) whose points all have |x| >= pole_x take the near-pole form
    int wait_probe = 0;          // test hook of the timeout path (pointsht_plan_set_wait_probe)
    int mixed_kernel = 0;        // weight-column contraction: 0 = mma.sync (default), 1 = tcgen05
    int tc_shape = 0;            // tcgen05 stage shape: 0 = 8 warps x 32 l, 1 = 4 x 64, 2 = 2 x 128
    unsigned long long* stats = nullptr;  // optional skip counters (pointsht_plan_set_skip_counters)
    double* alpha_d = nullptr;
    int64_t* colstart = nullptr;
    double* gamma = nullptr;
    float* log2c_hi = nullptr;
    float* log2c_lo = nullptr;
    double* log2c = nullptr;
    unsigned* err = nullptr;
    cudaEvent_t ev_start = nullptr;  // optional timing hook around the analysis kernel
    cudaEvent_t ev_stop = nullptr;
    int variant = 0;     // FP32 analysis kernel variant (0 = default)
    int chunk_log2 = 0;  // points per accumulation chunk (0 = automatic)
};

// ------------------------------------------------------------ errors --
static thread_local std::string g_last_error;

static pointsht_status fail(pointsht_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

// Sets the thread's last-error message (used by other translation units).
pointsht_status psht_set_error(pointsht_status s, const char* msg) { return fail(s, "%s", msg); }

#define CUDA_TRY(call)                                                                                  \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return fail(POINTSHT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static constexpr int64_t SHOT_NBLK = 64;
static constexpr int FLUSH_TILES = 16;

extern "C" const char* pointsht_version(void) { return "1.0.0"; }
extern "C" const char* pointsht_last_error(void) { return g_last_error.c_str(); }

// ------------------------------------------------------------ tables --
// Built in long double on the host: lambda-form recurrence coefficients
// (App. A divided through by sqrt((2l+1)/4pi)), their gamma rescaling and
// log2 c_m = log2 |lambda_mm| - m log2 sin(theta).
// Tables of the sign-folded FP32/FP64 recurrence (see analysis.cu): gamma_l =
// B_l gamma_{l-2} removes B from the recurrence on each parity chain of
// q = l - m (gamma_m = gamma_{m+1} = 1), alpha~ its coefficients.
//
// Near-pole table.  Near x = +-1 the recurrence mu_l = a_l x mu_{l-1} -
// mu_{l-2} (mu = lambda / gamma) has a double root at 1, where FP32 rounding
// of a_l and of x mu grows like l^1.5 eps.  Reinsch's form carries the
// difference d_l = mu_l - mu_{l-1} instead,
//   d_l = (a_l u + e_l) mu_{l-1} + d_{l-1},  mu_l = mu_{l-1} + d_l,
//   u = |x| - 1 (exact in FP32),  e_l = a_l - 2 (stored to full relative precision),
// so that only small quantities carry coefficient and product rounding.  It
// needs mu smooth in l, so there the odd chain of gamma is scaled by rho_m,
// chosen so that it meets the even chain at lmax (geometric mean of the
// neighbouring even values): a_l then tends to 2 instead of alternating
// between two constants.  Entry (m, q) of pae: (a_l, a_l, e_l, e_l) for
// l = m + q, q >= 1 (q = 0 unused); prho[m] = rho_m.
static void build_tables(int L, std::vector<int64_t>& colstart, std::vector<float>& af, std::vector<double>& ad,
                         std::vector<double>& gamma, std::vector<double>& l2c, std::vector<float4>& pae,
                         std::vector<float>& prho) {
    colstart.assign(L + 2, 0);
    for (int m = 0; m <= L; ++m) {
        const int64_t len = L - m + 1;
        colstart[m + 1] = colstart[m] + ((len + 15) / 16) * 16;
    }
    const int64_t acol = colstart[L + 1];
    af.assign(acol, 0.f);
    ad.assign(acol, 0.0);
    pae.assign(acol + 32, make_float4(0.f, 0.f, 0.f, 0.f));
    prho.assign(L + 1, 1.f);
    const int64_t M = (int64_t)(L + 1) * (L + 2) / 2;
    gamma.assign(M, 0.0);
    l2c.assign(L + 1, 0.0);
    long double sumlog = 0.0L;
    for (int m = 0; m <= L; ++m) {
        if (m > 0) sumlog += log2l(1.0L - 1.0L / (2.0L * m));
        l2c[m] = (double)(0.5L * log2l((2.0L * m + 1.0L) / (4.0L * 3.141592653589793238462643383279502884L)) +
                          0.5L * sumlog);
        const int64_t base = tri_base(m, L);
        const int n = L - m;
        std::vector<long double> g(n + 1, 1.0L);
        for (int l = m + 2; l <= L; ++l) {
            const long double ll = l, mm = m;
            const long double B = sqrtl((2 * ll + 1) * ((ll - 1) * (ll - 1) - mm * mm) /
                                        ((2 * ll - 3) * (ll * ll - mm * mm)));
            g[l - m] = B * g[l - m - 2];
        }
        long double rho = 1.0L;
        if (n >= 2) {
            const int qo = (n & 1) ? n : n - 1;  // last odd q
            const long double target = qo + 1 <= n ? sqrtl(g[qo - 1] * g[qo + 1]) : g[qo - 1];
            rho = target / g[qo];
        }
        prho[m] = (float)rho;
        // sigma_q = s_q mu_q with s_q = (-1)^floor(q/2), q = l - m, turns
        // mu_l = a_l x mu_{l-1} - mu_{l-2} into
        // sigma_l = (s_q/s_{q-1}) a_l x sigma_{l-1} + sigma_{l-2}
        // (no negation in the inner loop); s_q is folded into gamma.
        for (int l = m; l <= L; ++l) {
            const long double ll = l, mm = m;
            const int q = l - m;
            const int sq = ((q >> 1) & 1) ? -1 : 1;
            const int sq1 = q >= 1 ? ((((q - 1) >> 1) & 1) ? -1 : 1) : 1;
            long double A = 0.0L;
            if (l == m + 1) A = sqrtl(2 * mm + 3);
            if (l >= m + 2) A = sqrtl((4 * ll * ll - 1) / (ll * ll - mm * mm));
            if (q >= 1) {
                // smooth normalisation: gamma~_q = gamma_q (q even), rho gamma_q (q odd)
                const long double gs_prev = ((q - 1) & 1) ? g[q - 1] * rho : g[q - 1];
                const long double gs = (q & 1) ? g[q] * rho : g[q];
                const long double as = A * gs_prev / gs;
                const float pa = (float)as, pe = (float)(as - 2.0L);
                pae[colstart[m] + q] = make_float4(pa, pa, pe, pe);
            }
            long double a = q >= 1 ? A * g[q - 1] / g[q] : 0.0L;
            a *= (long double)(sq * sq1);
            af[colstart[m] + q] = (float)a;
            ad[colstart[m] + q] = (double)a;
            gamma[base + l] = (double)(g[q] * sq);
        }
    }
}

static bool device_is_sm103(int dev, int* sms) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return false;
    if (sms) *sms = prop.multiProcessorCount;
    return prop.major == 10 && prop.minor == 3;
}

extern "C" pointsht_status pointsht_plan_create(int32_t lmax, pointsht_plan* out) {
    if (!out) return fail(POINTSHT_EINVAL, "plan_create: out is NULL");
    *out = nullptr;
    if (lmax < 1 || lmax > 8192) return fail(POINTSHT_EINVAL, "plan_create: lmax=%d outside [1, 8192]", lmax);
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    int sms = 0;
    if (!device_is_sm103(dev, &sms))
        return fail(POINTSHT_EARCH, "plan_create: device %d is not compute capability 10.3 (sm_103)", dev);
    std::vector<int64_t> colstart;
    std::vector<float> af;
    std::vector<double> ad, gamma, l2c;
    std::vector<float4> pae;
    std::vector<float> prho;
    build_tables(lmax, colstart, af, ad, gamma, l2c, pae, prho);
    af.resize(af.size() + 256, 0.f);  // zeros past the last column, as for the pairs below
    std::vector<float> lh(lmax + 1), ll(lmax + 1);
    for (int m = 0; m <= lmax; ++m) {
        lh[m] = (float)l2c[m];
        ll[m] = (float)(l2c[m] - (double)lh[m]);
    }
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    // 256 zero entries past the last column: kernels read whole blocks of up to
    // 128 steps (the tcgen05 weight-column kernel's widest stage) past a column's end
    std::vector<float2> af2(af.size() + 256, make_float2(0.f, 0.f));
    for (size_t i = 0; i < af.size(); ++i) af2[i] = make_float2(af[i], af[i]);
    const size_t s_af2 = up(af2.size() * 8);
    const size_t s_af = up(af.size() * 4), s_ad = up(ad.size() * 8), s_cs = up(colstart.size() * 8),
                 s_g = up(gamma.size() * 8), s_lh = up(lh.size() * 4), s_l2 = up(l2c.size() * 8), s_err = 256;
    const size_t s_pae = up(pae.size() * 16), s_rho = up(prho.size() * 4);
    const size_t total = s_af + s_af2 + s_ad + s_cs + s_g + 2 * s_lh + s_l2 + s_err + s_pae + s_rho;
    pointsht_plan p = new pointsht_plan_s();
    p->lmax = lmax;
    p->device = dev;
    p->sm_count = sms;
    {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        p->smem_optin = (size_t)v;
    }
    p->nmodes = (int64_t)(lmax + 1) * (lmax + 2) / 2;
    p->acol = colstart[lmax + 1];
    if (cudaMalloc(&p->blob, total) != cudaSuccess) {
        delete p;
        cudaGetLastError();
        return fail(POINTSHT_ENOMEM, "plan_create: cudaMalloc(%zu) failed", total);
    }
    char* b = static_cast<char*>(p->blob);
    p->alpha_f = reinterpret_cast<float*>(b);
    b += s_af;
    p->alpha_f2 = reinterpret_cast<float2*>(b);
    b += s_af2;
    p->alpha_d = reinterpret_cast<double*>(b);
    b += s_ad;
    p->colstart = reinterpret_cast<int64_t*>(b);
    b += s_cs;
    p->gamma = reinterpret_cast<double*>(b);
    b += s_g;
    p->log2c_hi = reinterpret_cast<float*>(b);
    b += s_lh;
    p->log2c_lo = reinterpret_cast<float*>(b);
    b += s_lh;
    p->log2c = reinterpret_cast<double*>(b);
    b += s_l2;
    p->err = reinterpret_cast<unsigned*>(b);
    b += s_err;
    p->pole_ae = reinterpret_cast<float4*>(b);
    b += s_pae;
    p->pole_rho = reinterpret_cast<float*>(b);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpy(p->alpha_f, af.data(), af.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->alpha_f2, af2.data(), af2.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->alpha_d, ad.data(), ad.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->colstart, colstart.data(), colstart.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->gamma, gamma.data(), gamma.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->log2c_hi, lh.data(), lh.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->log2c_lo, ll.data(), ll.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->log2c, l2c.data(), l2c.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->err, 0, s_err);
    if (e == cudaSuccess) e = cudaMemcpy(p->pole_ae, pae.data(), pae.size() * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->pole_rho, prho.data(), prho.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->blob);
        delete p;
        return fail(POINTSHT_ECUDA, "plan_create: %s", cudaGetErrorString(e));
    }
    *out = p;
    return POINTSHT_OK;
}

extern "C" void pointsht_plan_destroy(pointsht_plan plan) {
    if (!plan) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    cudaFree(plan->blob);
    cudaSetDevice(cur);
    delete plan;
}

extern "C" int32_t pointsht_plan_lmax(pointsht_plan plan) { return plan ? plan->lmax : -1; }

extern "C" pointsht_status pointsht_plan_set_timing_events(pointsht_plan plan, void* start, void* stop) {
    if (!plan) return fail(POINTSHT_EINVAL, "set_timing_events: plan is NULL");
    if ((start == nullptr) != (stop == nullptr))
        return fail(POINTSHT_EINVAL, "set_timing_events: start and stop must both be set or both NULL");
    plan->ev_start = static_cast<cudaEvent_t>(start);
    plan->ev_stop = static_cast<cudaEvent_t>(stop);
    return POINTSHT_OK;
}

extern "C" pointsht_status pointsht_plan_set_tuning(pointsht_plan plan, int32_t variant, int32_t chunk_log2) {
    if (!plan) return fail(POINTSHT_EINVAL, "set_tuning: plan is NULL");
    if (!(variant == 0 || variant == 8 || variant == 12 || variant == 16 || variant == 108 || variant == 116))
        return fail(POINTSHT_EINVAL, "set_tuning: unknown variant %d", variant);
    if (!(chunk_log2 == 0 || (chunk_log2 >= 10 && chunk_log2 <= 22)))
        return fail(POINTSHT_EINVAL, "set_tuning: chunk_log2 %d outside {0} or [10, 22]", chunk_log2);
    plan->variant = variant;
    plan->chunk_log2 = chunk_log2;
    return POINTSHT_OK;
}

extern "C" pointsht_status pointsht_plan_set_pole_threshold(pointsht_plan plan, float pole_x) {
    if (!plan) return fail(POINTSHT_EINVAL, "set_pole_threshold: plan is NULL");
    if (!(pole_x >= 0.5f)) return fail(POINTSHT_EINVAL, "set_pole_threshold: %g is below 0.5 (or NaN)", pole_x);
    plan->pole_x = pole_x;
    return POINTSHT_OK;
}

extern "C" pointsht_status pointsht_plan_set_skip_counters(pointsht_plan plan, void* counters) {
    if (!plan) return fail(POINTSHT_EINVAL, "set_skip_counters: plan is NULL");
    if ((uintptr_t)counters % 8) return fail(POINTSHT_EINVAL, "set_skip_counters: counters not 8-byte aligned");
    plan->stats = static_cast<unsigned long long*>(counters);
    return POINTSHT_OK;
}

extern "C" pointsht_status pointsht_plan_set_mixed_kernel(pointsht_plan plan, int32_t which) {
    if (!plan) return fail(POINTSHT_EINVAL, "set_mixed_kernel: plan is NULL");
    if (which < 0 || which > 3) return fail(POINTSHT_EINVAL, "set_mixed_kernel: %d is not in 0..3", which);
    plan->mixed_kernel = which == 0 ? 0 : 1;
    plan->tc_shape = which == 0 ? 0 : which - 1;
    return POINTSHT_OK;
}

extern "C" pointsht_status pointsht_plan_set_wait_probe(pointsht_plan plan, int32_t enable) {
    if (!plan) return fail(POINTSHT_EINVAL, "set_wait_probe: plan is NULL");
    plan->wait_probe = enable ? 1 : 0;
    return POINTSHT_OK;
}

extern "C" pointsht_status pointsht_plan_check(pointsht_plan plan) {
    if (!plan) return fail(POINTSHT_EINVAL, "plan_check: plan is NULL");
    unsigned flags = 0;
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(&flags, plan->err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(plan->err, 0, sizeof(unsigned)));
    if (flags & ERR_TIMEOUT) return fail(POINTSHT_ETIMEOUT, "a bounded wait inside a kernel gave up");
    if (flags & ERR_RANGE) return fail(POINTSHT_ERANGE, "an input point had |x| > 1 or a non-finite value");
    if (flags & ERR_INTERNAL) return fail(POINTSHT_ECUDA, "internal kernel check failed");
    return POINTSHT_OK;
}

// ----------------------------------------------------------- layout --
struct Layout {
    int is_f64 = 0;
    int k32 = 116;      // FP32 kernel variant (see analysis_tile_points)
    int P = 0;          // tile points
    int narr = 0, abytes = 0;
    int64_t chunk = 0;  // points per chunk
    int ngroups = 0;    // m-groups
    int64_t ntot = 0;   // prepared points
    int64_t nunits = 0;
    int32_t nslots = 0;
    int64_t npad[PSHT_MAX_FIELDS] = {};
    int64_t off[PSHT_MAX_FIELDS] = {};
    int64_t nfpts[PSHT_MAX_FIELDS] = {};
    int32_t nchunk[PSHT_MAX_FIELDS] = {};
    int32_t slot0[PSHT_MAX_FIELDS] = {};
    int64_t unit0[PSHT_MAX_FIELDS] = {};
    // byte offsets in the workspace
    size_t pts_off = 0, slots_off = 0, counter_off = 0, hist_off = 0, fwd_end = 0;
    int64_t nranges = 0;
    size_t gtab_off = 0, bwd_end = 0, shot_off = 0, total = 0;
};

static const int WARPS = 4;

static inline size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

static pointsht_status check_common(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat, int32_t nfield,
                                    pointsht_precision prec, const char* who) {
    if (!plan) return fail(POINTSHT_EINVAL, "%s: plan is NULL", who);
    if (ncat < 0 || ncat > PSHT_MAX_CATS) return fail(POINTSHT_EINVAL, "%s: ncat=%d outside [0, %d]", who, ncat, PSHT_MAX_CATS);
    if (ncat > 0 && !cats) return fail(POINTSHT_EINVAL, "%s: cats is NULL", who);
    if (nfield < 1 || nfield > PSHT_MAX_FIELDS)
        return fail(POINTSHT_EINVAL, "%s: nfield=%d outside [1, %d]", who, nfield, PSHT_MAX_FIELDS);
    if (prec != POINTSHT_FP64 && prec != POINTSHT_FP32 && prec != POINTSHT_MIXED)
        return fail(POINTSHT_EINVAL, "%s: unknown precision %d", who, (int)prec);
    const size_t esz = prec == POINTSHT_FP64 ? 8 : 4;
    for (int c = 0; c < ncat; ++c) {
        const pointsht_catalog& k = cats[c];
        if (k.n < 0) return fail(POINTSHT_EINVAL, "%s: catalog %d has n=%lld < 0", who, c, (long long)k.n);
        if (k.field < 0 || k.field >= nfield)
            return fail(POINTSHT_EINVAL, "%s: catalog %d has field %d outside [0, %d)", who, c, k.field, nfield);
        if (!std::isfinite(k.coeff)) return fail(POINTSHT_EINVAL, "%s: catalog %d has a non-finite coeff", who, c);
        if (k.n > 0) {
            if (!k.x || !k.phi || !k.w) return fail(POINTSHT_EINVAL, "%s: catalog %d has a NULL array", who, c);
            if (((uintptr_t)k.x | (uintptr_t)k.phi | (uintptr_t)k.w) % esz)
                return fail(POINTSHT_EINVAL, "%s: catalog %d arrays are not %zu-byte aligned", who, c, esz);
        }
    }
    return POINTSHT_OK;
}

static pointsht_status make_layout(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat, int32_t nfield,
                                   pointsht_precision prec, Layout& lo) {
    const int is_f64 = prec == POINTSHT_FP64;
    lo.is_f64 = is_f64;
    lo.k32 = 116;  // the default FP32 variant; pointsht_plan_set_tuning selects another
    if (plan->variant) lo.k32 = plan->variant;
    lo.P = analysis_tile_points(is_f64, lo.k32);
    if (!is_f64) {  // fields padded to whole CTAs of the FP32 adjoint as well
        const int64_t q = adjoint_sorted_points_per_cta();
        while (lo.P % q) lo.P += analysis_tile_points(is_f64, lo.k32);
    }
    lo.narr = is_f64 ? 4 : 7;
    lo.abytes = is_f64 ? 8 : 4;
    const int L = plan->lmax;
    lo.ngroups = (L / 2 + 1 + WARPS - 1) / WARPS;
    for (int c = 0; c < ncat; ++c) lo.nfpts[cats[c].field] += cats[c].n;
    int64_t ntot = 0;
    for (int f = 0; f < nfield; ++f) {
        lo.npad[f] = (lo.nfpts[f] + lo.P - 1) / lo.P * lo.P;
        lo.off[f] = ntot;
        ntot += lo.npad[f];
    }
    lo.ntot = ntot;
    // Chunk size: the largest power-of-two multiple of the tile (at most
    // 2^18 points) that still gives >= 8 units per resident CTA slot.
    const int64_t target = (int64_t)8 * plan->sm_count * 2;
    const int64_t cmax = (int64_t)1 << 18;
    int64_t chunk = lo.P;
    while (chunk * 2 <= cmax) chunk *= 2;
    for (;;) {
        int64_t units = 0;
        for (int f = 0; f < nfield; ++f) units += (lo.npad[f] + chunk - 1) / chunk * lo.ngroups;
        if (units >= target || chunk <= lo.P) break;
        chunk /= 2;
    }
    if (plan->chunk_log2) chunk = std::max<int64_t>((int64_t)1 << plan->chunk_log2, lo.P);
    lo.chunk = chunk;
    int64_t units = 0;
    int32_t slots = 0;
    for (int f = 0; f < nfield; ++f) {
        lo.nchunk[f] = (int32_t)((lo.npad[f] + chunk - 1) / chunk);
        lo.slot0[f] = slots;
        lo.unit0[f] = units;
        slots += lo.nchunk[f];
        units += (int64_t)lo.nchunk[f] * lo.ngroups;
    }
    lo.nslots = slots;
    lo.nunits = units;
    size_t b = 0;
    lo.pts_off = b;
    b += up256((size_t)ntot * lo.narr * lo.abytes);
    lo.slots_off = b;
    b += up256((size_t)slots * plan->nmodes * 16);
    lo.counter_off = b;
    b += 256;
    lo.nranges = 0;
    for (int c = 0; c < ncat; ++c) lo.nranges += (cats[c].n + SORT_RANGE - 1) / SORT_RANGE;
    lo.hist_off = b;
    b += up256((size_t)std::max<int64_t>(lo.nranges, 1) * SORT_BUCKETS * 8);
    lo.fwd_end = b;
    if (is_f64) {  // catalog-order adjoint: the table alone
        lo.gtab_off = 0;
        lo.bwd_end = up256((size_t)nfield * plan->acol * 2 * lo.abytes);
    } else {  // sorted adjoint: the prepared points, then float4 table entries
        lo.gtab_off = lo.fwd_end;
        lo.bwd_end = lo.gtab_off + up256((size_t)nfield * plan->acol * 16);
    }
    lo.shot_off = 0;
    const size_t shot_end = up256((size_t)std::max(ncat, 1) * SHOT_NBLK * 8);
    lo.total = std::max(std::max(lo.fwd_end, lo.bwd_end), shot_end);
    return POINTSHT_OK;
}

extern "C" size_t pointsht_workspace_size(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat,
                                          int32_t nfield, pointsht_precision prec) {
    if (check_common(plan, cats, ncat, nfield, prec, "workspace_size") != POINTSHT_OK) return 0;
    Layout lo;
    if (make_layout(plan, cats, ncat, nfield, prec, lo) != POINTSHT_OK) return 0;
    return lo.total;
}

static pointsht_status check_device(pointsht_plan plan, const char* who) {
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev != plan->device)
        return fail(POINTSHT_EINVAL, "%s: current device %d differs from the plan's device %d", who, dev, plan->device);
    return POINTSHT_OK;
}

static pointsht_status check_ws(const Layout& lo, void* ws, size_t ws_bytes, size_t need, const char* who) {
    if (need > 0 && !ws) return fail(POINTSHT_EINVAL, "%s: workspace is NULL", who);
    if ((uintptr_t)ws % 256) return fail(POINTSHT_EINVAL, "%s: workspace is not 256-byte aligned", who);
    if (ws_bytes < need)
        return fail(POINTSHT_ENOMEM, "%s: workspace has %zu bytes, %zu needed", who, ws_bytes, need);
    (void)lo;
    return POINTSHT_OK;
}

static void fill_prep(const pointsht_catalog* cats, int32_t ncat, int32_t nfield, const Layout& lo, void* pts,
                      unsigned* err, PrepParams& pp) {
    memset(&pp, 0, sizeof(pp));
    pp.ncat = ncat;
    pp.nfield = nfield;
    pp.ntot = lo.ntot;
    pp.pts = pts;
    pp.err = err;
    int64_t run[PSHT_MAX_FIELDS] = {};
    int64_t id = 0;
    for (int c = 0; c < ncat; ++c) {
        const int f = cats[c].field;
        pp.cat[c].id0 = id;
        id += cats[c].n;
        pp.cat[c].x = cats[c].x;
        pp.cat[c].phi = cats[c].phi;
        pp.cat[c].w = cats[c].w;
        pp.cat[c].n = cats[c].n;
        pp.cat[c].coeff = cats[c].coeff;
        pp.cat[c].field = f;
        pp.cat[c].dst = lo.off[f] + run[f];
        run[f] += cats[c].n;
    }
    for (int f = 0; f < nfield; ++f) {
        pp.pad_off[f] = lo.off[f] + lo.nfpts[f];
        pp.pad_n[f] = lo.npad[f] - lo.nfpts[f];
    }
}

// ------------------------------------------------------------- a_lm --
extern "C" pointsht_status pointsht_alm(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat,
                                        int32_t nfield, pointsht_precision prec, double* alm_out, void* workspace,
                                        size_t ws_bytes, void* stream) {
    pointsht_status s = check_common(plan, cats, ncat, nfield, prec, "alm");
    if (s != POINTSHT_OK) return s;
    if (prec == POINTSHT_MIXED)
        return fail(POINTSHT_EINVAL,
                    "alm: POINTSHT_MIXED applies to weight columns on one point set: use pointsht_alm_columns");
    if (prec != POINTSHT_FP64 && plan->lmax > F32Scale::MAX_LMAX)
        return fail(POINTSHT_EINVAL, "alm: the FP32 path supports lmax <= %d (plan has %d)", F32Scale::MAX_LMAX,
                    plan->lmax);
    if (!alm_out || ((uintptr_t)alm_out % 16)) return fail(POINTSHT_EINVAL, "alm: alm_out NULL or not 16-byte aligned");
    if ((s = check_device(plan, "alm")) != POINTSHT_OK) return s;
    Layout lo;
    make_layout(plan, cats, ncat, nfield, prec, lo);
    if (plan->smem_optin && analysis_smem_need(lo.is_f64, lo.k32, plan->lmax) > plan->smem_optin) {
        // the per-warp accumulator rows of the analysis CTA live in shared memory
        int lm = 1;
        while (lm < plan->lmax && analysis_smem_need(lo.is_f64, lo.k32, lm + 1) <= plan->smem_optin) ++lm;
        return fail(POINTSHT_EINVAL, "alm: the %s path supports lmax <= %d on this device (plan has %d)",
                    lo.is_f64 ? "FP64" : "FP32", lm, plan->lmax);
    }
    if ((s = check_ws(lo, workspace, ws_bytes, lo.total, "alm")) != POINTSHT_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);

    PrepParams pp;
    fill_prep(cats, ncat, nfield, lo, ws + lo.pts_off, plan->err, pp);
    if (lo.ntot > 0) {
        SortParams sp;
        memset(&sp, 0, sizeof(sp));
        sp.prep = pp;
        int64_t r = 0;
        for (int c = 0; c < ncat; ++c) {
            sp.range0[c] = r;
            r += (cats[c].n + SORT_RANGE - 1) / SORT_RANGE;
        }
        sp.range0[ncat] = r;
        for (int f = 0; f < nfield; ++f) sp.field_off[f] = lo.off[f];
        sp.hist = reinterpret_cast<int64_t*>(ws + lo.hist_off);
        cudaError_t e = lo.is_f64 ? launch_prep_sorted<double>(sp, st) : launch_prep_sorted<float>(sp, st);
        if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "alm: prep launch: %s", cudaGetErrorString(e));
    }
    if (lo.nunits > 0) {
        CUDA_TRY(cudaMemsetAsync(ws + lo.counter_off, 0, 256, st));
        AnalysisParams ap;
        memset(&ap, 0, sizeof(ap));
        ap.lmax = plan->lmax;
        ap.nfield = nfield;
        ap.ngroups = lo.ngroups;
        ap.flush_tiles = FLUSH_TILES;
        ap.nmodes = plan->nmodes;
        ap.chunk = lo.chunk;
        ap.nunits = lo.nunits;
        ap.ntot = lo.ntot;
        for (int f = 0; f < nfield; ++f) {
            ap.fld[f].off = lo.off[f];
            ap.fld[f].npad = lo.npad[f];
            ap.fld[f].unit0 = lo.unit0[f];
            ap.fld[f].nchunk = lo.nchunk[f];
            ap.fld[f].slot0 = lo.slot0[f];
        }
        ap.pts = ws + lo.pts_off;
        ap.alpha_f = plan->alpha_f;
        ap.alpha_f2 = plan->alpha_f2;
        ap.alpha_d = plan->alpha_d;
        ap.colstart = plan->colstart;
        ap.log2c_hi = plan->log2c_hi;
        ap.log2c_lo = plan->log2c_lo;
        ap.log2c = plan->log2c;
        ap.pole_ae = plan->pole_ae;
        ap.pole_x = plan->pole_x;
        ap.pole_rho = plan->pole_rho;
        ap.pole_mmax = plan->pole_mmax;
        ap.wait_probe = plan->wait_probe;
        ap.stats = plan->stats;
        ap.slots = reinterpret_cast<double*>(ws + lo.slots_off);
        ap.counter = reinterpret_cast<int*>(ws + lo.counter_off);
        ap.err = plan->err;
        if (plan->ev_start) CUDA_TRY(cudaEventRecord(plan->ev_start, st));
        cudaError_t e = launch_analysis(ap, lo.is_f64, lo.k32, plan->sm_count, st, nullptr);
        if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "alm: analysis launch: %s", cudaGetErrorString(e));
        if (plan->ev_stop) CUDA_TRY(cudaEventRecord(plan->ev_stop, st));
    }
    ReduceParams rp;
    memset(&rp, 0, sizeof(rp));
    rp.nfield = nfield;
    rp.nmodes = plan->nmodes;
    for (int f = 0; f < nfield; ++f) {
        rp.slot0[f] = lo.slot0[f];
        rp.nchunk[f] = lo.nchunk[f];
    }
    rp.slots = reinterpret_cast<const double*>(ws + lo.slots_off);
    rp.gamma = plan->gamma;
    rp.out = alm_out;
    cudaError_t e = launch_reduce(rp, st);
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "alm: reduce launch: %s", cudaGetErrorString(e));
    return POINTSHT_OK;
}

// ---------------------------------------------------- weight columns --
// Workspace of the mixed column form.
struct ColLayout {
    int64_t ntot = 0, chunk = 0, nunits = 0, nranges = 0;
    int32_t nchunk = 0, npairs = 0, ncolp = 0, maxctas = 0;
    int64_t accstride = 0;
    size_t pts_off = 0, colmax_off = 0, hist_off = 0, slots_off = 0, acc_off = 0, counter_off = 0, total = 0;
};

static void make_col_layout(pointsht_plan plan, int64_t n, int32_t ncol, ColLayout& c) {
    const int P = mixed_tile_points();
    const int L = plan->lmax;
    c.ntot = (n + P - 1) / P * P;
    c.npairs = L / 2 + 1;
    c.ncolp = std::min(ncol, mixed_max_columns());
    // chunk: the largest power-of-two multiple of the tile (at most 2^22
    // points) that still gives >= 4 units per SM
    const int64_t target = (int64_t)4 * plan->sm_count;
    int64_t chunk = P;
    while (chunk * 2 <= ((int64_t)1 << 22)) chunk *= 2;
    while (chunk > P && (c.ntot + chunk - 1) / chunk * c.npairs < target) chunk /= 2;
    c.chunk = chunk;
    c.nchunk = (int32_t)((c.ntot + chunk - 1) / chunk);
    c.nunits = (int64_t)c.nchunk * c.npairs;
    c.nranges = (n + SORT_RANGE - 1) / SORT_RANGE;
    size_t b = 0;
    c.pts_off = b;
    b += up256((size_t)c.ntot * (mixed_geometry_arrays() + ncol) * 4);
    c.colmax_off = b;
    b += up256((size_t)ncol * 4);
    c.hist_off = b;
    b += up256((size_t)std::max<int64_t>(c.nranges, 1) * SORT_BUCKETS * 8);
    c.slots_off = b;
    b += up256((size_t)c.ncolp * c.nchunk * plan->nmodes * 16);
    // FP32 accumulator rows of each resident CTA (L2-resident; at most two per SM)
    c.maxctas = 2 * plan->sm_count;
    c.accstride = mixed_acc_stride(L);
    c.acc_off = b;
    b += up256((size_t)c.maxctas * c.accstride * 4);
    c.counter_off = b;
    b += 256;
    c.total = b;
}

static pointsht_status check_columns(pointsht_plan plan, const float* x, const float* phi, const float* w, int64_t n,
                                     int32_t ncol, pointsht_precision prec, const char* who) {
    if (!plan) return fail(POINTSHT_EINVAL, "%s: plan is NULL", who);
    if (n < 0) return fail(POINTSHT_EINVAL, "%s: n=%lld < 0", who, (long long)n);
    if (ncol < 1 || ncol > PSHT_MAX_FIELDS)
        return fail(POINTSHT_EINVAL, "%s: ncol=%d outside [1, %d]", who, ncol, PSHT_MAX_FIELDS);
    if (prec != POINTSHT_FP32 && prec != POINTSHT_MIXED)
        return fail(POINTSHT_EINVAL, "%s: precision must be POINTSHT_FP32 or POINTSHT_MIXED", who);
    if (n > 0 && (!x || !phi || !w)) return fail(POINTSHT_EINVAL, "%s: x, phi or w is NULL", who);
    if (((uintptr_t)x | (uintptr_t)phi | (uintptr_t)w) % 4)
        return fail(POINTSHT_EINVAL, "%s: x, phi, w are not 4-byte aligned", who);
    if (plan->lmax > F32Scale::MAX_LMAX)
        return fail(POINTSHT_EINVAL, "%s: the FP32 recurrence supports lmax <= %d (plan has %d)", who,
                    F32Scale::MAX_LMAX, plan->lmax);
    return POINTSHT_OK;
}

// the FP32 form of the columns: one catalog (and field) per column
static int32_t column_catalogs(const float* x, const float* phi, const float* w, int64_t n, int32_t ncol,
                               std::vector<pointsht_catalog>& cats) {
    cats.assign(ncol, pointsht_catalog{});
    for (int c = 0; c < ncol; ++c) {
        cats[c].x = x;
        cats[c].phi = phi;
        cats[c].w = w ? w + (size_t)c * n : nullptr;
        cats[c].n = n;
        cats[c].field = c;
        cats[c].coeff = 1.0;
    }
    return ncol;
}

extern "C" size_t pointsht_workspace_size_columns(pointsht_plan plan, int64_t n, int32_t ncol,
                                                  pointsht_precision prec) {
    if (!plan || n < 0 || ncol < 1 || ncol > PSHT_MAX_FIELDS || (prec != POINTSHT_FP32 && prec != POINTSHT_MIXED)) {
        fail(POINTSHT_EINVAL, "workspace_size_columns: bad plan, n, ncol or precision");
        return 0;
    }
    if (prec == POINTSHT_FP32) {
        std::vector<pointsht_catalog> cats;
        const float dummy = 0.f;
        column_catalogs(&dummy, &dummy, &dummy, n, ncol, cats);
        return pointsht_workspace_size(plan, cats.data(), ncol, ncol, prec);
    }
    ColLayout c;
    make_col_layout(plan, n, ncol, c);
    return c.total;
}

extern "C" pointsht_status pointsht_alm_columns(pointsht_plan plan, const float* x, const float* phi, const float* w,
                                                int64_t n, int32_t ncol, pointsht_precision prec, double* alm_out,
                                                void* workspace, size_t ws_bytes, void* stream) {
    pointsht_status s = check_columns(plan, x, phi, w, n, ncol, prec, "alm_columns");
    if (s != POINTSHT_OK) return s;
    if (prec == POINTSHT_FP32) {
        std::vector<pointsht_catalog> cats;
        column_catalogs(x, phi, w, n, ncol, cats);
        return pointsht_alm(plan, cats.data(), ncol, ncol, prec, alm_out, workspace, ws_bytes, stream);
    }
    if (!alm_out || ((uintptr_t)alm_out % 16))
        return fail(POINTSHT_EINVAL, "alm_columns: alm_out NULL or not 16-byte aligned");
    if ((s = check_device(plan, "alm_columns")) != POINTSHT_OK) return s;
    ColLayout c;
    make_col_layout(plan, n, ncol, c);
    if (!workspace && c.total > 0) return fail(POINTSHT_EINVAL, "alm_columns: workspace is NULL");
    if ((uintptr_t)workspace % 256) return fail(POINTSHT_EINVAL, "alm_columns: workspace is not 256-byte aligned");
    if (ws_bytes < c.total)
        return fail(POINTSHT_ENOMEM, "alm_columns: workspace has %zu bytes, %zu needed", ws_bytes, c.total);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    uint32_t* pts = reinterpret_cast<uint32_t*>(ws + c.pts_off);
    unsigned* colmax = reinterpret_cast<unsigned*>(ws + c.colmax_off);
    CUDA_TRY(cudaMemsetAsync(colmax, 0, (size_t)ncol * 4, st));
    PrepColsParams pp;
    memset(&pp, 0, sizeof(pp));
    pp.x = x;
    pp.phi = phi;
    pp.w = w;
    pp.n = n;
    pp.ncol = ncol;
    pp.ntot = c.ntot;
    pp.pts = pts;
    pp.hist = reinterpret_cast<const int64_t*>(ws + c.hist_off);
    pp.colmax = colmax;
    pp.err = plan->err;
    if (n > 0) {
        SortParams sp;
        memset(&sp, 0, sizeof(sp));
        sp.prep.ncat = 1;
        sp.prep.nfield = 1;
        sp.prep.cat[0].x = x;
        sp.prep.cat[0].phi = phi;
        sp.prep.cat[0].w = w;
        sp.prep.cat[0].n = n;
        sp.prep.cat[0].coeff = 1.0;
        sp.range0[0] = 0;
        sp.range0[1] = c.nranges;
        sp.field_off[0] = 0;
        sp.hist = reinterpret_cast<int64_t*>(ws + c.hist_off);
        cudaError_t e = launch_sort_offsets_f32(sp, st);
        if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "alm_columns: sort launch: %s", cudaGetErrorString(e));
    }
    if (c.ntot > 0) {
        cudaError_t e = launch_mixed_prep(pp, c.nranges, st);
        if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "alm_columns: prep launch: %s", cudaGetErrorString(e));
    }
    for (int col0 = 0; col0 < ncol; col0 += c.ncolp) {
        const int nc = std::min(c.ncolp, ncol - col0);
        if (c.nunits > 0) {
            CUDA_TRY(cudaMemsetAsync(ws + c.counter_off, 0, 256, st));
            MixedParams mp;
            memset(&mp, 0, sizeof(mp));
            mp.lmax = plan->lmax;
            mp.ncol = nc;
            mp.npairs = c.npairs;
            mp.flush_tiles = FLUSH_TILES;
            mp.nmodes = plan->nmodes;
            mp.chunk = c.chunk;
            mp.nunits = c.nunits;
            mp.ntot = c.ntot;
            mp.nchunk = c.nchunk;
            mp.pts = pts;
            mp.wcols = pts + (size_t)(mixed_geometry_arrays() + col0) * c.ntot;
            mp.colmax = colmax + col0;
            mp.alpha2 = plan->alpha_f2;
            mp.alpha_f = plan->alpha_f;
            mp.colstart = plan->colstart;
            mp.log2c_hi = plan->log2c_hi;
            mp.log2c_lo = plan->log2c_lo;
            mp.slots = reinterpret_cast<double*>(ws + c.slots_off);
            mp.accg = reinterpret_cast<float*>(ws + c.acc_off);
            mp.accstride = c.accstride;
            mp.maxctas = c.maxctas;
            mp.counter = reinterpret_cast<int*>(ws + c.counter_off);
            mp.err = plan->err;
            if (plan->ev_start && col0 == 0) CUDA_TRY(cudaEventRecord(plan->ev_start, st));
            cudaError_t e = plan->mixed_kernel == 0 ? launch_mixed(mp, plan->sm_count, st)
                                                    : launch_mixed_tc(mp, plan->sm_count, st, plan->tc_shape);
            if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "alm_columns: mixed launch: %s", cudaGetErrorString(e));
            if (plan->ev_stop && col0 + nc >= ncol) CUDA_TRY(cudaEventRecord(plan->ev_stop, st));
        }
        ReduceParams rp;
        memset(&rp, 0, sizeof(rp));
        rp.nfield = nc;
        rp.nmodes = plan->nmodes;
        for (int f = 0; f < nc; ++f) {
            rp.slot0[f] = f * c.nchunk;
            rp.nchunk[f] = c.nunits > 0 ? c.nchunk : 0;
        }
        rp.slots = reinterpret_cast<const double*>(ws + c.slots_off);
        rp.gamma = plan->gamma;
        rp.out = alm_out + (size_t)col0 * plan->nmodes * 2;
        cudaError_t e = launch_reduce(rp, st);
        if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "alm_columns: reduce launch: %s", cudaGetErrorString(e));
    }
    return POINTSHT_OK;
}

// ------------------------------------------------------ interpolated --
// Fields of one interpolated call are transformed in groups of up to
// INTERP_GROUP: each field of a group is sorted, binned and folded into its
// own sample table, then the group's 6 x fields weight columns share the
// transform passes of up to 8 columns (4 fields = 24 columns = 3 full passes).
constexpr int INTERP_GROUP = 4;
constexpr int INTERP_COLS = 6;

struct InterpLayout {
    int64_t npts_max = 0, nranges_max = 0, ntot = 0, chunk = 0, nunits = 0, vtab_fstride = 0;
    int32_t nb = 0, nchunk = 0, npairs = 0, maxctas = 0, group = 1;
    int64_t accstride = 0;
    size_t hist_off = 0, binoff_off = 0, total_off = 0, wc_off = 0, turn_off = 0, stage_off = 0, v_off = 0,
           vtab_off = 0,
           nodes_off = 0, colmax_off = 0, slots_off = 0, acc_off = 0, counter_off = 0, T_off = 0, total = 0;
};

static void make_interp_layout(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat, int32_t nfield,
                               int32_t ntheta, InterpLayout& c) {
    const int L = plan->lmax;
    const int P = mixed_tile_points();
    for (int f = 0; f < nfield; ++f) {
        int64_t n = 0, nr = 0;
        for (int k = 0; k < ncat; ++k)
            if (cats[k].field == f) {
                n += cats[k].n;
                nr += interp_nranges(cats[k].n);
            }
        c.npts_max = std::max(c.npts_max, n);
        c.nranges_max = std::max(c.nranges_max, nr);
    }
    c.nb = ntheta + 1;
    c.ntot = ((int64_t)ntheta / 2 + P - 1) / P * P;  // positions: north samples, the south ones mirrored
    c.npairs = L / 2 + 1;
    const int64_t target = (int64_t)4 * plan->sm_count;
    int64_t chunk = P;
    while (chunk * 2 <= ((int64_t)1 << 22)) chunk *= 2;
    while (chunk > P && (c.ntot + chunk - 1) / chunk * c.npairs < target) chunk /= 2;
    c.chunk = chunk;
    c.nchunk = (int32_t)((c.ntot + chunk - 1) / chunk);
    c.nunits = (int64_t)c.nchunk * c.npairs;
    c.maxctas = 2 * plan->sm_count;
    c.accstride = mixed_acc_stride(L);
    c.group = std::max(1, std::min(nfield, INTERP_GROUP));
    c.vtab_fstride = (int64_t)(L + 1) * c.ntot * 4;
    const int64_t np = std::max<int64_t>(c.npts_max, 1);
    size_t b = 0;
    c.hist_off = b;   b += up256((size_t)std::max<int64_t>(c.nranges_max, 1) * c.nb * 4);
    c.binoff_off = b; b += up256((size_t)(c.nb + 1) * 8);
    c.total_off = b;  b += up256((size_t)c.nb * 8);
    c.wc_off = b;     b += up256((size_t)np * 4 * 4);
    c.turn_off = b;   b += up256((size_t)np * 2 * 4);
    c.stage_off = b;  b += up256((size_t)std::max<int64_t>(c.nranges_max, 1) * interp_range() * 7 * 4);
    c.v_off = b;      b += up256((size_t)(L + 1) * c.nb * 4 * 8);
    c.vtab_off = b;   b += up256((size_t)c.group * c.vtab_fstride * 8);
    c.nodes_off = b;  b += up256((size_t)c.ntot * mixed_geometry_arrays() * 4);
    c.colmax_off = b; b += 256;
    c.slots_off = b;  b += up256((size_t)8 * c.nchunk * plan->nmodes * 16);
    c.acc_off = b;    b += up256((size_t)c.maxctas * c.accstride * 4);
    c.counter_off = b; b += 256;
    c.T_off = b;      b += up256((size_t)INTERP_COLS * c.group * plan->nmodes * 16);
    c.total = b;
}

static pointsht_status check_interp(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat, int32_t nfield,
                                    int32_t ntheta, const char* who) {
    pointsht_status s = check_common(plan, cats, ncat, nfield, POINTSHT_FP32, who);
    if (s != POINTSHT_OK) return s;
    if (ntheta < 2 || ntheta > 32768 || (ntheta & 1))
        return fail(POINTSHT_EINVAL, "%s: ntheta=%d must be even and in [2, 32768]", who, ntheta);
    if (plan->lmax > F32Scale::MAX_LMAX)
        return fail(POINTSHT_EINVAL, "%s: the FP32 recurrence supports lmax <= %d (plan has %d)", who,
                    F32Scale::MAX_LMAX, plan->lmax);
    for (int f = 0; f < nfield; ++f) {
        int64_t n = 0;
        for (int k = 0; k < ncat; ++k)
            if (cats[k].field == f) n += cats[k].n;
        if (n >= ((int64_t)1 << 31)) return fail(POINTSHT_EINVAL, "%s: field %d has 2^31 or more points", who, f);
    }
    return POINTSHT_OK;
}

extern "C" size_t pointsht_workspace_size_interp(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat,
                                                 int32_t nfield, int32_t ntheta) {
    if (check_interp(plan, cats, ncat, nfield, ntheta, "workspace_size_interp") != POINTSHT_OK) return 0;
    InterpLayout c;
    make_interp_layout(plan, cats, ncat, nfield, ntheta, c);
    return c.total;
}

extern "C" pointsht_status pointsht_alm_interp(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat,
                                               int32_t nfield, int32_t ntheta, double* alm_out, void* workspace,
                                               size_t ws_bytes, void* stream) {
    pointsht_status s = check_interp(plan, cats, ncat, nfield, ntheta, "alm_interp");
    if (s != POINTSHT_OK) return s;
    if (!alm_out || ((uintptr_t)alm_out % 16))
        return fail(POINTSHT_EINVAL, "alm_interp: alm_out NULL or not 16-byte aligned");
    if ((s = check_device(plan, "alm_interp")) != POINTSHT_OK) return s;
    InterpLayout c;
    make_interp_layout(plan, cats, ncat, nfield, ntheta, c);
    if (!workspace) return fail(POINTSHT_EINVAL, "alm_interp: workspace is NULL");
    if ((uintptr_t)workspace % 256) return fail(POINTSHT_EINVAL, "alm_interp: workspace is not 256-byte aligned");
    if (ws_bytes < c.total)
        return fail(POINTSHT_ENOMEM, "alm_interp: workspace has %zu bytes, %zu needed", ws_bytes, c.total);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    const int L = plan->lmax;
    float2* vtab = reinterpret_cast<float2*>(ws + c.vtab_off);
    unsigned* colmax = reinterpret_cast<unsigned*>(ws + c.colmax_off);
    for (int g0 = 0; g0 < nfield; g0 += c.group) {
        const int gn = std::min(c.group, nfield - g0);
        CUDA_TRY(cudaMemsetAsync(colmax, 0, 256, st));
        // ---- per field of the group: sort by interval, bin, fold into its table ----
        for (int gi = 0; gi < gn; ++gi) {
            const int f = g0 + gi;
            InterpParams ip;
            memset(&ip, 0, sizeof(ip));
            ip.lmax = L;
            ip.ntheta = ntheta;
            ip.nb = c.nb;
            ip.ntot = c.ntot;
            int64_t r = 0, n = 0;
            for (int k = 0; k < ncat; ++k) {
                if (cats[k].field != f) continue;
                ip.cat[ip.ncat].x = static_cast<const float*>(cats[k].x);
                ip.cat[ip.ncat].phi = static_cast<const float*>(cats[k].phi);
                ip.cat[ip.ncat].w = static_cast<const float*>(cats[k].w);
                ip.cat[ip.ncat].n = cats[k].n;
                ip.cat[ip.ncat].coeff = cats[k].coeff;
                ip.range0[ip.ncat] = r;
                r += interp_nranges(cats[k].n);
                n += cats[k].n;
                ++ip.ncat;
            }
            ip.range0[ip.ncat] = r;
            ip.nranges = r;
            ip.npts = n;
            ip.hist = reinterpret_cast<int32_t*>(ws + c.hist_off);
            ip.binoff = reinterpret_cast<int64_t*>(ws + c.binoff_off);
            ip.total = reinterpret_cast<int64_t*>(ws + c.total_off);
            ip.wc = reinterpret_cast<float*>(ws + c.wc_off);
            ip.turn = reinterpret_cast<uint32_t*>(ws + c.turn_off);
            ip.stage = reinterpret_cast<uint32_t*>(ws + c.stage_off);
            ip.v = reinterpret_cast<float2*>(ws + c.v_off);
            ip.vtab = vtab + (int64_t)gi * c.vtab_fstride;
            ip.nodes = reinterpret_cast<uint32_t*>(ws + c.nodes_off);
            ip.colmax = colmax + INTERP_COLS * gi;
            ip.err = plan->err;
            if (plan->ev_start && f == 0) CUDA_TRY(cudaEventRecord(plan->ev_start, st));
            cudaError_t e = launch_interp_sort(ip, st);
            if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "alm_interp: sort launch: %s", cudaGetErrorString(e));
            e = launch_interp_tables(ip, plan->sm_count, st);
            if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "alm_interp: binning launch: %s", cudaGetErrorString(e));
        }
        // ---- transform of the group's 6 gn sample-weight columns, up to 8 per pass
        // (mixed kernel, table mode), each pass reduced into its columns of T ----
        const int ncolg = INTERP_COLS * gn;
        for (int c0 = 0; c0 < ncolg; c0 += 8) {
            const int nc = std::min(8, ncolg - c0);
            CUDA_TRY(cudaMemsetAsync(ws + c.counter_off, 0, 256, st));
            MixedParams mp;
            memset(&mp, 0, sizeof(mp));
            mp.lmax = L;
            mp.ncol = nc;
            mp.npairs = c.npairs;
            mp.flush_tiles = FLUSH_TILES;
            mp.nmodes = plan->nmodes;
            mp.chunk = c.chunk;
            mp.nunits = c.nunits;
            mp.ntot = c.ntot;
            mp.nchunk = c.nchunk;
            mp.pts = reinterpret_cast<const uint32_t*>(ws + c.nodes_off);
            mp.wcols = nullptr;
            mp.colmax = colmax + c0;
            mp.alpha2 = plan->alpha_f2;
            mp.colstart = plan->colstart;
            mp.log2c_hi = plan->log2c_hi;
            mp.log2c_lo = plan->log2c_lo;
            mp.slots = reinterpret_cast<double*>(ws + c.slots_off);
            mp.accg = reinterpret_cast<float*>(ws + c.acc_off);
            mp.accstride = c.accstride;
            mp.maxctas = c.maxctas;
            mp.vtab = vtab;
            mp.vtab_fstride = c.vtab_fstride;
            mp.tcol0 = c0;
            // near-pole form of the sample recurrence for the positions next to the
            // north pole: the positions are in theta order, so a warp's 128 span a
            // theta range, and the threshold is min(pole_x, 0.75) (the form is at
            // least as accurate as the standard one from x = 0.7 up)
            mp.pole_ae = plan->pole_x <= 1.f ? plan->pole_ae : nullptr;
            mp.pole_rho = plan->pole_rho;
            mp.pole_x = std::min(plan->pole_x, 0.75f);
            mp.pole_mmax = std::min(plan->pole_mmax, 64);
            mp.vtab_h = (float)(3.14159265358979323846 / (double)ntheta);
            mp.counter = reinterpret_cast<int*>(ws + c.counter_off);
            mp.err = plan->err;
            cudaError_t e = launch_mixed(mp, plan->sm_count, st);
            if (e != cudaSuccess)
                return fail(POINTSHT_ECUDA, "alm_interp: grid transform launch: %s", cudaGetErrorString(e));
            ReduceParams rp;
            memset(&rp, 0, sizeof(rp));
            rp.nfield = nc;
            rp.nmodes = plan->nmodes;
            for (int k = 0; k < nc; ++k) {
                rp.slot0[k] = k * c.nchunk;
                rp.nchunk[k] = c.nchunk;
            }
            rp.slots = reinterpret_cast<const double*>(ws + c.slots_off);
            rp.gamma = plan->gamma;
            rp.out = reinterpret_cast<double*>(ws + c.T_off) + (size_t)c0 * plan->nmodes * 2;
            e = launch_reduce(rp, st);
            if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "alm_interp: reduce launch: %s", cudaGetErrorString(e));
        }
        // ---- per field: a_lm from its six transforms ----
        for (int gi = 0; gi < gn; ++gi) {
            const int f = g0 + gi;
            cudaError_t e = launch_interp_combine(
                L, plan->nmodes, reinterpret_cast<const double*>(ws + c.T_off) + (size_t)INTERP_COLS * gi * plan->nmodes * 2,
                alm_out + (size_t)f * plan->nmodes * 2, st);
            if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "alm_interp: combine launch: %s", cudaGetErrorString(e));
        }
    }
    if (plan->ev_stop) CUDA_TRY(cudaEventRecord(plan->ev_stop, st));
    return POINTSHT_OK;
}

// ------------------------------------------------------- shot noise --
extern "C" pointsht_status pointsht_shot_noise(const pointsht_catalog* cats, int32_t ncat, int32_t nfield,
                                               pointsht_precision prec, double* noise_out, void* workspace,
                                               size_t ws_bytes, void* stream) {
    if (ncat < 0 || ncat > PSHT_MAX_CATS || (ncat > 0 && !cats))
        return fail(POINTSHT_EINVAL, "shot_noise: bad catalog list");
    if (nfield < 1 || nfield > PSHT_MAX_FIELDS) return fail(POINTSHT_EINVAL, "shot_noise: nfield=%d", nfield);
    if (!noise_out) return fail(POINTSHT_EINVAL, "shot_noise: noise_out is NULL");
    const size_t esz = prec == POINTSHT_FP64 ? 8 : 4;
    for (int c = 0; c < ncat; ++c) {
        if (cats[c].n < 0 || cats[c].field < 0 || cats[c].field >= nfield)
            return fail(POINTSHT_EINVAL, "shot_noise: catalog %d: bad n or field", c);
        if (cats[c].n > 0 && (!cats[c].w || (uintptr_t)cats[c].w % esz))
            return fail(POINTSHT_EINVAL, "shot_noise: catalog %d: w NULL or misaligned", c);
    }
    const size_t need = up256((size_t)std::max(ncat, 1) * SHOT_NBLK * 8);
    if (!workspace || ws_bytes < need || (uintptr_t)workspace % 256)
        return fail(POINTSHT_ENOMEM, "shot_noise: workspace needs %zu bytes, 256-aligned", need);
    PrepParams pp;
    memset(&pp, 0, sizeof(pp));
    pp.ncat = ncat;
    pp.nfield = nfield;
    for (int c = 0; c < ncat; ++c) {
        pp.cat[c].w = cats[c].w;
        pp.cat[c].n = cats[c].n;
        pp.cat[c].coeff = cats[c].coeff;
        pp.cat[c].field = cats[c].field;
    }
    cudaError_t e = launch_shot_noise(pp, prec == POINTSHT_FP64, static_cast<double*>(workspace), (int)SHOT_NBLK,
                                      noise_out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "shot_noise: %s", cudaGetErrorString(e));
    return POINTSHT_OK;
}

// --------------------------------------------------- spectra & bins --
extern "C" pointsht_status pointsht_combine(int32_t lmax, const double* alm_src, int32_t nsrc, const double* coef,
                                            int32_t nout, const double* noise_src, double* alm_out,
                                            double* noise_out, void* stream) {
    if (lmax < 0 || nsrc < 1 || nout < 1 || !alm_src || !coef || !alm_out)
        return fail(POINTSHT_EINVAL, "combine: bad arguments");
    if ((noise_src == nullptr) != (noise_out == nullptr))
        return fail(POINTSHT_EINVAL, "combine: noise_src and noise_out must both be set or both NULL");
    cudaError_t e = launch_combine(lmax, alm_src, nsrc, coef, nout, noise_src, alm_out, noise_out,
                                   static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "combine: %s", cudaGetErrorString(e));
    return POINTSHT_OK;
}

extern "C" pointsht_status pointsht_cl(int32_t lmax, const double* alm, int32_t nfield, const double* noise,
                                       double* cl_out, void* stream) {
    if (lmax < 0 || nfield < 1 || nfield > 1024 || !alm || !cl_out) return fail(POINTSHT_EINVAL, "cl: bad arguments");
    cudaError_t e = launch_cl(lmax, alm, nfield, noise, cl_out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "cl: %s", cudaGetErrorString(e));
    return POINTSHT_OK;
}

extern "C" pointsht_status pointsht_cl_backward(int32_t lmax, const double* alm, int32_t nfield,
                                                const double* grad_cl, double* grad_alm, double* grad_noise,
                                                void* stream) {
    if (lmax < 0 || nfield < 1 || nfield > 1024 || !alm || !grad_cl || !grad_alm)
        return fail(POINTSHT_EINVAL, "cl_backward: bad arguments");
    cudaError_t e = launch_cl_backward(lmax, alm, nfield, grad_cl, grad_alm, grad_noise,
                                       static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "cl_backward: %s", cudaGetErrorString(e));
    return POINTSHT_OK;
}

extern "C" pointsht_status pointsht_bin(int32_t lmax, const double* cl, int32_t nspec, const int32_t* edges,
                                        int32_t nbin, double* out, void* stream) {
    if (lmax < 0 || nspec < 1 || nbin < 1 || !cl || !edges || !out) return fail(POINTSHT_EINVAL, "bin: bad arguments");
    cudaError_t e = launch_bin(lmax, cl, nspec, edges, nbin, out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "bin: %s", cudaGetErrorString(e));
    return POINTSHT_OK;
}

extern "C" pointsht_status pointsht_bin_backward(int32_t lmax, const double* grad_b, int32_t nspec,
                                                 const int32_t* edges, int32_t nbin, double* grad_cl, void* stream) {
    if (lmax < 0 || nspec < 1 || nbin < 1 || !grad_b || !edges || !grad_cl)
        return fail(POINTSHT_EINVAL, "bin_backward: bad arguments");
    cudaError_t e = launch_bin_backward(lmax, grad_b, nspec, edges, nbin, grad_cl, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "bin_backward: %s", cudaGetErrorString(e));
    return POINTSHT_OK;
}

// --------------------------------------------------------- adjoint --
// The point-evaluation kernels behind pointsht_alm_backward (synth = 0) and
// pointsht_synthesis (synth = 1: table factor c_m, coeff 1, no noise term).
// Arguments already checked; the layout is make_layout's for these catalogs.
static pointsht_status run_adjoint(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat, int32_t nfield,
                                   const Layout& lo, const double* grad_alm, const double* grad_noise,
                                   void* const* grad_w, char* ws, int synth, cudaStream_t st, const char* who) {
    void* gtab = ws + lo.gtab_off;
    cudaError_t e;
    AdjointParams ap;
    memset(&ap, 0, sizeof(ap));
    ap.lmax = plan->lmax;
    ap.ncat = ncat;
    ap.nfield = nfield;
    ap.gstride = plan->acol;
    ap.colstart = plan->colstart;
    ap.log2c_hi = plan->log2c_hi;
    ap.log2c_lo = plan->log2c_lo;
    ap.log2c = plan->log2c;
    ap.gnoise = grad_noise;
    ap.err = plan->err;
    ap.gtab = gtab;
    if (!lo.is_f64) {
        // FP32: the points are prepared and |x|-sorted as for the analysis
        // (point ids kept), then one warp runs 256 consecutive prepared points.
        int64_t npts = 0;
        for (int c = 0; c < ncat; ++c) npts += cats[c].n;
        if (npts >= (int64_t)0xffffffffLL)
            return fail(POINTSHT_EINVAL, "%s: %lld points; the FP32 path takes fewer than 2^32 - 1", who,
                        (long long)npts);
        PrepParams pp;
        fill_prep(cats, ncat, nfield, lo, ws + lo.pts_off, plan->err, pp);
        if (lo.ntot > 0) {
            SortParams sp;
            memset(&sp, 0, sizeof(sp));
            sp.prep = pp;
            int64_t r = 0;
            for (int c = 0; c < ncat; ++c) {
                sp.range0[c] = r;
                r += (cats[c].n + SORT_RANGE - 1) / SORT_RANGE;
            }
            sp.range0[ncat] = r;
            for (int f = 0; f < nfield; ++f) sp.field_off[f] = lo.off[f];
            sp.hist = reinterpret_cast<int64_t*>(ws + lo.hist_off);
            e = launch_prep_sorted<float>(sp, st);
            if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "%s: prep launch: %s", who, cudaGetErrorString(e));
        }
        for (int c = 0; c < ncat; ++c) {
            ap.cat[c] = pp.cat[c];
            ap.gradw[c] = grad_w[c];
        }
        ap.pts = reinterpret_cast<const uint32_t*>(ws + lo.pts_off);
        ap.ntot = lo.ntot;
        for (int f = 0; f < nfield; ++f) ap.fld[f].off = lo.off[f];
        ap.alpha2 = plan->alpha_f2;
        ap.pole_ae = plan->pole_ae;
        ap.pole_x = plan->pole_x;
        ap.pole_rho = plan->pole_rho;
        ap.pole_mmax = plan->pole_mmax;
        e = launch_adjoint_sorted(ap, grad_alm, plan->gamma, synth, st);
        if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "%s: adjoint: %s", who, cudaGetErrorString(e));
        return POINTSHT_OK;
    }
    e = launch_build_gtab(lo.is_f64, plan->lmax, nfield, grad_alm, plan->gamma, plan->colstart, plan->acol, synth,
                          gtab, st);
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "%s: table: %s", who, cudaGetErrorString(e));
    const int ppw = adjoint_points_per_warp(lo.is_f64);
    int64_t wsum = 0;
    for (int c = 0; c < ncat; ++c) {
        ap.cat[c].x = cats[c].x;
        ap.cat[c].phi = cats[c].phi;
        ap.cat[c].w = cats[c].w;
        ap.cat[c].n = cats[c].n;
        ap.cat[c].coeff = cats[c].coeff;
        ap.cat[c].field = cats[c].field;
        ap.gradw[c] = grad_w[c];
        ap.warp0[c] = wsum;
        wsum += (cats[c].n + ppw - 1) / ppw;
    }
    ap.warp0[ncat] = wsum;
    ap.alpha = plan->alpha_d;
    e = launch_adjoint(lo.is_f64, ap, st);
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "%s: adjoint: %s", who, cudaGetErrorString(e));
    return POINTSHT_OK;
}

extern "C" pointsht_status pointsht_alm_backward(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat,
                                                 int32_t nfield, pointsht_precision prec, const double* grad_alm,
                                                 const double* grad_noise, void* const* grad_w, void* workspace,
                                                 size_t ws_bytes, void* stream) {
    pointsht_status s = check_common(plan, cats, ncat, nfield, prec, "alm_backward");
    if (s != POINTSHT_OK) return s;
    if (prec == POINTSHT_MIXED) prec = POINTSHT_FP32;  // the adjoint has no per-m contraction to move
    if (!grad_alm || ((uintptr_t)grad_alm % 16)) return fail(POINTSHT_EINVAL, "alm_backward: grad_alm NULL/misaligned");
    if (ncat > 0 && !grad_w) return fail(POINTSHT_EINVAL, "alm_backward: grad_w is NULL");
    const size_t esz = prec == POINTSHT_FP64 ? 8 : 4;
    for (int c = 0; c < ncat; ++c)
        if (cats[c].n > 0 && (!grad_w[c] || (uintptr_t)grad_w[c] % esz))
            return fail(POINTSHT_EINVAL, "alm_backward: grad_w[%d] NULL or misaligned", c);
    if (prec != POINTSHT_FP64 && plan->lmax > F32Scale::MAX_LMAX)
        return fail(POINTSHT_EINVAL, "alm_backward: the FP32 path supports lmax <= %d (plan has %d)",
                    F32Scale::MAX_LMAX, plan->lmax);
    if ((s = check_device(plan, "alm_backward")) != POINTSHT_OK) return s;
    Layout lo;
    make_layout(plan, cats, ncat, nfield, prec, lo);
    if ((s = check_ws(lo, workspace, ws_bytes, lo.total, "alm_backward")) != POINTSHT_OK) return s;
    return run_adjoint(plan, cats, ncat, nfield, lo, grad_alm, grad_noise, grad_w, static_cast<char*>(workspace), 0,
                       static_cast<cudaStream_t>(stream), "alm_backward");
}

// ------------------------------------------------------- synthesis --
// The unit-weight catalog of a synthesis call: weights in the workspace
// after the adjoint's own layout.
static void synthesis_catalog(const void* x, const void* phi, int64_t n, pointsht_catalog& cat) {
    memset(&cat, 0, sizeof(cat));
    cat.x = x;
    cat.phi = phi;
    cat.w = nullptr;  // set to the workspace's ones once placed
    cat.n = n;
    cat.field = 0;
    cat.coeff = 1.0;
}

extern "C" size_t pointsht_workspace_size_synthesis(pointsht_plan plan, int64_t n, pointsht_precision prec) {
    if (!plan || n < 0 || (prec != POINTSHT_FP32 && prec != POINTSHT_FP64)) return 0;
    pointsht_catalog cat;
    synthesis_catalog(nullptr, nullptr, n, cat);
    Layout lo;
    if (make_layout(plan, &cat, 1, 1, prec, lo) != POINTSHT_OK) return 0;
    return up256(lo.total) + up256((size_t)n * (prec == POINTSHT_FP64 ? 8 : 4));
}

extern "C" pointsht_status pointsht_synthesis(pointsht_plan plan, const void* x, const void* phi, int64_t n,
                                              pointsht_precision prec, const double* alm, void* out, void* workspace,
                                              size_t ws_bytes, void* stream) {
    if (!plan) return fail(POINTSHT_EINVAL, "synthesis: plan is NULL");
    if (prec != POINTSHT_FP32 && prec != POINTSHT_FP64)
        return fail(POINTSHT_EINVAL, "synthesis: precision must be POINTSHT_FP32 or POINTSHT_FP64");
    if (n < 0) return fail(POINTSHT_EINVAL, "synthesis: n=%lld < 0", (long long)n);
    const size_t esz = prec == POINTSHT_FP64 ? 8 : 4;
    if (!alm || ((uintptr_t)alm % 16)) return fail(POINTSHT_EINVAL, "synthesis: alm NULL or not 16-byte aligned");
    if (n > 0 && (!x || !phi || !out || (((uintptr_t)x | (uintptr_t)phi | (uintptr_t)out) % esz)))
        return fail(POINTSHT_EINVAL, "synthesis: x, phi or out NULL or not %zu-byte aligned", esz);
    if (prec == POINTSHT_FP32 && plan->lmax > F32Scale::MAX_LMAX)
        return fail(POINTSHT_EINVAL, "synthesis: the FP32 path supports lmax <= %d (plan has %d)", F32Scale::MAX_LMAX,
                    plan->lmax);
    pointsht_status s = check_device(plan, "synthesis");
    if (s != POINTSHT_OK) return s;
    pointsht_catalog cat;
    synthesis_catalog(x, phi, n, cat);
    Layout lo;
    make_layout(plan, &cat, 1, 1, prec, lo);
    const size_t need = up256(lo.total) + up256((size_t)n * esz);
    if ((s = check_ws(lo, workspace, ws_bytes, need, "synthesis")) != POINTSHT_OK) return s;
    if (n == 0) return POINTSHT_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    void* ones = ws + up256(lo.total);
    cudaError_t e = launch_fill_ones(n, prec == POINTSHT_FP64, ones, st);
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "synthesis: %s", cudaGetErrorString(e));
    cat.w = ones;
    void* outs[1] = {out};
    return run_adjoint(plan, &cat, 1, 1, lo, alm, nullptr, outs, ws, 1, st, "synthesis");
}

// ------------------------------------------------------------ spin 2 --
static pointsht_status check_spin2(pointsht_plan plan, const pointsht_shear_catalog* cats, int32_t ncat,
                                   int32_t nfield, const char* who) {
    if (!plan) return fail(POINTSHT_EINVAL, "%s: plan is NULL", who);
    if (ncat < 0 || ncat > PSHT_MAX_CATS) return fail(POINTSHT_EINVAL, "%s: ncat=%d outside [0, %d]", who, ncat, PSHT_MAX_CATS);
    if (ncat > 0 && !cats) return fail(POINTSHT_EINVAL, "%s: cats is NULL", who);
    if (nfield < 1 || nfield > PSHT_MAX_FIELDS)
        return fail(POINTSHT_EINVAL, "%s: nfield=%d outside [1, %d]", who, nfield, PSHT_MAX_FIELDS);
    if (plan->lmax > F32Scale::MAX_LMAX)
        return fail(POINTSHT_EINVAL, "%s: the FP32 path supports lmax <= %d (plan has %d)", who, F32Scale::MAX_LMAX,
                    plan->lmax);
    for (int c = 0; c < ncat; ++c) {
        const pointsht_shear_catalog& k = cats[c];
        if (k.n < 0) return fail(POINTSHT_EINVAL, "%s: catalog %d has n=%lld < 0", who, c, (long long)k.n);
        if (k.field < 0 || k.field >= nfield)
            return fail(POINTSHT_EINVAL, "%s: catalog %d has field %d outside [0, %d)", who, c, k.field, nfield);
        if (!std::isfinite(k.coeff)) return fail(POINTSHT_EINVAL, "%s: catalog %d has a non-finite coeff", who, c);
        if (k.n > 0) {
            if (!k.x || !k.phi || !k.w || !k.g1 || !k.g2)
                return fail(POINTSHT_EINVAL, "%s: catalog %d has a NULL array", who, c);
            if (((uintptr_t)k.x | (uintptr_t)k.phi | (uintptr_t)k.w | (uintptr_t)k.g1 | (uintptr_t)k.g2) % 4)
                return fail(POINTSHT_EINVAL, "%s: catalog %d arrays are not 4-byte aligned", who, c);
        }
    }
    return POINTSHT_OK;
}

extern "C" size_t pointsht_workspace_size_spin2(pointsht_plan plan, const pointsht_shear_catalog* cats, int32_t ncat,
                                                int32_t nfield) {
    if (check_spin2(plan, cats, ncat, nfield, "workspace_size_spin2") != POINTSHT_OK) return 0;
    return spin2_workspace_bytes(plan->lmax, cats, ncat, nfield);
}

extern "C" pointsht_status pointsht_alm_spin2(pointsht_plan plan, const pointsht_shear_catalog* cats, int32_t ncat,
                                              int32_t nfield, double* E_out, double* B_out, void* workspace,
                                              size_t ws_bytes, void* stream) {
    pointsht_status s = check_spin2(plan, cats, ncat, nfield, "alm_spin2");
    if (s != POINTSHT_OK) return s;
    if (!E_out || !B_out || (((uintptr_t)E_out | (uintptr_t)B_out) % 16))
        return fail(POINTSHT_EINVAL, "alm_spin2: E_out or B_out NULL or not 16-byte aligned");
    if ((s = check_device(plan, "alm_spin2")) != POINTSHT_OK) return s;
    const size_t need = spin2_workspace_bytes(plan->lmax, cats, ncat, nfield);
    if (need == 0) return fail(POINTSHT_EINVAL, "alm_spin2: too many points for the chunk table");
    if (!workspace || ((uintptr_t)workspace % 256))
        return fail(POINTSHT_EINVAL, "alm_spin2: workspace NULL or not 256-byte aligned");
    if (ws_bytes < need) return fail(POINTSHT_ENOMEM, "alm_spin2: workspace has %zu bytes, %zu needed", ws_bytes, need);
    cudaError_t e = spin2_run(plan->lmax, cats, ncat, nfield, workspace, plan->err, plan->sm_count, E_out, B_out,
                              static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "alm_spin2: %s", cudaGetErrorString(e));
    return POINTSHT_OK;
}

// ------------------------------------------------------- mode coupling --
static const int COUPLING_MAX_LMAX = 8192;
static const int DECOUPLE_MAX_NBIN = 512;

extern "C" size_t pointsht_workspace_size_coupling(int32_t lmax) {
    if (lmax < 0 || lmax > COUPLING_MAX_LMAX) return 0;
    return up256((size_t)(2 * lmax + 1) * 8) * 2;
}

extern "C" pointsht_status pointsht_coupling(int32_t lmax, int32_t lmax_w, const double* W, double* M,
                                             void* workspace, size_t ws_bytes, void* stream) {
    if (lmax < 0 || lmax > COUPLING_MAX_LMAX)
        return fail(POINTSHT_EINVAL, "coupling: lmax=%d outside [0, %d]", lmax, COUPLING_MAX_LMAX);
    if (lmax_w < 0) return fail(POINTSHT_EINVAL, "coupling: lmax_w=%d < 0", lmax_w);
    if (!W || !M || !workspace) return fail(POINTSHT_EINVAL, "coupling: NULL pointer");
    if (((uintptr_t)W | (uintptr_t)M) % 8) return fail(POINTSHT_EINVAL, "coupling: W or M not 8-byte aligned");
    const size_t need = pointsht_workspace_size_coupling(lmax);
    if (ws_bytes < need || ((uintptr_t)workspace % 256))
        return fail(POINTSHT_EINVAL, "coupling: workspace of %zu bytes (need %zu, 256-byte aligned)", ws_bytes, need);
    // W beyond 2 lmax never enters (lambda <= l + l')
    const int lw = std::min(lmax_w, 2 * lmax);
    double* b = static_cast<double*>(workspace);
    double* ib = reinterpret_cast<double*>(static_cast<char*>(workspace) + need / 2);
    cudaError_t e = launch_coupling(lmax, lw, W, M, b, ib, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "coupling: %s", cudaGetErrorString(e));
    return POINTSHT_OK;
}

extern "C" pointsht_status pointsht_coupling_binned(int32_t lmax, const double* M, const int32_t* edges, int32_t nbin,
                                                    double* R, double* Mbb, void* stream) {
    if (lmax < 0 || nbin < 1 || nbin > DECOUPLE_MAX_NBIN)
        return fail(POINTSHT_EINVAL, "coupling_binned: lmax=%d, nbin=%d (1..%d)", lmax, nbin, DECOUPLE_MAX_NBIN);
    if (!M || !edges || !R || !Mbb) return fail(POINTSHT_EINVAL, "coupling_binned: NULL pointer");
    cudaError_t e = launch_coupling_binned(lmax, M, edges, nbin, R, Mbb, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "coupling_binned: %s", cudaGetErrorString(e));
    return POINTSHT_OK;
}

extern "C" size_t pointsht_workspace_size_decouple(int32_t nbin) {
    if (nbin < 1 || nbin > DECOUPLE_MAX_NBIN) return 0;
    return up256(decouple_workspace_bytes(nbin));
}

extern "C" pointsht_status pointsht_decouple(int32_t lmax, int32_t nbin, const double* Mbb, const double* R,
                                             const double* cl_binned, int32_t nspec, double* Minv, double* Mcal,
                                             double* cl_dec, void* workspace, size_t ws_bytes, void* stream) {
    if (lmax < 0 || nbin < 1 || nbin > DECOUPLE_MAX_NBIN || nspec < 0)
        return fail(POINTSHT_EINVAL, "decouple: lmax=%d, nbin=%d (1..%d), nspec=%d", lmax, nbin, DECOUPLE_MAX_NBIN,
                    nspec);
    if (!Mbb || !Minv || !workspace) return fail(POINTSHT_EINVAL, "decouple: NULL pointer");
    if ((!R) != (!Mcal)) return fail(POINTSHT_EINVAL, "decouple: R and Mcal must be given together");
    if ((!cl_binned) != (!cl_dec)) return fail(POINTSHT_EINVAL, "decouple: cl_binned and cl_dec must be given together");
    const size_t need = pointsht_workspace_size_decouple(nbin);
    if (ws_bytes < need || ((uintptr_t)workspace % 256))
        return fail(POINTSHT_EINVAL, "decouple: workspace of %zu bytes (need %zu, 256-byte aligned)", ws_bytes, need);
    cudaError_t e = launch_decouple(lmax, nbin, Mbb, R, cl_binned, nspec, Minv, Mcal, cl_dec,
                                    static_cast<double*>(workspace), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "decouple: %s", cudaGetErrorString(e));
    return POINTSHT_OK;
}

extern "C" pointsht_status pointsht_fkp_normalise(int32_t lmax_w, const double* W, int32_t lmax, int32_t nbin,
                                                  const double* R, const double* cl_binned, int32_t nspec,
                                                  double* norm, double* Mprime, double* cl_norm, void* stream) {
    if (lmax_w < 0 || !W || !norm) return fail(POINTSHT_EINVAL, "fkp_normalise: lmax_w=%d, W or norm NULL", lmax_w);
    if ((!R) != (!Mprime)) return fail(POINTSHT_EINVAL, "fkp_normalise: R and Mprime must be given together");
    if ((!cl_binned) != (!cl_norm))
        return fail(POINTSHT_EINVAL, "fkp_normalise: cl_binned and cl_norm must be given together");
    if ((R || cl_binned) && (nbin < 1 || lmax < 0 || nspec < 0))
        return fail(POINTSHT_EINVAL, "fkp_normalise: lmax=%d, nbin=%d, nspec=%d", lmax, nbin, nspec);
    cudaError_t e = launch_fkp_normalise(lmax_w, W, lmax, nbin, R, cl_binned, nspec, norm, Mprime, cl_norm,
                                         static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(POINTSHT_ECUDA, "fkp_normalise: %s", cudaGetErrorString(e));
    return POINTSHT_OK;
}
