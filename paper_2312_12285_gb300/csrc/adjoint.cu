// adjoint.cu -- vector-Jacobian product of the point-catalog SHT with respect
// to the weights (point-evaluation synthesis).
//
// From Eq. alm_def, a_lm = sum_i coeff w_i lambda_lm(x_i) e^{-i m phi_i}, so for
// a real loss L with g_lm = dL/dRe a_lm + i dL/dIm a_lm:
//   dL/dw_i = coeff sum_{l, m>=0} lambda_lm(x_i) Re(g_lm e^{i m phi_i}).
// With lambda = gamma' sigma (see analysis.cu) the table holds gamma'_lm g_lm
// and each lane runs the same seed and sigma-recurrence as the analysis for its
// K points, accumulating sum_l sigma_l (gamma' g)_l in registers: no cross-lane
// reduction.  Contributions made while a point's state is still below the
// floating-point range (exponent block E < 0) are dropped by clearing that
// point's accumulators when E reaches 0, and at the end of a column if it
// never does.  Sums over m are carried in FP64 per point.
//
// Two kernels: adjoint_kernel (FP64, catalog order, K = 2 points per lane)
// and adjoint_sorted_kernel (FP32, over the analysis's |x|-sorted prepared
// points, 8 per lane as f32x2 pairs).  Point-evaluation synthesis is the same
// computation with unit weights (see build_gtab_kernel).
#include "common.cuh"

#include <math_constants.h>

#include <algorithm>

namespace psht {

// Seed, phase and coefficient loads for the FP64 adjoint, from per-point
// values held in registers (the analysis reads them from its shared-memory
// tile).
namespace adj {

struct F64 {
    using real = double;
    using real2 = double2;
    __device__ static __forceinline__ void seed(int m, double ls, double lc, double, double& mant, int& E) {
        const double e = fma((double)m, ls, lc);
        const bool pole = e < -1.0e7;
        const double Ef = pole ? -1048576.0 : fmin(0.0, ceil((e - (double)F64Scale::CHECK_EXP) * (1.0 / F64Scale::SCALE_BITS)));
        E = (int)Ef;
        const double eh = pole ? 0.0 : e - (double)F64Scale::SCALE_BITS * Ef;
        const double n = floor(eh);
        mant = pole ? 0.0 : ldexp(exp2(eh - n), (int)n);
        if (m & 1) mant = -mant;
    }
    __device__ static __forceinline__ void phase(int m, uint64_t turn, double& cs, double& sn) {
        const uint64_t t = (uint64_t)m * turn;
        sincospi((double)(int64_t)t * 0x1p-63, &sn, &cs);
    }
    __device__ static __forceinline__ double down(double v) { return v * 0x1p-600; }
    __device__ static __forceinline__ double thresh() { return 0x1p-200; }
    __device__ static __forceinline__ void load16(const double2* g, double2 (&v)[16]) {
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = __ldg(g + c);
    }
    __device__ static __forceinline__ void load16a(const double* a, double (&v)[16]) {
        const double2* a2 = reinterpret_cast<const double2*>(a);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const double2 t = __ldg(a2 + c);
            v[2 * c] = t.x;
            v[2 * c + 1] = t.y;
        }
    }
};

}  // namespace adj

__device__ __forceinline__ uint64_t adj_turn(double ph) {
    double t = ph * (1.0 / (2.0 * CUDART_PI));
    t -= floor(t);
    if (!(t >= 0.0 && t < 1.0)) t = 0.0;
    return __double2ull_rn(t * 18446744073709551616.0);
}

template <typename Tr, typename TIn, int K>
__global__ void __launch_bounds__(128) adjoint_kernel(const __grid_constant__ AdjointParams p) {
    using real = typename Tr::real;
    using real2 = typename Tr::real2;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= p.warp0[p.ncat]) return;
    int c = 0;
    while (c + 1 < p.ncat && p.warp0[c + 1] <= gw) ++c;
    const CatDesc cd = p.cat[c];
    const int64_t base = (gw - p.warp0[c]) * (32 * K);
    const int L = p.lmax;
    const TIn* xs = static_cast<const TIn*>(cd.x);
    const TIn* ps = static_cast<const TIn*>(cd.phi);

    real x[K];
    double ls[K];
    uint64_t turn[K];
    double tot[K];
    bool valid[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t i = base + k * 32 + lane;
        valid[k] = i < cd.n;
        double xd = valid[k] ? (double)xs[i] : 0.0;
        double ph = valid[k] ? (double)ps[i] : 0.0;
        if (!(isfinite(xd) && isfinite(ph) && fabs(xd) <= 1.0)) {
            if (valid[k]) atomicOr(p.err, ERR_RANGE);
            xd = 0.0;
            ph = 0.0;
            valid[k] = false;
        }
        x[k] = (real)xd;
        const double xr = (double)x[k];
        const double s2 = (1.0 - xr) * (1.0 + xr);
        ls[k] = s2 > 0.0 ? 0.5 * log2(s2) : -1.0e30;
        turn[k] = adj_turn(ph);
        tot[k] = 0.0;
    }
    const real2* gtab = static_cast<const real2*>(p.gtab) + (int64_t)cd.field * p.gstride;
    const real* alpha_all = static_cast<const real*>(p.alpha);

    for (int m = 0; m <= L; ++m) {
        real lch, lcl;
        if constexpr (sizeof(real) == 4) {
            lch = p.log2c_hi[m];
            lcl = p.log2c_lo[m];
        } else {
            lch = p.log2c[m];
            lcl = 0;
        }
        real p1[K], p2[K], ar[K], ai[K], cs[K], sn[K];
        int E[K];
        bool lane_neg = false, lane_dead = true;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            real mant;
            Tr::seed(m, ls[k], lch, lcl, mant, E[k]);
            Tr::phase(m, turn[k], cs[k], sn[k]);
            p1[k] = real(0);   // sigma_{m-1}
            p2[k] = mant;      // sigma_{m-2}: with alpha_m = 0 the first step gives sigma_m = mant
            ar[k] = real(0);
            ai[k] = real(0);
            lane_neg |= E[k] < 0;
            lane_dead &= E[k] < 0;
        }
        bool any_neg = __any_sync(0xffffffffu, lane_neg);
        bool all_dead = __all_sync(0xffffffffu, lane_dead);
        const int64_t cs0 = p.colstart[m];
        const real* alpha = alpha_all + cs0;
        const real2* gcol = gtab + cs0;
        const int len = L - m + 1;
        const int nblk = (len + 15) >> 4;
        for (int bk = 0; bk < nblk; ++bk) {
            real av[16];
            real2 gv[16];
            Tr::load16a(alpha + 16 * bk, av);
            Tr::load16(gcol + 16 * bk, gv);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (all_dead) {
#pragma unroll
                    for (int j = 8 * h; j < 8 * h + 8; ++j)
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            const real mu = fma(av[j], x[k] * p1[k], p2[k]);
                            p2[k] = p1[k];
                            p1[k] = mu;
                        }
                } else {
#pragma unroll
                    for (int j = 8 * h; j < 8 * h + 8; ++j)
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            const real mu = fma(av[j], x[k] * p1[k], p2[k]);
                            p2[k] = p1[k];
                            p1[k] = mu;
                            ar[k] = fma(mu, gv[j].x, ar[k]);
                            ai[k] = fma(mu, gv[j].y, ai[k]);
                        }
                }
                if (any_neg) {
                    lane_neg = false;
                    lane_dead = true;
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        if (E[k] < 0) {
                            const real mx = fmax(fabs(p1[k]), fabs(p2[k]));
                            if (mx > Tr::thresh()) {
                                p1[k] = Tr::down(p1[k]);
                                p2[k] = Tr::down(p2[k]);
                                E[k] += 1;
                                if (E[k] == 0) {  // drop what was summed below range
                                    ar[k] = real(0);
                                    ai[k] = real(0);
                                }
                            }
                        }
                        lane_neg |= E[k] < 0;
                        lane_dead &= E[k] < 0;
                    }
                    any_neg = __any_sync(0xffffffffu, lane_neg);
                    all_dead = __all_sync(0xffffffffu, lane_dead);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (E[k] == 0) tot[k] += (double)cs[k] * (double)ar[k] - (double)sn[k] * (double)ai[k];
    }
    const double gn = p.gnoise ? p.gnoise[(int64_t)cd.field * (p.nfield + 1)] : 0.0;
    const TIn* ws = static_cast<const TIn*>(cd.w);
    TIn* out = static_cast<TIn*>(p.gradw[c]);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t i = base + k * 32 + lane;
        if (i < cd.n) {
            const double w = valid[k] ? (double)ws[i] : 0.0;
            const double g = cd.coeff * tot[k] + 2.0 * cd.coeff * cd.coeff * w * gn / (4.0 * CUDART_PI);
            out[i] = (TIn)g;
        }
    }
}

__device__ __forceinline__ float2 adj_fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)),
          "l"(reinterpret_cast<unsigned long long&>(c)));
    return d;
}
__device__ __forceinline__ float2 adj_add2(float2 a, float2 b) {
    float2 d;
    asm("add.rn.f32x2 %0, %1, %2;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)));
    return d;
}
__device__ __forceinline__ float2 adj_mul2(float2 a, float2 b) {
    float2 d;
    asm("mul.rn.f32x2 %0, %1, %2;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)));
    return d;
}

// FP32 adjoint over the points as prepared (and |x|-sorted) for the analysis:
// a warp takes 32 K consecutive prepared points of one field, K = 8 per lane
// as four f32x2 pairs, so that the points of a warp cross into the FP32
// range together and a warp all of whose points are below it runs the
// recurrence only.  Per step and pair: x sigma (mul2), the recurrence (fma2)
// and the two accumulations (fma2 with (gamma g re, same) and (im, im)).
// The four warps of a CTA (1024 points; fields are padded to whole CTAs, so a
// CTA lies in one field) walk the orders and steps together: the table
// entries, recurrence coefficients and near-pole coefficients of 64 steps at a
// time are copied into shared memory (cp.async, zero-filled past the column)
// while the previous 64 steps run, one barrier per 64 steps.
// The gradient goes back to each point's catalog and index through the
// prepared point id.
constexpr int ADJ_KP = 4;                 // f32x2 pairs per lane
constexpr int ADJ_PW = 32 * 2 * ADJ_KP;   // points per warp (256)
constexpr int ADJ_WARPS = 4;              // warps per CTA
constexpr int ADJ_CH = 64;                // steps per staged chunk

__device__ __forceinline__ void adj_cp_async(void* dst, const void* src, int bytes, bool in) {
    // bytes 8 or 16; src-size 0 fills the destination with zeros and reads nothing
    const uint32_t d = smem_u32(dst);
    if (bytes == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(in ? 16 : 0) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(in ? 8 : 0) : "memory");
}

__global__ void __launch_bounds__(ADJ_WARPS * 32) adjoint_sorted_kernel(const __grid_constant__ AdjointParams p) {
    constexpr int KP = ADJ_KP, K = 2 * ADJ_KP;
    __shared__ __align__(16) float4 s_g[2][ADJ_CH];   // (gamma g re, same, gamma g im, same)
    __shared__ __align__(16) float4 s_pe[2][ADJ_CH];  // near-pole coefficients (a, a, e, e)
    __shared__ __align__(16) float2 s_a[2][ADJ_CH];   // (alpha, alpha)
    const int lane = threadIdx.x & 31;
    const int64_t cta0 = (int64_t)blockIdx.x * ADJ_WARPS * ADJ_PW;
    const int64_t start = cta0 + (int64_t)(threadIdx.x >> 5) * ADJ_PW;
    // the launch covers whole CTAs of prepared points: every warp has its 256
    int f = 0;
    while (f + 1 < p.nfield && p.fld[f + 1].off <= cta0) ++f;
    const float* tf = reinterpret_cast<const float*>(p.pts);
    const uint32_t* tu = p.pts;
    const int64_t N = p.ntot;
    const int L = p.lmax;

    float2 x2[KP];
    float lh[K], ll[K];
    uint32_t thi[K], tlo[K];
    double tot[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t i = start + 32 * k + lane;
        const float xv = tf[i];
        if (k & 1) x2[k >> 1].y = xv;
        else x2[k >> 1].x = xv;
        lh[k] = tf[2 * N + i];
        ll[k] = tf[3 * N + i];
        thi[k] = tu[4 * N + i];
        tlo[k] = tu[5 * N + i];
        tot[k] = 0.0;
    }
    const float4* gtab = static_cast<const float4*>(p.gtab) + (int64_t)f * p.gstride;
    // Near a pole (every point of the warp at x >= pole_x, or every point at
    // x <= -pole_x) and for m < pole_mmax the recurrence runs in the
    // analysis's near-pole form (column_f32x2_pole): Reinsch's difference form
    // of the unfolded recurrence on |x|, with p1 = y_{q-1}, p2 = d_{q-1}, and
    // the factor s_q sgn^q (q odd ? rho_m : 1) of sigma_q applied to the
    // table entry of step j.
    // (padding points do not count: their gradient is not written)
    bool np = true, sp = true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float xv = (k & 1) ? x2[k >> 1].y : x2[k >> 1].x;
        const bool idle = tu[6 * N + start + 32 * k + lane] == 0xffffffffu;
        np &= idle | (xv >= p.pole_x);
        sp &= idle | (xv <= -p.pole_x);
    }
    const float sgn = __all_sync(0xffffffffu, np) ? 1.f : (__all_sync(0xffffffffu, sp) ? -1.f : 0.f);
    const bool pole = sgn != 0.f;
    float2 u2[KP];
#pragma unroll
    for (int kp = 0; kp < KP; ++kp) u2[kp] = make_float2(fabsf(x2[kp].x) - 1.f, fabsf(x2[kp].y) - 1.f);

    // copy of the 64 steps [64 ch, 64 ch + 64) of order m into buffer b: thread
    // t < 64 the table entry t, thread 64 + t the coefficients of entry t
    auto stage = [&](int m, int ch, int b) {
        const int64_t c0 = p.colstart[m];
        const int colpad = (int)(p.colstart[m + 1] - c0);
        const int t = threadIdx.x & (ADJ_CH - 1);
        const int q = ch * ADJ_CH + t;
        const bool in = q < colpad;
        const int64_t e = c0 + (in ? q : 0);
        if (threadIdx.x < ADJ_CH) {
            adj_cp_async(&s_g[b][t], gtab + e, 16, in);
        } else {
            adj_cp_async(&s_a[b][t], p.alpha2 + e, 8, in);
            if (m < p.pole_mmax) adj_cp_async(&s_pe[b][t], p.pole_ae + e, 16, in);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    int buf = 0;
    stage(0, 0, 0);

    for (int m = 0; m <= L; ++m) {
        const float lch = p.log2c_hi[m], lcl = p.log2c_lo[m];
        const bool pole_m = pole && m < p.pole_mmax;
        const float sr = pole_m ? sgn * p.pole_rho[m] : 0.f;
        const float sj[4] = {1.f, sr, -1.f, -sr};  // s_q sgn^q (q odd ? rho : 1), q = j (mod 4)
        float2 p1[KP], p2[KP], ar[KP], ai[KP];
        float cs[K], sn[K];
        int E[K];
        bool lane_neg = false, lane_dead = true;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float mant;
            seed_f32(m, lh[k], ll[k], lch, lcl, mant, E[k]);
            phase_f32(m, thi[k], tlo[k], cs[k], sn[k]);
            if (k & 1) {
                p2[k >> 1].y = mant;  // with alpha_m = 0 the first step gives sigma_m = mant
                p1[k >> 1].y = 0.f;
            } else {
                p2[k >> 1].x = mant;
                p1[k >> 1].x = 0.f;
            }
            lane_neg |= E[k] < 0;
            lane_dead &= E[k] < 0;
        }
#pragma unroll
        for (int kp = 0; kp < KP; ++kp) ar[kp] = ai[kp] = make_float2(0.f, 0.f);
        bool any_neg = __any_sync(0xffffffffu, lane_neg);
        bool all_dead = __all_sync(0xffffffffu, lane_dead);
        const int nblk = (L - m + 1 + 7) >> 3;
        const int nch = (nblk + 7) >> 3;
        for (int ch = 0; ch < nch; ++ch) {
            // this thread's copies of chunk (m, ch) are complete; after the barrier
            // everyone's are, and nobody reads the other buffer any more
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            if (ch + 1 < nch) stage(m, ch + 1, buf ^ 1);
            else if (m < L) stage(m + 1, 0, buf ^ 1);
            const float4* gcs = s_g[buf];
            const float2* als = s_a[buf];
            const float4* pas = s_pe[buf];
            const int bend = min(8, nblk - 8 * ch);
            for (int b = 0; b < bend; ++b) {
                if (pole_m) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float4 cv[4], gq[4];
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            cv[jj] = pas[8 * b + 4 * h + jj];
                            gq[jj] = gcs[8 * b + 4 * h + jj];
                        }
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const float2 a2 = make_float2(cv[jj].x, cv[jj].y), e2 = make_float2(cv[jj].z, cv[jj].w);
                            const float s = sj[jj];  // q = 8 bk + 4 h + jj = jj (mod 4)
                            const float2 gr = make_float2(s * gq[jj].x, s * gq[jj].y);
                            const float2 gi = make_float2(s * gq[jj].z, s * gq[jj].w);
#pragma unroll
                            for (int kp = 0; kp < KP; ++kp) {
                                const float2 c = adj_fma2(a2, u2[kp], e2);
                                p2[kp] = adj_fma2(c, p1[kp], p2[kp]);
                                p1[kp] = adj_add2(p1[kp], p2[kp]);
                                if (!all_dead) {
                                    ar[kp] = adj_fma2(p1[kp], gr, ar[kp]);
                                    ai[kp] = adj_fma2(p1[kp], gi, ai[kp]);
                                }
                            }
                        }
                    }
                } else {
                    float4 gv[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) gv[j] = gcs[8 * b + j];
                    float2 av[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) av[j] = als[8 * b + j];
                    if (all_dead) {
#pragma unroll
                        for (int j = 0; j < 8; ++j)
#pragma unroll
                            for (int kp = 0; kp < KP; ++kp) {
                                const float2 mu = adj_fma2(av[j], adj_mul2(x2[kp], p1[kp]), p2[kp]);
                                p2[kp] = p1[kp];
                                p1[kp] = mu;
                            }
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j)
#pragma unroll
                            for (int kp = 0; kp < KP; ++kp) {
                                const float2 mu = adj_fma2(av[j], adj_mul2(x2[kp], p1[kp]), p2[kp]);
                                p2[kp] = p1[kp];
                                p1[kp] = mu;
                                ar[kp] = adj_fma2(mu, make_float2(gv[j].x, gv[j].y), ar[kp]);
                                ai[kp] = adj_fma2(mu, make_float2(gv[j].z, gv[j].w), ai[kp]);
                            }
                    }
                }
                if (any_neg) {
                    // rescale check every 8 steps (F32Scale; 8-step growth <= 2^42)
                    lane_neg = false;
                    lane_dead = true;
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        float& a = (k & 1) ? p1[k >> 1].y : p1[k >> 1].x;
                        float& bb = (k & 1) ? p2[k >> 1].y : p2[k >> 1].x;
                        if (E[k] < 0 && fmaxf(fabsf(a), fabsf(bb)) > 0x1p-61f) {
                            a *= 0x1p-64f;
                            bb *= 0x1p-64f;
                            E[k] += 1;
                            if (E[k] == 0) {  // drop what was summed below range
                                if (k & 1) {
                                    ar[k >> 1].y = 0.f;
                                    ai[k >> 1].y = 0.f;
                                } else {
                                    ar[k >> 1].x = 0.f;
                                    ai[k >> 1].x = 0.f;
                                }
                            }
                        }
                        lane_neg |= E[k] < 0;
                        lane_dead &= E[k] < 0;
                    }
                    any_neg = __any_sync(0xffffffffu, lane_neg);
                    all_dead = __all_sync(0xffffffffu, lane_dead);
                }
            }
            buf ^= 1;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float r = (k & 1) ? ar[k >> 1].y : ar[k >> 1].x;
            const float im = (k & 1) ? ai[k >> 1].y : ai[k >> 1].x;
            if (E[k] == 0) tot[k] += (double)cs[k] * (double)r - (double)sn[k] * (double)im;
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    const double gn = p.gnoise ? p.gnoise[(int64_t)f * (p.nfield + 1)] : 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t i = start + 32 * k + lane;
        const uint32_t id = tu[6 * N + i];
        if (id == 0xffffffffu) continue;  // padding
        int c = 0;
        while (c + 1 < p.ncat && (uint64_t)p.cat[c + 1].id0 <= (uint64_t)id) ++c;
        const int64_t idx = (int64_t)id - p.cat[c].id0;
        const double cw = (double)tf[N + i];  // coeff * w (0 for a point flagged out of range)
        const double coeff = p.cat[c].coeff;
        const double g = coeff * tot[k] + 2.0 * coeff * cw * gn / (4.0 * CUDART_PI);
        static_cast<float*>(p.gradw[c])[idx] = (float)g;
    }
}

// gtab entries for the sorted FP32 adjoint: (gamma g re, same, gamma g im, same)
__global__ void build_gtab4_kernel(int L, const double2* __restrict__ galm, const double* __restrict__ gamma,
                                   const int64_t* __restrict__ colstart, int64_t gstride, int synth,
                                   float4* __restrict__ gtab) {
    const int m = blockIdx.y, f = blockIdx.z;
    const double cm = (synth && m > 0) ? 2.0 : 1.0;
    const int64_t w = colstart[m + 1] - colstart[m];
    const int64_t M = (int64_t)(L + 1) * (L + 2) / 2;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < w; q += (int64_t)gridDim.x * blockDim.x) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m + q <= L) {
            const int64_t idx = tri_base(m, L) + m + q;
            const double2 g = galm[(int64_t)f * M + idx];
            const double gm = cm * gamma[idx];
            v = make_float4((float)(g.x * gm), (float)(g.x * gm), (float)(g.y * gm), (float)(g.y * gm));
        }
        gtab[(int64_t)f * gstride + colstart[m] + q] = v;
    }
}

// prepared FP32 points of a field are padded to a multiple of this (one CTA)
int adjoint_sorted_points_per_cta() { return ADJ_WARPS * ADJ_PW; }

cudaError_t launch_adjoint_sorted(const AdjointParams& ap, const double* galm, const double* gamma, int synth,
                                  cudaStream_t st) {
    dim3 grid(4, ap.lmax + 1, ap.nfield);
    build_gtab4_kernel<<<grid, 256, 0, st>>>(ap.lmax, reinterpret_cast<const double2*>(galm), gamma, ap.colstart,
                                             ap.gstride, synth, (float4*)ap.gtab);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // ntot is a multiple of the CTA's 1024 points (every field is padded to it)
    if (ap.ntot % (ADJ_WARPS * ADJ_PW)) return cudaErrorInvalidValue;
    const int64_t ncta = ap.ntot / (ADJ_WARPS * ADJ_PW);
    if (ncta == 0) return cudaSuccess;
    adjoint_sorted_kernel<<<(unsigned)ncta, ADJ_WARPS * 32, 0, st>>>(ap);
    return cudaGetLastError();
}

// gtab[f][colstart[m] + q] = c_m gamma(l, m) * g^f(l, m), zero in the padding;
// c_m = 1, or for point-evaluation synthesis (the real field
// sum_{l, |m| <= l} a_lm Y_lm = sum_l [a_l0 Y_l0 + 2 sum_{m>0} Re(a_lm Y_lm)])
// c_m = 2 for m > 0.
template <typename R2>
__global__ void build_gtab_kernel(int L, const double2* __restrict__ galm, const double* __restrict__ gamma,
                                  const int64_t* __restrict__ colstart, int64_t gstride, int synth,
                                  R2* __restrict__ gtab) {
    const int m = blockIdx.y, f = blockIdx.z;
    const double cm = (synth && m > 0) ? 2.0 : 1.0;
    const int64_t w = colstart[m + 1] - colstart[m];
    const int64_t M = (int64_t)(L + 1) * (L + 2) / 2;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < w; q += (int64_t)gridDim.x * blockDim.x) {
        R2 v;
        v.x = 0;
        v.y = 0;
        if (m + q <= L) {
            const int64_t idx = tri_base(m, L) + m + q;
            const double2 g = galm[(int64_t)f * M + idx];
            const double gm = cm * gamma[idx];
            v.x = g.x * gm;
            v.y = g.y * gm;
        }
        gtab[(int64_t)f * gstride + colstart[m] + q] = v;
    }
}

cudaError_t launch_build_gtab(int is_f64, int L, int nfield, const double* galm, const double* gamma,
                              const int64_t* colstart, int64_t gstride, int synth, void* gtab, cudaStream_t st) {
    dim3 grid(4, L + 1, nfield);
    if (!is_f64) return cudaErrorInvalidValue;  // FP32 uses build_gtab4_kernel (sorted adjoint)
    build_gtab_kernel<double2><<<grid, 256, 0, st>>>(L, reinterpret_cast<const double2*>(galm), gamma, colstart,
                                                     gstride, synth, static_cast<double2*>(gtab));
    return cudaGetLastError();
}

int adjoint_points_per_warp(int is_f64) { return is_f64 ? 32 * 2 : 0; }

cudaError_t launch_adjoint(int is_f64, const AdjointParams& ap, cudaStream_t st) {
    const int64_t nwarps = ap.warp0[ap.ncat];
    if (nwarps == 0) return cudaSuccess;
    const int64_t nblocks = (nwarps + 3) / 4;
    if (!is_f64) return cudaErrorInvalidValue;  // FP32 runs adjoint_sorted_kernel
    adjoint_kernel<adj::F64, double, 2><<<(unsigned)nblocks, 128, 0, st>>>(ap);
    return cudaGetLastError();
}

}  // namespace psht

namespace psht {
// Unit weights for point-evaluation synthesis (the catalog form needs a
// weight array; synthesis has none).
__global__ void fill_ones_kernel(int64_t n, int is_f64, void* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (is_f64) static_cast<double*>(out)[i] = 1.0;
        else static_cast<float*>(out)[i] = 1.0f;
    }
}

cudaError_t launch_fill_ones(int64_t n, int is_f64, void* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    fill_ones_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, is_f64, out);
    return cudaGetLastError();
}
}  // namespace psht
