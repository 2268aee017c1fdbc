// analysis.cu -- the direct point-catalog SHT on GB300 (sm_103a).
//
//   a_lm = sum_i w_i Y*_lm(theta_i, phi_i)                        (Eq. alm_def)
//   Y_lm = lambda_lm(x) e^{i m phi},  lambda_lm = sqrt((2l+1)/4pi) Pbar_l^m (App. A)
//
// Per (point, m) the sectoral seed lambda_mm and the phase e^{-i m phi} are
// formed directly (no carry over m):
//   log2 |lambda_mm| = log2 c_m + m log2 sin(theta),
//   c_m^2 = (2m+1)/(4pi) prod_{k<=m} (1 - 1/(2k)),  sign (-1)^m,
// which is the App. A sectoral recurrence summed in log space.  Then the
// three-term recurrence in l (App. A, rewritten for lambda:
// lambda_l = A_l x lambda_{l-1} - B_l lambda_{l-2}) runs in the rescaled,
// sign-folded variable sigma_l = s_q lambda_l / gamma_l (q = l - m,
// s_q = (-1)^floor(q/2), gamma_l = B_l gamma_{l-2}):
//   sigma_l = alpha~_l x sigma_{l-1} + sigma_{l-2},
//   alpha~_l = (s_q / s_{q-1}) A_l gamma_{l-1} / gamma_l,
// i.e. one multiply and one FMA per step with no negation.  The per-(l, m)
// factor gamma' = s_q gamma_l is applied once, in FP64, when chunks are
// reduced.  The FP32 kernel runs two points per instruction (f32x2).
//
// Thread mapping of the analysis kernel: a CTA owns one tile of points in
// shared memory (filled by bulk TMA copies, double-buffered on mbarriers) and
// W warps; warp w runs the order pair (m, lmax - m) so that every warp does
// lmax + 2 recurrence steps per point.  A lane carries K points; the products
// for 16 consecutive l are reduced over the warp by a shared-memory transpose
// and added to a per-warp FP32 accumulator row in shared memory, which is
// flushed every few tiles into the unit's FP64 slot in global memory.
#include "common.cuh"

#include <math_constants.h>

#include <map>
#include <mutex>
#include <utility>

namespace psht {

// ====================================================================
//                           point preparation
// ====================================================================
// FP32 layout (7 arrays of 4 bytes, stride ntot):
//   0 x, 1 coeff*w, 2 log2 sin(theta) hi, 3 lo, 4 turn[63:32], 5 turn[31:0],
//   6 point id (catalog id0 + index; 0xffffffff for padding; read by the adjoint)
// FP64 layout (4 arrays of 8 bytes): 0 x, 1 coeff*w, 2 log2 sin(theta), 3 turn

template <typename T>
__device__ __forceinline__ void prep_one(const PrepParams& p, int64_t j, T x, T ph, T w, double coeff,
                                         uint32_t id = 0xffffffffu) {
    bool ok = isfinite((double)x) && isfinite((double)ph) && isfinite((double)w) && fabs((double)x) <= 1.0;
    if (!ok) {
        atomicOr(p.err, ERR_RANGE);
        x = T(0);
        ph = T(0);
        w = T(0);
    }
    const double xd = (double)x;
    const double s2 = (1.0 - xd) * (1.0 + xd);
    const double ls = s2 > 0.0 ? 0.5 * log2(s2) : -1.0e30;
    const uint64_t turn = phi_to_turn((double)ph);
    const double ww = coeff * (double)w;
    if constexpr (sizeof(T) == 4) {
        float* b = static_cast<float*>(p.pts);
        uint32_t* bu = static_cast<uint32_t*>(p.pts);
        const float lh = (float)ls;
        b[j] = (float)xd;
        b[p.ntot + j] = (float)ww;
        b[2 * p.ntot + j] = lh;
        b[3 * p.ntot + j] = (float)(ls - (double)lh);
        bu[4 * p.ntot + j] = (uint32_t)(turn >> 32);
        bu[5 * p.ntot + j] = (uint32_t)(turn & 0xffffffffu);
        bu[6 * p.ntot + j] = id;
    } else {
        double* b = static_cast<double*>(p.pts);
        uint64_t* bu = static_cast<uint64_t*>(p.pts);
        b[j] = xd;
        b[p.ntot + j] = ww;
        b[2 * p.ntot + j] = ls;
        bu[3 * p.ntot + j] = turn;
    }
}

template <typename T>
__global__ void prep_kernel(const __grid_constant__ PrepParams p) {
    const int seg = blockIdx.y;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (seg < p.ncat) {
        const CatDesc& c = p.cat[seg];
        const T* xs = static_cast<const T*>(c.x);
        const T* ps = static_cast<const T*>(c.phi);
        const T* ws = static_cast<const T*>(c.w);
        for (int64_t i = i0; i < c.n; i += stride)
            prep_one<T>(p, c.dst + i, xs[i], ps[i], ws[i], c.coeff, (uint32_t)(c.id0 + i));
    } else {
        const int f = seg - p.ncat;
        for (int64_t i = i0; i < p.pad_n[f]; i += stride) prep_one<T>(p, p.pad_off[f] + i, T(0), T(0), T(0), 0.0);
    }
}

// ====================================================================
//           ordering points by |x| (deterministic counting sort)
// ====================================================================
// Whether a point's recurrence state is still below the floating-point range
// at (l, m) depends on sin(theta), i.e. on |x|.  Points of a field are
// therefore laid out by |x| bucket (256 buckets), stable within a bucket, so
// that the 32*K points of one warp cross into range at nearly the same l:
// rescaling becomes warp-coherent and warps whose points are all below range
// skip the accumulation.  The order changes only the summation order.
//
//   hist:    per CTA range (SORT_RANGE points of one catalog) bucket counts
//   scan:    per field, bucket-major exclusive offsets over (bucket, CTA range)
//   scatter: each range, in index order, writes its prepared points to
//            offset(bucket, range) + rank, ranks taken warp by warp in order.

template <typename T>
__device__ __forceinline__ bool range_of(const SortParams& sp, int r, int& c, int64_t& i0, int64_t& i1) {
    c = 0;
    while (c + 1 < sp.prep.ncat && sp.range0[c + 1] <= r) ++c;
    const int64_t j = r - sp.range0[c];
    i0 = j * SORT_RANGE;
    i1 = min(sp.prep.cat[c].n, i0 + SORT_RANGE);
    return i0 < i1;
}

template <typename T>
__global__ void __launch_bounds__(256) sort_hist_kernel(const __grid_constant__ SortParams sp) {
    __shared__ int cnt[SORT_BUCKETS];
    const int r = blockIdx.x;
    for (int b = threadIdx.x; b < SORT_BUCKETS; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    int c;
    int64_t i0, i1;
    if (range_of<T>(sp, r, c, i0, i1)) {
        const T* xs = static_cast<const T*>(sp.prep.cat[c].x);
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) atomicAdd(&cnt[x_bucket((double)xs[i])], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < SORT_BUCKETS; b += blockDim.x) sp.hist[(int64_t)r * SORT_BUCKETS + b] = cnt[b];
}

// one CTA per field; thread b owns bucket b
__global__ void __launch_bounds__(SORT_BUCKETS) sort_scan_kernel(const __grid_constant__ SortParams sp) {
    const int f = blockIdx.x;
    const int b = threadIdx.x;
    __shared__ int64_t tot[SORT_BUCKETS];
    int64_t t = 0;
    for (int c = 0; c < sp.prep.ncat; ++c) {
        if (sp.prep.cat[c].field != f) continue;
        for (int64_t r = sp.range0[c]; r < sp.range0[c + 1]; ++r) t += sp.hist[r * SORT_BUCKETS + b];
    }
    tot[b] = t;
    __syncthreads();
    int64_t base = sp.field_off[f];
    for (int k = 0; k < b; ++k) base += tot[k];
    for (int c = 0; c < sp.prep.ncat; ++c) {
        if (sp.prep.cat[c].field != f) continue;
        for (int64_t r = sp.range0[c]; r < sp.range0[c + 1]; ++r) {
            const int64_t h = sp.hist[r * SORT_BUCKETS + b];
            sp.hist[r * SORT_BUCKETS + b] = base;  // becomes the range's first slot in bucket b
            base += h;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) sort_scatter_kernel(const __grid_constant__ SortParams sp) {
    __shared__ int64_t next[SORT_BUCKETS];
    __shared__ int wcnt[8][SORT_BUCKETS];
    const int r = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = threadIdx.x; b < SORT_BUCKETS; b += blockDim.x) next[b] = sp.hist[(int64_t)r * SORT_BUCKETS + b];
    int c;
    int64_t i0, i1;
    const bool any = range_of<T>(sp, r, c, i0, i1);
    __syncthreads();
    if (!any) return;
    const CatDesc& cd = sp.prep.cat[c];
    const T* xs = static_cast<const T*>(cd.x);
    const T* ps = static_cast<const T*>(cd.phi);
    const T* ws = static_cast<const T*>(cd.w);
    for (int64_t base = i0; base < i1; base += 256) {
        for (int b = lane; b < SORT_BUCKETS; b += 32) wcnt[warp][b] = 0;
        __syncwarp();
        const int64_t i = base + threadIdx.x;
        const bool valid = i < i1;
        T x = valid ? xs[i] : T(0);
        const int bk = valid ? x_bucket((double)x) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, bk);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[warp][bk] = __popc(peers);
        __syncthreads();
        if (valid) {
            int64_t dst = next[bk] + rank;
            for (int w = 0; w < warp; ++w) dst += wcnt[w][bk];
            prep_one<T>(sp.prep, dst, x, ps[i], ws[i], cd.coeff, (uint32_t)(cd.id0 + i));
        }
        __syncthreads();
        for (int b = threadIdx.x; b < SORT_BUCKETS; b += blockDim.x) {
            int s = 0;
            for (int w = 0; w < 8; ++w) s += wcnt[w][b];
            next[b] += s;
        }
        __syncthreads();
    }
}

// ====================================================================
//                      precision-specific pieces
// ====================================================================
struct TraitsF32 {
    using real = float;
    using real2 = float2;
    static constexpr int NARR = 6;   // arrays per prepared point
    static constexpr int ABYTES = 4; // bytes per array element
    static constexpr int SB = F32Scale::SCALE_BITS;
    static constexpr int CE = F32Scale::CHECK_EXP;

    // Seed mantissa (with sign) and exponent block E <= 0 such that
    // lambda_mm = mant * 2^(SB*E); Y phase e^{-i m phi} = (cs, -sn).
    __device__ static __forceinline__ void setup(const uint32_t* tile, int P, int i, int m, float lch, float lcl,
                                                 float& x, float& mant, int& E, float& cs, float& sn, float& w) {
        const float* tf = reinterpret_cast<const float*>(tile);
        x = tf[i];
        w = tf[P + i];
        seed_f32(m, tf[2 * P + i], tf[3 * P + i], lch, lcl, mant, E);
        phase(tile, P, i, m, cs, sn);
    }
    __device__ static __forceinline__ void phase(const uint32_t* tile, int P, int i, int m, float& cs, float& sn) {
        phase_f32(m, tile[4 * P + i], tile[5 * P + i], cs, sn);
    }
    __device__ static __forceinline__ float weight(const uint32_t* tile, int P, int i) {
        return reinterpret_cast<const float*>(tile)[P + i];
    }
    __device__ static __forceinline__ float down(float v) { return v * 0x1p-64f; }
    __device__ static __forceinline__ float thresh() { return 0x1p-61f; }
    // transpose-buffer row stride (float2 units): even, so rows are 16-byte
    // aligned for 128-bit loads, and 34 keeps both the 64-bit stores and the
    // 128-bit loads free of bank conflicts
    static constexpr int XSTRIDE = 34;
    __device__ static __forceinline__ void row_sum16(const float2* r, float& sr, float& si) {
        const float4* r4 = reinterpret_cast<const float4*>(r);
        float a = 0.f, b = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float4 v = r4[c];
            a += v.x + v.z;
            b += v.y + v.w;
        }
        sr = a;
        si = b;
    }
};

struct TraitsF64 {
    using real = double;
    using real2 = double2;
    static constexpr int NARR = 4;
    static constexpr int ABYTES = 8;
    static constexpr int SB = F64Scale::SCALE_BITS;
    static constexpr int CE = F64Scale::CHECK_EXP;

    __device__ static __forceinline__ void setup(const uint32_t* tile32, int P, int i, int m, double lc, double,
                                                 double& x, double& mant, int& E, double& cs, double& sn,
                                                 double& w) {
        const double* t = reinterpret_cast<const double*>(tile32);
        x = t[i];
        w = t[P + i];
        const double e = fma((double)m, t[2 * P + i], lc);
        const bool pole = e < -1.0e7;  // sin theta = 0 and m > 0: lambda_mm = 0
        const double Ef = pole ? -1048576.0 : fmin(0.0, ceil((e - (double)CE) * (1.0 / SB)));
        E = (int)Ef;
        const double eh = pole ? 0.0 : e - (double)SB * Ef;
        const double n = floor(eh);
        mant = pole ? 0.0 : ldexp(exp2(eh - n), (int)n);
        if (m & 1) mant = -mant;
        phase(tile32, P, i, m, cs, sn);
    }
    __device__ static __forceinline__ void phase(const uint32_t* tile32, int P, int i, int m, double& cs,
                                                 double& sn) {
        const uint64_t* tu = reinterpret_cast<const uint64_t*>(tile32);
        const uint64_t t = (uint64_t)m * tu[3 * P + i];
        const double y = (double)(int64_t)t * 0x1p-63;
        sincospi(y, &sn, &cs);
    }
    __device__ static __forceinline__ double weight(const uint32_t* tile32, int P, int i) {
        return reinterpret_cast<const double*>(tile32)[P + i];
    }
    __device__ static __forceinline__ double down(double v) { return v * 0x1p-600; }
    __device__ static __forceinline__ double thresh() { return 0x1p-200; }
    static constexpr int XSTRIDE = 33;  // odd: conflict-free for 16-byte elements
    __device__ static __forceinline__ void row_sum16(const double2* r, double& sr, double& si) {
        double a = 0.0, b = 0.0;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const double2 v = r[c];
            a += v.x;
            b += v.y;
        }
        sr = a;
        si = b;
    }
};

template <typename Tr>
__device__ __forceinline__ const typename Tr::real* alpha_base(const AnalysisParams& p, int m);
template <>
__device__ __forceinline__ const float* alpha_base<TraitsF32>(const AnalysisParams& p, int m) {
    return p.alpha_f + p.colstart[m];
}
template <>
__device__ __forceinline__ const double* alpha_base<TraitsF64>(const AnalysisParams& p, int m) {
    return p.alpha_d + p.colstart[m];
}

// Load 16 consecutive coefficients (16-byte aligned) into registers.
__device__ __forceinline__ void load16(const float* a, float (&v)[16]) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float4 t = __ldg(a4 + c);
        v[4 * c] = t.x;
        v[4 * c + 1] = t.y;
        v[4 * c + 2] = t.z;
        v[4 * c + 3] = t.w;
    }
}
__device__ __forceinline__ void load16(const double* a, double (&v)[16]) {
    const double2* a2 = reinterpret_cast<const double2*>(a);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        double2 t = __ldg(a2 + c);
        v[2 * c] = t.x;
        v[2 * c + 1] = t.y;
    }
}

// ====================================================================
//                one order m over the K*32 points of a tile
// ====================================================================
// acc: this warp's accumulator row for the column (len = lmax-m+1 entries);
// xb: this warp's 16-row transpose buffer (row stride Tr::XSTRIDE).
// Rare path (a point's state reaches the floating-point range): recompute its
// weighted phase.  Kept out of line so the hot loop stays small.
template <typename Tr>
__device__ __noinline__ typename Tr::real2 restore_weight(const uint32_t* tile, int P, int i, int m) {
    typename Tr::real cs, sn;
    Tr::phase(tile, P, i, m, cs, sn);
    const typename Tr::real w = Tr::weight(tile, P, i);
    typename Tr::real2 r;
    r.x = w * cs;
    r.y = -w * sn;
    return r;
}

template <typename Tr, int K>
__device__ __forceinline__ void analysis_column(const uint32_t* tile, int P, int m, int L,
                                                const typename Tr::real* __restrict__ alpha,
                                                typename Tr::real lch, typename Tr::real lcl,
                                                typename Tr::real2* acc, typename Tr::real2* xb, int lane) {
    using real = typename Tr::real;
    using real2 = typename Tr::real2;
    constexpr int XS = Tr::XSTRIDE;
    const int len = L - m + 1;
    real x[K], p1[K], p2[K], wc[K], ws[K];
    int E[K];
    bool lane_neg = false, lane_dead = true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        real mant, cs, sn, w;
        Tr::setup(tile, P, k * 32 + lane, m, lch, lcl, x[k], mant, E[k], cs, sn, w);
        const bool live = E[k] == 0;
        wc[k] = live ? w * cs : real(0);
        ws[k] = live ? -w * sn : real(0);
        p1[k] = real(0);   // sigma_{m-1}
        p2[k] = mant;      // sigma_{m-2}: with alpha_m = 0 the first step gives sigma_m = mant
        lane_neg |= !live;
        lane_dead &= !live;
    }
    bool any_neg = __any_sync(0xffffffffu, lane_neg);
    bool all_dead = __all_sync(0xffffffffu, lane_dead);

    const int nblk = (len + 15) >> 4;
    real an[16];
    load16(alpha, an);
    for (int bk = 0; bk < nblk; ++bk) {
        real av[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) av[j] = an[j];
        if (bk + 1 < nblk) load16(alpha + 16 * (bk + 1), an);
        real re[16], im[16];
        if (all_dead) {  // every point of the warp is still below range: recurrence only
#pragma unroll
            for (int j = 0; j < 16; ++j) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const real mu = fma(av[j], x[k] * p1[k], p2[k]);
                    p2[k] = p1[k];
                    p1[k] = mu;
                }
                re[j] = real(0);
                im[j] = real(0);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                real r = real(0), ii = real(0);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const real mu = fma(av[j], x[k] * p1[k], p2[k]);
                    p2[k] = p1[k];
                    p1[k] = mu;
                    r = fma(mu, wc[k], r);
                    ii = fma(mu, ws[k], ii);
                }
                re[j] = r;
                im[j] = ii;
            }
        }
        if (any_neg) {
            // Rescale check once per 16 steps.  Fast path: one predicate per
            // point and one vote; the branchy rescale runs only if some lane
            // has a point to rescale.
            bool need = false;
#pragma unroll
            for (int k = 0; k < K; ++k) need |= (E[k] < 0) & (fmax(fabs(p1[k]), fabs(p2[k])) > Tr::thresh());
            if (__any_sync(0xffffffffu, need)) {
                lane_neg = false;
                lane_dead = true;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if ((E[k] < 0) & (fmax(fabs(p1[k]), fabs(p2[k])) > Tr::thresh())) {
                        p1[k] = Tr::down(p1[k]);
                        p2[k] = Tr::down(p2[k]);
                        E[k] += 1;
                        if (E[k] == 0) {
                            const real2 rw = restore_weight<Tr>(tile, P, k * 32 + lane, m);
                            wc[k] = rw.x;
                            ws[k] = rw.y;
                        }
                    }
                    lane_neg |= E[k] < 0;
                    lane_dead &= E[k] < 0;
                }
                any_neg = __any_sync(0xffffffffu, lane_neg);
                all_dead = __all_sync(0xffffffffu, lane_dead);
            }
        }
        // ---- reduce the 16 (re, im) rows over the 32 lanes ----
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            real2 v;
            v.x = re[j];
            v.y = im[j];
            xb[j * XS + lane] = v;
        }
        __syncwarp();
        const int row = lane & 15, half = lane >> 4;
        real sr, si;
        Tr::row_sum16(xb + row * XS + half * 16, sr, si);
        sr += __shfl_xor_sync(0xffffffffu, sr, 16);
        si += __shfl_xor_sync(0xffffffffu, si, 16);
        const int q = bk * 16 + row;
        if (half == 0 && q < len) {
            real2 a = acc[q];
            a.x += sr;
            a.y += si;
            acc[q] = a;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------
// FP32 column on packed pairs: lanes carry K points as K/2 (f32x2) pairs, so
// each recurrence / accumulation instruction advances two points.
// ---------------------------------------------------------------------
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    float2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)),
          "l"(reinterpret_cast<unsigned long long&>(c)));
    return d;
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
    float2 d;
    asm("mul.rn.f32x2 %0, %1, %2;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)));
    return d;
}

__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    float2 d;
    asm("add.rn.f32x2 %0, %1, %2;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)));
    return d;
}

__device__ __forceinline__ bool needs_rescale(int E, float a, float b) {
    return (E < 0) & (fmaxf(fabsf(a), fabsf(b)) > TraitsF32::thresh());
}

template <int K>
__device__ __forceinline__ int column_f32x2(const uint32_t* tile, int P, int m, int L,
                                             const float2* __restrict__ alpha2, float lch, float lcl, float2* acc,
                                             float2* xb, int lane) {
    constexpr int KP = K / 2;
    constexpr int XS = TraitsF32::XSTRIDE;
    const int len = L - m + 1;
    float2 x2[KP], p1[KP], p2[KP], wc2[KP], ws2[KP];
    int E[K];
    bool lane_neg = false, lane_dead = true;
#pragma unroll
    for (int kp = 0; kp < KP; ++kp) {
        float xv[2], mant[2], cs[2], sn[2], w[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * kp + h;
            TraitsF32::setup(tile, P, k * 32 + lane, m, lch, lcl, xv[h], mant[h], E[k], cs[h], sn[h], w[h]);
            lane_neg |= E[k] != 0;
            lane_dead &= E[k] != 0;
        }
        x2[kp] = make_float2(xv[0], xv[1]);
        p1[kp] = make_float2(0.f, 0.f);          // sigma_{m-1}
        p2[kp] = make_float2(mant[0], mant[1]);  // sigma_{m-2}
        wc2[kp] = make_float2(E[2 * kp] == 0 ? w[0] * cs[0] : 0.f, E[2 * kp + 1] == 0 ? w[1] * cs[1] : 0.f);
        ws2[kp] = make_float2(E[2 * kp] == 0 ? -w[0] * sn[0] : 0.f, E[2 * kp + 1] == 0 ? -w[1] * sn[1] : 0.f);
    }
    bool any_neg = __any_sync(0xffffffffu, lane_neg);
    bool all_dead = __all_sync(0xffffffffu, lane_dead);

    int nskip = 0;  // blocks of 16 steps whose accumulation was skipped
    const int nblk = (len + 15) >> 4;
    // coefficients of the next block are fetched while the current one runs
    float4 an[8];
    {
        const float4* a4 = reinterpret_cast<const float4*>(alpha2);
#pragma unroll
        for (int c = 0; c < 8; ++c) an[c] = __ldg(a4 + c);
    }
    for (int bk = 0; bk < nblk; ++bk) {
        float2 av[16];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            av[2 * c] = make_float2(an[c].x, an[c].y);
            av[2 * c + 1] = make_float2(an[c].z, an[c].w);
        }
        if (bk + 1 < nblk) {
            const float4* a4 = reinterpret_cast<const float4*>(alpha2 + 16 * (bk + 1));
#pragma unroll
            for (int c = 0; c < 8; ++c) an[c] = __ldg(a4 + c);
        }
        const bool skip = all_dead;
        nskip += skip;  // decided for this whole block of 16 steps
        if (skip) {  // every point of the warp is still below range: recurrence only
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                float2 t[KP];
#pragma unroll
                for (int kp = 0; kp < KP; ++kp) t[kp] = f2_mul(x2[kp], p1[kp]);
#pragma unroll
                for (int kp = 0; kp < KP; ++kp) {
                    const float2 sg = f2_fma(av[j], t[kp], p2[kp]);
                    p2[kp] = p1[kp];
                    p1[kp] = sg;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                // stage order: all products, all recurrence FMAs, then the
                // accumulation
                float2 t[KP];
#pragma unroll
                for (int kp = 0; kp < KP; ++kp) t[kp] = f2_mul(x2[kp], p1[kp]);
#pragma unroll
                for (int kp = 0; kp < KP; ++kp) {
                    const float2 sg = f2_fma(av[j], t[kp], p2[kp]);
                    p2[kp] = p1[kp];
                    p1[kp] = sg;
                }
                // one packed chain per component (the next step's recurrence
                // does not depend on it, so its latency overlaps), then one
                // add per component
                float2 r0 = f2_mul(p1[0], wc2[0]), i0 = f2_mul(p1[0], ws2[0]);
#pragma unroll
                for (int kp = 1; kp < KP; ++kp) {
                    r0 = f2_fma(p1[kp], wc2[kp], r0);
                    i0 = f2_fma(p1[kp], ws2[kp], i0);
                }
                xb[j * XS + lane] = make_float2(r0.x + r0.y, i0.x + i0.y);
            }
        }
        if (any_neg) {
            // Rescale check once per 16 steps, branch-free: points whose state
            // is still below range and above the threshold are scaled down by
            // 2^-64 (exact).  Only a point reaching E == 0 needs its weights,
            // which is rare and handled behind one vote.
            bool reached = false;
            lane_neg = false;
            lane_dead = true;
#pragma unroll
            for (int kp = 0; kp < KP; ++kp) {
                const bool nx = needs_rescale(E[2 * kp], p1[kp].x, p2[kp].x);
                const bool ny = needs_rescale(E[2 * kp + 1], p1[kp].y, p2[kp].y);
                const float2 f = make_float2(nx ? 0x1p-64f : 1.f, ny ? 0x1p-64f : 1.f);
                p1[kp] = f2_mul(p1[kp], f);
                p2[kp] = f2_mul(p2[kp], f);
                E[2 * kp] += nx;
                E[2 * kp + 1] += ny;
                reached |= (nx & (E[2 * kp] == 0)) | (ny & (E[2 * kp + 1] == 0));
                lane_neg |= (E[2 * kp] != 0) | (E[2 * kp + 1] != 0);
                lane_dead &= (E[2 * kp] != 0) & (E[2 * kp + 1] != 0);
            }
            if (__any_sync(0xffffffffu, reached)) {
#pragma unroll
                for (int kp = 0; kp < KP; ++kp) {
                    if (E[2 * kp] == 0 && wc2[kp].x == 0.f && ws2[kp].x == 0.f) {
                        const float2 rw = restore_weight<TraitsF32>(tile, P, (2 * kp) * 32 + lane, m);
                        wc2[kp].x = rw.x;
                        ws2[kp].x = rw.y;
                    }
                    if (E[2 * kp + 1] == 0 && wc2[kp].y == 0.f && ws2[kp].y == 0.f) {
                        const float2 rw = restore_weight<TraitsF32>(tile, P, (2 * kp + 1) * 32 + lane, m);
                        wc2[kp].y = rw.x;
                        ws2[kp].y = rw.y;
                    }
                }
            }
            any_neg = __any_sync(0xffffffffu, lane_neg);
            all_dead = __all_sync(0xffffffffu, lane_dead);
        }
        if (!skip) {
            __syncwarp();
            const int row = lane & 15, half = lane >> 4;
            float sr, si;
            TraitsF32::row_sum16(xb + row * XS + half * 16, sr, si);
            sr += __shfl_xor_sync(0xffffffffu, sr, 16);
            si += __shfl_xor_sync(0xffffffffu, si, 16);
            const int q = bk * 16 + row;
            if (half == 0 && q < len) {
                float2 a = acc[q];
                a.x += sr;
                a.y += si;
                acc[q] = a;
            }
            __syncwarp();
        }
    }
    return nskip;
}


// ---------------------------------------------------------------------
// FP32 column near a pole: every point of the tile has x >= pole_x (sgn = 1)
// or every point has x <= -pole_x (sgn = -1), and m < pole_mmax.  Near
// x = +-1 the three-term recurrence has a double root and FP32 rounding of its
// coefficients and of x sigma grows like l^1.5 eps (1e-3 of lambda_max by
// l = 2048 at theta ~ 1e-3, mostly at low m).  Here the unfolded recurrence
// runs in Reinsch's difference form on |x| in the smooth normalisation of the
// near-pole table (per step and pair: c = a u + e, d = c y + d, y = y + d;
// u = |x| - 1; tables in build_tables):
//   y_q = lambda_l(|x|) / gamma~_l  (q = l - m),  d_q = y_q - y_{q-1},
// gamma~_l = gamma_l (q even), rho gamma_l (q odd).  lambda_l(x) =
// sgn^q lambda_l(|x|) (mirror symmetry), and the sign-folded accumulators of
// column_f32x2 hold sigma_q = s_q lambda_l / gamma_l with s_q =
// (-1)^floor(q/2): the factor s_q sgn^q (q odd ? rho : 1) depends on
// q mod 4 = j mod 4, sgn and m only, so it is applied to the warp's row
// value of step j.
// ---------------------------------------------------------------------
template <int K>
__device__ __forceinline__ int column_f32x2_pole(const uint32_t* tile, int P, int m, int L,
                                                  const float4* __restrict__ ae, float sgn, float rho, float lch,
                                                  float lcl, float2* acc, float2* xb, int lane) {
    constexpr int KP = K / 2;
    constexpr int XS = TraitsF32::XSTRIDE;
    const int len = L - m + 1;
    float2 u2[KP], y2[KP], d2[KP], wc2[KP], ws2[KP];
    int E[K];
    bool lane_neg = false, lane_dead = true;
#pragma unroll
    for (int kp = 0; kp < KP; ++kp) {
        float xv[2], mant[2], cs[2], sn[2], w[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * kp + h;
            TraitsF32::setup(tile, P, k * 32 + lane, m, lch, lcl, xv[h], mant[h], E[k], cs[h], sn[h], w[h]);
            lane_neg |= E[k] != 0;
            lane_dead &= E[k] != 0;
        }
        u2[kp] = make_float2(fabsf(xv[0]) - 1.f, fabsf(xv[1]) - 1.f);
        y2[kp] = make_float2(0.f, 0.f);          // y_{-1}
        d2[kp] = make_float2(mant[0], mant[1]);  // d_{-1}: the first step gives y_0 = mant
        wc2[kp] = make_float2(E[2 * kp] == 0 ? w[0] * cs[0] : 0.f, E[2 * kp + 1] == 0 ? w[1] * cs[1] : 0.f);
        ws2[kp] = make_float2(E[2 * kp] == 0 ? -w[0] * sn[0] : 0.f, E[2 * kp + 1] == 0 ? -w[1] * sn[1] : 0.f);
    }
    bool any_neg = __any_sync(0xffffffffu, lane_neg);
    bool all_dead = __all_sync(0xffffffffu, lane_dead);
    // row factor of step j: s_q sgn^q (q odd ? rho : 1), q = j (mod 4)
    const float fr = sgn * rho;
    const float sj[4] = {1.f, fr, -1.f, -fr};

    int nskip = 0;  // blocks of 16 steps whose accumulation was skipped
    const int nblk = (len + 15) >> 4;
    for (int bk = 0; bk < nblk; ++bk) {
        const bool skip = all_dead;
        nskip += skip;
#pragma unroll
        for (int j4 = 0; j4 < 4; ++j4) {
            float4 cv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) cv[c] = __ldg(ae + 16 * bk + 4 * j4 + c);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int j = 4 * j4 + jj;
                const float2 a2 = make_float2(cv[jj].x, cv[jj].y), e2 = make_float2(cv[jj].z, cv[jj].w);
#pragma unroll
                for (int kp = 0; kp < KP; ++kp) {
                    const float2 c = f2_fma(a2, u2[kp], e2);
                    d2[kp] = f2_fma(c, y2[kp], d2[kp]);
                    y2[kp] = f2_add(y2[kp], d2[kp]);
                }
                if (!skip) {
                    float2 r0 = f2_mul(y2[0], wc2[0]), i0 = f2_mul(y2[0], ws2[0]);
#pragma unroll
                    for (int kp = 1; kp < KP; ++kp) {
                        r0 = f2_fma(y2[kp], wc2[kp], r0);
                        i0 = f2_fma(y2[kp], ws2[kp], i0);
                    }
                    xb[j * XS + lane] = make_float2(sj[jj] * (r0.x + r0.y), sj[jj] * (i0.x + i0.y));
                }
            }
        }
        if (any_neg) {
            // rescale check once per 16 steps (as column_f32x2, on (y, d))
            bool reached = false;
            lane_neg = false;
            lane_dead = true;
#pragma unroll
            for (int kp = 0; kp < KP; ++kp) {
                const bool nx = needs_rescale(E[2 * kp], y2[kp].x, d2[kp].x);
                const bool ny = needs_rescale(E[2 * kp + 1], y2[kp].y, d2[kp].y);
                const float2 f = make_float2(nx ? 0x1p-64f : 1.f, ny ? 0x1p-64f : 1.f);
                y2[kp] = f2_mul(y2[kp], f);
                d2[kp] = f2_mul(d2[kp], f);
                E[2 * kp] += nx;
                E[2 * kp + 1] += ny;
                reached |= (nx & (E[2 * kp] == 0)) | (ny & (E[2 * kp + 1] == 0));
                lane_neg |= (E[2 * kp] != 0) | (E[2 * kp + 1] != 0);
                lane_dead &= (E[2 * kp] != 0) & (E[2 * kp + 1] != 0);
            }
            if (__any_sync(0xffffffffu, reached)) {
#pragma unroll
                for (int kp = 0; kp < KP; ++kp) {
                    if (E[2 * kp] == 0 && wc2[kp].x == 0.f && ws2[kp].x == 0.f) {
                        const float2 rw = restore_weight<TraitsF32>(tile, P, (2 * kp) * 32 + lane, m);
                        wc2[kp].x = rw.x;
                        ws2[kp].x = rw.y;
                    }
                    if (E[2 * kp + 1] == 0 && wc2[kp].y == 0.f && ws2[kp].y == 0.f) {
                        const float2 rw = restore_weight<TraitsF32>(tile, P, (2 * kp + 1) * 32 + lane, m);
                        wc2[kp].y = rw.x;
                        ws2[kp].y = rw.y;
                    }
                }
            }
            any_neg = __any_sync(0xffffffffu, lane_neg);
            all_dead = __all_sync(0xffffffffu, lane_dead);
        }
        if (!skip) {
            __syncwarp();
            const int row = lane & 15, half = lane >> 4;
            float sr, si;
            TraitsF32::row_sum16(xb + row * XS + half * 16, sr, si);
            sr += __shfl_xor_sync(0xffffffffu, sr, 16);
            si += __shfl_xor_sync(0xffffffffu, si, 16);
            const int q = bk * 16 + row;
            if (half == 0 && q < len) {
                float2 a = acc[q];
                a.x += sr;
                a.y += si;
                acc[q] = a;
            }
            __syncwarp();
        }
    }
    return nskip;
}

// +1 if every point of the tile has x >= pole_x, -1 if every point has
// x <= -pole_x, 0 otherwise; points of weight zero (padding among them)
// contribute nothing and do not count.  The same answer in every warp of the
// CTA: all warps read the same tile.
template <int K>
__device__ __forceinline__ int tile_near_pole(const uint32_t* tile, int P, float pole_x, int lane) {
    const float* tf = reinterpret_cast<const float*>(tile);
    bool np = true, sp = true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float x = tf[k * 32 + lane];
        const bool idle = tf[P + k * 32 + lane] == 0.f;
        np &= idle | (x >= pole_x);
        sp &= idle | (x <= -pole_x);
    }
    return __all_sync(0xffffffffu, np) ? 1 : (__all_sync(0xffffffffu, sp) ? -1 : 0);
}

// ---------------------------------------------------------------------
// FP32 column, scalar FMAs (the default): K points per lane.  The hot loop
// is a straight 16-step block per branch outcome: recurrence (mul + FMA per
// point), accumulation in two chains per component, one 64-bit store per
// step for the warp transpose.  The rescale test is a predicate per point
// and one vote every 16 steps; only a lane that has to rescale takes the
// branch.
// ---------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void column_f32s(const uint32_t* tile, int P, int m, int L,
                                            const float* __restrict__ alpha, float lch, float lcl, float2* acc,
                                            float2* xb, int lane) {
    constexpr int XS = TraitsF32::XSTRIDE;
    const int len = L - m + 1;
    float x[K], p1[K], p2[K], wc[K], ws[K];
    int E[K];
    bool lane_neg = false, lane_dead = true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float mant, cs, sn, w;
        TraitsF32::setup(tile, P, k * 32 + lane, m, lch, lcl, x[k], mant, E[k], cs, sn, w);
        const bool live = E[k] == 0;
        wc[k] = live ? w * cs : 0.f;
        ws[k] = live ? -w * sn : 0.f;
        p1[k] = 0.f;   // sigma_{m-1}
        p2[k] = mant;  // sigma_{m-2}
        lane_neg |= !live;
        lane_dead &= !live;
    }
    bool any_neg = __any_sync(0xffffffffu, lane_neg);
    bool all_dead = __all_sync(0xffffffffu, lane_dead);
    const int row = lane & 15, half = lane >> 4;

    const int nblk = (len + 15) >> 4;
    float an[16];
    load16(alpha, an);
    for (int bk = 0; bk < nblk; ++bk) {
        float av[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) av[j] = an[j];
        if (bk + 1 < nblk) load16(alpha + 16 * (bk + 1), an);
        const bool skip = all_dead;
        if (skip) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float sg = fmaf(av[j], x[k] * p1[k], p2[k]);
                    p2[k] = p1[k];
                    p1[k] = sg;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float sg = fmaf(av[j], x[k] * p1[k], p2[k]);
                    p2[k] = p1[k];
                    p1[k] = sg;
                }
                float r0 = p1[0] * wc[0], i0 = p1[0] * ws[0], r1 = p1[1] * wc[1], i1 = p1[1] * ws[1];
#pragma unroll
                for (int k = 2; k < K; k += 2) {
                    r0 = fmaf(p1[k], wc[k], r0);
                    i0 = fmaf(p1[k], ws[k], i0);
                    r1 = fmaf(p1[k + 1], wc[k + 1], r1);
                    i1 = fmaf(p1[k + 1], ws[k + 1], i1);
                }
                xb[j * XS + lane] = make_float2(r0 + r1, i0 + i1);
            }
        }
        if (any_neg) {
            bool need = false;
#pragma unroll
            for (int k = 0; k < K; ++k) need |= needs_rescale(E[k], p1[k], p2[k]);
            if (__any_sync(0xffffffffu, need)) {
                lane_neg = false;
                lane_dead = true;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if (needs_rescale(E[k], p1[k], p2[k])) {
                        p1[k] *= 0x1p-64f;
                        p2[k] *= 0x1p-64f;
                        E[k] += 1;
                        if (E[k] == 0) {
                            const float2 rw = restore_weight<TraitsF32>(tile, P, k * 32 + lane, m);
                            wc[k] = rw.x;
                            ws[k] = rw.y;
                        }
                    }
                    lane_neg |= E[k] != 0;
                    lane_dead &= E[k] != 0;
                }
                any_neg = __any_sync(0xffffffffu, lane_neg);
                all_dead = __all_sync(0xffffffffu, lane_dead);
            }
        }
        if (!skip) {
            __syncwarp();
            float sr, si;
            TraitsF32::row_sum16(xb + row * XS + half * 16, sr, si);
            sr += __shfl_xor_sync(0xffffffffu, sr, 16);
            si += __shfl_xor_sync(0xffffffffu, si, 16);
            const int q = bk * 16 + row;
            if (half == 0 && q < len) {
                float2 a = acc[q];
                a.x += sr;
                a.y += si;
                acc[q] = a;
            }
            __syncwarp();
        }
    }
}

template <typename Tr>
__device__ __forceinline__ void flush_acc(typename Tr::real2* acc, int lena, int lenb, int ma, int mb, int L,
                                          double* slot, bool first, int lane) {
    using real2 = typename Tr::real2;
    for (int i = lane; i < lena + lenb; i += 32) {
        const int m = i < lena ? ma : mb;
        const int l = i < lena ? ma + i : mb + (i - lena);
        const int64_t idx = tri_base(m, L) + l;
        const real2 a = acc[i];
        real2 z;
        z.x = 0;
        z.y = 0;
        acc[i] = z;
        double2* sp = reinterpret_cast<double2*>(slot) + idx;
        double2 v = first ? make_double2(0.0, 0.0) : *sp;
        v.x += (double)a.x;
        v.y += (double)a.y;
        *sp = v;
    }
    __syncwarp();
}

template <typename Tr>
__device__ __forceinline__ void log2c_of(const AnalysisParams& p, int m, typename Tr::real& hi,
                                         typename Tr::real& lo);
template <>
__device__ __forceinline__ void log2c_of<TraitsF32>(const AnalysisParams& p, int m, float& hi, float& lo) {
    hi = p.log2c_hi[m];
    lo = p.log2c_lo[m];
}
template <>
__device__ __forceinline__ void log2c_of<TraitsF64>(const AnalysisParams& p, int m, double& hi, double& lo) {
    hi = p.log2c[m];
    lo = 0.0;
}

// ====================================================================
//                  persistent analysis kernel (a_lm)
// ====================================================================
template <typename Tr, int K, int W, bool PACKED = false>
__global__ void __launch_bounds__(W * 32) analysis_kernel(const __grid_constant__ AnalysisParams p) {
    using real = typename Tr::real;
    using real2 = typename Tr::real2;
    constexpr int P = 32 * K;
    constexpr int ARR_BYTES = P * Tr::ABYTES;
    constexpr int TILE_BYTES = Tr::NARR * ARR_BYTES;
    const int L = p.lmax;
    const int accw = (L + 2 + 3) & ~3;

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    int64_t* s_unit = reinterpret_cast<int64_t*>(smem + 16);
    unsigned char* tiles = smem + 128;
    real2* xbuf = reinterpret_cast<real2*>(tiles + 2 * TILE_BYTES);
    real2* accb = xbuf + W * 16 * Tr::XSTRIDE;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    real2* my_acc = accb + warp * accw;
    real2* my_xb = xbuf + warp * 16 * Tr::XSTRIDE;

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (p.wait_probe && blockIdx.x == 0) {
        // Test hook for the timeout path: a bounded wait on a barrier that no
        // copy and no thread ever arrives at gives up, the CTA records
        // ERR_TIMEOUT and leaves before it takes a work unit or issues a copy
        // (the other CTAs take every unit).
        if (threadIdx.x == 0) {
            uint64_t* probe = reinterpret_cast<uint64_t*>(smem + 32);
            mbar_init(probe, 1);
            fence_mbar_init();
            if (!mbar_wait_bounded(probe, 0, 1u << 10)) atomicOr(p.err, ERR_TIMEOUT);
        }
        __syncthreads();
        return;
    }
    uint32_t blk_skip = 0, blk_all = 0;  // 16-step blocks skipped below range / run (PACKED)
    uint32_t parity0 = 0, parity1 = 0;

    for (;;) {
        if (threadIdx.x == 0) s_unit[0] = (int64_t)atomicAdd(p.counter, 1);
        __syncthreads();
        const int64_t u = s_unit[0];
        __syncthreads();
        if (u >= p.nunits) break;

        int f = 0;
        while (f + 1 < p.nfield && p.fld[f + 1].unit0 <= u) ++f;
        const FieldDesc fd = p.fld[f];
        const int64_t q = u - fd.unit0;
        const int64_t r = q / p.ngroups;
        const int g = (int)(q - r * p.ngroups);
        const int64_t pt0 = fd.off + r * p.chunk;
        const int64_t npts = min(p.chunk, fd.npad - r * p.chunk);
        const int ntiles = (int)(npts / P);
        double* slot = p.slots + (int64_t)(fd.slot0 + r) * p.nmodes * 2;

        const int pi = g * W + warp;
        const int ma = pi, mb = L - pi;
        const bool active = ma <= mb;
        const bool single = ma == mb;
        const int lena = active ? L - ma + 1 : 0;
        const int lenb = (active && !single) ? L - mb + 1 : 0;
        real lca = 0, lcla = 0, lcb = 0, lclb = 0;
        const real* alpha_a = nullptr;
        const real* alpha_b = nullptr;
        if (active) {
            log2c_of<Tr>(p, ma, lca, lcla);
            alpha_a = alpha_base<Tr>(p, ma);
            if (!single) {
                log2c_of<Tr>(p, mb, lcb, lclb);
                alpha_b = alpha_base<Tr>(p, mb);
            }
        }
        for (int i = lane; i < lena + lenb; i += 32) {
            real2 z;
            z.x = 0;
            z.y = 0;
            my_acc[i] = z;
        }
        __syncwarp();
        bool first_flush = true;

        auto issue = [&](int t, int b) {
            uint64_t* bar = &bars[b];
            unsigned char* dst = tiles + b * TILE_BYTES;
            mbar_expect_tx(bar, TILE_BYTES);
            const unsigned char* src = static_cast<const unsigned char*>(p.pts);
            const int64_t first = pt0 + (int64_t)t * P;
            for (int a = 0; a < Tr::NARR; ++a)
                bulk_g2s(dst + a * ARR_BYTES, src + ((int64_t)a * p.ntot + first) * Tr::ABYTES, ARR_BYTES, bar);
        };
        if (threadIdx.x == 0 && ntiles > 0) issue(0, 0);

        for (int t = 0; t < ntiles; ++t) {
            const int b = t & 1;
            if (threadIdx.x == 0 && t + 1 < ntiles) issue(t + 1, b ^ 1);
            const uint32_t par = b ? parity1 : parity0;
            const bool ok = mbar_wait_bounded(&bars[b], par);
            if (b) parity1 ^= 1u; else parity0 ^= 1u;
            if (__syncthreads_or(!ok)) {
                // give up on this unit: record the timeout, then wait (bounded)
                // for every copy this CTA still has in flight, on both buffers
                if (threadIdx.x == 0) {
                    atomicOr(p.err, ERR_TIMEOUT);
                    mbar_drain(&bars[b], par);
                    if (t + 1 < ntiles) mbar_drain(&bars[b ^ 1], b ? parity0 : parity1);
                }
                __syncthreads();
                return;
            }
            const uint32_t* tile = reinterpret_cast<const uint32_t*>(tiles + b * TILE_BYTES);
            if (active) {
                int pole = 0;
                if constexpr (PACKED) pole = tile_near_pole<K>(tile, P, p.pole_x, lane);
                // one inlined copy of the column body, run for both orders of the pair
                for (int c = 0; c < (single ? 1 : 2); ++c) {
                    const int m = c ? mb : ma;
                    if constexpr (sizeof(real) == 4) {
                        if constexpr (PACKED) {
                            const int nb = (L - m + 16) >> 4;
                            int sk;
                            if (pole && m < p.pole_mmax)
                                sk = column_f32x2_pole<K>(tile, P, m, L, p.pole_ae + p.colstart[m], (float)pole,
                                                           p.pole_rho[m], c ? lcb : lca, c ? lclb : lcla,
                                                           my_acc + (c ? lena : 0), my_xb, lane);
                            else
                                sk = column_f32x2<K>(tile, P, m, L, p.alpha_f2 + p.colstart[m], c ? lcb : lca,
                                                     c ? lclb : lcla, my_acc + (c ? lena : 0), my_xb, lane);
                            blk_skip += (uint32_t)sk;
                            blk_all += (uint32_t)nb;
                        } else
                            column_f32s<K>(tile, P, m, L, p.alpha_f + p.colstart[m], c ? lcb : lca, c ? lclb : lcla,
                                           my_acc + (c ? lena : 0), my_xb, lane);
                    } else
                        analysis_column<Tr, K>(tile, P, m, L, c ? alpha_b : alpha_a, c ? lcb : lca, c ? lclb : lcla,
                                               my_acc + (c ? lena : 0), my_xb, lane);
                }
                if (t == ntiles - 1 || (t + 1) % p.flush_tiles == 0) {
                    flush_acc<Tr>(my_acc, lena, lenb, ma, mb, L, slot, first_flush, lane);
                    first_flush = false;
                }
            }
            __syncthreads();
        }
    }
    if (p.stats && lane == 0 && blk_all) {
        atomicAdd(p.stats, (unsigned long long)blk_skip);
        atomicAdd(p.stats + 1, (unsigned long long)blk_all);
    }
}

// ====================================================================
//     FP32 analysis kernel: groups of WG warps share one order pair
// ====================================================================
// A CTA holds G groups of WG warps (G*WG warps, 16 for G = WG = 4) and one
// tile of P = 32*K*WG points.  Group g runs the order pair (m, lmax - m) of
// the unit's m-group; warp w of the group runs the recurrence for points
// [w*32K, (w+1)*32K) of the tile (K per lane, in f32x2 pairs).  After each
// block of 16 steps every warp reduces its 32 lanes (shared-memory
// transpose) to 16 partial (re, im) sums, a named barrier joins the group,
// and one warp adds the WG partials, in warp order, into the group's FP32
// accumulator row.  Partials are double-buffered so one barrier per block
// suffices.  Sharing the row lets 16 warps fit per SM.
__device__ __forceinline__ void group_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int K, int WG>
__device__ __forceinline__ void column_f32g(const uint32_t* tile, int P, int pt0, int m, int L,
                                            const float2* __restrict__ alpha2, float lch, float lcl, float2* acc,
                                            float2* xb, float2* part, int wig, int lane, int bar_id) {
    constexpr int KP = K / 2;
    constexpr int XS = TraitsF32::XSTRIDE;
    const int len = L - m + 1;
    float2 x2[KP], p1[KP], p2[KP], wc2[KP], ws2[KP];
    int E[K];
    bool lane_neg = false, lane_dead = true;
#pragma unroll
    for (int kp = 0; kp < KP; ++kp) {
        float xv[2], mant[2], cs[2], sn[2], w[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * kp + h;
            TraitsF32::setup(tile, P, pt0 + k * 32 + lane, m, lch, lcl, xv[h], mant[h], E[k], cs[h], sn[h], w[h]);
            lane_neg |= E[k] != 0;
            lane_dead &= E[k] != 0;
        }
        x2[kp] = make_float2(xv[0], xv[1]);
        p1[kp] = make_float2(0.f, 0.f);          // sigma_{m-1}
        p2[kp] = make_float2(mant[0], mant[1]);  // sigma_{m-2}
        wc2[kp] = make_float2(E[2 * kp] == 0 ? w[0] * cs[0] : 0.f, E[2 * kp + 1] == 0 ? w[1] * cs[1] : 0.f);
        ws2[kp] = make_float2(E[2 * kp] == 0 ? -w[0] * sn[0] : 0.f, E[2 * kp + 1] == 0 ? -w[1] * sn[1] : 0.f);
    }
    bool any_neg = __any_sync(0xffffffffu, lane_neg);
    bool all_dead = __all_sync(0xffffffffu, lane_dead);
    const int row = lane & 15, half = lane >> 4;

    const int nblk = (len + 15) >> 4;
    for (int bk = 0; bk < nblk; ++bk) {
        const float4* a4 = reinterpret_cast<const float4*>(alpha2 + 16 * bk);
        const bool skip = all_dead;  // decided for this whole block of 16 steps
#pragma unroll
        for (int j4 = 0; j4 < 4; ++j4) {
            const float4 u = __ldg(a4 + 2 * j4), v = __ldg(a4 + 2 * j4 + 1);
            const float2 av[4] = {make_float2(u.x, u.y), make_float2(u.z, u.w), make_float2(v.x, v.y),
                                  make_float2(v.z, v.w)};
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int j = 4 * j4 + jj;
                float2 t[KP];
#pragma unroll
                for (int kp = 0; kp < KP; ++kp) t[kp] = f2_mul(x2[kp], p1[kp]);
#pragma unroll
                for (int kp = 0; kp < KP; ++kp) {
                    const float2 sg = f2_fma(av[jj], t[kp], p2[kp]);
                    p2[kp] = p1[kp];
                    p1[kp] = sg;
                }
                if (!skip) {
                    float2 r0 = f2_mul(p1[0], wc2[0]), i0 = f2_mul(p1[0], ws2[0]);
                    float2 r1 = f2_mul(p1[1], wc2[1]), i1 = f2_mul(p1[1], ws2[1]);
#pragma unroll
                    for (int kp = 2; kp < KP; kp += 2) {
                        r0 = f2_fma(p1[kp], wc2[kp], r0);
                        i0 = f2_fma(p1[kp], ws2[kp], i0);
                        r1 = f2_fma(p1[kp + 1], wc2[kp + 1], r1);
                        i1 = f2_fma(p1[kp + 1], ws2[kp + 1], i1);
                    }
                    xb[j * XS + lane] =
                        make_float2((r0.x + r1.x) + (r0.y + r1.y), (i0.x + i1.x) + (i0.y + i1.y));
                }
            }
        }
        if (any_neg) {
            // rescale check once per 16 steps (branch-free; see column_f32x2)
            bool reached = false;
            lane_neg = false;
            lane_dead = true;
#pragma unroll
            for (int kp = 0; kp < KP; ++kp) {
                const bool nx = needs_rescale(E[2 * kp], p1[kp].x, p2[kp].x);
                const bool ny = needs_rescale(E[2 * kp + 1], p1[kp].y, p2[kp].y);
                const float2 f = make_float2(nx ? 0x1p-64f : 1.f, ny ? 0x1p-64f : 1.f);
                p1[kp] = f2_mul(p1[kp], f);
                p2[kp] = f2_mul(p2[kp], f);
                E[2 * kp] += nx;
                E[2 * kp + 1] += ny;
                reached |= (nx & (E[2 * kp] == 0)) | (ny & (E[2 * kp + 1] == 0));
                lane_neg |= (E[2 * kp] != 0) | (E[2 * kp + 1] != 0);
                lane_dead &= (E[2 * kp] != 0) & (E[2 * kp + 1] != 0);
            }
            if (__any_sync(0xffffffffu, reached)) {
#pragma unroll
                for (int kp = 0; kp < KP; ++kp) {
                    if (E[2 * kp] == 0 && wc2[kp].x == 0.f && ws2[kp].x == 0.f) {
                        const float2 rw = restore_weight<TraitsF32>(tile, P, pt0 + (2 * kp) * 32 + lane, m);
                        wc2[kp].x = rw.x;
                        ws2[kp].x = rw.y;
                    }
                    if (E[2 * kp + 1] == 0 && wc2[kp].y == 0.f && ws2[kp].y == 0.f) {
                        const float2 rw = restore_weight<TraitsF32>(tile, P, pt0 + (2 * kp + 1) * 32 + lane, m);
                        wc2[kp].y = rw.x;
                        ws2[kp].y = rw.y;
                    }
                }
            }
            any_neg = __any_sync(0xffffffffu, lane_neg);
            all_dead = __all_sync(0xffffffffu, lane_dead);
        }
        float sr = 0.f, si = 0.f;
        if (!skip) {
            __syncwarp();
            TraitsF32::row_sum16(xb + row * XS + half * 16, sr, si);
            sr += __shfl_xor_sync(0xffffffffu, sr, 16);
            si += __shfl_xor_sync(0xffffffffu, si, 16);
            __syncwarp();
        }
        float2* pb = part + (bk & 1) * (WG * 16);
        if (half == 0) pb[wig * 16 + row] = make_float2(sr, si);
        group_bar(bar_id, WG * 32);
        const int q = bk * 16 + row;
        if (wig == 0 && half == 0 && q < len) {
            float2 a = acc[q];
#pragma unroll
            for (int w = 0; w < WG; ++w) {
                const float2 v = pb[w * 16 + row];
                a.x += v.x;
                a.y += v.y;
            }
            acc[q] = a;
        }
    }
    group_bar(bar_id, WG * 32);  // the accumulator row is complete for this tile
}

template <int K, int G, int WG>
__global__ void __launch_bounds__(G * WG * 32, 1) analysis_f32g_kernel(const __grid_constant__ AnalysisParams p) {
    constexpr int NW = G * WG;
    constexpr int P = 32 * K * WG;
    constexpr int ARR_BYTES = P * 4;
    constexpr int TILE_BYTES = TraitsF32::NARR * ARR_BYTES;
    constexpr int XS = TraitsF32::XSTRIDE;
    const int L = p.lmax;
    const int accw = (L + 2 + 3) & ~3;

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    int64_t* s_unit = reinterpret_cast<int64_t*>(smem + 16);
    unsigned char* tiles = smem + 128;
    float2* xbuf = reinterpret_cast<float2*>(tiles + 2 * TILE_BYTES);
    float2* partb = xbuf + NW * 16 * XS;
    float2* accb = partb + G * 2 * WG * 16;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = warp / WG, wig = warp % WG;
    float2* my_acc = accb + grp * accw;
    float2* my_xb = xbuf + warp * 16 * XS;
    float2* my_part = partb + grp * 2 * WG * 16;
    const int bar_id = 1 + grp;

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t parity0 = 0, parity1 = 0;

    for (;;) {
        if (threadIdx.x == 0) s_unit[0] = (int64_t)atomicAdd(p.counter, 1);
        __syncthreads();
        const int64_t u = s_unit[0];
        __syncthreads();
        if (u >= p.nunits) break;

        int f = 0;
        while (f + 1 < p.nfield && p.fld[f + 1].unit0 <= u) ++f;
        const FieldDesc fd = p.fld[f];
        const int64_t q = u - fd.unit0;
        const int64_t r = q / p.ngroups;
        const int g = (int)(q - r * p.ngroups);
        const int64_t pt0 = fd.off + r * p.chunk;
        const int64_t npts = min(p.chunk, fd.npad - r * p.chunk);
        const int ntiles = (int)(npts / P);
        double* slot = p.slots + (int64_t)(fd.slot0 + r) * p.nmodes * 2;

        const int pi = g * G + grp;
        const int ma = pi, mb = L - pi;
        const bool active = ma <= mb;
        const bool single = ma == mb;
        const int lena = active ? L - ma + 1 : 0;
        const int lenb = (active && !single) ? L - mb + 1 : 0;
        for (int i = threadIdx.x - grp * WG * 32; i < lena + lenb; i += WG * 32) my_acc[i] = make_float2(0.f, 0.f);
        bool first_flush = true;

        auto issue = [&](int t, int b) {
            uint64_t* bar = &bars[b];
            unsigned char* dst = tiles + b * TILE_BYTES;
            mbar_expect_tx(bar, TILE_BYTES);
            const unsigned char* src = static_cast<const unsigned char*>(p.pts);
            const int64_t first = pt0 + (int64_t)t * P;
            for (int a = 0; a < TraitsF32::NARR; ++a)
                bulk_g2s(dst + a * ARR_BYTES, src + ((int64_t)a * p.ntot + first) * 4, ARR_BYTES, bar);
        };
        __syncthreads();  // accumulator rows cleared before any warp adds to them
        if (threadIdx.x == 0 && ntiles > 0) issue(0, 0);

        for (int t = 0; t < ntiles; ++t) {
            const int b = t & 1;
            if (threadIdx.x == 0 && t + 1 < ntiles) issue(t + 1, b ^ 1);
            const uint32_t par = b ? parity1 : parity0;
            const bool ok = mbar_wait_bounded(&bars[b], par);
            if (b) parity1 ^= 1u; else parity0 ^= 1u;
            if (__syncthreads_or(!ok)) {
                // give up on this unit: record the timeout, then wait (bounded)
                // for every copy this CTA still has in flight, on both buffers
                if (threadIdx.x == 0) {
                    atomicOr(p.err, ERR_TIMEOUT);
                    mbar_drain(&bars[b], par);
                    if (t + 1 < ntiles) mbar_drain(&bars[b ^ 1], b ? parity0 : parity1);
                }
                __syncthreads();
                return;
            }
            const uint32_t* tile = reinterpret_cast<const uint32_t*>(tiles + b * TILE_BYTES);
            if (active) {
                for (int c = 0; c < (single ? 1 : 2); ++c) {
                    const int m = c ? mb : ma;
                    float lch, lcl;
                    log2c_of<TraitsF32>(p, m, lch, lcl);
                    column_f32g<K, WG>(tile, P, wig * 32 * K, m, L, p.alpha2_col(m), lch, lcl,
                                       my_acc + (c ? lena : 0), my_xb, my_part, wig, lane, bar_id);
                }
            }
            const bool do_flush = t == ntiles - 1 || (t + 1) % p.flush_tiles == 0;
            if (do_flush) __syncthreads();  // the group's last additions are visible to all its warps
            if (active && do_flush) {
                for (int i = threadIdx.x - grp * WG * 32; i < lena + lenb; i += WG * 32) {
                    const int m = i < lena ? ma : mb;
                    const int l = i < lena ? ma + i : mb + (i - lena);
                    const int64_t idx = tri_base(m, L) + l;
                    const float2 a = my_acc[i];
                    my_acc[i] = make_float2(0.f, 0.f);
                    double2* sp = reinterpret_cast<double2*>(slot) + idx;
                    double2 v = first_flush ? make_double2(0.0, 0.0) : *sp;
                    v.x += (double)a.x;
                    v.y += (double)a.y;
                    *sp = v;
                }
                first_flush = false;
            }
            __syncthreads();
        }
    }
}

template <int K, int G, int WG>
size_t analysis_f32g_smem_bytes(int lmax) {
    const int accw = (lmax + 2 + 3) & ~3;
    return 128 + 2 * (size_t)TraitsF32::NARR * 32 * K * WG * 4 + (size_t)G * WG * 16 * TraitsF32::XSTRIDE * 8 +
           (size_t)G * 2 * WG * 16 * 8 + (size_t)G * accw * 8;
}

template <int K, int G, int WG>
cudaError_t launch_analysis_f32g(const AnalysisParams& ap, int sm_count, cudaStream_t st, int* grid_out) {
    const size_t smem = analysis_f32g_smem_bytes<K, G, WG>(ap.lmax);
    auto kern = analysis_f32g_kernel<K, G, WG>;
    int occ = 0;
    cudaError_t e = configure_once(kern, G * WG * 32, smem, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)sm_count * occ;
    if (grid > ap.nunits) grid = ap.nunits;
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = (int)grid;
    kern<<<(int)grid, G * WG * 32, smem, st>>>(ap);
    return cudaGetLastError();
}

// ====================================================================
//            reduction over chunks, times the gamma factors
// ====================================================================
__global__ void reduce_kernel(const __grid_constant__ ReduceParams p) {
    const int64_t total = (int64_t)p.nfield * p.nmodes;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(t / p.nmodes);
        const int64_t idx = t - (int64_t)f * p.nmodes;
        const double2* s = reinterpret_cast<const double2*>(p.slots);
        double re = 0.0, im = 0.0;
        for (int r = 0; r < p.nchunk[f]; ++r) {
            const double2 v = s[(int64_t)(p.slot0[f] + r) * p.nmodes + idx];
            re += v.x;
            im += v.y;
        }
        const double gm = p.gamma[idx];
        reinterpret_cast<double2*>(p.out)[t] = make_double2(re * gm, im * gm);
    }
}

// ====================================================================
//                          host-side launchers
// ====================================================================
template <typename T>
cudaError_t launch_prep(const PrepParams& pp, int nseg, cudaStream_t st) {
    dim3 grid(256, nseg);
    prep_kernel<T><<<grid, 256, 0, st>>>(pp);
    return cudaGetLastError();
}
template cudaError_t launch_prep<float>(const PrepParams&, int, cudaStream_t);
template cudaError_t launch_prep<double>(const PrepParams&, int, cudaStream_t);

// Sorted preparation: padding by prep_kernel (catalog segments empty), then
// hist / scan / scatter.  nranges = sp.range0[ncat].
template <typename T>
cudaError_t launch_prep_sorted(const SortParams& sp, cudaStream_t st) {
    const int ncat = sp.prep.ncat;
    const int64_t nr = sp.range0[ncat];
    {
        PrepParams pads = sp.prep;  // pad segments only
        for (int c = 0; c < ncat; ++c) pads.cat[c].n = 0;
        dim3 grid(64, ncat + sp.prep.nfield);
        prep_kernel<T><<<grid, 256, 0, st>>>(pads);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (nr == 0) return cudaSuccess;
    sort_hist_kernel<T><<<(unsigned)nr, 256, 0, st>>>(sp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sort_scan_kernel<<<sp.prep.nfield, SORT_BUCKETS, 0, st>>>(sp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sort_scatter_kernel<T><<<(unsigned)nr, 256, 0, st>>>(sp);
    return cudaGetLastError();
}
template cudaError_t launch_prep_sorted<float>(const SortParams&, cudaStream_t);
template cudaError_t launch_prep_sorted<double>(const SortParams&, cudaStream_t);

// Bucket offsets only (hist + scan), for callers that scatter the points
// into a layout of their own.  nranges = sp.range0[ncat].
cudaError_t launch_sort_offsets_f32(const SortParams& sp, cudaStream_t st) {
    const int64_t nr = sp.range0[sp.prep.ncat];
    if (nr == 0) return cudaSuccess;
    sort_hist_kernel<float><<<(unsigned)nr, 256, 0, st>>>(sp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sort_scan_kernel<<<sp.prep.nfield, SORT_BUCKETS, 0, st>>>(sp);
    return cudaGetLastError();
}

template <typename KernelT>
cudaError_t configure_once(KernelT kern, int threads, size_t smem, int* occ_out) {
    return configure_kernel(reinterpret_cast<const void*>(kern), threads, smem, occ_out);
}

template <typename Tr, int K, int W>
size_t analysis_smem_bytes(int lmax) {
    const int accw = (lmax + 2 + 3) & ~3;
    return 128 + 2 * (size_t)Tr::NARR * 32 * K * Tr::ABYTES + (size_t)W * 16 * Tr::XSTRIDE * sizeof(typename Tr::real2) +
           (size_t)W * accw * sizeof(typename Tr::real2);
}

template <typename Tr, int K, int W, bool PACKED = false>
cudaError_t launch_analysis_t(const AnalysisParams& ap, int sm_count, cudaStream_t st, int* grid_out) {
    const size_t smem = analysis_smem_bytes<Tr, K, W>(ap.lmax);
    auto kern = analysis_kernel<Tr, K, W, PACKED>;
    int occ = 0;
    cudaError_t e = configure_once(kern, W * 32, smem, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)sm_count * occ;
    if (grid > ap.nunits) grid = ap.nunits;
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = (int)grid;
    kern<<<(int)grid, W * 32, smem, st>>>(ap);
    return cudaGetLastError();
}

// FP32 variants (k32): 8, 12, 16 = scalar FMAs with that many points per lane,
// 4 warps per CTA, one order pair per warp; 116 = 16 points per lane in packed
// f32x2 pairs (the default); 108 = grouped kernel (K = 8, 4 groups of 4 warps
// sharing accumulator rows, 1024-point tiles).  FP64 uses K = 4.
int analysis_tile_points(int prec_is_f64, int k32) {
    if (prec_is_f64) return 32 * 4;
    if (k32 == 108) return 32 * 8 * 4;
    if (k32 == 116) return 32 * 16;
    return 32 * k32;
}

// shared memory one CTA of the analysis launch needs at this lmax (the per-warp
// accumulator rows grow with lmax)
size_t analysis_smem_need(int prec_is_f64, int k32, int lmax) {
    if (prec_is_f64) return analysis_smem_bytes<TraitsF64, 4, 4>(lmax);
    switch (k32) {
        case 8: return analysis_smem_bytes<TraitsF32, 8, 4>(lmax);
        case 12: return analysis_smem_bytes<TraitsF32, 12, 4>(lmax);
        case 108: return analysis_f32g_smem_bytes<8, 4, 4>(lmax);
        default: return analysis_smem_bytes<TraitsF32, 16, 4>(lmax);
    }
}

cudaError_t launch_analysis(const AnalysisParams& ap, int prec_is_f64, int k32, int sm_count, cudaStream_t st,
                            int* grid) {
    if (prec_is_f64) return launch_analysis_t<TraitsF64, 4, 4>(ap, sm_count, st, grid);
    switch (k32) {
        case 8: return launch_analysis_t<TraitsF32, 8, 4>(ap, sm_count, st, grid);
        case 12: return launch_analysis_t<TraitsF32, 12, 4>(ap, sm_count, st, grid);
        case 116: return launch_analysis_t<TraitsF32, 16, 4, true>(ap, sm_count, st, grid);
        case 108: return launch_analysis_f32g<8, 4, 4>(ap, sm_count, st, grid);
        default: return launch_analysis_t<TraitsF32, 16, 4>(ap, sm_count, st, grid);
    }
}

cudaError_t launch_reduce(const ReduceParams& rp, cudaStream_t st) {
    reduce_kernel<<<1024, 256, 0, st>>>(rp);
    return cudaGetLastError();
}

}  // namespace psht
