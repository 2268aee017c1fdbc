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
// three-term recurrence in l (App. A, rewritten for lambda) runs for
// l = m+2..lmax in the rescaled variable mu_l = lambda_l / gamma_l:
//   mu_l = alpha_l x mu_{l-1} - mu_{l-2}
// (gamma_l = B_l gamma_{l-2}, alpha_l = A_l gamma_{l-1}/gamma_l, with A_l, B_l
// the lambda-form coefficients), i.e. one multiply and one FMA per step.  The
// per-(l, m) factor gamma is applied once, in FP64, when chunks are reduced.
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

namespace psht {

// ====================================================================
//                           point preparation
// ====================================================================
// FP32 layout (6 arrays of 4 bytes, stride ntot):
//   0 x, 1 coeff*w, 2 log2 sin(theta) hi, 3 lo, 4 turn[63:32], 5 turn[31:0]
// FP64 layout (4 arrays of 8 bytes): 0 x, 1 coeff*w, 2 log2 sin(theta), 3 turn
__device__ __forceinline__ uint64_t phi_to_turn(double ph) {
    double t = ph * (1.0 / (2.0 * CUDART_PI));
    t -= floor(t);
    if (!(t >= 0.0 && t < 1.0)) t = 0.0;
    return __double2ull_rn(t * 18446744073709551616.0);
}

template <typename T>
__device__ __forceinline__ void prep_one(const PrepParams& p, int64_t j, T x, T ph, T w, double coeff) {
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
        for (int64_t i = i0; i < c.n; i += stride) prep_one<T>(p, c.dst + i, xs[i], ps[i], ws[i], c.coeff);
    } else {
        const int f = seg - p.ncat;
        for (int64_t i = i0; i < p.pad_n[f]; i += stride) prep_one<T>(p, p.pad_off[f] + i, T(0), T(0), T(0), 0.0);
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
        const float lh = tf[2 * P + i], ll = tf[3 * P + i];
        const float mf = (float)m;
        // e = log2 c_m + m (lh + ll), carried as a float pair
        const float pr = mf * lh;
        float pe = fmaf(mf, lh, -pr);
        pe = fmaf(mf, ll, pe);
        f2 s = two_sum(pr, lch);
        f2 e = fast_two_sum(s.hi, s.lo + pe + lcl);
        // A point at a pole (sin theta = 0, log2 stored as -1e30) has
        // lambda_mm = 0 for m > 0: it is marked dead for good (E at the floor,
        // zero mantissa).  Every other point has |e| < 5e4.
        const bool pole = e.hi < -1.0e7f;
        const float Ef = pole ? -1048576.f : fminf(0.f, ceilf((e.hi - (float)CE) * (1.0f / SB)));
        E = (int)Ef;
        const float eh = pole ? 0.f : e.hi - (float)SB * Ef;
        f2 ep = fast_two_sum(eh, pole ? 0.f : e.lo);
        const float n = floorf(ep.hi);
        const float fr = (ep.hi - n) + ep.lo;
        mant = pole ? 0.f : ldexpf(exp2f(fr), (int)n);
        if (m & 1) mant = -mant;
        phase(tile, P, i, m, cs, sn);
    }
    __device__ static __forceinline__ void phase(const uint32_t* tile, int P, int i, int m, float& cs, float& sn) {
        const uint32_t t = (uint32_t)m * tile[4 * P + i] + __umulhi((uint32_t)m, tile[5 * P + i]);
        const float y = (float)(int32_t)t * 0x1p-31f;  // turns * 2 in [-1, 1)
        sincospif(y, &sn, &cs);
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
        p1[k] = real(0);   // mu_{m-1}
        p2[k] = -mant;     // mu_{m-2}: with alpha_m = 0 the first step gives mu_m = mant
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
                    const real mu = fma(av[j], x[k] * p1[k], -p2[k]);
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
                    const real mu = fma(av[j], x[k] * p1[k], -p2[k]);
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
template <typename Tr, int K, int W>
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
                if (threadIdx.x == 0) {
                    atomicOr(p.err, ERR_TIMEOUT);
                    if (t + 1 < ntiles) mbar_wait_bounded(&bars[b ^ 1], b ? parity0 : parity1);
                }
                return;
            }
            const uint32_t* tile = reinterpret_cast<const uint32_t*>(tiles + b * TILE_BYTES);
            if (active) {
                // one inlined copy of the column body, run for both orders of the pair
                for (int c = 0; c < (single ? 1 : 2); ++c) {
                    analysis_column<Tr, K>(tile, P, c ? mb : ma, L, c ? alpha_b : alpha_a, c ? lcb : lca,
                                           c ? lclb : lcla, my_acc + (c ? lena : 0), my_xb, lane);
                }
                if (t == ntiles - 1 || (t + 1) % p.flush_tiles == 0) {
                    flush_acc<Tr>(my_acc, lena, lenb, ma, mb, L, slot, first_flush, lane);
                    first_flush = false;
                }
            }
            __syncthreads();
        }
    }
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

template <typename Tr, int K, int W>
size_t analysis_smem_bytes(int lmax) {
    const int accw = (lmax + 2 + 3) & ~3;
    return 128 + 2 * (size_t)Tr::NARR * 32 * K * Tr::ABYTES + (size_t)W * 16 * Tr::XSTRIDE * sizeof(typename Tr::real2) +
           (size_t)W * accw * sizeof(typename Tr::real2);
}

template <typename Tr, int K, int W>
cudaError_t launch_analysis_t(const AnalysisParams& ap, int sm_count, cudaStream_t st, int* grid_out) {
    const size_t smem = analysis_smem_bytes<Tr, K, W>(ap.lmax);
    auto kern = analysis_kernel<Tr, K, W>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, W * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)sm_count * occ;
    if (grid > ap.nunits) grid = ap.nunits;
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = (int)grid;
    kern<<<(int)grid, W * 32, smem, st>>>(ap);
    return cudaGetLastError();
}

// FP32 points per lane (K): 8, 12 or 16 (tile = 32 K points); FP64 uses K = 4.
int analysis_tile_points(int prec_is_f64, int k32) { return prec_is_f64 ? 32 * 4 : 32 * k32; }

cudaError_t launch_analysis(const AnalysisParams& ap, int prec_is_f64, int k32, int sm_count, cudaStream_t st,
                            int* grid) {
    if (prec_is_f64) return launch_analysis_t<TraitsF64, 4, 4>(ap, sm_count, st, grid);
    switch (k32) {
        case 8: return launch_analysis_t<TraitsF32, 8, 4>(ap, sm_count, st, grid);
        case 12: return launch_analysis_t<TraitsF32, 12, 4>(ap, sm_count, st, grid);
        default: return launch_analysis_t<TraitsF32, 16, 4>(ap, sm_count, st, grid);
    }
}

cudaError_t launch_reduce(const ReduceParams& rp, cudaStream_t st) {
    reduce_kernel<<<1024, 256, 0, st>>>(rp);
    return cudaGetLastError();
}

}  // namespace psht
