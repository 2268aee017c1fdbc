// spin2.cu -- spin-2 (shear) transform of weighted point catalogs: E_lm, B_lm
// of the field (g1, g2) carried by the points (the paper's named
// generalisation to fields of non-zero spin, Sec. 4).
//
//   _{+-2}a_lm = sum_i w_i (g1 +- i g2)_i _{+-2}Y*_lm(n_i),
//   E_lm = -(_{2}a_lm + _{-2}a_lm)/2,   B_lm = i (_{2}a_lm - _{-2}a_lm)/2,
//   _{+2}Y*_lm = lambda_lm(x) e^{-i m phi},  _{-2}Y*_lm = lambda^-_lm(x) e^{-i m phi},
//   lambda_lm = sqrt((2l+1)/4pi) d^l_{m,-2}(theta),
//   lambda^-_lm(x) = sqrt((2l+1)/4pi) d^l_{m,+2}(theta) = (-1)^(l+m) lambda_lm(-x).
//
// The last identity (d at pi - theta) lets one recurrence serve both spins:
// each point is carried as the f32x2 pair (lambda(x), lambda(-x)) through
// the same coefficients, and the sign (-1)^(l+m) is applied to the second
// component's sums at the end.  Recurrence in l at fixed m (Wigner's d,
// written for lambda), from the seed at l0 = max(m, 2):
//   lambda_{l+1} = (A_l x + B_l) lambda_l - C_l lambda_{l-1}
//   seed = (-1)^m sqrt((2 l0 + 1)/4pi) sqrt((2 l0)! / ((l0+k)! (l0-k)!))
//          cos^|m-2|(theta/2) sin^(m+2)(theta/2),  k = -2 (m >= 2) or -m,
// taken in log2 (FP32 hi + lo) with the same exponent blocks as the scalar
// path.  As for the scalar path, the recurrence runs in a rescaled,
// sign-folded variable tau_l = lambda_l / (g_l eps_l) with g_{l+1} = C_l g_{l-1}
// (g = 1 at l0, l0 + 1) and eps_{l+1} = -eps_{l-1}, so that
//   tau_{l+1} = (A'_l x + B'_l) tau_l + tau_{l-1},
//   A'_l, B'_l = (A_l, B_l) g_l eps_l / (g_{l+1} eps_{l+1}),
// and g_l eps_l multiplies the FP32 row sums when they are added into the
// FP64 slots.  Per point and step: t = A' (x, -x) + B', tau = t p1 + p2, and
// two accumulations (re of both spins, im of both spins): four packed f32x2
// FMAs.
//
// Points are laid out per field in |x|-bucket order (as for the scalar
// path), so warps whose points are all still below the FP32 range skip the
// accumulation.  Work: a unit is (order m, chunk of points of one field); a CTA of 4 warps
// takes units from a global counter (largest l-range first).  Each warp runs
// 256 points (8 per lane) of a round of 1024; per 16 steps a warp reduces its
// lanes by a shared-memory transpose, the four warps' block sums are added in
// fixed order into the unit's FP32 row, and the row is added into the unit's
// FP64 slot every 16 rounds.  A reduction over chunks in fixed order then
// forms E and B.  Deterministic run to run.
#include "common.cuh"
#include "pointsht.h"

#include <math_constants.h>

#include <algorithm>
#include <cstring>

namespace psht {

constexpr int S2_NARR = 9;                     // prepared arrays
constexpr int S2_K = 8;                        // points per lane
constexpr int S2_WARPS = 4;                    // warps per CTA
constexpr int S2_TILE = 32 * S2_K;             // points per warp and round
constexpr int S2_ROUND = S2_WARPS * S2_TILE;   // points per CTA round
constexpr int S2_FLUSH = 16;                   // rounds per FP32 -> FP64 flush
constexpr int S2_XS = 33;                      // transpose row stride (float4)

struct S2Cat {
    const float* x;
    const float* phi;
    const float* w;
    const float* g1;
    const float* g2;
    int64_t n;
    int64_t dst;  // first prepared point
    double coeff;
};

struct S2PrepParams {
    int32_t ncat, nfield;
    int64_t ntot;
    S2Cat cat[PSHT_MAX_CATS];
    int64_t pad_off[PSHT_MAX_FIELDS];
    int64_t pad_n[PSHT_MAX_FIELDS];
    float* pts;
    unsigned* err;
};

struct S2Chunk {
    int64_t first;  // first prepared point
    int32_t n;      // points, a multiple of S2_ROUND
    int32_t field;
};

constexpr int S2_MAXCHUNK = 512;

struct S2Params {
    int32_t lmax, nchunk;
    int64_t ntot, nmodes, cstride;
    const float* pts;
    const float4* coef;   // [lmax+1][cstride] (A', A', B', B') per step (f32x2 operand pairs)
    const double* scale;  // [lmax+1][cstride] g_l eps_l per step
    const float4* seedc;  // [lmax+1] (log2 c hi, lo, |m-2|, m+2)
    double4* slots;       // [nchunk][nmodes] (re+, im+, re-, im-)
    int* counter;
    unsigned* err;
    S2Chunk chunk[S2_MAXCHUNK];
};

struct S2ReduceParams {
    int32_t lmax, nfield;
    int64_t nmodes;
    int32_t chunk0[PSHT_MAX_FIELDS + 1];  // chunks of field f: [chunk0[f], chunk0[f+1])
    const double4* slots;
    double2* E;
    double2* B;
};

__device__ __forceinline__ float2 s2_fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)),
          "l"(reinterpret_cast<unsigned long long&>(c)));
    return d;
}
__device__ __forceinline__ float2 s2_mul2(float2 a, float2 b) {
    float2 d;
    asm("mul.rn.f32x2 %0, %1, %2;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)));
    return d;
}
__device__ __forceinline__ float2 s2_add2(float2 a, float2 b) {
    float2 d;
    asm("add.rn.f32x2 %0, %1, %2;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)));
    return d;
}

// ------------------------------------------------------------ preparation --
// FP32 layout (9 arrays of ntot): 0 x, 1/2 log2 cos(theta/2) hi/lo,
// 3/4 log2 sin(theta/2) hi/lo, 5/6 turn hi/lo, 7 coeff w g1, 8 coeff w g2.
__device__ __forceinline__ void s2_prep_one(const S2PrepParams& p, int64_t j, float x, float ph, float w, float g1,
                                            float g2, double coeff) {
    const bool ok = isfinite(x) && isfinite(ph) && isfinite(w) && isfinite(g1) && isfinite(g2) && fabsf(x) <= 1.f;
    if (!ok) {
        atomicOr(p.err, ERR_RANGE);
        x = ph = w = g1 = g2 = 0.f;
    }
    const double xd = (double)x;
    const double c2 = 0.5 * (1.0 + xd), s2 = 0.5 * (1.0 - xd);  // cos^2, sin^2 of theta/2
    const double lc = c2 > 0.0 ? 0.5 * log2(c2) : -1.0e30;
    const double ls = s2 > 0.0 ? 0.5 * log2(s2) : -1.0e30;
    const uint64_t turn = phi_to_turn((double)ph);
    const int64_t N = p.ntot;
    float* b = p.pts;
    uint32_t* bu = reinterpret_cast<uint32_t*>(p.pts);
    const float lch = (float)lc, lsh = (float)ls;
    b[j] = x;
    b[N + j] = lch;
    b[2 * N + j] = (float)(lc - (double)lch);
    b[3 * N + j] = lsh;
    b[4 * N + j] = (float)(ls - (double)lsh);
    bu[5 * N + j] = (uint32_t)(turn >> 32);
    bu[6 * N + j] = (uint32_t)(turn & 0xffffffffu);
    b[7 * N + j] = (float)(coeff * (double)w * (double)g1);
    b[8 * N + j] = (float)(coeff * (double)w * (double)g2);
}

__global__ void s2_prep_kernel(const __grid_constant__ S2PrepParams p) {
    const int seg = blockIdx.y;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (seg < p.ncat) {
        const S2Cat& c = p.cat[seg];
        for (int64_t i = i0; i < c.n; i += stride)
            s2_prep_one(p, c.dst + i, c.x[i], c.phi[i], c.w[i], c.g1[i], c.g2[i], c.coeff);
    } else {
        const int f = seg - p.ncat;
        for (int64_t i = i0; i < p.pad_n[f]; i += stride) s2_prep_one(p, p.pad_off[f] + i, 0.f, 0.f, 0.f, 0.f, 0.f, 0.0);
    }
}

// Points of a field in |x|-bucket order (the scalar path's counting sort:
// bucket offsets from its hist + scan, then this scatter), so that the 256
// points of a warp cross into the FP32 range at nearly the same l and whole
// warps below range skip the accumulation.  The order changes only the
// summation order; ranks within a bucket follow the input order.
__global__ void __launch_bounds__(256) s2_scatter_kernel(const __grid_constant__ SortParams sp,
                                                         const __grid_constant__ S2PrepParams p) {
    __shared__ int64_t next[SORT_BUCKETS];
    __shared__ int wcnt[8][SORT_BUCKETS];
    const int r = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = threadIdx.x; b < SORT_BUCKETS; b += blockDim.x) next[b] = sp.hist[(int64_t)r * SORT_BUCKETS + b];
    int c = 0;
    while (c + 1 < sp.prep.ncat && sp.range0[c + 1] <= r) ++c;
    const int64_t i0 = (int64_t)(r - sp.range0[c]) * SORT_RANGE;
    const int64_t i1 = min(p.cat[c].n, i0 + SORT_RANGE);
    __syncthreads();
    if (i0 >= i1) return;
    const S2Cat& cd = p.cat[c];
    for (int64_t base = i0; base < i1; base += 256) {
        for (int b = lane; b < SORT_BUCKETS; b += 32) wcnt[warp][b] = 0;
        __syncwarp();
        const int64_t i = base + threadIdx.x;
        const bool valid = i < i1;
        const float x = valid ? cd.x[i] : 0.f;
        const int bk = valid ? x_bucket((double)x) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, bk);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[warp][bk] = __popc(peers);
        __syncthreads();
        if (valid) {
            int64_t dst = next[bk] + rank;
            for (int w = 0; w < warp; ++w) dst += wcnt[w][bk];
            s2_prep_one(p, dst, x, cd.phi[i], cd.w[i], cd.g1[i], cd.g2[i], cd.coeff);
        }
        __syncthreads();
        for (int b = threadIdx.x; b < SORT_BUCKETS; b += blockDim.x) {
            int t = 0;
            for (int w = 0; w < 8; ++w) t += wcnt[w][b];
            next[b] += t;
        }
        __syncthreads();
    }
}

cudaError_t launch_sort_offsets_f32(const SortParams& sp, cudaStream_t st);  // analysis.cu

// Recurrence coefficients, row scales and seed constants, FP64 (the
// coefficients then rounded once).  Step q of order m produces tau_{l0+q}:
// q = 0 is the seed (p1 = 0, p2 = seed: tau = t 0 + p2), step q >= 1 applies
// the coefficients of l = l0 + q - 1.  One thread per order (g is a running
// product along l); entries past the column are zero.
__global__ void s2_coef_kernel(int L, int64_t cstride, float4* __restrict__ coef, double* __restrict__ scale,
                               float4* __restrict__ seedc) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > L) return;
    const int l0 = max(m, 2);
    const int len = L - l0 + 1;
    const double mm = (double)m * m, nn = 4.0;
    float4* cm = coef + (int64_t)m * cstride;
    double* sm = scale + (int64_t)m * cstride;
    double g2 = 1.0, g1 = 1.0;  // g eps of l - 1 and l (signed)
    for (int64_t q = 0; q < cstride; ++q) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        double sc = 0.0;
        if (q == 0 && len > 0) {
            sc = 1.0;
        } else if (q < len) {
            const double l = (double)(l0 + q - 1);
            const double r1 = sqrt(((l + 1) * (l + 1) - mm) * ((l + 1) * (l + 1) - nn));
            const double qq = sqrt((2 * l + 3) * (2 * l + 1));
            const double A = qq * (l + 1) / r1;
            const double B = 2.0 * qq * (double)m / (l * r1);  // -qq m n / (l R), n = -2
            // g eps of l + 1: 1 at l0 + 1, else -C_l (g eps of l - 1)
            const double gn = q == 1 ? 1.0
                                     : -(sqrt((2 * l + 3) / (2 * l - 1)) * (l + 1) * sqrt((l * l - mm) * (l * l - nn)) /
                                         (l * r1)) * g2;
            const double f = g1 / gn;
            const float a = (float)(A * f), b = (float)(B * f);
            v = make_float4(a, a, b, b);
            sc = gn;
            g2 = g1;
            g1 = gn;
        }
        cm[q] = v;
        sm[q] = sc;
    }
    const int k = m >= 2 ? -2 : -m;
    const double lg = 0.5 * log2((2.0 * l0 + 1.0) / (4.0 * CUDART_PI)) +
                      0.5 * (lgamma(2.0 * l0 + 1.0) - lgamma((double)(l0 + k) + 1.0) - lgamma((double)(l0 - k) + 1.0)) /
                          CUDART_LN2;
    const float hi = (float)lg;
    seedc[m] = make_float4(hi, (float)(lg - (double)hi), (float)(l0 + k), (float)(l0 - k));
}

// log2 of the seed magnitude c + pc a + ps b (a, b = log2 cos, log2 sin of the
// half angle as hi + lo) with compensated products, then the mantissa and
// exponent block (value = mant 2^(64 E), E <= 0) as for the scalar seed.
__device__ __forceinline__ void s2_seed(float4 sc, float ah, float al, float bh, float bl, bool neg, float& mant,
                                        int& E) {
    const float pc = sc.z, ps = sc.w;
    const bool pole = (pc > 0.f && ah < -1.0e29f) || (ps > 0.f && bh < -1.0e29f);
    const float pa = pc * ah;
    float ea = fmaf(pc, ah, -pa);
    ea = fmaf(pc, al, ea);
    const float pb = ps * bh;
    float eb = fmaf(ps, bh, -pb);
    eb = fmaf(ps, bl, eb);
    const f2 s1 = two_sum(pa, pb);
    const f2 s2 = two_sum(s1.hi, sc.x);
    const f2 e = fast_two_sum(s2.hi, s2.lo + s1.lo + ea + eb + sc.y);
    const float Ef =
        pole ? -1048576.f : fminf(0.f, ceilf((e.hi - (float)F32Scale::CHECK_EXP) * (1.0f / F32Scale::SCALE_BITS)));
    E = (int)Ef;
    const float eh = pole ? 0.f : e.hi - (float)F32Scale::SCALE_BITS * Ef;
    const f2 ep = fast_two_sum(eh, pole ? 0.f : e.lo);
    const float n = floorf(ep.hi);
    const float fr = (ep.hi - n) + ep.lo;
    mant = pole ? 0.f : ldexpf(exp2f(fr), (int)n);
    if (neg) mant = -mant;
}

// weights of a point for order m: (W+ re, W- re), (W+ im, W- im) with
// W+- = coeff w (g1 +- i g2) e^{-i m phi}
__device__ __forceinline__ void s2_weights(int m, uint32_t thi, uint32_t tlo, float g1, float g2, float2& wr,
                                           float2& wi) {
    float cs, sn;
    phase_f32(m, thi, tlo, cs, sn);
    const float c = cs, s = -sn;
    wr = make_float2(g1 * c - g2 * s, g1 * c + g2 * s);
    wi = make_float2(g1 * s + g2 * c, g1 * s - g2 * c);
}

__global__ void __launch_bounds__(S2_WARPS * 32, 3) s2_analysis_kernel(const __grid_constant__ S2Params p) {
    extern __shared__ float4 s2_smem[];
    const int L = p.lmax;
    float4* acc = s2_smem;                            // [L + 17] row of the current unit, index l - l0
    float4* stage = acc + (L + 17);                   // [2][S2_WARPS][16], double-buffered
    float4* xb = stage + 2 * S2_WARPS * 16 + (threadIdx.x >> 5) * 16 * S2_XS;  // this warp's [16][S2_XS]
    // the unit index lives in dynamic shared memory too (no static shared
    // memory, so the launch may use the device's whole opt-in size)
    int& unit_s = *reinterpret_cast<int*>(stage + 2 * S2_WARPS * 16 + S2_WARPS * 16 * S2_XS);
    // [2][16] recurrence coefficients of a block, copied (cp.async) during the
    // previous block and completed before that block's barrier
    float4* cst = stage + 2 * S2_WARPS * 16 + S2_WARPS * 16 * S2_XS + 1;
    int cbuf = 0;
    auto cstage = [&](const float4* src, int b) {
        if (threadIdx.x < 16) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(cst + b * 16 + threadIdx.x)),
                         "l"(src + threadIdx.x) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    int sbuf = 0;  // stage buffer of the next block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t N = p.ntot;
    const float* X = p.pts;
    const uint32_t* XU = reinterpret_cast<const uint32_t*>(p.pts);
    const int64_t nunits = (int64_t)(L + 1) * p.nchunk;

    for (;;) {
        if (threadIdx.x == 0) unit_s = atomicAdd(p.counter, 1);
        __syncthreads();
        const int64_t u = unit_s;
        __syncthreads();
        if (u >= nunits) break;
        const int m = (int)(u / p.nchunk);
        const int ci = (int)(u - (int64_t)m * p.nchunk);
        const S2Chunk ch = p.chunk[ci];
        const int l0 = max(m, 2);
        const int len = L - l0 + 1;
        if (len <= 0) continue;
        const int nblk = (len + 15) >> 4;
        const float4* coef = p.coef + (int64_t)m * p.cstride;  // nblk * 16 <= cstride entries
        cstage(coef, cbuf);  // block 0 of the first round
        for (int q = threadIdx.x; q < nblk * 16; q += blockDim.x) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        const float4 sc = p.seedc[m];
        const double* rowscale = p.scale + (int64_t)m * p.cstride;
        double4* slot = p.slots + (int64_t)ci * p.nmodes + tri_base(m, L) + l0;
        const int nround = ch.n / S2_ROUND;
        bool first_flush = true;
        for (int r = 0; r < nround; ++r) {
            const int64_t tb = ch.first + (int64_t)r * S2_ROUND + warp * S2_TILE;
            float2 x2[S2_K], p1[S2_K], p2[S2_K], wr[S2_K], wi[S2_K];
            int Ep[S2_K], Em[S2_K];
            bool lane_neg = false, lane_dead = true;
#pragma unroll
            for (int k = 0; k < S2_K; ++k) {
                const int64_t i = tb + k * 32 + lane;
                const float x = X[i];
                const float ah = X[N + i], al = X[2 * N + i], bh = X[3 * N + i], bl = X[4 * N + i];
                float mp, mq;
                s2_seed(sc, ah, al, bh, bl, m & 1, mp, Ep[k]);  // at x
                s2_seed(sc, bh, bl, ah, al, m & 1, mq, Em[k]);  // at -x: half angles swap
                float2 a, b;
                s2_weights(m, XU[5 * N + i], XU[6 * N + i], X[7 * N + i], X[8 * N + i], a, b);
                wr[k] = make_float2(Ep[k] == 0 ? a.x : 0.f, Em[k] == 0 ? a.y : 0.f);
                wi[k] = make_float2(Ep[k] == 0 ? b.x : 0.f, Em[k] == 0 ? b.y : 0.f);
                x2[k] = make_float2(x, -x);
                p1[k] = make_float2(0.f, 0.f);
                p2[k] = make_float2(mp, mq);
                lane_neg |= (Ep[k] != 0) | (Em[k] != 0);
                lane_dead &= (Ep[k] != 0) & (Em[k] != 0);
            }
            bool any_neg = __any_sync(0xffffffffu, lane_neg);
            bool all_dead = __all_sync(0xffffffffu, lane_dead);
            for (int bk = 0; bk < nblk; ++bk) {
                const float4* cb = cst + cbuf * 16;
                // the next block's coefficients into the other buffer (read by every
                // warp before the previous block's barrier, so free)
                if (bk + 1 < nblk) cstage(coef + (bk + 1) * 16, cbuf ^ 1);
                else if (r + 1 < nround) cstage(coef, cbuf ^ 1);
                const bool skip = all_dead;
                if (skip) {
#pragma unroll 4
                    for (int j = 0; j < 16; ++j) {
                        const float4 c = cb[j];
                        const float2 A2 = make_float2(c.x, c.y), B2 = make_float2(c.z, c.w);
#pragma unroll
                        for (int k = 0; k < S2_K; ++k) {
                            const float2 t = s2_fma2(A2, x2[k], B2);
                            const float2 lam = s2_fma2(t, p1[k], p2[k]);
                            p2[k] = p1[k];
                            p1[k] = lam;
                        }
                    }
                } else {
#pragma unroll 4
                    for (int j = 0; j < 16; ++j) {
                        const float4 c = cb[j];
                        const float2 A2 = make_float2(c.x, c.y), B2 = make_float2(c.z, c.w);
                        float2 ra = make_float2(0.f, 0.f), ia = ra, rb = ra, ib = ra;
#pragma unroll
                        for (int k = 0; k < S2_K; ++k) {
                            const float2 t = s2_fma2(A2, x2[k], B2);
                            const float2 lam = s2_fma2(t, p1[k], p2[k]);
                            p2[k] = p1[k];
                            p1[k] = lam;
                            if (k & 1) {
                                rb = s2_fma2(lam, wr[k], rb);
                                ib = s2_fma2(lam, wi[k], ib);
                            } else {
                                ra = s2_fma2(lam, wr[k], ra);
                                ia = s2_fma2(lam, wi[k], ia);
                            }
                        }
                        const float2 rs = s2_add2(ra, rb), is = s2_add2(ia, ib);
                        xb[j * S2_XS + lane] = make_float4(rs.x, is.x, rs.y, is.y);
                    }
                }
                if (any_neg) {
                    bool reached = false;
                    lane_neg = false;
                    lane_dead = true;
#pragma unroll
                    for (int k = 0; k < S2_K; ++k) {
                        const bool nx = Ep[k] < 0 && fmaxf(fabsf(p1[k].x), fabsf(p2[k].x)) > 0x1p-61f;
                        const bool ny = Em[k] < 0 && fmaxf(fabsf(p1[k].y), fabsf(p2[k].y)) > 0x1p-61f;
                        const float2 f = make_float2(nx ? 0x1p-64f : 1.f, ny ? 0x1p-64f : 1.f);
                        p1[k] = s2_mul2(p1[k], f);
                        p2[k] = s2_mul2(p2[k], f);
                        Ep[k] += nx;
                        Em[k] += ny;
                        reached |= (nx & (Ep[k] == 0)) | (ny & (Em[k] == 0));
                        lane_neg |= (Ep[k] != 0) | (Em[k] != 0);
                        lane_dead &= (Ep[k] != 0) & (Em[k] != 0);
                    }
                    if (__any_sync(0xffffffffu, reached)) {
#pragma unroll
                        for (int k = 0; k < S2_K; ++k) {
                            const bool rx = Ep[k] == 0 && wr[k].x == 0.f && wi[k].x == 0.f;
                            const bool ry = Em[k] == 0 && wr[k].y == 0.f && wi[k].y == 0.f;
                            if (rx || ry) {
                                const int64_t i = tb + k * 32 + lane;
                                float2 a, b;
                                s2_weights(m, XU[5 * N + i], XU[6 * N + i], X[7 * N + i], X[8 * N + i], a, b);
                                if (rx) {
                                    wr[k].x = a.x;
                                    wi[k].x = b.x;
                                }
                                if (ry) {
                                    wr[k].y = a.y;
                                    wi[k].y = b.y;
                                }
                            }
                        }
                    }
                    any_neg = __any_sync(0xffffffffu, lane_neg);
                    all_dead = __all_sync(0xffffffffu, lane_dead);
                }
                // this warp's 16 block sums -> stage[warp]
                const int row = lane & 15, half = lane >> 4;
                float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
                if (!skip) {
                    __syncwarp();
                    // four independent partial sums, then a fixed tree
                    float4 t4[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) t4[c] = xb[row * S2_XS + half * 16 + c];
#pragma unroll
                    for (int c = 4; c < 16; ++c) {
                        const float4 v = xb[row * S2_XS + half * 16 + c];
                        t4[c & 3].x += v.x;
                        t4[c & 3].y += v.y;
                        t4[c & 3].z += v.z;
                        t4[c & 3].w += v.w;
                    }
                    s.x = (t4[0].x + t4[1].x) + (t4[2].x + t4[3].x);
                    s.y = (t4[0].y + t4[1].y) + (t4[2].y + t4[3].y);
                    s.z = (t4[0].z + t4[1].z) + (t4[2].z + t4[3].z);
                    s.w = (t4[0].w + t4[1].w) + (t4[2].w + t4[3].w);
                    s.x += __shfl_xor_sync(0xffffffffu, s.x, 16);
                    s.y += __shfl_xor_sync(0xffffffffu, s.y, 16);
                    s.z += __shfl_xor_sync(0xffffffffu, s.z, 16);
                    s.w += __shfl_xor_sync(0xffffffffu, s.w, 16);
                    __syncwarp();
                }
                // One barrier per block: the stage is double-buffered, and the
                // barrier of the next block orders this block's combine before
                // the buffer is written again.
                float4* sb = stage + sbuf * S2_WARPS * 16;
                if (half == 0) sb[warp * 16 + row] = s;
                asm volatile("cp.async.wait_group 0;" ::: "memory");  // the next block's coefficients
                __syncthreads();
                if (threadIdx.x < 64) {
                    const int q = threadIdx.x >> 2, comp = threadIdx.x & 3;
                    const float* st = reinterpret_cast<const float*>(sb);
                    const float v = ((st[(0 * 16 + q) * 4 + comp] + st[(1 * 16 + q) * 4 + comp]) +
                                     st[(2 * 16 + q) * 4 + comp]) + st[(3 * 16 + q) * 4 + comp];
                    reinterpret_cast<float*>(acc)[(bk * 16 + q) * 4 + comp] += v;
                }
                sbuf ^= 1;
                cbuf ^= 1;
            }
            if ((r + 1) % S2_FLUSH == 0 || r + 1 == nround) {
                __syncthreads();  // the last block's combine is in acc
                for (int q = threadIdx.x; q < len; q += blockDim.x) {
                    const float4 a = acc[q];
                    const double g = rowscale[q];
                    double4 s = first_flush ? make_double4(0.0, 0.0, 0.0, 0.0) : slot[q];
                    s.x += g * (double)a.x;
                    s.y += g * (double)a.y;
                    s.z += g * (double)a.z;
                    s.w += g * (double)a.w;
                    slot[q] = s;
                    acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                first_flush = false;
                __syncthreads();
            }
        }
    }
}

// E and B from the chunk slots: sum over a field's chunks in order, the
// (-1)^(l+m) of the -x component, then the E/B combination; zero for l < 2.
__global__ void s2_reduce_kernel(const __grid_constant__ S2ReduceParams p) {
    const int m = blockIdx.y, f = blockIdx.z;
    const int L = p.lmax;
    const int64_t base = tri_base(m, L);
    for (int l = m + blockIdx.x * blockDim.x + threadIdx.x; l <= L; l += gridDim.x * blockDim.x) {
        const int64_t idx = base + l;
        double ar = 0, ai = 0, br = 0, bi = 0;
        if (l >= 2) {
            for (int c = p.chunk0[f]; c < p.chunk0[f + 1]; ++c) {
                const double4 s = p.slots[(int64_t)c * p.nmodes + idx];
                ar += s.x;
                ai += s.y;
                br += s.z;
                bi += s.w;
            }
            if ((l + m) & 1) {
                br = -br;
                bi = -bi;
            }
        }
        p.E[(int64_t)f * p.nmodes + idx] = make_double2(-0.5 * (ar + br), -0.5 * (ai + bi));
        p.B[(int64_t)f * p.nmodes + idx] = make_double2(-0.5 * (ai - bi), 0.5 * (ar - br));
    }
}

// ------------------------------------------------------------- host side --
using S2Catalog = pointsht_shear_catalog;

struct S2Layout {
    int64_t ntot = 0, cstride = 0, nmodes = 0;
    int64_t off[PSHT_MAX_FIELDS] = {}, npad[PSHT_MAX_FIELDS] = {}, nfpts[PSHT_MAX_FIELDS] = {};
    int nchunk = 0;
    S2Chunk chunk[S2_MAXCHUNK];
    int32_t chunk0[PSHT_MAX_FIELDS + 1] = {};
    int64_t nranges = 0;
    size_t pts_off = 0, hist_off = 0, coef_off = 0, scale_off = 0, seed_off = 0, slots_off = 0, counter_off = 0,
           total = 0;
};

static size_t s2_up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Returns false when the points need more than S2_MAXCHUNK chunks.
static bool spin2_layout(int L, const S2Catalog* cats, int ncat, int nfield, S2Layout& lo) {
    lo = S2Layout();
    lo.nmodes = (int64_t)(L + 1) * (L + 2) / 2;
    lo.cstride = ((int64_t)(L + 1) + 15) / 16 * 16 + 16;
    for (int c = 0; c < ncat; ++c) lo.nfpts[cats[c].field] += cats[c].n;
    int64_t ntot = 0;
    for (int f = 0; f < nfield; ++f) {
        lo.npad[f] = (lo.nfpts[f] + S2_ROUND - 1) / S2_ROUND * S2_ROUND;
        lo.off[f] = ntot;
        ntot += lo.npad[f];
    }
    lo.ntot = ntot;
    // chunks of at most cmax points (a multiple of the round), cmax doubled
    // until the chunk table fits
    int64_t cmax = (int64_t)1 << 20;
    for (;;) {
        int n = 0;
        for (int f = 0; f < nfield; ++f) n += (int)((lo.npad[f] + cmax - 1) / cmax);
        if (n <= S2_MAXCHUNK) break;
        cmax *= 2;
        if (cmax > ((int64_t)1 << 40)) return false;
    }
    int n = 0;
    for (int f = 0; f < nfield; ++f) {
        lo.chunk0[f] = n;
        const int64_t k = (lo.npad[f] + cmax - 1) / cmax;
        if (k == 0) continue;
        const int64_t per = ((lo.npad[f] + k - 1) / k + S2_ROUND - 1) / S2_ROUND * S2_ROUND;
        for (int64_t s = 0; s < lo.npad[f]; s += per) {
            lo.chunk[n].first = lo.off[f] + s;
            lo.chunk[n].n = (int32_t)std::min<int64_t>(per, lo.npad[f] - s);
            lo.chunk[n].field = f;
            ++n;
        }
    }
    lo.chunk0[nfield] = n;
    lo.nchunk = n;
    size_t b = 0;
    lo.pts_off = b;
    b += s2_up256((size_t)ntot * S2_NARR * 4);
    for (int c = 0; c < ncat; ++c) lo.nranges += (cats[c].n + SORT_RANGE - 1) / SORT_RANGE;
    lo.hist_off = b;
    b += s2_up256((size_t)std::max<int64_t>(lo.nranges, 1) * SORT_BUCKETS * 8);
    lo.coef_off = b;
    b += s2_up256((size_t)(L + 1) * lo.cstride * 16);
    lo.scale_off = b;
    b += s2_up256((size_t)(L + 1) * lo.cstride * 8);
    lo.seed_off = b;
    b += s2_up256((size_t)(L + 1) * 16);
    lo.slots_off = b;
    b += s2_up256((size_t)std::max(n, 1) * lo.nmodes * 32);
    lo.counter_off = b;
    b += 256;
    lo.total = b;
    return true;
}

static size_t spin2_smem_bytes(int L) {
    return (size_t)(L + 17 + 2 * S2_WARPS * 16 + S2_WARPS * 16 * S2_XS + 1 + 2 * 16) * 16;
}

static cudaError_t launch_spin2(int L, const S2Catalog* cats, int ncat, int nfield, const S2Layout& lo, char* ws,
                                unsigned* err, int sm_count, double* E, double* B, cudaStream_t st) {
    cudaError_t e;
    if (lo.ntot > 0) {
        S2PrepParams pp;
        memset(&pp, 0, sizeof(pp));
        pp.ncat = ncat;
        pp.nfield = nfield;
        pp.ntot = lo.ntot;
        pp.pts = reinterpret_cast<float*>(ws + lo.pts_off);
        pp.err = err;
        int64_t run[PSHT_MAX_FIELDS] = {};
        int64_t nmax = 1;
        for (int c = 0; c < ncat; ++c) {
            const int f = cats[c].field;
            pp.cat[c] = S2Cat{static_cast<const float*>(cats[c].x), static_cast<const float*>(cats[c].phi),
                              static_cast<const float*>(cats[c].w), static_cast<const float*>(cats[c].g1),
                              static_cast<const float*>(cats[c].g2), cats[c].n, lo.off[f] + run[f], cats[c].coeff};
            run[f] += cats[c].n;
            nmax = std::max(nmax, cats[c].n);
        }
        for (int f = 0; f < nfield; ++f) {
            pp.pad_off[f] = lo.off[f] + lo.nfpts[f];
            pp.pad_n[f] = lo.npad[f] - lo.nfpts[f];
            nmax = std::max(nmax, pp.pad_n[f]);
        }
        // padding first (the catalogs' segments of the prep kernel are empty)
        S2PrepParams* pads = new S2PrepParams(pp);
        for (int c = 0; c < ncat; ++c) pads->cat[c].n = 0;
        const int64_t bx = std::min<int64_t>((nmax + 255) / 256, 1024);
        s2_prep_kernel<<<dim3((unsigned)bx, ncat + nfield), 256, 0, st>>>(*pads);
        delete pads;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (lo.nranges > 0) {
            SortParams* sp = new SortParams;
            memset(sp, 0, sizeof(SortParams));
            sp->prep.ncat = ncat;
            sp->prep.nfield = nfield;
            int64_t r = 0;
            for (int c = 0; c < ncat; ++c) {
                sp->prep.cat[c].x = cats[c].x;
                sp->prep.cat[c].n = cats[c].n;
                sp->prep.cat[c].field = cats[c].field;
                sp->range0[c] = r;
                r += (cats[c].n + SORT_RANGE - 1) / SORT_RANGE;
            }
            sp->range0[ncat] = r;
            for (int f = 0; f < nfield; ++f) sp->field_off[f] = lo.off[f];
            sp->hist = reinterpret_cast<int64_t*>(ws + lo.hist_off);
            e = launch_sort_offsets_f32(*sp, st);
            if (e == cudaSuccess) {
                s2_scatter_kernel<<<(unsigned)lo.nranges, 256, 0, st>>>(*sp, pp);
                e = cudaGetLastError();
            }
            delete sp;
            if (e != cudaSuccess) return e;
        }
    }
    float4* coef = reinterpret_cast<float4*>(ws + lo.coef_off);
    double* scale = reinterpret_cast<double*>(ws + lo.scale_off);
    float4* seedc = reinterpret_cast<float4*>(ws + lo.seed_off);
    s2_coef_kernel<<<(L + 1 + 63) / 64, 64, 0, st>>>(L, lo.cstride, coef, scale, seedc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    double4* slots = reinterpret_cast<double4*>(ws + lo.slots_off);
    if (lo.nchunk > 0 && L >= 2) {
        if ((e = cudaMemsetAsync(ws + lo.counter_off, 0, 256, st)) != cudaSuccess) return e;
        S2Params* kp = new S2Params;
        memset(kp, 0, sizeof(S2Params));
        kp->lmax = L;
        kp->nchunk = lo.nchunk;
        kp->ntot = lo.ntot;
        kp->nmodes = lo.nmodes;
        kp->cstride = lo.cstride;
        kp->pts = reinterpret_cast<const float*>(ws + lo.pts_off);
        kp->coef = coef;
        kp->scale = scale;
        kp->seedc = seedc;
        kp->slots = slots;
        kp->counter = reinterpret_cast<int*>(ws + lo.counter_off);
        kp->err = err;
        for (int c = 0; c < lo.nchunk; ++c) kp->chunk[c] = lo.chunk[c];
        const size_t smem = spin2_smem_bytes(L);
        int occ = 0;
        e = configure_kernel((const void*)s2_analysis_kernel, S2_WARPS * 32, smem, &occ);
        if (e == cudaSuccess && occ < 1) e = cudaErrorInvalidConfiguration;
        if (e == cudaSuccess) {
            const int64_t units = (int64_t)(L + 1) * lo.nchunk;
            const int64_t grid = std::min<int64_t>((int64_t)sm_count * occ, units);
            s2_analysis_kernel<<<(unsigned)grid, S2_WARPS * 32, smem, st>>>(*kp);
            e = cudaGetLastError();
        }
        delete kp;
        if (e != cudaSuccess) return e;
    }
    S2ReduceParams rp;
    memset(&rp, 0, sizeof(rp));
    rp.lmax = L;
    rp.nfield = nfield;
    rp.nmodes = lo.nmodes;
    for (int f = 0; f <= nfield; ++f) rp.chunk0[f] = lo.chunk0[f];
    rp.slots = slots;
    rp.E = reinterpret_cast<double2*>(E);
    rp.B = reinterpret_cast<double2*>(B);
    s2_reduce_kernel<<<dim3(4, L + 1, nfield), 256, 0, st>>>(rp);
    return cudaGetLastError();
}

// Workspace bytes for these catalogs, 0 if they need more chunks than the
// kernel parameters hold.
size_t spin2_workspace_bytes(int L, const pointsht_shear_catalog* cats, int ncat, int nfield) {
    S2Layout* lo = new S2Layout;
    const size_t t = spin2_layout(L, cats, ncat, nfield, *lo) ? lo->total : 0;
    delete lo;
    return t;
}

cudaError_t spin2_run(int L, const pointsht_shear_catalog* cats, int ncat, int nfield, void* ws, unsigned* err,
                      int sm_count, double* E, double* B, cudaStream_t st) {
    S2Layout* lo = new S2Layout;
    cudaError_t e = cudaErrorInvalidValue;
    if (spin2_layout(L, cats, ncat, nfield, *lo))
        e = launch_spin2(L, cats, ncat, nfield, *lo, static_cast<char*>(ws), err, sm_count, E, B, st);
    delete lo;
    return e;
}

}  // namespace psht
