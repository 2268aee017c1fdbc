// mixed.cu -- per-m contraction on tensor cores for several weight columns
// sharing one point set (POINTSHT_MIXED).
//
// For order m the transform of F weight columns is the contraction over points
//   a_m[l, f] = sum_i lambda_lm(x_i) W_m[i, f],  W_m[i, f] = w_f,i e^{-i m phi_i}
// (Eq. alm_def for each column).  lambda comes from the same FP32 sign-folded
// recurrence as the FP32 kernel (App. A); the contraction runs on the tensor
// cores in fp16 with a hi + lo split of both operands and FP32 accumulation:
//   a = W_hi lambda_hi + W_lo lambda_hi + W_hi lambda_lo   (lo x lo dropped,
// about 2^-22 of each product).
//
// Shape of one warp-level mma.sync.m16n8k16 (fp16 in, fp32 accumulate):
//   A (16 x 16) = W^T of one 16-point group: rows 0..7 = (field f, re/im) of
//                 W_hi (f = row/2), rows 8..15 = the same of W_lo; kept in
//                 registers for the whole column (W does not depend on l);
//   B (16 x 8)  = lambda of those 16 points at 8 consecutive l, staged as fp16
//                 hi and lo rows in shared memory and read with ldmatrix.trans;
//   D (16 x 8)  = sums over the warp's points; rows r and r + 8 are added.
// Only 8 l are staged at a time (4 KB per warp): the recurrence hands its
// values to the tensor cores every 8 steps.
//
// CTA: 8 warps on one order pair (m, lmax - m), tiles of 1024 points (128 per
// warp, 4 per lane as two f32x2 pairs).  Every 32 steps the warps' partial
// sums meet in shared memory and are added, in warp order, to the CTA's FP32
// accumulator rows (deterministic); rows are flushed to FP64 slots per chunk.
// Rounds of 8 steps are software-pipelined: the MMAs of round r - 1 are issued
// together with the recurrence of round r, and their sums stored one round
// later, so the tensor-core latency is covered by FP32 work.  Points still below the FP32
// range contribute nothing: their hi part is masked to zero and their lo part
// multiplied by zero in the split itself, and a warp whose points are all
// below range skips the split and the MMAs (its partial sums are exact zeros).
//
// Each weight column is scaled by a power of two (exact) so that its largest
// |w| lies in [1, 2): fp16 then holds every W without overflow, and the scale
// is undone in FP64 when the rows are flushed.
#include "common.cuh"

#include <cuda_fp16.h>

namespace psht {

constexpr int MX_WARPS = 8;
constexpr int MX_KQ = 4;                       // points per lane
constexpr int MX_PW = 32 * MX_KQ;              // points per warp (128)
constexpr int MX_P = MX_WARPS * MX_PW;         // points per tile (1024)
constexpr int MX_MAXCOL = 8;                   // weight columns per pass (kernels for 4 and 8)
constexpr int MX_NGEO = 5;                     // x, lsh, lsl, turn hi, turn lo
constexpr int MX_BLK = 32;                     // steps between CTA combines
// The near-pole form in column mode (catalog points next to a pole) is compiled
// out: its second code path slows the standard one (250 registers instead of
// 232; 12.1 -> 13.2 s at 8 columns on 1e7 points) for an error (6e-5 of the
// m = 0 column) already inside the mixed path's tolerance.  Table mode keeps it.
constexpr bool COLPOLE = false;

// ---------------------------------------------------------------- prep --
__device__ __forceinline__ void mx_write(const PrepColsParams& p, int64_t j, float x, float ph, int64_t src) {
    bool ok = isfinite(x) && isfinite(ph) && fabsf(x) <= 1.f;
    for (int f = 0; f < p.ncol && src >= 0; ++f) ok &= isfinite(p.w[(int64_t)f * p.n + src]);
    if (!ok) {
        atomicOr(p.err, ERR_RANGE);
        x = 0.f;
        ph = 0.f;
    }
    const double xd = (double)x;
    const double s2 = (1.0 - xd) * (1.0 + xd);
    const double ls = s2 > 0.0 ? 0.5 * log2(s2) : -1.0e30;
    const uint64_t turn = phi_to_turn((double)ph);
    float* b = reinterpret_cast<float*>(p.pts);
    const float lh = (float)ls;
    b[j] = x;
    b[p.ntot + j] = lh;
    b[2 * p.ntot + j] = (float)(ls - (double)lh);
    p.pts[3 * p.ntot + j] = (uint32_t)(turn >> 32);
    p.pts[4 * p.ntot + j] = (uint32_t)(turn & 0xffffffffu);
    for (int f = 0; f < p.ncol; ++f)
        b[(MX_NGEO + f) * p.ntot + j] = (ok && src >= 0) ? p.w[(int64_t)f * p.n + src] : 0.f;
}

// stable counting-sort scatter of the points into |x| order (offsets from
// the histogram / scan kernels of analysis.cu), plus the column maxima
__global__ void __launch_bounds__(256) mx_scatter_kernel(const __grid_constant__ PrepColsParams p) {
    __shared__ int64_t next[SORT_BUCKETS];
    __shared__ int wcnt[8][SORT_BUCKETS];
    const int r = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = threadIdx.x; b < SORT_BUCKETS; b += blockDim.x) next[b] = p.hist[(int64_t)r * SORT_BUCKETS + b];
    const int64_t i0 = (int64_t)r * SORT_RANGE, i1 = min(p.n, i0 + SORT_RANGE);
    __syncthreads();
    for (int64_t base = i0; base < i1; base += 256) {
        for (int b = lane; b < SORT_BUCKETS; b += 32) wcnt[warp][b] = 0;
        __syncwarp();
        const int64_t i = base + threadIdx.x;
        const bool valid = i < i1;
        const float x = valid ? p.x[i] : 0.f;
        const int bk = valid ? x_bucket((double)x) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, bk);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[warp][bk] = __popc(peers);
        __syncthreads();
        if (valid) {
            int64_t dst = next[bk] + rank;
            for (int w = 0; w < warp; ++w) dst += wcnt[w][bk];
            mx_write(p, dst, x, p.phi[i], i);
        }
        for (int f = 0; f < p.ncol; ++f) {
            const float v = valid ? fabsf(p.w[(int64_t)f * p.n + i]) : 0.f;
            const unsigned bits = isfinite(v) ? __float_as_uint(v) : 0u;
            const unsigned mx = __reduce_max_sync(0xffffffffu, bits);
            if (lane == 0 && mx) atomicMax(&p.colmax[f], mx);
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

__global__ void mx_pad_kernel(const __grid_constant__ PrepColsParams p) {
    for (int64_t j = p.n + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p.ntot;
         j += (int64_t)gridDim.x * blockDim.x)
        mx_write(p, j, 0.f, 0.f, -1);
}

// ------------------------------------------------------ PTX helpers --
__device__ __forceinline__ float2 mx_fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)),
          "l"(reinterpret_cast<unsigned long long&>(c)));
    return d;
}
__device__ __forceinline__ float2 mx_mul2(float2 a, float2 b) {
    float2 d;
    asm("mul.rn.f32x2 %0, %1, %2;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)));
    return d;
}
__device__ __forceinline__ float2 mx_add2(float2 a, float2 b) {
    float2 d;
    asm("add.rn.f32x2 %0, %1, %2;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)));
    return d;
}
// two f32 -> packed f16x2 with `a` in the low half, saturating to the finite range
__device__ __forceinline__ uint32_t mx_pack(float a, float b) {
    uint32_t r;
    asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}
__device__ __forceinline__ void mx_ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr)
                 : "memory");
}
__device__ __forceinline__ void mx_mma(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                       uint32_t b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// the same with a zero accumulator (first product of a chain)
__device__ __forceinline__ void mx_mma0(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                        uint32_t b0, uint32_t b1) {
    const float z = 0.f;
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%10,%10,%10};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(z));
}

// exponent e with max|w| * 2^-e in [1, 2) (0 for an all-zero column)
__device__ __forceinline__ int mx_col_exp(unsigned bits) {
    if (bits == 0u) return 0;
    const int e = ilogbf(__uint_as_float(bits));
    return e < -120 ? -120 : (e > 120 ? 120 : e);
}

// ------------------------------------------------------------ kernel --
// One round: 8 recurrence steps of the lane's 4 points (two f32x2 pairs; point
// k = 2 kp + {0: .x, 1: .y}).  With UF the point is carried as u = x - 1 and
// the product x sigma formed as fma(u, sigma, sigma): u keeps full relative
// precision next to the north pole, where x itself is within an FP32 spacing
// of 1 (the interpolated route's samples, whose u is computed in FP64);
// without UF (catalog points, whose x is an FP32 input) as x * sigma.  With
// SPLIT each value v is also split into
//   hi  = v with its low 13 mantissa bits cleared (exact in fp16), 0 below range
//   lo' = hi - v (the negated low part, exact in FP32, rounded to fp16), 0 below range
// packed as fp16 pairs of consecutive steps.
template <bool SPLIT, bool UF>
__device__ __forceinline__ void mx_round(const float4 (&alr)[4], const float2 (&u2)[2], float2 (&p1)[2],
                                         float2 (&p2)[2], const float2 (&nal)[2], const uint32_t (&mask)[4],
                                         uint32_t (&hi)[4][4], uint32_t (&lo)[4][4]) {
#pragma unroll
    for (int j2 = 0; j2 < 4; ++j2) {
        const float4 av4 = alr[j2];
        const float2 av0 = make_float2(av4.x, av4.y), av1 = make_float2(av4.z, av4.w);
        float2 s0[2];
#pragma unroll
        for (int kp = 0; kp < 2; ++kp) {
            const float2 sg = mx_fma2(av0, UF ? mx_fma2(u2[kp], p1[kp], p1[kp]) : mx_mul2(u2[kp], p1[kp]), p2[kp]);
            p2[kp] = p1[kp];
            p1[kp] = sg;
            s0[kp] = sg;
        }
#pragma unroll
        for (int kp = 0; kp < 2; ++kp) {
            const float2 sg = mx_fma2(av1, UF ? mx_fma2(u2[kp], p1[kp], p1[kp]) : mx_mul2(u2[kp], p1[kp]), p2[kp]);
            p2[kp] = p1[kp];
            p1[kp] = sg;
        }
        if (SPLIT) {
#pragma unroll
            for (int kp = 0; kp < 2; ++kp) {
                const float hax = __uint_as_float(__float_as_uint(s0[kp].x) & mask[2 * kp]);
                const float hay = __uint_as_float(__float_as_uint(s0[kp].y) & mask[2 * kp + 1]);
                const float hbx = __uint_as_float(__float_as_uint(p1[kp].x) & mask[2 * kp]);
                const float hby = __uint_as_float(__float_as_uint(p1[kp].y) & mask[2 * kp + 1]);
                const float2 la = mx_fma2(s0[kp], nal[kp], make_float2(hax, hay));
                const float2 lb = mx_fma2(p1[kp], nal[kp], make_float2(hbx, hby));
                hi[2 * kp][j2] = mx_pack(hax, hbx);
                hi[2 * kp + 1][j2] = mx_pack(hay, hby);
                lo[2 * kp][j2] = mx_pack(la.x, lb.x);
                lo[2 * kp + 1][j2] = mx_pack(la.y, lb.y);
            }
        }
    }
}

// The same round in the near-pole form (a warp of points next to one pole,
// orders m < pole_mmax): Reinsch's difference form of the recurrence in the
// smooth normalisation of the near-pole table, on u = |x| - 1: per step and
// pair c = a u + e, d = c y + d, y = y + d, with (p1, p2) holding (y, d).  y is
// the value that is split and staged; the step factor s_q sgn^q (q odd ? rho : 1)
// of the normalisation and the mirror is applied to the sums.
// alr: the round's table entries 0..3 (a, a, e, e); cv4: entries 4..7.
template <bool SPLIT>
__device__ __forceinline__ void mx_round_pole(const float4 (&alr)[4], const float4* __restrict__ cv4,
                                              const float2 (&u2)[2], float2 (&p1)[2], float2 (&p2)[2],
                                              const float2 (&nal)[2], const uint32_t (&mask)[4],
                                              uint32_t (&hi)[4][4], uint32_t (&lo)[4][4]) {
    // entries 0..3 were fetched a round ahead (alr); 4..7 are fetched two at a
    // time, each pair one step pair ahead of its use
    float4 cn0 = __ldg(cv4), cn1 = __ldg(cv4 + 1);
#pragma unroll
    for (int j2 = 0; j2 < 4; ++j2) {
        float4 ca, cb;
        if (j2 < 2) {
            ca = alr[2 * j2];
            cb = alr[2 * j2 + 1];
        } else {
            ca = cn0;
            cb = cn1;
            if (j2 == 2) {
                cn0 = __ldg(cv4 + 2);
                cn1 = __ldg(cv4 + 3);
            }
        }
        const float2 a0 = make_float2(ca.x, ca.y), e0 = make_float2(ca.z, ca.w);
        const float2 a1 = make_float2(cb.x, cb.y), e1 = make_float2(cb.z, cb.w);
        float2 s0[2];
#pragma unroll
        for (int kp = 0; kp < 2; ++kp) {
            const float2 c = mx_fma2(a0, u2[kp], e0);
            p2[kp] = mx_fma2(c, p1[kp], p2[kp]);
            p1[kp] = mx_add2(p1[kp], p2[kp]);
            s0[kp] = p1[kp];
        }
#pragma unroll
        for (int kp = 0; kp < 2; ++kp) {
            const float2 c = mx_fma2(a1, u2[kp], e1);
            p2[kp] = mx_fma2(c, p1[kp], p2[kp]);
            p1[kp] = mx_add2(p1[kp], p2[kp]);
        }
        if (SPLIT) {
#pragma unroll
            for (int kp = 0; kp < 2; ++kp) {
                const float hax = __uint_as_float(__float_as_uint(s0[kp].x) & mask[2 * kp]);
                const float hay = __uint_as_float(__float_as_uint(s0[kp].y) & mask[2 * kp + 1]);
                const float hbx = __uint_as_float(__float_as_uint(p1[kp].x) & mask[2 * kp]);
                const float hby = __uint_as_float(__float_as_uint(p1[kp].y) & mask[2 * kp + 1]);
                const float2 la = mx_fma2(s0[kp], nal[kp], make_float2(hax, hay));
                const float2 lb = mx_fma2(p1[kp], nal[kp], make_float2(hbx, hby));
                hi[2 * kp][j2] = mx_pack(hax, hbx);
                hi[2 * kp + 1][j2] = mx_pack(hay, hby);
                lo[2 * kp][j2] = mx_pack(la.x, lb.x);
                lo[2 * kp + 1][j2] = mx_pack(la.y, lb.y);
            }
        }
    }
}

// fp16 hi / lo of one float: hi = round-to-nearest fp16, lo = the remainder
__device__ __forceinline__ void mx_split_w(float v, float& h, float& l) {
    h = __half2float(__float2half_rn(v));
    l = v - h;
}

// NF = weight columns per pass (4 or 8).  NF = 4: A rows 0..7 = W_hi of fields
// 0..3 (re, im), rows 8..15 = W_lo of the same; per 16-point group
//   D1 += A . B_hi,   D2 += [W_hi; 0] . B_lo'
// and row g of the result is (D1 - D2)[g] + D1[g + 8].  NF = 8: rows 0..15 =
// fields 0..7 (re, im); A_hi and A_lo are separate fragments and
//   D1 += A_hi . B_hi + A_lo . B_hi,   D2 += A_hi . B_lo',   result D1 - D2.
template <int NF, bool UF>
__global__ void __launch_bounds__(MX_WARPS * 32, 1) analysis_mixed_kernel(const __grid_constant__ MixedParams p) {
    constexpr int NV = 2 * NF;                 // values per l: (field, re/im)
    constexpr int PS = NV + 4;                 // row stride of the partial sums (bank-conflict-free stores)
    constexpr int AR = NF == 4 ? 4 : 8;        // A registers per 16-point group
    constexpr int ITEMS = MX_BLK * NV / (MX_WARPS * 32);  // combine items per thread
    constexpr int ARR = MX_P * 4;              // bytes of one array in a tile
    const int narr = MX_NGEO + (p.vtab ? 0 : p.ncol);  // table mode: weights come from p.vtab
    const int L = p.lmax;

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    int64_t* s_unit = reinterpret_cast<int64_t*>(smem + 16);
    unsigned char* tile = smem + 128;
    uint4* stage = reinterpret_cast<uint4*>(tile + (MX_NGEO + NF) * ARR);  // [warp][plane][128]
    float2* phs = reinterpret_cast<float2*>(stage + MX_WARPS * 2 * MX_PW);  // [warp][128]
    float* part = reinterpret_cast<float*>(phs + MX_WARPS * MX_PW);         // [2][warp][32][PS]
    if ((int)blockIdx.x >= p.maxctas) return;
    float* accg = p.accg + (int64_t)blockIdx.x * p.accstride;               // [(L+2)][NV], this CTA's

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, c4 = lane & 3;
    const int qbase = warp * MX_PW;
    uint4* my_stage = stage + warp * 2 * MX_PW;
    float2* my_ph = phs + warp * MX_PW;
    const uint32_t ld_addr = smem_u32(my_stage) + (uint32_t)(((lane >> 4) * MX_PW + (lane & 15)) * 16);

    // fields of this lane's A rows and their column scales
    const int comp = g & 1;
    const int fa = g >> 1;
    const int fb = NF == 4 ? fa : 4 + (g >> 1);
    const float sca = fa < p.ncol ? ldexpf(1.f, -mx_col_exp(p.colmax[fa])) : 0.f;
    const float scb = fb < p.ncol ? ldexpf(1.f, -mx_col_exp(p.colmax[fb])) : 0.f;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t parity = 0;

    for (;;) {
        if (threadIdx.x == 0) s_unit[0] = (int64_t)atomicAdd(p.counter, 1);
        __syncthreads();
        const int64_t u = s_unit[0];
        if (u >= p.nunits) break;
        const int64_t r = u / p.npairs;
        const int pi = (int)(u - r * p.npairs);
        const int64_t pt0 = r * p.chunk;
        const int64_t npts = min(p.chunk, p.ntot - pt0);
        const int ntiles = (int)(npts / MX_P);
        const int ma = pi, mb = L - pi;
        const bool single = ma == mb;
        const int ncols = single ? 1 : 2;
        const int lena = L - ma + 1, lenb = single ? 0 : L - mb + 1;
        for (int i = threadIdx.x; i < (lena + lenb) * NV; i += blockDim.x) accg[i] = 0.f;
        bool first_flush = true;

        auto issue = [&](int t) {
            mbar_expect_tx(bar, narr * ARR);
            const int64_t first = pt0 + (int64_t)t * MX_P;
            for (int a = 0; a < MX_NGEO; ++a) bulk_g2s(tile + a * ARR, p.pts + (int64_t)a * p.ntot + first, ARR, bar);
            // weight arrays only in column mode (narr counts them); table mode reads p.vtab
            for (int f = 0; f < narr - MX_NGEO; ++f)
                bulk_g2s(tile + (MX_NGEO + f) * ARR, p.wcols + (int64_t)f * p.ntot + first, ARR, bar);
        };
        __syncthreads();  // s_unit read, accumulator rows zeroed
        if (threadIdx.x == 0 && ntiles > 0) issue(0);

        for (int t = 0; t < ntiles; ++t) {
            const bool ok = mbar_wait_bounded(bar, parity);
            parity ^= 1u;
            if (__syncthreads_or(!ok)) {
                // record the timeout and wait (bounded) for the copy in flight
                if (threadIdx.x == 0) {
                    atomicOr(p.err, ERR_TIMEOUT);
                    mbar_drain(bar, parity ^ 1u);
                }
                __syncthreads();
                return;
            }
            const float* tf = reinterpret_cast<const float*>(tile);
            const uint32_t* tu = reinterpret_cast<const uint32_t*>(tile);

            for (int col = 0; col < ncols; ++col) {
                const int m = col ? mb : ma;
                const int len = L - m + 1;
                float* cacc = accg + (col ? lena : 0) * NV;
                const float2* alpha2 = p.alpha2 + p.colstart[m];
                const float lch = p.log2c_hi[m], lcl = p.log2c_lo[m];
                // ---- per-point seed, phase and state (4 points per lane) ----
                float2 u2[2], p1[2], p2[2], nal[2];
                uint32_t mask[4];
                int E[4];
#pragma unroll
                for (int k = 0; k < MX_KQ; ++k) {
                    const int q = 32 * k + lane, i = qbase + q;
                    float mant, cs, sn;
                    seed_f32(m, tf[MX_P + i], tf[2 * MX_P + i], lch, lcl, mant, E[k]);
                    if (!p.vtab) {
                        phase_f32(m, tu[3 * MX_P + i], tu[4 * MX_P + i], cs, sn);
                        my_ph[q] = make_float2(cs, sn);
                    }
                    const float xv = tf[i];
                    const float na = E[k] == 0 ? -1.f : 0.f;
                    if (k & 1) {
                        u2[k >> 1].y = xv;
                        p2[k >> 1].y = mant;
                        p1[k >> 1].y = 0.f;
                        nal[k >> 1].y = na;
                    } else {
                        u2[k >> 1].x = xv;
                        p2[k >> 1].x = mant;
                        p1[k >> 1].x = 0.f;
                        nal[k >> 1].x = na;
                    }
                    mask[k] = E[k] == 0 ? 0xffffe000u : 0u;
                }
                // Near-pole form for orders m < pole_mmax when every point of the warp
                // lies next to one pole.  Table mode: the tile holds u = x - 1 of the
                // north samples (padding u = -1), x >= pole_x.  Column mode: the tile
                // holds x; every |x| >= pole_x with one sign sgn (the |x| order keeps the
                // signs apart there; padding has x = 0), and the recurrence runs on
                // u = |x| - 1, mirrored by sgn^q.
                bool pole = false;
                float sgn = 1.f;
                if (COLPOLE || UF) {
                    if (p.pole_ae != nullptr && m < p.pole_mmax) {
                        if (UF) {
                            const float umin = p.pole_x - 1.f;
                            pole = __all_sync(0xffffffffu, (u2[0].x >= umin) & (u2[0].y >= umin) &
                                                               (u2[1].x >= umin) & (u2[1].y >= umin));
                        } else {
                            const float px = p.pole_x;
                            const bool np = __all_sync(0xffffffffu, (u2[0].x >= px) & (u2[0].y >= px) &
                                                                        (u2[1].x >= px) & (u2[1].y >= px));
                            const bool sp = __all_sync(0xffffffffu, (u2[0].x <= -px) & (u2[0].y <= -px) &
                                                                        (u2[1].x <= -px) & (u2[1].y <= -px));
                            pole = np | sp;
                            sgn = np ? 1.f : -1.f;
                            if (pole) {
#pragma unroll
                                for (int kp = 0; kp < 2; ++kp)
                                    u2[kp] = make_float2(fabsf(u2[kp].x) - 1.f, fabsf(u2[kp].y) - 1.f);
                            }
                        }
                    }
                }
                const float4* pae = pole ? p.pole_ae + p.colstart[m] : nullptr;
                // step factor s_q sgn^q (q odd ? rho : 1) of the near-pole normalisation;
                // this lane's sums are of steps q = 2 c4 + (e & 1) (mod 4)
                const float rho = pole ? sgn * p.pole_rho[m] : 1.f;
                const float fac_even = pole ? ((c4 & 1) ? -1.f : 1.f) : 1.f;
                const float fac_odd = pole ? ((c4 & 1) ? -rho : rho) : 1.f;
                __syncwarp();
                // ---- A fragments ----
                uint32_t A[8][AR];
#pragma unroll
                for (int gi = 0; gi < 8; ++gi) {
                    float ha[4], la[4], hb[4], lb[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int q = 16 * gi + 2 * c4 + (e & 1) + (e >> 1) * 8;
                        float wa, wb = 0.f;
                        if (p.vtab) {
                            // table mode: column 6 fg + 3 half + {0: Vy^(m), 1: h Vd^(m-1),
                            // 2: h Vd^(m+1)} of the group is that of field fg's sample pair at this
                            // position (half 0 north, 1 south)
                            const int64_t node = pt0 + (int64_t)t * MX_P + qbase + q;
                            auto tab = [&](int c) {
                                const int gc = p.tcol0 + c, fg = gc / 6, c6 = gc - 6 * fg;
                                const int half = c6 >= 3, ty = c6 - 3 * half;
                                const float2* vt = p.vtab + (int64_t)fg * p.vtab_fstride;
                                float2 wt = make_float2(0.f, 0.f);
                                float f = 1.f;
                                if (ty == 0) {
                                    wt = vt[((int64_t)m * p.ntot + node) * 4 + 2 * half];
                                } else if (ty == 1 && m >= 1) {
                                    wt = vt[((int64_t)(m - 1) * p.ntot + node) * 4 + 2 * half + 1];
                                    f = p.vtab_h;
                                } else if (ty == 2 && m < L) {
                                    wt = vt[((int64_t)(m + 1) * p.ntot + node) * 4 + 2 * half + 1];
                                    f = p.vtab_h;
                                }
                                return (comp ? wt.y : wt.x) * f;
                            };
                            wa = fa < p.ncol ? tab(fa) * sca : 0.f;
                            if (NF == 8) wb = fb < p.ncol ? tab(fb) * scb : 0.f;
                        } else {
                            const float2 ph = my_ph[q];
                            const float trig = comp ? -ph.y : ph.x;
                            wa = fa < p.ncol ? tf[(MX_NGEO + fa) * MX_P + qbase + q] * sca * trig : 0.f;
                            if (NF == 8)
                                wb = fb < p.ncol ? tf[(MX_NGEO + fb) * MX_P + qbase + q] * scb * trig : 0.f;
                        }
                        mx_split_w(wa, ha[e], la[e]);
                        if (NF == 8) mx_split_w(wb, hb[e], lb[e]);
                    }
                    if (NF == 4) {
                        A[gi][0] = mx_pack(ha[0], ha[1]);
                        A[gi][1] = mx_pack(la[0], la[1]);
                        A[gi][2] = mx_pack(ha[2], ha[3]);
                        A[gi][3] = mx_pack(la[2], la[3]);
                    } else {
                        A[gi][0] = mx_pack(ha[0], ha[1]);
                        A[gi][1] = mx_pack(hb[0], hb[1]);
                        A[gi][2] = mx_pack(ha[2], ha[3]);
                        A[gi][3] = mx_pack(hb[2], hb[3]);
                        A[gi][AR / 2 + 0] = mx_pack(la[0], la[1]);
                        A[gi][AR / 2 + 1] = mx_pack(lb[0], lb[1]);
                        A[gi][AR / 2 + 2] = mx_pack(la[2], la[3]);
                        A[gi][AR / 2 + 3] = mx_pack(lb[2], lb[3]);
                    }
                }
                if (col == ncols - 1) {
                    // every warp has read the tile: fetch the next one behind this column
                    __syncthreads();
                    if (threadIdx.x == 0 && t + 1 < ntiles) issue(t + 1);
                }
                bool lane_neg = (E[0] | E[1] | E[2] | E[3]) != 0;
                bool any_neg = __any_sync(0xffffffffu, lane_neg);
                // a warp all of whose points are still below range contributes
                // exact zeros: it runs the recurrence only
                bool warp_alive = __any_sync(0xffffffffu, (E[0] == 0) | (E[1] == 0) | (E[2] == 0) | (E[3] == 0));
                const int nrounds = 4 * ((len + MX_BLK - 1) / MX_BLK);
                float D1[4], D2[4];
                float accv[ITEMS];
                // recurrence coefficients of the next round, loaded one round ahead:
                // 4 float4 per round, the (alpha, alpha) pairs of 8 steps, or the first
                // 4 near-pole entries (a, a, e, e)
                float4 aln[4];
                const float4* apf = pole ? pae : reinterpret_cast<const float4*>(alpha2);
                const int astride = pole ? 8 : 4;
#pragma unroll
                for (int j = 0; j < 4; ++j) aln[j] = __ldg(apf + j);
                // Rounds of 8 steps in a three-stage pipeline.  Iteration r8:
                //   store the sums of round r8-2 (its MMAs were issued one iteration ago),
                //   load the B fragments of round r8-1 and issue its MMAs in the same
                //   basic block as round r8's recurrence and split, so that the MMA
                //   latency is covered by FP32 work, then stage round r8.
                bool mm_prev = false;  // round r8-2 had its MMAs issued
                bool st_prev = false;  // round r8-1 is staged
                for (int r8 = 0; r8 < nrounds + 2; ++r8) {
                    if (r8 >= 2) {
                        // round r8-2: columns l = 8 (r8-2) + 2 c4 (+1) of this order
                        const int rp = r8 - 2;
                        float* pb = part + ((rp >> 2) & 1) * (MX_WARPS * MX_BLK * PS);
                        const int row = warp * MX_BLK + 8 * (rp & 3) + 2 * c4;
                        if (NF == 4) {
                            // columns 2 c4 (steps q even mod 2) and 2 c4 + 1 (odd); the step
                            // factors are 1 outside the near-pole form
                            pb[row * PS + g] = mm_prev ? ((D1[0] - D2[0]) + D1[2]) * fac_even : 0.f;
                            pb[(row + 1) * PS + g] = mm_prev ? ((D1[1] - D2[1]) + D1[3]) * fac_odd : 0.f;
                        } else if (pole) {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                pb[(row + (e & 1)) * PS + (e >> 1) * 8 + g] =
                                    mm_prev ? (D1[e] - D2[e]) * ((e & 1) ? fac_odd : fac_even) : 0.f;
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                pb[(row + (e & 1)) * PS + (e >> 1) * 8 + g] = mm_prev ? D1[e] - D2[e] : 0.f;
                        }
                        if ((rp & 3) == 3) {
                            // block rp/4 complete in every warp: add the warps'
                            // partial sums, in warp order
                            __syncthreads();
                            const int bk = rp >> 2;
                            const float* pbb = part + (bk & 1) * (MX_WARPS * MX_BLK * PS);
#pragma unroll
                            for (int j = 0; j < ITEMS; ++j) {
                                const int it = threadIdx.x + j * MX_WARPS * 32;
                                const int li = it / NV, v = it % NV;
                                const int q = MX_BLK * bk + li;
                                if (q < len) {
                                    float sacc = accv[j];
#pragma unroll
                                    for (int w = 0; w < MX_WARPS; ++w) sacc += pbb[(w * MX_BLK + li) * PS + v];
                                    cacc[q * NV + v] = sacc;
                                }
                            }
                        }
                    }
                    if ((r8 & 3) == 2 && r8 - 2 < nrounds) {
                        // accumulator rows of block (r8-2)/4, read ahead of its combine
#pragma unroll
                        for (int j = 0; j < ITEMS; ++j) {
                            const int it = threadIdx.x + j * MX_WARPS * 32;
                            const int q = MX_BLK * ((r8 - 2) >> 2) + it / NV;
                            accv[j] = q < len ? cacc[q * NV + it % NV] : 0.f;
                        }
                    }
                    const bool have = r8 < nrounds;
                    const bool act = have && warp_alive;
                    const bool mm = st_prev;
                    uint32_t bf[8][4];
                    if (mm) {
#pragma unroll
                        for (int gi = 0; gi < 8; ++gi)
                            mx_ldsm_x4_t(ld_addr + (uint32_t)(16 * gi * 16), bf[gi][0], bf[gi][1], bf[gi][2], bf[gi][3]);
                    }
                    __syncwarp();  // every lane has read the stage before it is rewritten
                    float4 alr[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) alr[j] = aln[j];
                    if (r8 + 1 < nrounds) {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            aln[j] = __ldg(apf + astride * (r8 + 1) + j);
                    }
                    uint32_t hi[4][4], lo[4][4];
                    auto mmas = [&]() {
#pragma unroll
                        for (int gi = 0; gi < 8; ++gi) {
                            if (NF == 4) {
                                if (gi == 0) {
                                    mx_mma0(D1, A[gi][0], A[gi][1], A[gi][2], A[gi][3], bf[gi][0], bf[gi][1]);
                                    mx_mma0(D2, A[gi][0], 0u, A[gi][2], 0u, bf[gi][2], bf[gi][3]);
                                } else {
                                    mx_mma(D1, A[gi][0], A[gi][1], A[gi][2], A[gi][3], bf[gi][0], bf[gi][1]);
                                    mx_mma(D2, A[gi][0], 0u, A[gi][2], 0u, bf[gi][2], bf[gi][3]);
                                }
                            } else {
                                if (gi == 0) {
                                    mx_mma0(D1, A[gi][0], A[gi][1], A[gi][2], A[gi][3], bf[gi][0], bf[gi][1]);
                                    mx_mma0(D2, A[gi][0], A[gi][1], A[gi][2], A[gi][3], bf[gi][2], bf[gi][3]);
                                } else {
                                    mx_mma(D1, A[gi][0], A[gi][1], A[gi][2], A[gi][3], bf[gi][0], bf[gi][1]);
                                    mx_mma(D2, A[gi][0], A[gi][1], A[gi][2], A[gi][3], bf[gi][2], bf[gi][3]);
                                }
                                mx_mma(D1, A[gi][AR / 2], A[gi][AR / 2 + 1], A[gi][AR / 2 + 2], A[gi][AR / 2 + 3],
                                       bf[gi][0], bf[gi][1]);
                            }
                        }
                    };
                    // (each form in its own branch, so that the MMAs and the round's
                    // FP32 work stay in one basic block)
                    if (pole) {
                        if (mm && act) {
                            mmas();
                            mx_round_pole<true>(alr, pae + 8 * r8 + 4, u2, p1, p2, nal, mask, hi, lo);
                        } else if (act) {
                            mx_round_pole<true>(alr, pae + 8 * r8 + 4, u2, p1, p2, nal, mask, hi, lo);
                        } else {
                            if (mm) mmas();
                            if (have) mx_round_pole<false>(alr, pae + 8 * r8 + 4, u2, p1, p2, nal, mask, hi, lo);
                        }
                    } else {
                        if (mm && act) {
                            mmas();
                            mx_round<true, UF>(alr, u2, p1, p2, nal, mask, hi, lo);
                        } else if (act) {
                            mx_round<true, UF>(alr, u2, p1, p2, nal, mask, hi, lo);
                        } else {
                            if (mm) mmas();
                            if (have) mx_round<false, UF>(alr, u2, p1, p2, nal, mask, hi, lo);
                        }
                    }
                    if (act) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            my_stage[32 * k + lane] = make_uint4(hi[k][0], hi[k][1], hi[k][2], hi[k][3]);
                            my_stage[MX_PW + 32 * k + lane] = make_uint4(lo[k][0], lo[k][1], lo[k][2], lo[k][3]);
                        }
                    }
                    __syncwarp();  // the stage is complete before the next iteration reads it
                    if (have && any_neg && (r8 & 1)) {
                        // rescale check every 16 steps (F32Scale: 2^64 blocks)
                        lane_neg = false;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            float& a = (k & 1) ? p1[k >> 1].y : p1[k >> 1].x;
                            float& b = (k & 1) ? p2[k >> 1].y : p2[k >> 1].x;
                            const bool nd = (E[k] < 0) & (fmaxf(fabsf(a), fabsf(b)) > 0x1p-61f);
                            const float sc = nd ? 0x1p-64f : 1.f;
                            a *= sc;
                            b *= sc;
                            E[k] += nd;
                            mask[k] = E[k] == 0 ? 0xffffe000u : 0u;
                            if (k & 1) nal[k >> 1].y = E[k] == 0 ? -1.f : 0.f;
                            else nal[k >> 1].x = E[k] == 0 ? -1.f : 0.f;
                            lane_neg |= E[k] != 0;
                        }
                        any_neg = __any_sync(0xffffffffu, lane_neg);
                        warp_alive = __any_sync(0xffffffffu, (E[0] == 0) | (E[1] == 0) | (E[2] == 0) | (E[3] == 0));
                    }
                    mm_prev = mm;
                    st_prev = act;
                }
                __syncthreads();  // the column's rows are complete; phases may be rewritten
            }
            // ---- flush the accumulator rows into this chunk's FP64 slots ----
            if (t == ntiles - 1 || (t + 1) % p.flush_tiles == 0) {
                for (int i = threadIdx.x; i < (lena + lenb) * NV; i += blockDim.x) {
                    const int q = i / NV, v = i % NV;
                    const int f = v >> 1;
                    if (f < p.ncol) {
                        const int m = q < lena ? ma : mb;
                        const int l = q < lena ? ma + q : mb + (q - lena);
                        double* sp =
                            p.slots + (((int64_t)f * p.nchunk + r) * p.nmodes + tri_base(m, L) + l) * 2 + (v & 1);
                        const double val = ldexp((double)accg[i], mx_col_exp(p.colmax[f]));
                        *sp = (first_flush ? 0.0 : *sp) + val;
                    }
                    accg[i] = 0.f;
                }
                first_flush = false;
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------ launchers --
size_t mixed_smem_bytes(int nf) {
    return 128 + (size_t)(MX_NGEO + nf) * MX_P * 4 + (size_t)MX_WARPS * 2 * MX_PW * 16 + (size_t)MX_WARPS * MX_PW * 8 +
           (size_t)2 * MX_WARPS * MX_BLK * (2 * nf + 4) * 4;
}

int mixed_tile_points() { return MX_P; }
int mixed_max_columns() { return MX_MAXCOL; }
int mixed_geometry_arrays() { return MX_NGEO; }
// floats of one CTA's accumulator rows (the widest pass, 2 x MX_MAXCOL values per l)
int64_t mixed_acc_stride(int lmax) { return ((int64_t)(lmax + 2) * 2 * MX_MAXCOL + 63) / 64 * 64; }

cudaError_t launch_mixed_prep(const PrepColsParams& pp, int64_t nranges, cudaStream_t st) {
    mx_pad_kernel<<<64, 256, 0, st>>>(pp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nranges == 0) return e;
    mx_scatter_kernel<<<(unsigned)nranges, 256, 0, st>>>(pp);
    return cudaGetLastError();
}

cudaError_t launch_mixed(const MixedParams& mp, int sm_count, cudaStream_t st) {
    // exactly one weight source: prepared weight arrays or a table
    if ((mp.wcols == nullptr) == (mp.vtab == nullptr) || mp.ncol < 1 || mp.ncol > MX_MAXCOL ||
        (mp.vtab && (mp.tcol0 < 0 || mp.vtab_fstride < 0)))
        return cudaErrorInvalidValue;
    // table mode always runs the 8-column instantiation, whatever this pass's column count
    const int nf = (mp.vtab || mp.ncol > 4) ? 8 : 4;
    const size_t smem = mixed_smem_bytes(nf);
    // column mode: x from the catalogs; table mode: u = x - 1 of the interpolation samples
    const void* kern = mp.vtab ? reinterpret_cast<const void*>(analysis_mixed_kernel<8, true>)
                       : nf == 4 ? reinterpret_cast<const void*>(analysis_mixed_kernel<4, false>)
                                 : reinterpret_cast<const void*>(analysis_mixed_kernel<8, false>);
    int occ = 0;
    cudaError_t e = configure_kernel(kern, MX_WARPS * 32, smem, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)sm_count * occ;
    if (grid > mp.nunits) grid = mp.nunits;
    if (grid > mp.maxctas) grid = mp.maxctas;
    if (grid < 1) grid = 1;
    if (mp.vtab) analysis_mixed_kernel<8, true><<<(int)grid, MX_WARPS * 32, smem, st>>>(mp);
    else if (nf == 4) analysis_mixed_kernel<4, false><<<(int)grid, MX_WARPS * 32, smem, st>>>(mp);
    else analysis_mixed_kernel<8, false><<<(int)grid, MX_WARPS * 32, smem, st>>>(mp);
    return cudaGetLastError();
}

}  // namespace psht
