// mixed_tc.cu -- per-m contraction of weight columns on the fifth-generation
// tensor cores (tcgen05: operands in shared and tensor memory, accumulators in
// tensor memory), POINTSHT_MIXED for pointsht_alm_columns.
//
// For order m the transform of F <= 8 weight columns sharing one point set is
//   a_m[l, f] = sum_i lambda_lm(x_i) W_m[i, f],  W_m[i, f] = w_f,i e^{-i m phi_i}
// (Eq. alm_def for each column; lambda from the FP32 sign-folded recurrence of
// App. A, as in the FP32 kernel).  As one MMA chain per block of 32 multipoles:
//   D[r, l] = sum_k A[r, k] B[k, l],   k = point of a 512-point tile,
//   A (tensor memory, 128 x 512 fp16): row r < 16 = W_hi[(f, re/im)], row
//     16 + r = W_lo of the same (hi = fp16 rounding, lo = fp16 of the rest),
//     rows 32..127 zero; written once per (tile, m);
//   B (shared memory, MN-major, 512 x 32 fp16): lambda_hi (low 13 mantissa
//     bits cleared, exact in fp16) and, in a second MMA with B negated,
//     lo' = hi - lambda (the negated remainder), both 0 while a point is still
//     below the FP32 range;
//   so rows r and 16 + r of D add up to (W_hi + W_lo)(lambda_hi + lambda_lo)
//   for (field, re/im) r: FP32 accumulation, all four hi/lo products kept.
// A block's hi and lo' MMA chains go into one accumulator; two blocks'
// accumulators live in tensor memory.  A block's 32 x 32 useful sums are read
// back (tcgen05.ld), the hi and lo rows added, and accumulated in block order
// into the CTA's FP32 rows in global memory (fire-and-forget atomics, one lane
// per entry), flushed into FP64 slots every flush_tiles tiles.  Each column is
// scaled by a power of two so that its largest |w| lies in [1, 2) (exact;
// undone at the flush).
//
// CTA (one per SM, 288 threads for 8 x 32): warp 0 controls: it writes A into
// tensor memory (lanes 0..31), issues the MMAs from one thread (stage full ->
// MMAs -> tcgen05.commit on the stage's "empty" barrier) and reads D back;
// warps 1..PW produce: lane l of producer warp w runs the recurrence for tile
// points k = 64 w + 2 l and k + 1 as one f32x2 pair, and every 8 steps stores
// each point's 8 fp16 hi and lo values as one 16-byte row of B (core matrices
// of 8 points x 8 multipoles).  The two orders of a unit (m, lmax - m) have
// their coefficient columns copied into shared memory once per unit.  B is
// double-buffered on mbarriers, so the recurrence of block b + 1 runs while
// the tensor cores work on block b.  A block in which no producer warp has a
// point inside the FP32 range issues no MMA (its sums are exact zeros).  Every
// wait is bounded; a CTA that gives up records ERR_TIMEOUT, waits (bounded)
// for its copies and MMAs in flight, frees its tensor memory and returns.
//
// Cost model (why this kernel is not the default).  With M = 128 only 32 rows
// of A carry W (F = 8), N is limited to the 32 multipoles a stage holds (the
// two stages of P x N hi and lo values take 128 KB), and the hi / lo' split
// doubles the MMAs: one M = 128, N = 32, K = 16 instruction per 16 x 32
// point-steps and operand half.  Issued from one thread such an instruction
// costs more than the tensor core's own time for it, so the MMA stream, not
// the recurrence, sets the pace; and the 512 points in flight per SM that the
// stages allow leave the producer warps latency-bound.  The warp-level
// mma.sync kernel (mixed.cu), whose operands never leave registers and
// 4 KB per warp of shared memory, is faster on the same work.
#include "common.cuh"

#include <cuda_fp16.h>

namespace psht {

constexpr int TC_NGEO = 5;                        // x, log2 sin theta hi, lo, turn hi, lo
constexpr int TC_MAXCOL = 8;
constexpr int TC_TMEM_COLS = 512;
constexpr int TC_DRING = 2;                       // blocks whose accumulators live in tensor memory

// Shape of a configuration: PW producer warps (one f32x2 pair of points per
// lane, P = 64 PW points per tile) and NB multipoles per B stage (N of one
// MMA).  A stage holds P x NB fp16 hi and lo values (P NB = 16384 for every
// shape, 32 KB per array); the MMA instructions per stage are P / 8, so a
// wider NB issues fewer, larger MMAs for the same work.
template <int PW, int NB>
struct TcShape {
    static constexpr int P = 64 * PW;
    static constexpr int WARPS = PW + 1 < 4 ? 4 : PW + 1;  // warp 0 controls; 1..PW produce; the rest idle
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int PT = 32 * (PW + 1);                // threads of the producer/control barriers
    static constexpr int KCS = (NB / 8) * 128 + 16;         // bytes between B core-matrix rows of 8 points (LBO)
    static constexpr int BARR = (P / 8) * KCS;              // bytes of one B array (hi or lo) of a stage
    static constexpr int ACOLS = P / 2;                     // tensor-memory columns of A (fp16 pairs)
    static constexpr int OFF_TILE = 128;
    static constexpr int TILE_BYTES = (TC_NGEO + TC_MAXCOL) * P * 4;
    static constexpr int OFF_WST = OFF_TILE + TILE_BYTES;   // [P / 2 pairs][32 rows] uint32 (fp16 pairs)
    static constexpr int WST_BYTES = ACOLS * 32 * 4;
    static constexpr int OFF_B = ((OFF_WST + WST_BYTES + 1023) / 1024) * 1024;  // [stage][hi, lo][BARR]
    static constexpr int OFF_COEF = OFF_B + 4 * BARR;       // the unit's two coefficient columns (floats)
    // entries of one column's copy: its length, a stage past it and the group
    // prefetched after that, rounded to 16 (64 bytes for the bulk copy)
    __host__ __device__ static constexpr int coef_entries(int len) { return (len + NB + 16 + 15) / 16 * 16; }
    // a unit pairs orders m and lmax - m (lengths summing to lmax + 2); each copy
    // adds at most NB + 31 entries to its length
    static size_t smem(int lmax) { return OFF_COEF + (size_t)(lmax + 2 + 2 * (NB + 31)) * 4; }
    static_assert(ACOLS + TC_DRING * NB <= TC_TMEM_COLS, "tensor memory");
    static_assert(NB % 32 == 0 && NB <= 256, "N of one MMA");
};

// ------------------------------------------------------------ PTX helpers --
__device__ __forceinline__ float2 tc_fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)),
          "l"(reinterpret_cast<unsigned long long&>(c)));
    return d;
}
__device__ __forceinline__ float2 tc_mul2(float2 a, float2 b) {
    float2 d;
    asm("mul.rn.f32x2 %0, %1, %2;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)));
    return d;
}
// two f32 -> f16x2, a in the low half
__device__ __forceinline__ uint32_t tc_pack(float a, float b) {
    uint32_t r;
    asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}
// shared-memory matrix descriptor (no swizzle): start, LBO (stride between core
// matrices along K), SBO (stride along M/N), all in 16-byte units; bit 46 =
// descriptor version of this architecture family
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void named_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
        "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
        "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&f)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) f[i] = __uint_as_float(r[i]);
}

// The CTA's FP32 accumulator rows in global memory: during a tile, entry (q, v)
// is only added to by one lane of the control warp, in block order, with a
// fire-and-forget device-scope atomic (so the readout never waits for memory;
// the sum is the same bit for bit on every run); flushes read and clear the
// rows behind a fence and a barrier.
__device__ __forceinline__ void tc_acc_add(float* a, float v) { atomicAdd(a, v); }
// exponent e with max|w| * 2^-e in [1, 2) (0 for an all-zero column)
__device__ __forceinline__ int tc_col_exp(unsigned bits) {
    if (bits == 0u) return 0;
    const int e = ilogbf(__uint_as_float(bits));
    return e < -120 ? -120 : (e > 120 ? 120 : e);
}

struct TcShared {
    uint64_t tile_bar, full[2], empty[2], coef_bar;
    int64_t unit;
    int alive[2];
    volatile int abort;
    uint32_t tmem;
};

// ------------------------------------------------------------------ kernel --
template <int PW, int NB>
__global__ void __launch_bounds__(TcShape<PW, NB>::THREADS, 1)
    analysis_tc_kernel(const __grid_constant__ MixedParams p) {
    using S = TcShape<PW, NB>;
    constexpr int P = S::P;
    extern __shared__ __align__(1024) unsigned char smem[];
    TcShared* sh = reinterpret_cast<TcShared*>(smem);
    unsigned char* tile = smem + S::OFF_TILE;
    uint32_t* wst = reinterpret_cast<uint32_t*>(smem + S::OFF_WST);
    unsigned char* bst = smem + S::OFF_B;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool ctl = warp == 0;                   // tensor-memory lanes 0..31
    const bool prod = warp >= 1 && warp <= PW;
    const int L = p.lmax;
    constexpr int NV = 2 * TC_MAXCOL;  // accumulator values per l: (field, re/im)
    if ((int)blockIdx.x >= p.maxctas) return;
    float* accg = p.accg + (int64_t)blockIdx.x * p.accstride;  // [(L+2)][NV]

    float* coef = reinterpret_cast<float*>(smem + S::OFF_COEF);
    uint32_t coef_parity = 0;
    if (threadIdx.x == 0) {
        mbar_init(&sh->coef_bar, 1);
        mbar_init(&sh->tile_bar, 1);
        mbar_init(&sh->full[0], PW);
        mbar_init(&sh->full[1], PW);
        mbar_init(&sh->empty[0], 1);
        mbar_init(&sh->empty[1], 1);
        sh->alive[0] = sh->alive[1] = -1;
        sh->abort = 0;
        fence_mbar_init();
    }
    if (ctl) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = sh->tmem;
    // rows 32..127 of A stay zero: warps 1..3 own tensor-memory lanes 32..127
    if (warp >= 1 && warp <= 3) {
        uint32_t z[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) z[i] = 0u;
        for (int c = 0; c < S::ACOLS; c += 32) tmem_st32(tbase + ((uint32_t)(32 * warp) << 16) + c, z);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (ctl) named_arrive(2, S::PT);  // the W staging area is free

    // instruction descriptors: D f32, A and B f16, A K-major, B MN-major,
    // N = NB, M = 128; the second one negates B (for lo' = hi - lambda)
    const uint32_t idesc = (1u << 4) | (1u << 16) | ((uint32_t)(NB >> 3) << 17) | ((128u >> 4) << 24);
    const uint32_t idesc_neg = idesc | (1u << 14);

    uint32_t gb = 0;            // blocks of this CTA so far (stage gb & 1, phase (gb >> 1) & 1)
    uint32_t tile_parity = 0;
    bool tile_pending = false;  // a tile copy is owed to tile_bar (thread 32, which issues the copies)
    bool coef_owed = false;     // thread 32 gave up on a coefficient copy: owed to coef_bar
    uint32_t coef_owed_parity = 0;

    for (;;) {
        if (threadIdx.x == 0) sh->unit = (int64_t)atomicAdd(p.counter, 1);
        __syncthreads();
        const int64_t u = sh->unit;
        __syncthreads();  // every thread has read the unit before the next one is fetched
        if (u >= p.nunits) break;
        const int64_t r = u / p.npairs;
        const int pi = (int)(u - r * p.npairs);
        const int64_t pt0 = r * p.chunk;
        const int64_t npts = min(p.chunk, p.ntot - pt0);
        const int ntiles = (int)(npts / P);
        const int ma = pi, mb = L - pi;
        const bool single = ma == mb;
        const int ncols = single ? 1 : 2;
        const int lena = L - ma + 1, lenb = single ? 0 : L - mb + 1;
        // clear the accumulator rows (in L2, where the control warp's atomics land)
        for (int i = threadIdx.x; i < (lena + lenb) * NV; i += S::THREADS) __stcg(accg + i, 0.f);
        __threadfence();
        __syncthreads();
        bool first_flush = true;
        const int narr = TC_NGEO + p.ncol;
        auto issue = [&](int t) {
            mbar_expect_tx(&sh->tile_bar, narr * P * 4);
            const int64_t first = pt0 + (int64_t)t * P;
            for (int a = 0; a < TC_NGEO; ++a)
                bulk_g2s(tile + a * P * 4, p.pts + (int64_t)a * p.ntot + first, P * 4, &sh->tile_bar);
            for (int f = 0; f < p.ncol; ++f)
                bulk_g2s(tile + (TC_NGEO + f) * P * 4, p.wcols + (int64_t)f * p.ntot + first, P * 4, &sh->tile_bar);
        };
        // the coefficients of both orders of the pair, copied once per unit
        const int na = S::coef_entries(lena);
        if (threadIdx.x == 32) {
            const int nb2 = single ? 0 : S::coef_entries(lenb);
            mbar_expect_tx(&sh->coef_bar, (na + nb2) * 4);
            bulk_g2s(coef, p.alpha_f + p.colstart[ma], na * 4, &sh->coef_bar);
            if (!single) bulk_g2s(coef + na, p.alpha_f + p.colstart[mb], nb2 * 4, &sh->coef_bar);
        }
        if (threadIdx.x == 32 && ntiles > 0) {
            issue(0);
            tile_pending = true;
        }
        if (prod && !mbar_wait_bounded(&sh->coef_bar, coef_parity)) {
            atomicOr(p.err, ERR_TIMEOUT);
            sh->abort = 1;
            if (threadIdx.x == 32) {  // the copy may still land: drained before the CTA leaves
                coef_owed = true;
                coef_owed_parity = coef_parity;
            }
        }
        coef_parity ^= 1u;

        for (int t = 0; t < ntiles; ++t) {
            if (prod) {
                const bool ok = mbar_wait_bounded(&sh->tile_bar, tile_parity);
                if (!ok) {
                    atomicOr(p.err, ERR_TIMEOUT);
                    sh->abort = 1;
                }
                // a copy thread 32 gave up on stays owed, on this phase, until
                // the drain below (no further tile is issued once aborted)
                if (threadIdx.x == 32 && ok) tile_pending = false;
            }
            if (!tile_pending) tile_parity ^= 1u;
            const float* tf = reinterpret_cast<const float*>(tile);
            const uint32_t* tu = reinterpret_cast<const uint32_t*>(tile);

            for (int col = 0; col < ncols; ++col) {
                const int m = col ? mb : ma;
                const int len = L - m + 1;
                const int nblk = (len + NB - 1) / NB;
                const int qoff = col ? lena : 0;
                if (prod) {
                    // ------------------------------ producer warps --
                    const int k0 = 64 * (warp - 1) + 2 * lane;  // this lane's points k0, k0 + 1 of the tile
                    const float lch = p.log2c_hi[m], lcl = p.log2c_lo[m];
                    float xv[2], mant[2], cs[2], sn[2];
                    int E[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int i = k0 + h;
                        xv[h] = tf[i];
                        seed_f32(m, tf[P + i], tf[2 * P + i], lch, lcl, mant[h], E[h]);
                        phase_f32(m, tu[3 * P + i], tu[4 * P + i], cs[h], sn[h]);
                    }
                    // W rows of both points, packed as fp16 pairs (k0, k0 + 1)
                    named_sync(2, S::PT);  // the control warp has read the previous W
                    {
                        uint32_t* wrow = wst + (size_t)(k0 >> 1) * 32;
#pragma unroll
                        for (int f = 0; f < TC_MAXCOL; ++f) {
                            const float sc = f < p.ncol ? ldexpf(1.f, -tc_col_exp(p.colmax[f])) : 0.f;
                            float wh[2][2], wl[2][2];
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const float w = f < p.ncol ? tf[(TC_NGEO + f) * P + k0 + h] * sc : 0.f;
                                const float re = w * cs[h], im = -w * sn[h];
                                wh[h][0] = __half2float(__float2half_rn(re));
                                wh[h][1] = __half2float(__float2half_rn(im));
                                wl[h][0] = re - wh[h][0];
                                wl[h][1] = im - wh[h][1];
                            }
                            wrow[2 * f] = tc_pack(wh[0][0], wh[1][0]);
                            wrow[2 * f + 1] = tc_pack(wh[0][1], wh[1][1]);
                            wrow[16 + 2 * f] = tc_pack(wl[0][0], wl[1][0]);
                            wrow[16 + 2 * f + 1] = tc_pack(wl[0][1], wl[1][1]);
                        }
                    }
                    named_arrive(1, S::PT);  // W written
                    if (col == ncols - 1) {
                        // every producer has read the tile: fetch the next one
                        named_sync(3, 32 * PW);
                        if (threadIdx.x == 32 && t + 1 < ntiles && !sh->abort) {
                            issue(t + 1);
                            tile_pending = true;
                        }
                    }
                    // recurrence state (sign-folded sigma, as the FP32 kernel)
                    const float2 x2 = make_float2(xv[0], xv[1]);
                    float2 p1 = make_float2(0.f, 0.f), p2 = make_float2(mant[0], mant[1]);
                    uint32_t mask[2] = {E[0] == 0 ? 0xffffe000u : 0u, E[1] == 0 ? 0xffffe000u : 0u};
                    float2 nlive = make_float2(E[0] == 0 ? -1.f : 0.f, E[1] == 0 ? -1.f : 0.f);
                    bool any_neg = __any_sync(0xffffffffu, (E[0] | E[1]) != 0);
                    bool warp_alive = __any_sync(0xffffffffu, (E[0] == 0) | (E[1] == 0));
                    // coefficients from the unit's shared-memory copy; those of the next 8
                    // steps are read while the current 8 run (the copy extends a stage and a
                    // group past the column: the next column's values or the table's zeros)
                    const float4* a4 = reinterpret_cast<const float4*>(coef + (col ? na : 0));
                    float4 an[2] = {a4[0], a4[1]};
                    // B rows of this lane's points: core-matrix row k0 / 8 (+ k0 % 8 rows of 16 bytes)
                    const uint32_t brow = (uint32_t)((k0 >> 3) * S::KCS + (k0 & 7) * 16);
                    for (int b = 0; b < nblk; ++b, ++gb) {
                        const int s = gb & 1;
                        if (gb >= 2 && !sh->abort) {
                            if (!mbar_wait_bounded(&sh->empty[s], ((gb >> 1) - 1) & 1u)) {
                                atomicOr(p.err, ERR_TIMEOUT);
                                sh->abort = 1;
                            }
                        }
                        uint4* bhi = reinterpret_cast<uint4*>(bst + (2 * s) * S::BARR + brow);
                        uint4* blo = reinterpret_cast<uint4*>(bst + (2 * s + 1) * S::BARR + brow);
                        bool blk_alive = false;
#pragma unroll 1
                        for (int nc = 0; nc < NB / 8; ++nc) {
                            const bool act = warp_alive;  // re-evaluated at every rescale check
                            blk_alive |= act;
                            uint32_t hw[2][4], lw[2][4];
                            const float4 ac[2] = {an[0], an[1]};
                            {
                                const float4* nx = a4 + 2 * ((NB / 8) * b + nc + 1);
                                an[0] = nx[0];
                                an[1] = nx[1];
                            }
#pragma unroll
                            for (int j2 = 0; j2 < 4; ++j2) {
                                // coefficients of steps (2 j2, 2 j2 + 1), as (alpha, alpha) pairs
                                const float4 c4 = ac[j2 >> 1];
                                const float ca = (j2 & 1) ? c4.z : c4.x, cb = (j2 & 1) ? c4.w : c4.y;
                                const float4 av = make_float4(ca, ca, cb, cb);
                                float2 s0;
                                {
                                    const float2 sg = tc_fma2(make_float2(av.x, av.y), tc_mul2(x2, p1), p2);
                                    p2 = p1;
                                    p1 = sg;
                                    s0 = sg;
                                }
                                {
                                    const float2 sg = tc_fma2(make_float2(av.z, av.w), tc_mul2(x2, p1), p2);
                                    p2 = p1;
                                    p1 = sg;
                                }
                                if (act) {
                                    const float h0x = __uint_as_float(__float_as_uint(s0.x) & mask[0]);
                                    const float h0y = __uint_as_float(__float_as_uint(s0.y) & mask[1]);
                                    const float h1x = __uint_as_float(__float_as_uint(p1.x) & mask[0]);
                                    const float h1y = __uint_as_float(__float_as_uint(p1.y) & mask[1]);
                                    const float2 l0 = tc_fma2(s0, nlive, make_float2(h0x, h0y));  // hi - lambda
                                    const float2 l1 = tc_fma2(p1, nlive, make_float2(h1x, h1y));
                                    hw[0][j2] = tc_pack(h0x, h1x);
                                    hw[1][j2] = tc_pack(h0y, h1y);
                                    lw[0][j2] = tc_pack(l0.x, l1.x);
                                    lw[1][j2] = tc_pack(l0.y, l1.y);
                                } else {
                                    hw[0][j2] = hw[1][j2] = lw[0][j2] = lw[1][j2] = 0u;
                                }
                            }
                            // rows of points k0 (.x) and k0 + 1 (.y), multipoles 8 nc .. 8 nc + 7
                            bhi[nc * 8] = make_uint4(hw[0][0], hw[0][1], hw[0][2], hw[0][3]);
                            bhi[nc * 8 + 1] = make_uint4(hw[1][0], hw[1][1], hw[1][2], hw[1][3]);
                            blo[nc * 8] = make_uint4(lw[0][0], lw[0][1], lw[0][2], lw[0][3]);
                            blo[nc * 8 + 1] = make_uint4(lw[1][0], lw[1][1], lw[1][2], lw[1][3]);
                            if (any_neg && (nc & 1)) {
                                // rescale check every 16 steps (F32Scale: 2^64 blocks)
                                bool lane_neg = false;
#pragma unroll
                                for (int h = 0; h < 2; ++h) {
                                    float& a = h ? p1.y : p1.x;
                                    float& c = h ? p2.y : p2.x;
                                    const bool nd = (E[h] < 0) & (fmaxf(fabsf(a), fabsf(c)) > 0x1p-61f);
                                    const float sc = nd ? 0x1p-64f : 1.f;
                                    a *= sc;
                                    c *= sc;
                                    E[h] += nd;
                                    mask[h] = E[h] == 0 ? 0xffffe000u : 0u;
                                    lane_neg |= E[h] != 0;
                                }
                                nlive = make_float2(E[0] == 0 ? -1.f : 0.f, E[1] == 0 ? -1.f : 0.f);
                                any_neg = __any_sync(0xffffffffu, lane_neg);
                                warp_alive = __any_sync(0xffffffffu, (E[0] == 0) | (E[1] == 0));
                            }
                        }
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) {
                            if (blk_alive) sh->alive[s] = (int)gb;
                            mbar_arrive(&sh->full[s]);
                        }
                    }
                } else if (ctl) {
                    // ---------------------------------- control warp --
                    named_sync(1, S::PT);  // W of this column is in shared memory
                    {
                        uint32_t v[32];
                        for (int c0 = 0; c0 < S::ACOLS; c0 += 32) {
#pragma unroll
                            for (int i = 0; i < 32; ++i) v[i] = wst[(size_t)(c0 + i) * 32 + lane];
                            tmem_st32(tbase + c0, v);  // lanes 0..31 = rows 0..31 of A
                        }
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    }
                    named_arrive(2, S::PT);  // W may be rewritten
                    tc_fence_before();
                    __syncwarp();
                    tc_fence_after();
                    const int ec0 = gb;  // first block of this column
                    // whether the previous block issued MMAs (decided when they were issued:
                    // the alive word of its stage is reused by the block after next)
                    bool had_prev = false;
                    for (int b = 0; b <= nblk; ++b) {
                        const uint32_t g = (uint32_t)ec0 + b;
                        bool had_now = false;
                        if (b < nblk) {
                            // issue the MMAs of block b (hi and lo' chains into one accumulator)
                            const int s = g & 1;
                            bool ok = true;
                            if (!sh->abort) ok = mbar_wait_bounded(&sh->full[s], (g >> 1) & 1u);
                            had_now = ok && !sh->abort && sh->alive[s] == (int)g;
                            had_now = __shfl_sync(0xffffffffu, had_now, 0);
                            if (!ok || sh->abort) {
                                if (lane == 0 && !ok) atomicOr(p.err, ERR_TIMEOUT);
                                sh->abort = 1;
                                had_now = false;
                                if (lane == 0) mbar_arrive(&sh->empty[s]);  // release the producers
                            } else if (lane == 0) {
                                if (had_now) {
                                    tc_fence_after();
                                    const uint32_t d = tbase + S::ACOLS + (g % TC_DRING) * NB;
                                    const uint64_t dh = tc_sdesc(smem_u32(bst + (2 * s) * S::BARR), S::KCS, 128);
                                    const uint64_t dl = tc_sdesc(smem_u32(bst + (2 * s + 1) * S::BARR), S::KCS, 128);
#pragma unroll
                                    for (int kk = 0; kk < P / 16; ++kk) {
                                        const uint64_t step = (uint64_t)((2 * kk * S::KCS) >> 4);  // start field
                                        tc_mma(d, tbase + 8 * kk, dh + step, idesc, kk > 0 ? 1u : 0u);
                                        tc_mma(d, tbase + 8 * kk, dl + step, idesc_neg, 1u);
                                    }
                                    tc_commit(&sh->empty[s]);
                                } else {
                                    mbar_arrive(&sh->empty[s]);  // no point in range: nothing to add
                                }
                            }
                            __syncwarp();
                        }
                        if (b >= 1) {
                            // read back block b - 1 once its MMAs are complete
                            const uint32_t gp = g - 1;
                            const int sp = gp & 1;
                            const bool okw = mbar_wait_bounded(&sh->empty[sp], (gp >> 1) & 1u);
                            if (!okw) {
                                if (lane == 0) atomicOr(p.err, ERR_TIMEOUT);
                                sh->abort = 1;
                            }
                            tc_fence_after();
                            const bool had = okw && !sh->abort && had_prev;
                            if (had) {
                                const uint32_t dcol = tbase + S::ACOLS + (gp % TC_DRING) * NB;
                                // lane r < 16: row r (hi) + row r + 16 (lo) for the first 16 of
                                // each 32 multipoles; lane r + 16 the other 16
                                const bool up = lane >= 16;
                                const int row = lane & 15;
#pragma unroll 1
                                for (int c32 = 0; c32 < NB / 32; ++c32) {
                                    float dv[32];
                                    tmem_ld32(dcol + 32 * c32, dv);
                                    const int l0 = NB * (b - 1) + 32 * c32 + (up ? 16 : 0);
#pragma unroll
                                    for (int j = 0; j < 16; ++j) {
                                        const float send = up ? dv[j] : dv[16 + j];
                                        const float recv = __shfl_xor_sync(0xffffffffu, send, 16);
                                        const float sum = (up ? dv[16 + j] : dv[j]) + recv;
                                        if (l0 + j < len) tc_acc_add(accg + (size_t)(qoff + l0 + j) * NV + row, sum);
                                    }
                                }
                            }
                            tc_fence_before();
                            __syncwarp();
                        }
                        had_prev = had_now;
                    }
                    gb += nblk;
                } else {
                    gb += nblk;  // idle warp
                }
            }
            // ---- flush the accumulator rows into this chunk's FP64 slots ----
            if (t == ntiles - 1 || (t + 1) % p.flush_tiles == 0) {
                // the control warp's atomics are performed before the barrier; then every
                // thread of the CTA reads rows from L2, adds them into the FP64 slots and
                // clears them (the next atomics come after the next barrier)
                __threadfence();
                __syncthreads();
                for (int i = threadIdx.x; i < (lena + lenb) * NV; i += S::THREADS) {
                    const int q = i / NV, v = i % NV;
                    const int f = v >> 1;
                    const float val = __ldcg(accg + i);
                    __stcg(accg + i, 0.f);
                    if (f < p.ncol) {
                        const int m = q < lena ? ma : mb;
                        const int l = q < lena ? ma + q : mb + (q - lena);
                        double* sp =
                            p.slots + (((int64_t)f * p.nchunk + r) * p.nmodes + tri_base(m, L) + l) * 2 + (v & 1);
                        *sp = (first_flush ? 0.0 : *sp) + ldexp((double)val, tc_col_exp(p.colmax[f]));
                    }
                }
                __threadfence();
                first_flush = false;
            }
            // one decision for the whole CTA (every thread reaches this point
            // once per tile): leave after a wait gave up anywhere
            if (__syncthreads_or(sh->abort)) break;
        }
        if (__syncthreads_or(sh->abort)) break;
    }
    // ---- leave: nothing in flight, tensor memory freed ----
    if (prod) named_sync(2, S::PT);  // the control warp's last "W read" arrival
    __syncthreads();
    if (threadIdx.x == 32 && tile_pending) mbar_drain(&sh->tile_bar, tile_parity);
    if (threadIdx.x == 32 && coef_owed) mbar_drain(&sh->coef_bar, coef_owed_parity);
    if (ctl) {
        // the last issued block's MMAs: its empty phase (if any block was issued)
        if (gb > 0) {
            const uint32_t gl = gb - 1;
            mbar_drain(&sh->empty[gl & 1], (gl >> 1) & 1u);
        }
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TC_TMEM_COLS));
    }
}

// ------------------------------------------------------------ launcher --
template <int PW, int NB>
cudaError_t launch_tc_shape(const MixedParams& mp, int sm_count, cudaStream_t st) {
    using S = TcShape<PW, NB>;
    if (mp.ntot % S::P || mp.chunk % S::P) return cudaErrorInvalidValue;
    auto kern = analysis_tc_kernel<PW, NB>;
    const size_t smem = S::smem(mp.lmax);
    int occ = 0;
    cudaError_t e = configure_kernel(reinterpret_cast<const void*>(kern), S::THREADS, smem, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = sm_count;  // one CTA per SM: 512 tensor-memory columns each
    if (grid > mp.nunits) grid = mp.nunits;
    if (grid > mp.maxctas) grid = mp.maxctas;
    if (grid < 1) grid = 1;
    kern<<<(int)grid, S::THREADS, smem, st>>>(mp);
    return cudaGetLastError();
}

// shape: 0 = (8 producer warps, 32 multipoles per stage), 1 = (4, 64), 2 = (2, 128)
cudaError_t launch_mixed_tc(const MixedParams& mp, int sm_count, cudaStream_t st, int shape) {
    if (mp.wcols == nullptr || mp.vtab != nullptr || mp.ncol < 1 || mp.ncol > TC_MAXCOL) return cudaErrorInvalidValue;
    switch (shape) {
        case 1: return launch_tc_shape<4, 64>(mp, sm_count, st);
        case 2: return launch_tc_shape<2, 128>(mp, sm_count, st);
        default: return launch_tc_shape<8, 32>(mp, sm_count, st);
    }
}

}  // namespace psht
