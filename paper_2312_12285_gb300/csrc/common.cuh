// common.cuh -- types and device helpers shared by the libpointsht kernels.
//
// Kernel-side layout of the work (arXiv:2312.12285, Eq. alm_def, App. A):
//   * "prepared points": every catalog of a field is copied once into a
//     structure of arrays (x, signed weight coeff*w, log2 sin(theta) as a
//     float pair, phi/2pi as a 64-bit fixed-point turn), padded with zero
//     weights to a whole number of tiles;
//   * a work unit is (field, chunk of points, group of W order-pairs); the
//     persistent analysis kernel pulls units from an atomic counter;
//   * each unit accumulates into its own FP64 slot (full packed triangle per
//     (field, chunk)), so no two CTAs ever add to the same address and the
//     final reduction over chunks runs in a fixed order.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <utility>

#define PSHT_MAX_FIELDS 64
#define PSHT_MAX_CATS 128

namespace psht {

enum ErrBits : unsigned { ERR_RANGE = 1u, ERR_TIMEOUT = 2u, ERR_INTERNAL = 4u };

// Launch configuration of a kernel with dynamic shared memory.  The
// function's maximum dynamic shared memory is raised once per (device,
// kernel) to the device's opt-in limit, so that no later launch of a smaller
// size can lower it below a size already in use; occupancy is cached per
// (device, kernel, size).  After the first call for a size, no runtime call is
// made, so launches made while a stream is being captured into a CUDA graph
// only enqueue kernels.
inline cudaError_t configure_kernel(const void* kern, int threads, size_t smem, int* occ_out) {
    static std::mutex mu;
    static std::set<std::pair<int, const void*>> raised;
    static std::map<std::tuple<int, const void*, size_t>, int> occ_cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    auto it = occ_cache.find(std::make_tuple(dev, kern, smem));
    if (it != occ_cache.end()) {
        *occ_out = it->second;
        return cudaSuccess;
    }
    if (!raised.count({dev, kern})) {
        int optin = 0;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e != cudaSuccess) return e;
        raised.insert({dev, kern});
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return e;
    occ_cache[std::make_tuple(dev, kern, smem)] = occ;
    *occ_out = occ;
    return cudaSuccess;
}

// Rescaling of the recurrence state below the floating-point range (the
// paper does not discuss underflow; Pbar_m^m ~ sin^m(theta) leaves the FP32
// range already at m ~ 1000 for sin(theta) ~ 0.9).  A value is carried as
// mantissa * 2^(SCALE_BITS * E) with E <= 0; contributions are counted only
// once E == 0.  Every 16 recurrence steps a lane with E < 0 whose state
// exceeds 2^CHECK_EXP is rescaled by 2^-SCALE_BITS.  Over 16 steps the state
// grows by at most prod(alpha_l + 1) <= 2^84 for lmax <= 4096, so while E < 0
// it stays below 2^(CHECK_EXP + 84): for FP32 that is 2^23, i.e. a dropped
// value is below 2^-41 of its true size, and a rescaled value is at least
// 2^(CHECK_EXP - SCALE_BITS) = 2^-125, still a normal float.
struct F32Scale {
    static constexpr int SCALE_BITS = 64;
    static constexpr int CHECK_EXP = -61;
    static constexpr int MAX_LMAX = 4096;
};
struct F64Scale {
    static constexpr int SCALE_BITS = 600;
    static constexpr int CHECK_EXP = -200;
    static constexpr int MAX_LMAX = 8192;
};

struct FieldDesc {
    int64_t off;     // first prepared point of the field
    int64_t npad;    // prepared points of the field (multiple of the tile)
    int64_t unit0;   // first work unit of the field
    int32_t nchunk;  // chunks (= accumulation slots) of the field
    int32_t slot0;   // first slot of the field
};

struct AnalysisParams {
    int32_t lmax, nfield, ngroups, flush_tiles;
    int64_t nmodes;   // (lmax+1)(lmax+2)/2
    int64_t chunk;    // points per chunk (multiple of the tile)
    int64_t nunits;   // total work units
    int64_t ntot;     // prepared points over all fields (SoA stride)
    FieldDesc fld[PSHT_MAX_FIELDS];
    const void* pts;        // prepared points, SoA with stride ntot
    const float* alpha_f;   // padded columns, FP32
    const float2* alpha_f2; // padded columns, FP32 (alpha, alpha) pairs
    const double* alpha_d;  // padded columns, FP64
    const int64_t* colstart;
    const float* log2c_hi;  // log2 c_m as float pair
    const float* log2c_lo;
    const double* log2c;    // log2 c_m in FP64
    const float4* pole_ae;  // near-pole form: (a, a, a - 2, a - 2) per (m, q), padded columns
    float pole_x;           // a tile whose points all have |x| >= pole_x takes the near-pole form
    const float* pole_rho;  // near-pole form: odd-chain scale per m
    int32_t pole_mmax;      // ... for orders m < pole_mmax
    int32_t wait_probe;     // test hook: CTA 0 waits on a barrier nothing arrives at, then leaves
    double* slots;          // [slot][nmodes][2]
    unsigned long long* stats;  // optional: [0] += 16-step blocks whose accumulation was skipped, [1] += all
    int* counter;
    unsigned* err;
#ifdef __CUDACC__
    __device__ __forceinline__ const float2* alpha2_col(int m) const { return alpha_f2 + colstart[m]; }
#endif
};

struct CatDesc {
    const void* x;
    const void* phi;
    const void* w;
    int64_t n;
    int64_t dst;   // first prepared point (prep) / unused (adjoint)
    double coeff;
    int32_t field;
    int32_t pad_;
    int64_t id0;   // point id of this catalog's first point (catalogs numbered consecutively)
};

struct PrepParams {
    int32_t ncat, nfield;
    int64_t ntot;
    CatDesc cat[PSHT_MAX_CATS];
    int64_t pad_off[PSHT_MAX_FIELDS];
    int64_t pad_n[PSHT_MAX_FIELDS];
    void* pts;
    unsigned* err;
};

#define SORT_XBINS 256          // bins of |x| in [0, 1]
#define SORT_SPLIT 224          // from |x| >= 224/256 on, x < 0 and x > 0 get separate buckets
#define SORT_BUCKETS (SORT_XBINS + SORT_XBINS - SORT_SPLIT)
#define SORT_RANGE 4096  // points per CTA range of the counting sort

#ifdef __CUDACC__
// Bucket of the counting sort: points are ordered by |x| (see analysis.cu);
// near the poles the two signs of x are kept apart, so that a tile of points
// near a pole lies on one side (the near-pole form mirrors x < 0 onto |x|).
__device__ __forceinline__ int x_bucket(double x) {
    const double a = fabs(x);
    int b = (int)(a * SORT_XBINS);
    b = b < 0 ? 0 : (b >= SORT_XBINS ? SORT_XBINS - 1 : b);
    return (b >= SORT_SPLIT && x < 0.0) ? b + SORT_XBINS - SORT_SPLIT : b;
}

// phi (radians, any finite value) as a 64-bit fixed-point fraction of a turn
__device__ __forceinline__ uint64_t phi_to_turn(double ph) {
    double t = ph * (1.0 / (2.0 * 3.14159265358979323846));
    t -= floor(t);
    if (!(t >= 0.0 && t < 1.0)) t = 0.0;
    return __double2ull_rn(t * 18446744073709551616.0);
}
#endif

struct SortParams {
    PrepParams prep;                     // catalogs (dst unused), pads, output
    int64_t range0[PSHT_MAX_CATS + 1];   // first CTA range of each catalog
    int64_t field_off[PSHT_MAX_FIELDS];  // first prepared point of each field
    int64_t* hist;                       // [nranges][SORT_BUCKETS] counts, then offsets
};

struct ReduceParams {
    int32_t nfield;
    int64_t nmodes;
    int32_t slot0[PSHT_MAX_FIELDS];
    int32_t nchunk[PSHT_MAX_FIELDS];
    const double* slots;
    const double* gamma;
    double* out;
};

// Weight-column form (mixed.cu).  Layout written by its preparation: five
// geometry arrays (x, log2 sin theta hi, lo, turn hi, turn lo) and then ncol
// weight arrays, each of ntot 4-byte values, points in |x| order.
struct PrepColsParams {
    const float* x;
    const float* phi;
    const float* w;        // [ncol][n]
    int64_t n;
    int32_t ncol, pad_;
    int64_t ntot;          // padded points (multiple of the tile)
    uint32_t* pts;         // (5 + ncol) arrays of ntot
    const int64_t* hist;   // sorted offsets per (range, bucket)
    unsigned* colmax;      // [ncol] bits of max |w| (non-negative floats order as integers)
    unsigned* err;
};

struct MixedParams {
    int32_t lmax, ncol, npairs, flush_tiles;
    int64_t nmodes, chunk, nunits, ntot;
    int32_t nchunk, pad_;
    const uint32_t* pts;      // geometry arrays (5 x ntot)
    const uint32_t* wcols;    // this pass's first weight array (ncol x ntot)
    const unsigned* colmax;   // this pass's columns
    const float2* alpha2;
    const float* alpha_f;     // the same coefficients as single floats (tcgen05 kernel)
    const int64_t* colstart;
    const float* log2c_hi;
    const float* log2c_lo;
    double* slots;            // [col][chunk][nmodes] complex
    float* accg;              // per-CTA FP32 accumulator rows, accstride floats each
    int64_t accstride;
    int32_t maxctas;          // CTAs the accumulator buffer provides for
    float vtab_h;             // table mode: sample spacing h
    const float2* vtab;       // table mode (interpolated route): per field [(lmax+1)][ntot][4] = (Vy, Vd) of
                              // the north and the mirrored south sample at each position; a field's six
                              // columns at order m are Vy^(m), h Vd^(m-1), h Vd^(m+1) of each instead of
                              // w e^{-i m phi}
    int64_t vtab_fstride;     // table mode: float2 entries between two fields' tables
    int32_t tcol0;            // table mode: column 6 f + j of the group is this pass's column tcol0 + c
    int32_t pole_mmax;        // table mode: near-pole form for orders m < pole_mmax ...
    float pole_x;             // ... in warps whose positions all have x >= pole_x
    int32_t pad3_;
    const float4* pole_ae;    // near-pole coefficients (a, a, e, e) in the column layout (NULL: off)
    const float* pole_rho;    // per order: the odd-step factor of the near-pole normalisation
    int* counter;
    unsigned* err;
};

// Interpolated transform (interp.cu)
struct InterpCat {
    const float* x;
    const float* phi;
    const float* w;
    int64_t n;
    double coeff;
};

struct InterpParams {
    int32_t lmax, ntheta, nb, ncat;  // nb = ntheta + 1 intervals
    int64_t npts, nranges, ntot;     // ntot = samples padded to the grid-transform tile
    InterpCat cat[PSHT_MAX_CATS];
    int64_t range0[PSHT_MAX_CATS + 1];  // first range of each catalog
    int32_t* hist;                      // [nranges][nb]: counts, then first slots
    int64_t* binoff;                    // [nb + 1]
    int64_t* total;                     // [nb]
    float* wc;                          // [4][npts] w coeff c_alpha, interval order
    uint32_t* turn;                     // [2][npts]
    uint32_t* stage;                    // [7][npts] bucket, w coeff c_alpha, turn; catalog order
    float2* v;                          // [(lmax+1)][nb][4]
    float2* vtab;                       // [(lmax+1)][ntot][4]: (Vy, Vd) north, (Vy, Vd) south per position
    uint32_t* nodes;                    // [5][ntot] sample geometry (x, lsh, lsl, turn hi, lo)
    unsigned* colmax;                   // [6]
    unsigned* err;
};

struct AdjointParams {
    int32_t lmax, ncat, nfield, pad_;
    CatDesc cat[PSHT_MAX_CATS];
    int64_t warp0[PSHT_MAX_CATS + 1];  // first warp of each catalog (prefix)
    const void* gtab;                   // [nfield][gstride] real2: gamma * g, padded columns
    int64_t gstride;
    const void* alpha;                  // padded columns (float or double)
    const int64_t* colstart;
    const float* log2c_hi;
    const float* log2c_lo;
    const double* log2c;
    const double* gnoise;               // [nfield][nfield] dL/dN (diagonal used) or null
    void* gradw[PSHT_MAX_CATS];
    unsigned* err;
    // FP32: the points as prepared for the analysis (|x| order, 7 arrays of
    // ntot, array 6 = point id), fields at fld[].off; gtab entries float4
    // (gamma g re, same, gamma g im, same)
    const uint32_t* pts;
    int64_t ntot;
    FieldDesc fld[PSHT_MAX_FIELDS];
    const float2* alpha2;
    const float4* pole_ae;   // near-pole form (see the analysis)
    const float* pole_rho;
    float pole_x;
    int32_t pole_mmax;
};

__host__ __device__ inline int64_t tri_base(int64_t m, int64_t lmax) {
    return m * (2 * lmax + 1 - m) / 2;
}

#ifdef __CUDACC__
// ------------------------------------------------------ PTX wrappers --
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bulk (non-tensor) TMA copy global -> shared, completing on an mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after `limit` polls (each try_wait may itself
// suspend for a hardware-defined time) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit = 1u << 22) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// After a bounded wait gave up: wait once more, bounded but far longer, for
// the copy still owed to `bar` (the phase of parity `parity`), so that no bulk
// copy lands in the shared memory of a CTA that has exited.  Called by the one
// thread that issues the copies, before the CTA returns.
__device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t parity) {
    return mbar_wait_bounded(bar, parity, 1u << 26);
}

// -------------------------------------------- float-pair arithmetic --
// Error-free transformations (Knuth two-sum, FMA two-product) for the
// log2 of the sectoral seed, where e = log2 c_m + m log2 sin(theta) must be
// known to ~1e-12 absolute for |e| up to 2e4.
struct f2 { float hi, lo; };

__device__ __forceinline__ f2 two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
    float s = a + b;
    return {s, b - (s - a)};
}

// ------------------------------------------ FP32 seed and phase (App. A) --
// lambda_mm = mant * 2^(64 E): log2 |lambda_mm| = log2 c_m + m log2 sin(theta)
// carried as a float pair (lh + ll for log2 sin theta, lch + lcl for
// log2 c_m), split into an exponent block E <= 0 and a mantissa in
// [2^-125, 2^-61] (E < 0) or (2^-125, ~1] (E = 0).  A point at a pole
// (log2 sin theta stored as -1e30) gets E at the floor and mantissa 0.
__device__ __forceinline__ void seed_f32(int m, float lh, float ll, float lch, float lcl, float& mant, int& E) {
    const float mf = (float)m;
    const float pr = mf * lh;
    float pe = fmaf(mf, lh, -pr);
    pe = fmaf(mf, ll, pe);
    const f2 s = two_sum(pr, lch);
    const f2 e = fast_two_sum(s.hi, s.lo + pe + lcl);
    const bool pole = e.hi < -1.0e7f;
    const float Ef =
        pole ? -1048576.f : fminf(0.f, ceilf((e.hi - (float)F32Scale::CHECK_EXP) * (1.0f / F32Scale::SCALE_BITS)));
    E = (int)Ef;
    const float eh = pole ? 0.f : e.hi - (float)F32Scale::SCALE_BITS * Ef;
    const f2 ep = fast_two_sum(eh, pole ? 0.f : e.lo);
    const float n = floorf(ep.hi);
    const float fr = (ep.hi - n) + ep.lo;
    mant = pole ? 0.f : ldexpf(exp2f(fr), (int)n);
    if (m & 1) mant = -mant;
}

// e^{i m phi} from phi as a 64-bit fixed-point turn (hi, lo words):
// (m * turn) mod 2^64, top 32 bits as a signed fraction of a half turn.
__device__ __forceinline__ void phase_f32(int m, uint32_t thi, uint32_t tlo, float& cs, float& sn) {
    const uint32_t t = (uint32_t)m * thi + __umulhi((uint32_t)m, tlo);
    sincospif((float)(int32_t)t * 0x1p-31f, &sn, &cs);
}
#endif

}  // namespace psht
