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

#define PSHT_MAX_FIELDS 64
#define PSHT_MAX_CATS 128

namespace psht {

enum ErrBits : unsigned { ERR_RANGE = 1u, ERR_TIMEOUT = 2u, ERR_INTERNAL = 4u };

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
    double* slots;          // [slot][nmodes][2]
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

#define SORT_BUCKETS 256
#define SORT_RANGE 4096  // points per CTA range of the counting sort

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
#endif

}  // namespace psht
