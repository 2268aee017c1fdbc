// noalloc.cu -- pointsht_alm for callers that cannot allocate device memory.
//
// Some callers of this library have no way to obtain device memory for a
// workspace: code running inside a host framework that owns all device
// allocations, or real-time pipelines that forbid allocation after start-up.
// For them, pointsht_alm_noalloc runs the same transform with its scratch in
// a fixed array that lives in this library's device image.
//
// The array is a file-scope __device__ variable.  In host code its name is
// only a host-side stand-in, not a device address, so the device address is
// obtained here with cudaGetSymbolAddress, once per device, with that device
// current, and then passed to the kernels as an ordinary pointer.
#include <mutex>

#include "pointsht.h"

#define NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[POINTSHT_NOALLOC_SCRATCH_BYTES];

// error-message slot of the library (defined in api.cu)
pointsht_status psht_set_error(pointsht_status s, const char* msg);

static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on `dev` (the current device), looked up
// on first use.  Returns nullptr and sets *err on failure.
static void* scratch_address(int dev, cudaError_t* err) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            *err = e;
            return nullptr;
        }
        g_noalloc_ptr[dev] = p;
    }
    return g_noalloc_ptr[dev];
}

extern "C" pointsht_status pointsht_alm_noalloc(pointsht_plan plan, const pointsht_catalog* cats, int32_t ncat,
                                                int32_t nfield, pointsht_precision prec, double* alm_out,
                                                void* stream) {
    const size_t need = pointsht_workspace_size(plan, cats, ncat, nfield, prec);
    if (need == 0) return POINTSHT_EINVAL;  // the size query has set the message
    if (need > (size_t)POINTSHT_NOALLOC_SCRATCH_BYTES)
        return psht_set_error(POINTSHT_ENOMEM,
                              "alm_noalloc: this transform needs more scratch than the fixed no-allocation array "
                              "(POINTSHT_NOALLOC_SCRATCH_BYTES); use pointsht_alm with a caller workspace");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return psht_set_error(POINTSHT_ECUDA, "alm_noalloc: no usable current device");
    cudaError_t err = cudaSuccess;
    void* scratch = scratch_address(dev, &err);
    if (!scratch)
        return psht_set_error(POINTSHT_ECUDA, "alm_noalloc: cudaGetSymbolAddress of the scratch array failed");
    return pointsht_alm(plan, cats, ncat, nfield, prec, alm_out, scratch, (size_t)POINTSHT_NOALLOC_SCRATCH_BYTES,
                        stream);
}
