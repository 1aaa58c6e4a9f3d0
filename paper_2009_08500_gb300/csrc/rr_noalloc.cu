// rr_evaluate_noalloc: rr_evaluate with library-owned, statically allocated
// scratch memory, for callers that cannot allocate device memory at call time.
//
// The scratch is a file-scope __device__ array: every GPU that loads this
// library holds RR_NOALLOC_SCRATCH_BYTES for it until the process exits.
// Host code cannot use the array's name as a device address, so its address
// is looked up once per device with cudaGetSymbolAddress (with that device
// current) and then passed to the kernels like any other workspace.
#include <mutex>
#include <string>

#include "rr_internal.h"

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[RR_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Address of the scratch array on `dev`; looked up on the first call for that device.
cudaError_t scratch_on(int dev, void** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        int prev = 0;
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) return e;
        if ((e = cudaSetDevice(dev)) != cudaSuccess) return e;
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        cudaError_t e2 = cudaSetDevice(prev);
        if (e != cudaSuccess) return e;
        if (e2 != cudaSuccess) return e2;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" rr_status rr_evaluate_noalloc(rr_ctx* c, const double* times, const int32_t* pb_index, int32_t npt,
                                         const double* params, int32_t npv, const int32_t* supersampling,
                                         const double* exptime, void* flux, int32_t* pv_status, void* stream) {
    if (!c) return rr_evaluate(c, times, pb_index, npt, params, npv, supersampling, exptime, flux, pv_status,
                               nullptr, 0, stream);
    const int dev = c->cfg.device;
    if (dev < 0 || dev >= kMaxDevices) {
        c->err = "rr_evaluate_noalloc: device ordinal beyond the library's table of scratch arrays";
        return RR_EINVAL;
    }
    const size_t need = rr_workspace_bytes(c, npv < 0 ? 0 : npv, npt < 0 ? 0 : npt, 0);
    if (npv > 0 && npt >= 0 && need > (size_t)RR_NOALLOC_SCRATCH_BYTES) {
        c->err = "rr_evaluate_noalloc: " + std::to_string(npv) + " parameter vectors x " + std::to_string(npt) +
                 " times need " + std::to_string(need) + " bytes of scratch, more than the fixed " +
                 std::to_string((size_t)RR_NOALLOC_SCRATCH_BYTES) +
                 " (RR_NOALLOC_SCRATCH_BYTES); use rr_evaluate with a caller-owned workspace or split the batch";
        return RR_EINVAL;
    }
    void* scratch = nullptr;
    cudaError_t e = scratch_on(dev, &scratch);
    if (e != cudaSuccess) {
        c->err = std::string("rr_evaluate_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorName(e);
        return RR_ECUDA;
    }
    // Every call writes all the scratch it reads (per-pv records and per-time
    // inputs are rebuilt by the first kernels of the call), so nothing has to
    // be cleared between calls.
    return rr_evaluate(c, times, pb_index, npt, params, npv, supersampling, exptime, flux, pv_status, scratch,
                       (size_t)RR_NOALLOC_SCRATCH_BYTES, stream);
}
