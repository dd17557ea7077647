// ddm_structure_function_static: the structure-function path with its spectrum scratch
// in a fixed device array of this library instead of memory obtained with cudaMalloc.
//
// Some callers cannot allocate device memory at the moment they need D: a host that
// hands all device memory to its own pool allocator up front (so a fresh cudaMalloc
// fails or fragments that pool), code running under a strict no-allocation policy in
// a latency-critical loop, or code whose only device memory is what it was handed
// (the frames and the output).  They create the plan once, during set-up, and call
// this entry point afterwards: it allocates nothing and takes no workspace.
//
// The scratch is a file-scope device array of DDM_STATIC_SCRATCH_BYTES; every GPU that
// loads this library holds it until the process exits.  Its name is only a host-side
// stand-in in host code, so the device address is fetched once per device with
// cudaGetSymbolAddress (on the first call made with that device current) and cached.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ddm_internal.h"

namespace {

static __device__ __align__(256) float2 g_static_spectrum[DDM_STATIC_SCRATCH_BYTES / sizeof(float2)];

constexpr int kMaxDevices = 256;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_spectrum on the current device, or nullptr on error.
void* scratch_address(int device) {
    if (device < 0 || device >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[device]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_spectrum) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_ptr[device] = ptr;
    }
    return g_scratch_ptr[device];
}

}  // namespace

extern "C" ddm_status ddm_structure_function_static(ddm_plan p, const void* frames, float* D,
                                                    void* stream) {
    if (!p || !frames || !D) return DDM_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(D) & 3) != 0) return DDM_ERR_INVALID_ARG;
    if (p->d.precision == DDM_PREC_FP64) return DDM_ERR_UNSUPPORTED;
    const size_t need = (size_t)p->n_q * (size_t)p->d.N * sizeof(float2);
    if (need > (size_t)DDM_STATIC_SCRATCH_BYTES) return DDM_ERR_UNSUPPORTED;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return DDM_ERR_CUDA;
    }
    if (dev != p->device) return DDM_ERR_INVALID_ARG;
    float2* spec = static_cast<float2*>(scratch_address(dev));
    if (!spec) return DDM_ERR_CUDA;
    // Every spectrum element the time-sequence stage reads is written by the spatial
    // stage of this same call, so nothing in the scratch has to start at zero.
    ddm_status st = ddm::launch_spatial(p, frames, spec, (cudaStream_t)stream);
    if (st != DDM_OK) return st;
    return ddm::launch_temporal(p, spec, D, (cudaStream_t)stream);
}
