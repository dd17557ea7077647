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
// stand-in in host code, so its device address is fetched with cudaGetSymbolAddress, on
// the first call made in a given CUDA context, and cached per context: the array lives in
// the context's copy of this library's module, so a device reset (or any other way the
// context is destroyed and created again) moves it, and the cache must not outlive the
// context it was filled in.  Contexts are told apart by the driver's process-unique
// context id (cuCtxGetId), not by device ordinal.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "ddm_internal.h"

namespace {

static __device__ __align__(256) float2 g_static_spectrum[DDM_STATIC_SCRATCH_BYTES / sizeof(float2)];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

struct ScratchEntry {
    unsigned long long ctx_id;
    void* ptr;
};

std::mutex g_setup_mutex;
std::vector<ScratchEntry> g_scratch;     // one entry per CUDA context seen, never reused
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

template <typename Fn>
bool driver_entry(const char* name, Fn* out) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f) {
        cudaGetLastError();
        return false;
    }
    *out = reinterpret_cast<Fn>(f);
    return true;
}

// Process-unique id of the current CUDA context (the runtime's primary context of the
// current device once a runtime call has made it current), or false on error.
bool current_context_id(unsigned long long* id) {
    if (!g_ctx_get_current && !driver_entry("cuCtxGetCurrent", &g_ctx_get_current)) return false;
    if (!g_ctx_get_id && !driver_entry("cuCtxGetId", &g_ctx_get_id)) return false;
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return g_ctx_get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of g_static_spectrum in the current context, or nullptr on error.
void* scratch_address() {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = 0;
    if (!current_context_id(&id)) return nullptr;
    for (const ScratchEntry& e : g_scratch)
        if (e.ctx_id == id) return e.ptr;
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_spectrum) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return nullptr;
    }
    g_scratch.push_back({id, ptr});
    return ptr;
}

}  // namespace

extern "C" ddm_status ddm_structure_function_static(ddm_plan p, const void* frames, float* D,
                                                    void* stream) {
    if (!p || !frames || !D) return DDM_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(D) & 3) != 0) return DDM_ERR_INVALID_ARG;
    if (p->d.precision == DDM_PREC_FP64) return DDM_ERR_UNSUPPORTED;
    if (p->nk > 0) return DDM_ERR_UNSUPPORTED;   // a kx-column range needs its workspace
    const size_t need = (size_t)p->n_q * (size_t)p->d.N * sizeof(float2);
    if (need > (size_t)DDM_STATIC_SCRATCH_BYTES) return DDM_ERR_UNSUPPORTED;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return DDM_ERR_CUDA;
    }
    if (dev != p->device) return DDM_ERR_INVALID_ARG;
    float2* spec = static_cast<float2*>(scratch_address());
    if (!spec) return DDM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // stage timing as in ddm_structure_function: events before step one, between the steps
    // and after step two, so that ddm_plan_stats reports this call
    const bool stats = p->stats_ev[0] != nullptr;
    p->stats_recorded = false;
    if (stats && cudaEventRecord(p->stats_ev[0], s) != cudaSuccess) return DDM_ERR_CUDA;
    // Every spectrum element the time-sequence stage reads is written by the spatial
    // stage of this same call, so nothing in the scratch has to start at zero.
    ddm_status st = ddm::launch_spatial(p, frames, spec, s);
    if (st != DDM_OK) return st;
    if (stats && cudaEventRecord(p->stats_ev[1], s) != cudaSuccess) return DDM_ERR_CUDA;
    st = ddm::launch_temporal(p, spec, D, s);
    if (st == DDM_OK && stats && cudaEventRecord(p->stats_ev[2], s) != cudaSuccess) return DDM_ERR_CUDA;
    p->stats_recorded = stats && st == DDM_OK;
    return st;
}
