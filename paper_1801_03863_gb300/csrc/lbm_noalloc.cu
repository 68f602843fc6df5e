// lbm_noalloc.cu -- lbm_conservation_noalloc: the per-instance FP64
// mass/momentum reduction with its scratch in a fixed device array, for
// callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc at the point where it
// wants the totals -- a host application that owns and budgets all device
// memory through its own pool (framework caching allocators, plugin hosts),
// a real-time loop that cannot afford the implicit synchronisation an
// allocation may cause, or code that runs while another component forbids
// new allocations.  The regular entry points take their scratch from the
// context's block; this one takes it from the array below instead, so the
// call itself allocates nothing.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lbm.h"
#include "lbm_aux.h"

namespace lbm {
int ctx_conservation_inputs(const lbm_ctx* ctx, AuxArgs* args, const void** src, int* count);
}

namespace {

// Largest context (in instances) the fixed scratch serves.  64 partial sums
// of 3 doubles per instance: 4096 instances = 6 MiB, held by every device
// that loads the library until the process exits.
constexpr int NOALLOC_MAX_INSTANCES = 4096;

static __device__ __align__(256) double g_cons_scratch[NOALLOC_MAX_INSTANCES *
                                                       lbm::CONS_PARTIALS * 3];

constexpr int MAX_DEVICES = 64;
double* g_scratch_addr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mu;

// Device address of g_cons_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
int scratch_on_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return LBM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_cons_scratch) != cudaSuccess) return LBM_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_conservation_noalloc(lbm_ctx* ctx, double* out) {
    if (!ctx || !out) return LBM_ERR_ARG;
    lbm::AuxArgs a;
    const void* src = nullptr;
    int count = 0;
    int rc = lbm::ctx_conservation_inputs(ctx, &a, &src, &count);
    if (rc != LBM_OK) return rc;
    if (count > NOALLOC_MAX_INSTANCES) return LBM_ERR_ARG;
    double* scratch = nullptr;
    rc = scratch_on_current_device(&scratch);
    if (rc != LBM_OK) return rc;
    // Every partial the final pass reads is written by the first pass of the
    // same call, so the array needs no clearing between calls.
    if (lbm::run_aux(lbm::AuxOp::Conservation, a, src, nullptr, nullptr, nullptr, nullptr, out,
                     scratch, nullptr) != cudaSuccess)
        return LBM_ERR_CUDA;
    return LBM_OK;
}
