// tmm_noalloc.cu -- tmm_coh_batched_noalloc: the persistent (ragged,
// longest-first) forward launch with its scratch memory in a fixed, statically
// sized device array instead of a caller-provided workspace.
//
// Who needs it: callers that must not allocate device memory at call time --
// services whose request path may not take cudaMalloc's implicit device-wide
// synchronisation, and host programs whose device memory is owned by another
// allocator or fixed at start-up and cannot hand this library a workspace.
// The scratch (work counter, error flag, counting-sort buckets, stack order) is
// a file-scope __device__ array that every GPU loading this library keeps until
// the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "tmm_internal.h"

namespace tmm {

constexpr size_t kNoAllocScratchBytes = 1u << 20;  // 1 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch for the current device, looked up once
// per device (host code cannot use the symbol itself as a device pointer).
// The cached address belongs to the device's primary context: after
// cudaDeviceReset the module is loaded anew and the address may change, so
// the entry point must not be used after a reset of a device it ran on.
static tmm_status noalloc_scratch(void **out)
{
    static std::mutex mu;
    static void *addr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= 64) return TMM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e);
        addr[dev] = p;
    }
    *out = addr[dev];
    return TMM_OK;
}

}  // namespace tmm

using namespace tmm;

extern "C" TMM_API tmm_status tmm_coh_batched_noalloc(const tmm_problem *p, const tmm_launch_cfg *cfg, void *R,
                                                      void *T, void *stream)
{
    TraceRange trace("tmm_coh_batched_noalloc");
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if ((long long)p->S * p->n_lambda * p->n_theta == 0) return TMM_OK;
    if (p->prec == TMM_F64X) return TMM_ERR_UNSUPPORTED;  // the double-float kernel has no persistent form
    if (!R) return TMM_ERR_INVALID_ARG;
    tmm_launch_cfg c = cfg ? *cfg : tmm_launch_cfg{};
    if (c.tile_lambda < 0 || c.tile_theta < 0 || c.blocks_per_sm < 0 || c.max_items_per_block != 0)
        return TMM_ERR_INVALID_ARG;
    c.persistent = 1;
    if (persistent_ws_layout(p).total > kNoAllocScratchBytes) return TMM_ERR_NOMEM;
    void *scratch = nullptr;
    s = noalloc_scratch(&scratch);
    if (s != TMM_OK) return s;
    // launch_forward zeroes the counter, error flag and buckets it uses on
    // `stream` before the kernels run; the stack order is rewritten in full.
    return launch_forward(p, &c, scratch, kNoAllocScratchBytes, R, T, static_cast<cudaStream_t>(stream));
}
