// tmm_grad.cu -- adjoint (reverse-sweep) gradient of the per-stack merit.
#include <cuda_runtime.h>

#include "tmm_device.cuh"
#include "tmm_internal.h"

namespace tmm {

size_t grad_ws_bytes(const tmm_problem *) { return 0; }

tmm_status launch_grad(const tmm_problem *, const void *, void *, void *, void *, void *, size_t, cudaStream_t)
{
    return TMM_ERR_UNSUPPORTED;
}

}  // namespace tmm
