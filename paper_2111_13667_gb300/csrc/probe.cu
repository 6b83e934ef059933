// probe.cu -- issue-rate probe: independent FMA chains in the working type on
// every SM, timed with CUDA events.  Used to put a measured figure beside the
// unit-count peak when reporting the arithmetic roofline.
#include <cuda_runtime.h>

#include "tmm_internal.h"

namespace tmm {

constexpr int kChains = 8;

// Store target that keeps the chains from being optimised away.
__device__ double tmm_probe_sink;

template <typename R>
__global__ void __launch_bounds__(256) fma_chains(int iters, R a, R b)
{
    R v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = R(threadIdx.x + c) * R(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
    }
    R acc = R(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += v[c];
    if (acc == R(12345.678)) tmm_probe_sink = (double)acc;
}

template <typename R>
static tmm_status probe(double *flops, float *ms_out, cudaStream_t st, int iters)
{
    DeviceInfo di;
    tmm_status s = device_info(&di);
    if (s != TMM_OK) return s;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(e); }
    const int blocks = di.sms * 8, threads = 256;
    // warm-up launch, then the timed one
    fma_chains<R><<<blocks, threads, 0, st>>>(iters / 8 + 1, R(0.999999), R(1e-7));
    cudaEventRecord(e0, st);
    fma_chains<R><<<blocks, threads, 0, st>>>(iters, R(0.999999), R(1e-7));
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e);
    s = check_launch();
    if (s != TMM_OK) return s;
    *flops = 2.0 * kChains * (double)iters * blocks * threads / (ms * 1e-3);
    *ms_out = ms;
    return TMM_OK;
}

}  // namespace tmm

extern "C" tmm_status tmm_probe_fma_rate(int32_t prec, double *flops_per_s, float *ms, void *stream)
{
    if (!flops_per_s || !ms) return TMM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (prec == TMM_F64) return tmm::probe<double>(flops_per_s, ms, st, 1 << 12);
    if (prec == TMM_F32) return tmm::probe<float>(flops_per_s, ms, st, 1 << 16);
    return TMM_ERR_INVALID_ARG;
}
