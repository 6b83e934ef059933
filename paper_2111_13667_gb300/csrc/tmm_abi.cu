// tmm_abi.cu -- the extern "C" boundary of libtmm: host-side argument checks,
// status and error reporting, and dispatch to the launchers.
#include <cuda_runtime.h>

#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "tmm_internal.h"

namespace tmm {

static thread_local char g_last_cuda_error[256] = "no error";

tmm_status cuda_fail(cudaError_t e)
{
    std::snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", cudaGetErrorName(e),
                  cudaGetErrorString(e));
    return TMM_ERR_CUDA;
}

tmm_status check_launch()
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TMM_OK : cuda_fail(e);
}

tmm_status device_info(DeviceInfo *out)
{
    static std::mutex mu;
    static DeviceInfo cache[64];
    static bool have[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= 64) return TMM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(mu);
    if (!have[dev]) {
        DeviceInfo di;
        e = cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e);
        e = cudaDeviceGetAttribute(&di.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return cuda_fail(e);
        // leave room for the kernels' static shared memory
        di.max_smem_optin -= 1024;
        cache[dev] = di;
        have[dev] = true;
    }
    *out = cache[dev];
    return TMM_OK;
}

tmm_status ensure_dynamic_smem(const void *fn, size_t bytes)
{
    if (bytes <= 48 * 1024) return TMM_OK;
    if (bytes > (size_t)0x7fffffff) return TMM_ERR_UNSUPPORTED;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    struct Granted {
        const void *fn;
        int dev;
        size_t bytes;
    };
    static std::mutex mu;
    static std::vector<Granted> granted;
    std::lock_guard<std::mutex> lk(mu);
    Granted *g = nullptr;
    for (auto &x : granted)
        if (x.fn == fn && x.dev == dev) g = &x;
    if (g && g->bytes >= bytes) return TMM_OK;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(e);
    if (g)
        g->bytes = bytes;
    else
        granted.push_back(Granted{fn, dev, bytes});
    return TMM_OK;
}

int npol(uint32_t pol_mask) { return (int)(pol_mask & 1u) + (int)((pol_mask >> 1) & 1u); }

size_t real_size(int prec) { return (prec == TMM_F32 || prec == TMM_F32D) ? sizeof(float) : sizeof(double); }

tmm_status validate_problem(const tmm_problem *p)
{
    if (!p) return TMM_ERR_INVALID_ARG;
    if (p->S < 0 || p->L_max < 0 || p->n_lambda < 0 || p->n_theta < 0) return TMM_ERR_INVALID_ARG;
    if (p->pol_mask == 0 || p->pol_mask > 7u) return TMM_ERR_INVALID_ARG;
    if ((p->pol_mask & TMM_POL_AVG) && (p->pol_mask & 3u) != 3u) return TMM_ERR_INVALID_ARG;
    if (p->prec != TMM_F64 && p->prec != TMM_F32 && p->prec != TMM_F64X && p->prec != TMM_F32D)
        return TMM_ERR_INVALID_ARG;
    if (p->n_direct_per_lambda != 0 && p->n_direct_per_lambda != 1) return TMM_ERR_INVALID_ARG;
    // an empty batch reads no array, so its pointers are not checked
    if ((long long)p->S * p->n_lambda * p->n_theta == 0) return TMM_OK;
    const bool direct = p->n_direct != nullptr;
    const bool gathered = p->mat_table != nullptr || p->mat_idx != nullptr;
    if (direct == gathered) return TMM_ERR_INVALID_ARG;
    if (gathered && (!p->mat_table || !p->mat_idx || p->n_materials < 1)) return TMM_ERR_INVALID_ARG;
    const bool any = (long long)p->S * p->n_lambda * p->n_theta > 0;
    if (any) {
        if (!p->theta || !p->lambda) return TMM_ERR_INVALID_ARG;
        if (p->L_max > 0 && !p->d) return TMM_ERR_INVALID_ARG;
    }
    if ((long long)p->L_max + 2 > (1 << 20)) return TMM_ERR_UNSUPPORTED;
    return TMM_OK;
}

}  // namespace tmm

using namespace tmm;

extern "C" {

tmm_status tmm_coh_batched_ex(const tmm_problem *p, const tmm_launch_cfg *cfg, void *workspace,
                              size_t workspace_bytes, void *R, void *T, void *stream)
{
    TraceRange trace("tmm_coh_batched_ex");
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if ((long long)p->S * p->n_lambda * p->n_theta == 0) return TMM_OK;
    if (!R) return TMM_ERR_INVALID_ARG;
    if (cfg && (cfg->tile_lambda < 0 || cfg->tile_theta < 0 || cfg->blocks_per_sm < 0 ||
                cfg->max_items_per_block < 0 || (cfg->persistent != 0 && cfg->persistent != 1)))
        return TMM_ERR_INVALID_ARG;
    return launch_forward(p, cfg, workspace, workspace_bytes, R, T, static_cast<cudaStream_t>(stream));
}

tmm_status tmm_coh_batched(const tmm_problem *p, void *R, void *T, void *stream)
{
    return tmm_coh_batched_ex(p, nullptr, nullptr, 0, R, T, stream);
}

tmm_status tmm_workspace_size(const tmm_problem *p, const tmm_launch_cfg *cfg, size_t *bytes)
{
    if (!bytes) return TMM_ERR_INVALID_ARG;
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    size_t need = grad_ws_bytes(p);
    if (cfg && cfg->persistent) need = std::max(need, persistent_ws_layout(p).total);
    *bytes = need;
    return TMM_OK;
}

tmm_status tmm_workspace_status(const void *workspace, void *stream)
{
    if (!workspace) return TMM_ERR_INVALID_ARG;
    int err = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned char *base = static_cast<const unsigned char *>(workspace);
    cudaError_t e = cudaMemcpyAsync(&err, base + 4, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    return err ? TMM_ERR_TIMEOUT : TMM_OK;
}

tmm_status tmm_coh_grad(const tmm_problem *p, const void *R_target, void *merit, void *dm_dd, void *dm_dn,
                        void *workspace, size_t workspace_bytes, void *stream)
{
    TraceRange trace("tmm_coh_grad");
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if (p->S == 0) return TMM_OK;
    if (p->n_lambda == 0 || p->n_theta == 0) return TMM_ERR_INVALID_ARG;
    if (!R_target || !merit || (p->L_max > 0 && !dm_dd)) return TMM_ERR_INVALID_ARG;
    if ((p->prec != TMM_F64 && p->prec != TMM_F32) || (p->pol_mask & TMM_POL_AVG)) return TMM_ERR_UNSUPPORTED;
    return launch_grad(p, R_target, merit, dm_dd, dm_dn, workspace, workspace_bytes,
                       static_cast<cudaStream_t>(stream));
}

tmm_status tmm_reward_workspace_size(const tmm_problem *p, const tmm_launch_cfg *cfg, size_t *bytes)
{
    if (!bytes) return TMM_ERR_INVALID_ARG;
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if (p->prec != TMM_F64 && p->prec != TMM_F32) return TMM_ERR_UNSUPPORTED;
    if (p->S == 0 || p->n_lambda == 0 || p->n_theta == 0) {
        *bytes = 0;
        return TMM_OK;
    }
    Tile t;
    size_t part = 0;
    return reward_layout(p, cfg, &t, &part, bytes);
}

tmm_status tmm_coh_reward(const tmm_problem *p, const tmm_launch_cfg *cfg, const void *R_target, void *reward,
                          void *workspace, size_t workspace_bytes, void *stream)
{
    TraceRange trace("tmm_coh_reward");
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if (p->prec != TMM_F64 && p->prec != TMM_F32) return TMM_ERR_UNSUPPORTED;
    if (cfg && (cfg->persistent < 0 || cfg->persistent > 1 || cfg->max_items_per_block != 0))
        return TMM_ERR_INVALID_ARG;
    if (p->S == 0) return TMM_OK;
    if (!R_target || !reward) return TMM_ERR_INVALID_ARG;
    if (p->n_lambda == 0 || p->n_theta == 0) {  // an empty sum
        cudaError_t e = cudaMemsetAsync(reward, 0, (size_t)p->S * real_size(p->prec), static_cast<cudaStream_t>(stream));
        return e == cudaSuccess ? TMM_OK : cuda_fail(e);
    }
    return launch_reward(p, cfg, R_target, reward, workspace, workspace_bytes, static_cast<cudaStream_t>(stream));
}

const char *tmm_status_string(int status)
{
    switch (status) {
    case TMM_OK: return "ok";
    case TMM_ERR_INVALID_ARG: return "invalid argument";
    case TMM_ERR_UNSUPPORTED: return "unsupported by this build";
    case TMM_ERR_CUDA: return "CUDA error";
    case TMM_ERR_TIMEOUT: return "device iteration limit reached";
    case TMM_ERR_NOMEM: return "workspace too small or out of memory";
    default: return "unknown status";
    }
}

const char *tmm_last_cuda_error(void) { return g_last_cuda_error; }

int32_t tmm_version(void) { return 100; }

}  // extern "C"
