// tmm_internal.h -- host-side declarations shared by the translation units of
// libtmm (launchers behind the C ABI).  Not part of the public interface.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/tmm.h"

namespace tmm {

// A named NVTX range around one ABI call, so that Nsight Systems timelines and
// ncu's range filters show the library's calls by name; with no tool
// attached the push and pop are no-ops.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

struct Tile {
    int TL = 0, TT = 0;        // wavelengths x angles per work item
    int n_lt = 0, n_tt = 0;    // tiles along lambda / theta
    long long n_items = 0;     // S * n_lt * n_tt
    size_t smem = 0;           // dynamic shared memory per block
};

// Device facts cached per device (SM count, opt-in shared memory limit).
struct DeviceInfo {
    int sms = 0;
    int max_smem_optin = 0;
};
tmm_status device_info(DeviceInfo *out);

// Largest dynamic shared memory a block of these kernels can be given on
// sm_103a (227 KiB opt-in); a stage larger than this is rejected before any
// device query.
constexpr size_t kSmemBlockCeiling = 227 * 1024;

// Allow the kernel fn to be launched with `bytes` of dynamic shared memory on
// the current device.  Above the 48 KiB default the attribute is raised to the
// largest size asked for so far and never lowered, under one process-wide
// lock: a launch of another size, in this host thread or another, cannot
// shrink the limit below what an earlier check granted.
tmm_status ensure_dynamic_smem(const void *fn, size_t bytes);

int npol(uint32_t pol_mask);
// Bytes of the working real type of the outputs (float for TMM_F32 and TMM_F32D).
size_t real_size(int prec);

// Host-side validation of a problem (sizes, pointers, modes).
tmm_status validate_problem(const tmm_problem *p);

// Tile choice for a forward launch (cfg fields of 0 take defaults).
tmm_status choose_tile(const tmm_problem *p, const tmm_launch_cfg *cfg, Tile *t);

// Workspace layout of a persistent forward launch.
struct PersistentWs {
    size_t counter = 0, err = 0, counts = 0, offsets = 0, order = 0, total = 0;
};
PersistentWs persistent_ws_layout(const tmm_problem *p);

tmm_status launch_forward(const tmm_problem *p, const tmm_launch_cfg *cfg, void *ws, size_t ws_bytes,
                          void *R, void *T, cudaStream_t st);
// Per-stack reward -sum |R_target - R| (forward kernels in reduction mode).
tmm_status reward_layout(const tmm_problem *p, const tmm_launch_cfg *cfg, Tile *t, size_t *partial_bytes,
                         size_t *total);
tmm_status launch_reward(const tmm_problem *p, const tmm_launch_cfg *cfg, const void *R_target, void *reward,
                         void *ws, size_t ws_bytes, cudaStream_t st);
// {sin, cos} of 2 pi k / 256 as float pairs (host-built, passed to kernels by value).
struct SinCosTable;
const SinCosTable &sincos_table();

tmm_status launch_forward_df64(const tmm_problem *p, const tmm_launch_cfg *cfg, void *R, void *T, cudaStream_t st);

// Adjoint / merit.
size_t grad_ws_bytes(const tmm_problem *p);
tmm_status launch_grad(const tmm_problem *p, const void *R_target, void *merit, void *dm_dd,
                       void *dm_dn, void *ws, size_t ws_bytes, cudaStream_t st);

// Record a CUDA error for tmm_last_cuda_error and map it to a status.
tmm_status cuda_fail(cudaError_t e);
tmm_status check_launch();

}  // namespace tmm
