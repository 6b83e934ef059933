// tmm_opt.cu -- merit-driven thickness optimisation (the use case of the
// paper's Fig. 1c): many-start Adam over d on top of the adjoint merit
// gradient (tmm_grad.cu).  Each step is two launches on the caller's stream:
// the merit/gradient kernel(s) and an element-wise Adam update of every
// finite layer of every stack; the moment estimates live in the caller's
// workspace between steps and calls.
#include <cuda_runtime.h>

#include <cmath>

#include "tmm_device.cuh"
#include "tmm_internal.h"

namespace tmm {

namespace {

// Workspace sections, each 256-byte aligned: m, v, g [S][L_max]; merit [S];
// the gradient launch's own workspace.
struct OptWs {
    size_t m = 0, v = 0, g = 0, merit = 0, grad = 0, grad_bytes = 0, total = 0;
};

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

OptWs opt_layout(const tmm_problem *p)
{
    const size_t r = real_size(p->prec);
    const size_t n = up256((size_t)p->S * p->L_max * r);
    OptWs w;
    w.m = 0;
    w.v = w.m + n;
    w.g = w.v + n;
    w.merit = w.g + n;
    w.grad = w.merit + up256((size_t)p->S * r);
    w.grad_bytes = grad_ws_bytes(p);
    w.total = w.grad + up256(w.grad_bytes);
    return w;
}

// One Adam step on element (s, j) of d [S][L_max] for j < L_s.  c1, c2 are the
// bias corrections 1 / (1 - beta^t), formed on the host in double.
template <typename R>
__global__ void adam_update(const tmm_problem p, const R *__restrict__ g, R *__restrict__ m, R *__restrict__ v,
                            R *__restrict__ d, R lr, R b1, R b2, R eps, R c1, R c2, R d_min, R d_max)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)p.S * p.L_max) return;
    const int s = (int)(i / p.L_max), j = (int)(i - (long long)s * p.L_max);
    if (j >= layers_of(p, s)) return;  // also skips stacks with an invalid L_s
    const R gi = g[i];
    const R mi = b1 * m[i] + (R(1) - b1) * gi;
    const R vi = b2 * v[i] + (R(1) - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const R step = lr * (mi * c1) / (sqrt(vi * c2) + eps);
    d[i] = fmin(fmax(d[i] - step, d_min), d_max);
}

template <typename R>
tmm_status launch_update(const tmm_problem *p, unsigned char *ws, const OptWs &L, const tmm_adam_cfg *cfg, int t,
                         cudaStream_t st)
{
    const long long n = (long long)p->S * p->L_max;
    if (n == 0) return TMM_OK;
    const double c1 = 1.0 / (1.0 - std::pow(cfg->beta1, (double)t));
    const double c2 = 1.0 / (1.0 - std::pow(cfg->beta2, (double)t));
    const unsigned blocks = (unsigned)((n + 255) / 256);
    adam_update<R><<<blocks, 256, 0, st>>>(*p, reinterpret_cast<const R *>(ws + L.g), reinterpret_cast<R *>(ws + L.m),
                                           reinterpret_cast<R *>(ws + L.v),
                                           const_cast<R *>(static_cast<const R *>(p->d)), (R)cfg->lr, (R)cfg->beta1,
                                           (R)cfg->beta2, (R)cfg->eps, (R)c1, (R)c2, (R)cfg->d_min, (R)cfg->d_max);
    return check_launch();
}

}  // namespace

}  // namespace tmm

using namespace tmm;

extern "C" TMM_API tmm_status tmm_optimize_workspace_size(const tmm_problem *p, size_t *bytes)
{
    if (!bytes) return TMM_ERR_INVALID_ARG;
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if ((p->prec != TMM_F64 && p->prec != TMM_F32) || (p->pol_mask & TMM_POL_AVG)) return TMM_ERR_UNSUPPORTED;
    *bytes = p->S == 0 ? 0 : opt_layout(p).total;
    return TMM_OK;
}

extern "C" TMM_API tmm_status tmm_optimize_adam(const tmm_problem *p, const void *R_target, const tmm_adam_cfg *cfg,
                                                int32_t steps, void *merit_hist, void *workspace,
                                                size_t workspace_bytes, void *stream)
{
    TraceRange trace("tmm_optimize_adam");
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if ((p->prec != TMM_F64 && p->prec != TMM_F32) || (p->pol_mask & TMM_POL_AVG)) return TMM_ERR_UNSUPPORTED;
    if (!cfg || steps < 0 || cfg->step0 < 0) return TMM_ERR_INVALID_ARG;
    if (!(cfg->lr > 0.0) || !(cfg->beta1 >= 0.0 && cfg->beta1 < 1.0) || !(cfg->beta2 >= 0.0 && cfg->beta2 < 1.0) ||
        !(cfg->eps > 0.0) || !(cfg->d_min <= cfg->d_max))
        return TMM_ERR_INVALID_ARG;
    if (p->S == 0 || steps == 0) return TMM_OK;
    if (p->n_lambda == 0 || p->n_theta == 0 || !R_target || !p->d) return TMM_ERR_INVALID_ARG;
    const OptWs L = opt_layout(p);
    if (!workspace || workspace_bytes < L.total) return TMM_ERR_NOMEM;
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return TMM_ERR_INVALID_ARG;
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t r = real_size(p->prec);
    if (cfg->step0 == 0) {
        cudaError_t e = cudaMemsetAsync(ws + L.m, 0, L.g - L.m, st);  // m and v
        if (e != cudaSuccess) return cuda_fail(e);
    }
    for (int k = 0; k < steps; ++k) {
        unsigned char *merit =
            merit_hist ? static_cast<unsigned char *>(merit_hist) + (size_t)k * p->S * r : ws + L.merit;
        s = launch_grad(p, R_target, merit, ws + L.g, nullptr, L.grad_bytes ? ws + L.grad : nullptr, L.grad_bytes,
                        st);
        if (s != TMM_OK) return s;
        const int t = cfg->step0 + k + 1;
        s = p->prec == TMM_F64 ? launch_update<double>(p, ws, L, cfg, t, st)
                               : launch_update<float>(p, ws, L, cfg, t, st);
        if (s != TMM_OK) return s;
    }
    return TMM_OK;
}
