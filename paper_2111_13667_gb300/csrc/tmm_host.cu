// tmm_host.cu -- tmm_coh_batched_host: the forward evaluation for a problem
// whose arrays live in host memory, with the device traffic pipelined against
// the kernels.
//
// The inputs go to the device once (they are small next to the outputs); the
// stacks then run in contiguous chunks on the caller's stream, each chunk
// writing R and T into one of three device slots, and a copy stream brings
// every finished slot back into the caller's host arrays while the next two
// chunks run.  A slot is reused only after its copy has finished (events), so
// the kernels never wait for the copies unless the copies are the slower side.
#include <cuda_runtime.h>

#include <algorithm>

#include "tmm_internal.h"

namespace tmm {

namespace {

constexpr int kSlots = 3;

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Bytes of every input array of p (host layout = device layout).
struct InputSizes {
    size_t n_direct = 0, table = 0, mat_idx = 0, d = 0, Ls = 0, theta = 0, lambda = 0;
};

size_t in_real(const tmm_problem *p) { return p->prec == TMM_F32 ? sizeof(float) : sizeof(double); }

InputSizes input_sizes(const tmm_problem *p)
{
    InputSizes z;
    const size_t r = in_real(p);
    const size_t rows = (size_t)p->S * (p->L_max + 2);
    if (p->n_direct) z.n_direct = rows * (p->n_direct_per_lambda ? (size_t)p->n_lambda : 1) * 2 * r;
    if (p->mat_table) z.table = (size_t)p->n_materials * p->n_lambda * 2 * r;
    if (p->mat_idx) z.mat_idx = rows * sizeof(int32_t);
    z.d = (size_t)p->S * p->L_max * r;
    if (p->L_per_stack) z.Ls = (size_t)p->S * sizeof(int32_t);
    z.theta = (size_t)p->n_theta * r;
    z.lambda = (size_t)p->n_lambda * r;
    return z;
}

struct HostLayout {
    size_t n_direct, table, mat_idx, d, Ls, theta, lambda, slots, slot_bytes, total;
    int chunk;  // stacks per chunk (the last may be shorter)
};

HostLayout host_layout(const tmm_problem *p, int n_chunks)
{
    const InputSizes z = input_sizes(p);
    HostLayout h;
    size_t o = 0;
    h.n_direct = o, o += align256(z.n_direct);
    h.table = o, o += align256(z.table);
    h.mat_idx = o, o += align256(z.mat_idx);
    h.d = o, o += align256(z.d);
    h.Ls = o, o += align256(z.Ls);
    h.theta = o, o += align256(z.theta);
    h.lambda = o, o += align256(z.lambda);
    h.chunk = (p->S + n_chunks - 1) / n_chunks;
    const int P = (p->pol_mask & TMM_POL_AVG) ? 1 : npol(p->pol_mask);
    // one slot holds a chunk's R and T: [2][P][chunk][n_theta][n_lambda]
    h.slot_bytes = align256((size_t)2 * P * h.chunk * p->n_theta * p->n_lambda * real_size(p->prec));
    h.slots = o;
    h.total = o + kSlots * h.slot_bytes;
    return h;
}

tmm_status copy_in(void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    if (!bytes) return TMM_OK;
    const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    return e == cudaSuccess ? TMM_OK : cuda_fail(e);
}

}  // namespace

}  // namespace tmm

using namespace tmm;

extern "C" {

TMM_API tmm_status tmm_host_workspace_size(const tmm_problem *p, int32_t n_chunks, size_t *bytes)
{
    if (!bytes) return TMM_ERR_INVALID_ARG;
    const tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if (p->S > 0 && (n_chunks < 1 || n_chunks > p->S)) return TMM_ERR_INVALID_ARG;
    *bytes = p->S > 0 ? host_layout(p, n_chunks).total : 0;
    return TMM_OK;
}

TMM_API tmm_status tmm_coh_batched_host(const tmm_problem *p, int32_t n_chunks, void *workspace,
                                        size_t workspace_bytes, void *R, void *T, void *stream)
{
    TraceRange trace("tmm_coh_batched_host");
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if ((long long)p->S * p->n_lambda * p->n_theta == 0) return TMM_OK;
    if (!R || n_chunks < 1 || n_chunks > p->S || !workspace) return TMM_ERR_INVALID_ARG;
    const HostLayout h = host_layout(p, n_chunks);
    if (workspace_bytes < h.total) return TMM_ERR_NOMEM;
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return TMM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    const InputSizes z = input_sizes(p);

    // the problem on the device
    tmm_problem dp = *p;
    if ((s = copy_in(ws + h.n_direct, p->n_direct, z.n_direct, st)) != TMM_OK) return s;
    if ((s = copy_in(ws + h.table, p->mat_table, z.table, st)) != TMM_OK) return s;
    if ((s = copy_in(ws + h.mat_idx, p->mat_idx, z.mat_idx, st)) != TMM_OK) return s;
    if ((s = copy_in(ws + h.d, p->d, z.d, st)) != TMM_OK) return s;
    if ((s = copy_in(ws + h.Ls, p->L_per_stack, z.Ls, st)) != TMM_OK) return s;
    if ((s = copy_in(ws + h.theta, p->theta, z.theta, st)) != TMM_OK) return s;
    if ((s = copy_in(ws + h.lambda, p->lambda, z.lambda, st)) != TMM_OK) return s;
    dp.n_direct = p->n_direct ? ws + h.n_direct : nullptr;
    dp.mat_table = p->mat_table ? ws + h.table : nullptr;
    dp.mat_idx = p->mat_idx ? reinterpret_cast<const int32_t *>(ws + h.mat_idx) : nullptr;
    dp.d = ws + h.d;
    dp.L_per_stack = p->L_per_stack ? reinterpret_cast<const int32_t *>(ws + h.Ls) : nullptr;
    dp.theta = ws + h.theta;
    dp.lambda = ws + h.lambda;

    cudaStream_t cs = nullptr;
    cudaEvent_t done[kSlots] = {}, freed[kSlots] = {};
    auto release = [&]() {
        for (int i = 0; i < kSlots; ++i) {
            if (done[i]) cudaEventDestroy(done[i]);
            if (freed[i]) cudaEventDestroy(freed[i]);
        }
        if (cs) cudaStreamDestroy(cs);  // releases once its queued copies have run
    };
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int i = 0; i < kSlots && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&freed[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        release();
        return cuda_fail(e);
    }

    const int P = (p->pol_mask & TMM_POL_AVG) ? 1 : npol(p->pol_mask);
    const size_t rs = real_size(p->prec);
    const size_t row = (size_t)p->n_theta * p->n_lambda * rs;  // one stack's plane
    const size_t full_plane = (size_t)p->S * row;
    const size_t lrow = (size_t)(p->L_max + 2);
    s = TMM_OK;
    for (int c = 0, s0 = 0; s0 < p->S && s == TMM_OK; ++c, s0 += h.chunk) {
        const int n = std::min(h.chunk, p->S - s0);
        const int slot = c % kSlots;
        unsigned char *Rd = ws + h.slots + (size_t)slot * h.slot_bytes;
        unsigned char *Td = Rd + (size_t)P * n * row;
        if (c >= kSlots && (e = cudaStreamWaitEvent(st, freed[slot], 0)) != cudaSuccess) {
            s = cuda_fail(e);
            break;
        }
        tmm_problem cp = dp;
        cp.S = n;
        cp.d = static_cast<const unsigned char *>(dp.d) + (size_t)s0 * p->L_max * in_real(p);
        if (dp.n_direct)
            cp.n_direct = static_cast<const unsigned char *>(dp.n_direct) +
                          (size_t)s0 * lrow * (p->n_direct_per_lambda ? (size_t)p->n_lambda : 1) * 2 * in_real(p);
        if (dp.mat_idx) cp.mat_idx = dp.mat_idx + (size_t)s0 * lrow;
        if (dp.L_per_stack) cp.L_per_stack = dp.L_per_stack + s0;
        if ((s = launch_forward(&cp, nullptr, nullptr, 0, Rd, T ? Td : nullptr, st)) != TMM_OK) break;
        if ((e = cudaEventRecord(done[slot], st)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, done[slot], 0)) != cudaSuccess) {
            s = cuda_fail(e);
            break;
        }
        // R (and T): P planes of n stacks each, into the host planes of S stacks
        for (int k = 0; k < (T ? 2 : 1) && e == cudaSuccess; ++k) {
            unsigned char *src = k ? Td : Rd;
            unsigned char *dst = static_cast<unsigned char *>(k ? T : R) + (size_t)s0 * row;
            e = cudaMemcpy2DAsync(dst, full_plane, src, (size_t)n * row, (size_t)n * row, P, cudaMemcpyDeviceToHost, cs);
        }
        if (e == cudaSuccess) e = cudaEventRecord(freed[slot], cs);
        if (e != cudaSuccess) s = cuda_fail(e);
    }
    // the caller's stream completes only after the last copy
    if (s == TMM_OK) {
        e = cudaEventRecord(freed[0], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, freed[0], 0);
        if (e != cudaSuccess) s = cuda_fail(e);
    }
    release();
    return s;
}

}  // extern "C"
