// surrogate.cu -- the learned surrogate: an MLP from layer thicknesses to the
// R spectra (s and p, every theta and lambda) of a fixed stack, trained on
// spectra that the library's own transfer-matrix kernel generates, run on the
// tcgen05 bf16 GEMM with fp32 accumulation, and judged by the exact
// transfer-matrix kernel with a per-row fallback.
//
// Network: x = (d - d_min) / (d_max - d_min) in [0, 1] (L inputs, zero-padded to
// 64), `depth` hidden layers of width `hidden` with GELU (erf form), a linear
// head of 2 n_theta n_lambda outputs (clamped to [0, 1] at inference).
// Training: MSE loss, Adam on fp32 master weights; every GEMM of the forward
// and backward pass is the tcgen05 kernel (weight gradients from transposed
// activations the forward epilogues write alongside).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "tcgen05_gemm.cuh"
#include "tmm_internal.h"

namespace tmm {
namespace gemm {
tmm_status gemm(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M, int N, int K, EpiArgs ep,
                cudaStream_t st);
tmm_status clear_error(cudaStream_t st);
tmm_status gemm_status(cudaStream_t st);
tmm_status flag_status(const int *flag, cudaStream_t st);
int *error_flag();
}  // namespace gemm

namespace sur {

constexpr int KIN = 64;  // padded input width (TMA rows must be 16-byte multiples)

struct Layer {
    int N = 0, K = 0, Kvalid = 0;
    float *W = nullptr, *b = nullptr, *mW = nullptr, *vW = nullptr, *mb = nullptr, *vb = nullptr;
    float *dW = nullptr, *db = nullptr;
    __nv_bfloat16 *Wb = nullptr, *WbT = nullptr;
};

// ---------------------------------------------------------------- kernels
__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    // splitmix64 finaliser (Steele, Lea, Flood 2014)
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__global__ void init_weights(float *W, int N, int K, int Kvalid, float stdv, uint64_t seed)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)N * K) return;
    const int k = (int)(i % K);
    if (k >= Kvalid) {
        W[i] = 0.0f;
        return;
    }
    // Box-Muller on two counter-based uniforms
    const uint64_t r = mix64(seed ^ mix64((uint64_t)i));
    const float u1 = ((r >> 40) + 0.5f) * (1.0f / 16777216.0f);
    const float u2 = (((r >> 16) & 0xFFFFFF) + 0.5f) * (1.0f / 16777216.0f);
    W[i] = stdv * sqrtf(-2.0f * logf(u1)) * cosf(6.2831853f * u2);
}

__global__ void to_bf16_pair(const float *W, __nv_bfloat16 *Wb, __nv_bfloat16 *WbT, int N, int K)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)N * K) return;
    const int n = (int)(i / K), k = (int)(i % K);
    const __nv_bfloat16 v = __float2bfloat16(W[i]);
    Wb[i] = v;
    WbT[(long long)k * N + n] = v;
}

__global__ void normalize_input(const float *d, int B, int L, float lo, float inv_span, __nv_bfloat16 *X,
                                __nv_bfloat16 *XT)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B * KIN) return;
    const int r = (int)(i / KIN), k = (int)(i % KIN);
    float x = 0.0f;
    if (k < L) x = (d[(long long)r * L + k] - lo) * inv_span;  // in [0, 1]
    const __nv_bfloat16 v = __float2bfloat16(x);
    X[i] = v;
    if (XT) XT[(long long)k * B + r] = v;
}

// dY = scale (Y - T) in bf16, row-major and transposed; loss += mean (Y - T)^2.
__global__ void loss_grad(const float *Y, const float *T, int B, int O, float scale, __nv_bfloat16 *dY,
                          __nv_bfloat16 *dYT, float *loss)
{
    __shared__ float tile[32][33];
    __shared__ float red[8];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    float acc = 0.0f;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        float g = 0.0f;
        if (r < B && c < O) {
            const float e = Y[(long long)r * O + c] - T[(long long)r * O + c];
            acc += e * e;
            g = scale * e;
            dY[(long long)r * O + c] = __float2bfloat16(g);
        }
        tile[k][threadIdx.x] = g;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < B && c < O) dYT[(long long)c * B + r] = __float2bfloat16(tile[threadIdx.x][k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) red[threadIdx.y] = acc;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        float s = 0.0f;
        for (int w = 0; w < 8; ++w) s += red[w];
        atomicAdd(loss, s / ((float)B * (float)O));
    }
}

// Column sums of a bf16 [B][N] matrix in two fixed-order passes.
__global__ void colsum_partial(const __nv_bfloat16 *X, int B, int N, int rows_per, float *part)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int r0 = blockIdx.y * rows_per, r1 = min(B, r0 + rows_per);
    float s = 0.0f;
    for (int r = r0; r < r1; ++r) s += __bfloat162float(X[(long long)r * N + c]);
    part[(long long)blockIdx.y * N + c] = s;
}

__global__ void colsum_final(const float *part, int chunks, int N, float *out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    float s = 0.0f;
    for (int k = 0; k < chunks; ++k) s += part[(long long)k * N + c];
    out[c] = s;
}

__global__ void adam_update(float *w, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

__global__ void gather_rows(const float *d, int L, int stride, int Bj, float *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)Bj * L) return;
    const int r = (int)(i / L), k = (int)(i % L);
    out[i] = d[((long long)r * stride) * L + k];
}

__global__ void fill_index(const float2 *row, int Lp2, int S, float2 *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (long long)S * Lp2) out[i] = row[i % Lp2];
}

// [P][S][nt][nl] (transfer-matrix output) -> [S][P nt nl]
__global__ void permute_spectra(const float *in, int P, int S, int per, float *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)P * S * per) return;
    const int p = (int)(i / ((long long)S * per));
    const long long rem = i - (long long)p * S * per;
    const int s = (int)(rem / per), k = (int)(rem % per);
    out[(long long)s * P * per + (long long)p * per + k] = in[i];
}

// One block per judged row: largest |R_surrogate - R_exact|; rows above tol
// are replaced by the exact spectrum.
__global__ void judge_rows(float *R, const float *exact, int P, int Bj, int per, int stride, float tol, int *n_fallback,
                           unsigned int *max_err_bits)
{
    __shared__ float red[32];
    const int k = blockIdx.x;
    const long long row = (long long)k * stride;
    const int O = P * per;
    float m = 0.0f;
    for (int c = threadIdx.x; c < O; c += blockDim.x) {
        const int p = c / per, q = c - p * per;
        const float e = exact[((long long)p * Bj + k) * per + q];
        m = fmaxf(m, fabsf(R[row * O + c] - e));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) {
            red[0] = m;
            atomicMax(max_err_bits, __float_as_uint(m));
            if (m > tol) atomicAdd(n_fallback, 1);
        }
    }
    __syncthreads();
    if (red[0] > tol) {
        for (int c = threadIdx.x; c < O; c += blockDim.x) {
            const int p = c / per, q = c - p * per;
            R[row * O + c] = exact[((long long)p * Bj + k) * per + q];
        }
    }
}

static unsigned blocks_for(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace sur
}  // namespace tmm

using namespace tmm;
using namespace tmm::sur;

struct tmm_surrogate {
    int L = 0, nl = 0, nt = 0, O = 0, hidden = 0, depth = 0;
    float d_min = 0, d_max = 1;
    uint64_t seed = 0;
    long long step = 0;
    float2 *n_row = nullptr;  // complex64 [L+2]
    float *theta = nullptr, *lam = nullptr;
    std::vector<Layer> layers;
    std::vector<void *> owned;  // every device allocation of the object
    // batch buffers (grown on demand)
    int cap = 0;
    std::vector<void *> batch;
    __nv_bfloat16 *X0 = nullptr, *X0T = nullptr, *dY = nullptr, *dYT = nullptr;
    std::vector<__nv_bfloat16 *> H, Z, HT;
    __nv_bfloat16 *dZ[2] = {nullptr, nullptr}, *dZT[2] = {nullptr, nullptr};
    float *Y = nullptr, *part = nullptr, *loss_tmp = nullptr;
    // judge buffers
    int jcap = 0;
    std::vector<void *> jbuf;
    float *jd = nullptr, *jout = nullptr;
    float2 *jn = nullptr;
    int *jcount = nullptr;
    unsigned int *jmax = nullptr;
    int *err = nullptr;  // this object's GEMM pipeline-timeout flag (device)
};

namespace {

template <typename T> tmm_status dalloc(std::vector<void *> &owner, T **p, size_t count)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
    if (e != cudaSuccess) return cuda_fail(e);
    owner.push_back(q);
    *p = static_cast<T *>(q);
    return TMM_OK;
}

void free_all(std::vector<void *> &v)
{
    for (void *p : v) cudaFree(p);
    v.clear();
}

tmm_status ensure_batch(tmm_surrogate *s, int B)
{
    if (B <= s->cap) return TMM_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e);
    free_all(s->batch);
    s->H.assign(s->depth, nullptr);
    s->Z.assign(s->depth, nullptr);
    s->HT.assign(s->depth, nullptr);
    const size_t b = (size_t)B, h = (size_t)s->hidden;
    tmm_status st = TMM_OK;
#define TRY(x)                   \
    if ((st = (x)) != TMM_OK) {  \
        free_all(s->batch);      \
        s->cap = 0;              \
        return st;               \
    }
    TRY(dalloc(s->batch, &s->X0, b * KIN));
    TRY(dalloc(s->batch, &s->X0T, b * KIN));
    for (int i = 0; i < s->depth; ++i) {
        TRY(dalloc(s->batch, &s->H[i], b * h));
        TRY(dalloc(s->batch, &s->Z[i], b * h));
        TRY(dalloc(s->batch, &s->HT[i], b * h));
    }
    for (int i = 0; i < 2; ++i) {
        TRY(dalloc(s->batch, &s->dZ[i], b * h));
        TRY(dalloc(s->batch, &s->dZT[i], b * h));
    }
    TRY(dalloc(s->batch, &s->Y, b * s->O));
    TRY(dalloc(s->batch, &s->dY, b * s->O));
    TRY(dalloc(s->batch, &s->dYT, b * s->O));
    TRY(dalloc(s->batch, &s->part, (size_t)64 * (s->O > (int)h ? s->O : (int)h)));
    TRY(dalloc(s->batch, &s->loss_tmp, 1));
#undef TRY
    s->cap = B;
    return TMM_OK;
}

tmm_status ensure_judge(tmm_surrogate *s, int Bj)
{
    if (Bj <= s->jcap) return TMM_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e);
    free_all(s->jbuf);
    tmm_status st;
    if ((st = dalloc(s->jbuf, &s->jd, (size_t)Bj * s->L)) != TMM_OK ||
        (st = dalloc(s->jbuf, &s->jn, (size_t)Bj * (s->L + 2))) != TMM_OK ||
        (st = dalloc(s->jbuf, &s->jout, (size_t)Bj * s->O)) != TMM_OK ||
        (st = dalloc(s->jbuf, &s->jcount, 1)) != TMM_OK || (st = dalloc(s->jbuf, &s->jmax, 1)) != TMM_OK) {
        free_all(s->jbuf);
        s->jcap = 0;
        return st;
    }
    s->jcap = Bj;
    return TMM_OK;
}

// Exact R (both polarisations) of Bj stacks with thicknesses `d`, written as
// [P][Bj][nt][nl] into s->jout (the transfer-matrix kernel, FP32).
tmm_status exact_spectra(tmm_surrogate *s, const float *d, int Bj, cudaStream_t st)
{
    fill_index<<<blocks_for((long long)Bj * (s->L + 2)), 256, 0, st>>>(s->n_row, s->L + 2, Bj, s->jn);
    tmm_status r = check_launch();
    if (r != TMM_OK) return r;
    tmm_problem p{};
    p.S = Bj;
    p.L_max = s->L;
    p.n_lambda = s->nl;
    p.n_theta = s->nt;
    p.pol_mask = TMM_POL_S | TMM_POL_P;
    p.prec = TMM_F32;
    p.n_direct = s->jn;
    p.n_direct_per_lambda = 0;
    p.d = d;
    p.theta = s->theta;
    p.lambda = s->lam;
    return launch_forward(&p, nullptr, nullptr, 0, s->jout, nullptr, st);
}

// Forward pass.  train: keep pre-activations and transposed activations.
tmm_status forward(tmm_surrogate *s, const float *d, int B, float *out, bool train, cudaStream_t st)
{
    normalize_input<<<blocks_for((long long)B * KIN), 256, 0, st>>>(d, B, s->L, s->d_min, 1.0f / (s->d_max - s->d_min),
                                                                     s->X0, train ? s->X0T : nullptr);
    tmm_status r = check_launch();
    if (r != TMM_OK) return r;
    const __nv_bfloat16 *A = s->X0;
    int K = KIN;
    for (int i = 0; i < s->depth; ++i) {
        gemm::EpiArgs ep{};
        ep.err = s->err;
        ep.epi = gemm::EPI_GELU;
        ep.bias = s->layers[i].b;
        ep.out_bf = s->H[i];
        ep.aux = train ? s->Z[i] : nullptr;
        ep.out_bfT = train ? s->HT[i] : nullptr;
        ep.ldo = s->hidden;
        ep.ldoT = B;
        r = gemm::gemm(A, K, s->layers[i].Wb, K, B, s->hidden, K, ep, st);
        if (r != TMM_OK) return r;
        A = s->H[i];
        K = s->hidden;
    }
    gemm::EpiArgs ep{};
    ep.err = s->err;
    ep.epi = train ? gemm::EPI_F32 : gemm::EPI_F32_CLAMP;
    ep.bias = s->layers[s->depth].b;
    ep.out_f32 = out;
    ep.ldo = s->O;
    return gemm::gemm(A, K, s->layers[s->depth].Wb, K, B, s->O, K, ep, st);
}

tmm_status colsum(tmm_surrogate *s, const __nv_bfloat16 *X, int B, int N, float *out, cudaStream_t st)
{
    const int chunks = 64;
    const int rows_per = (B + chunks - 1) / chunks;
    colsum_partial<<<dim3(sur::blocks_for(N), chunks), 256, 0, st>>>(X, B, N, rows_per, s->part);
    colsum_final<<<sur::blocks_for(N), 256, 0, st>>>(s->part, chunks, N, out);
    return check_launch();
}

tmm_status refresh_bf16(tmm_surrogate *s, cudaStream_t st)
{
    for (auto &l : s->layers) {
        to_bf16_pair<<<blocks_for((long long)l.N * l.K), 256, 0, st>>>(l.W, l.Wb, l.WbT, l.N, l.K);
    }
    return check_launch();
}

}  // namespace

extern "C" {

TMM_API tmm_status tmm_surrogate_create(const tmm_surrogate_desc *desc, tmm_surrogate **out)
{
    if (!desc || !out) return TMM_ERR_INVALID_ARG;
    *out = nullptr;
    if (desc->n_layers < 1 || desc->n_layers > KIN || !desc->n_media || desc->n_lambda < 1 || !desc->lambda ||
        desc->n_theta < 1 || !desc->theta || !(desc->d_max > desc->d_min) || desc->hidden < 64 ||
        desc->hidden % 64 != 0 || desc->depth < 1 || desc->depth > 16)
        return TMM_ERR_INVALID_ARG;
    if (desc->n_media[1] != 0.0) return TMM_ERR_INVALID_ARG;  // real injection medium
    tmm_surrogate *s = new (std::nothrow) tmm_surrogate();
    if (!s) return TMM_ERR_NOMEM;
    s->L = desc->n_layers;
    s->nl = desc->n_lambda;
    s->nt = desc->n_theta;
    s->O = 2 * s->nl * s->nt;
    s->hidden = desc->hidden;
    s->depth = desc->depth;
    s->d_min = (float)desc->d_min;
    s->d_max = (float)desc->d_max;
    s->seed = desc->seed;
    if (s->O % 8 != 0) {
        delete s;
        return TMM_ERR_UNSUPPORTED;
    }
    tmm_status st = TMM_OK;
    std::vector<float2> row(s->L + 2);
    for (int j = 0; j < s->L + 2; ++j) row[j] = make_float2((float)desc->n_media[2 * j], (float)desc->n_media[2 * j + 1]);
    std::vector<float> th(desc->theta, desc->theta + s->nt), la(desc->lambda, desc->lambda + s->nl);
    if ((st = dalloc(s->owned, &s->n_row, row.size())) != TMM_OK || (st = dalloc(s->owned, &s->theta, th.size())) != TMM_OK ||
        (st = dalloc(s->owned, &s->lam, la.size())) != TMM_OK || (st = dalloc(s->owned, &s->err, 1)) != TMM_OK ||
        cudaMemset(s->err, 0, sizeof(int)) != cudaSuccess) {
        if (st == TMM_OK) st = cuda_fail(cudaGetLastError());
        tmm_surrogate_destroy(s);
        return st;
    }
    cudaMemcpy(s->n_row, row.data(), row.size() * sizeof(float2), cudaMemcpyHostToDevice);
    cudaMemcpy(s->theta, th.data(), th.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(s->lam, la.data(), la.size() * sizeof(float), cudaMemcpyHostToDevice);
    // layers: depth hidden (GELU) + linear head
    for (int i = 0; i <= s->depth; ++i) {
        Layer l;
        l.K = i == 0 ? KIN : s->hidden;
        l.Kvalid = i == 0 ? s->L : s->hidden;
        l.N = i == s->depth ? s->O : s->hidden;
        const size_t nw = (size_t)l.N * l.K;
        if ((st = dalloc(s->owned, &l.W, nw)) != TMM_OK || (st = dalloc(s->owned, &l.mW, nw)) != TMM_OK ||
            (st = dalloc(s->owned, &l.vW, nw)) != TMM_OK || (st = dalloc(s->owned, &l.dW, nw)) != TMM_OK ||
            (st = dalloc(s->owned, &l.b, l.N)) != TMM_OK || (st = dalloc(s->owned, &l.mb, l.N)) != TMM_OK ||
            (st = dalloc(s->owned, &l.vb, l.N)) != TMM_OK || (st = dalloc(s->owned, &l.db, l.N)) != TMM_OK ||
            (st = dalloc(s->owned, &l.Wb, nw)) != TMM_OK || (st = dalloc(s->owned, &l.WbT, nw)) != TMM_OK) {
            tmm_surrogate_destroy(s);
            return st;
        }
        const float stdv = (i == s->depth ? 0.5f : 1.0f) / sqrtf((float)l.Kvalid);
        init_weights<<<blocks_for((long long)nw), 256>>>(l.W, l.N, l.K, l.Kvalid, stdv, s->seed + 7919ull * (i + 1));
        cudaMemset(l.mW, 0, nw * sizeof(float));
        cudaMemset(l.vW, 0, nw * sizeof(float));
        cudaMemset(l.b, 0, l.N * sizeof(float));
        cudaMemset(l.mb, 0, l.N * sizeof(float));
        cudaMemset(l.vb, 0, l.N * sizeof(float));
        s->layers.push_back(l);
    }
    if ((st = refresh_bf16(s, nullptr)) != TMM_OK) {
        tmm_surrogate_destroy(s);
        return st;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        tmm_surrogate_destroy(s);
        return cuda_fail(e);
    }
    *out = s;
    return TMM_OK;
}

TMM_API void tmm_surrogate_destroy(tmm_surrogate *s)
{
    if (!s) return;
    cudaDeviceSynchronize();
    free_all(s->batch);
    free_all(s->jbuf);
    free_all(s->owned);
    delete s;
}

TMM_API int32_t tmm_surrogate_outputs(const tmm_surrogate *s) { return s ? s->O : 0; }

TMM_API int64_t tmm_surrogate_parameters(const tmm_surrogate *s)
{
    if (!s) return 0;
    int64_t n = 0;
    for (const auto &l : s->layers) n += (int64_t)l.N * l.Kvalid + l.N;
    return n;
}

TMM_API tmm_status tmm_surrogate_generate(tmm_surrogate *s, const float *d, int32_t B, float *R, void *stream)
{
    TraceRange trace("tmm_surrogate_generate");
    if (!s || !d || !R || B < 0) return TMM_ERR_INVALID_ARG;
    if (B == 0) return TMM_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    tmm_status r = ensure_judge(s, B);
    if (r != TMM_OK) return r;
    if ((r = exact_spectra(s, d, B, st)) != TMM_OK) return r;
    permute_spectra<<<blocks_for((long long)B * s->O), 256, 0, st>>>(s->jout, 2, B, s->nt * s->nl, R);
    return check_launch();
}

TMM_API tmm_status tmm_surrogate_train_step(tmm_surrogate *s, const float *d, const float *R_target, int32_t B,
                                            float lr, float *loss, void *stream)
{
    TraceRange trace("tmm_surrogate_train_step");
    if (!s || !d || !R_target || B < 128 || B % 8 != 0 || !(lr > 0)) return TMM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    tmm_status r = ensure_batch(s, B);
    if (r != TMM_OK) return r;
    if (cudaMemsetAsync(s->err, 0, sizeof(int), st) != cudaSuccess) return cuda_fail(cudaGetLastError());
    if ((r = forward(s, d, B, s->Y, true, st)) != TMM_OK) return r;
    float *lossp = loss ? loss : s->loss_tmp;
    cudaMemsetAsync(lossp, 0, sizeof(float), st);
    loss_grad<<<dim3((s->O + 31) / 32, (B + 31) / 32), dim3(32, 8), 0, st>>>(
        s->Y, R_target, B, s->O, 2.0f / ((float)B * (float)s->O), s->dY, s->dYT, lossp);
    if ((r = check_launch()) != TMM_OK) return r;
    // head
    Layer &head = s->layers[s->depth];
    {
        gemm::EpiArgs ep{};
        ep.err = s->err;
        ep.epi = gemm::EPI_F32;
        ep.out_f32 = head.dW;
        ep.ldo = head.K;
        if ((r = gemm::gemm(s->dYT, B, s->HT[s->depth - 1], B, head.N, head.K, B, ep, st)) != TMM_OK) return r;
        if ((r = colsum(s, s->dY, B, head.N, head.db, st)) != TMM_OK) return r;
        gemm::EpiArgs eb{};
        eb.err = s->err;
        eb.epi = gemm::EPI_DGELU;
        eb.aux = s->Z[s->depth - 1];
        eb.out_bf = s->dZ[0];
        eb.out_bfT = s->dZT[0];
        eb.ldo = s->hidden;
        eb.ldoT = B;
        if ((r = gemm::gemm(s->dY, s->O, head.WbT, s->O, B, s->hidden, s->O, eb, st)) != TMM_OK) return r;
    }
    int cur = 0;
    for (int i = s->depth - 1; i >= 0; --i) {
        Layer &l = s->layers[i];
        const __nv_bfloat16 *inT = i == 0 ? s->X0T : s->HT[i - 1];
        gemm::EpiArgs ep{};
        ep.err = s->err;
        ep.epi = gemm::EPI_F32;
        ep.out_f32 = l.dW;
        ep.ldo = l.K;
        if ((r = gemm::gemm(s->dZT[cur], B, inT, B, l.N, l.K, B, ep, st)) != TMM_OK) return r;
        if ((r = colsum(s, s->dZ[cur], B, l.N, l.db, st)) != TMM_OK) return r;
        if (i > 0) {
            gemm::EpiArgs eb{};
            eb.err = s->err;
            eb.epi = gemm::EPI_DGELU;
            eb.aux = s->Z[i - 1];
            eb.out_bf = s->dZ[cur ^ 1];
            eb.out_bfT = s->dZT[cur ^ 1];
            eb.ldo = s->hidden;
            eb.ldoT = B;
            if ((r = gemm::gemm(s->dZ[cur], s->hidden, l.WbT, l.N, B, s->hidden, s->hidden, eb, st)) != TMM_OK)
                return r;
            cur ^= 1;
        }
    }
    // Adam
    s->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f / (1.0f - powf(b1, (float)s->step)), c2 = 1.0f / (1.0f - powf(b2, (float)s->step));
    for (auto &l : s->layers) {
        const long long nw = (long long)l.N * l.K;
        adam_update<<<blocks_for(nw), 256, 0, st>>>(l.W, l.dW, l.mW, l.vW, nw, lr, b1, b2, eps, c1, c2);
        adam_update<<<blocks_for(l.N), 256, 0, st>>>(l.b, l.db, l.mb, l.vb, l.N, lr, b1, b2, eps, c1, c2);
    }
    if ((r = check_launch()) != TMM_OK) return r;
    return refresh_bf16(s, st);
}

TMM_API tmm_status tmm_surrogate_infer(tmm_surrogate *s, const float *d, int32_t B, float *R, float judge_fraction,
                                       float tol, int32_t *n_fallback, float *max_err, void *stream)
{
    TraceRange trace("tmm_surrogate_infer");
    if (!s || !d || !R || B < 0 || !(judge_fraction >= 0.0f) || judge_fraction > 1.0f || !(tol >= 0.0f))
        return TMM_ERR_INVALID_ARG;
    if (B == 0) return TMM_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    tmm_status r = ensure_batch(s, B);
    if (r != TMM_OK) return r;
    if (cudaMemsetAsync(s->err, 0, sizeof(int), st) != cudaSuccess) return cuda_fail(cudaGetLastError());
    if ((r = forward(s, d, B, R, false, st)) != TMM_OK) return r;
    if (judge_fraction <= 0.0f) return TMM_OK;
    const int stride = std::max(1, (int)lroundf(1.0f / judge_fraction));
    const int Bj = (B + stride - 1) / stride;
    if ((r = ensure_judge(s, Bj)) != TMM_OK) return r;
    cudaMemsetAsync(s->jcount, 0, sizeof(int), st);
    cudaMemsetAsync(s->jmax, 0, sizeof(unsigned int), st);
    const float *dj = d;
    if (stride > 1) {
        gather_rows<<<blocks_for((long long)Bj * s->L), 256, 0, st>>>(d, s->L, stride, Bj, s->jd);
        dj = s->jd;
    }
    if ((r = exact_spectra(s, dj, Bj, st)) != TMM_OK) return r;
    judge_rows<<<Bj, 256, 0, st>>>(R, s->jout, 2, Bj, s->nt * s->nl, stride, tol, s->jcount, s->jmax);
    if ((r = check_launch()) != TMM_OK) return r;
    if (n_fallback) cudaMemcpyAsync(n_fallback, s->jcount, sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (max_err) cudaMemcpyAsync(max_err, s->jmax, sizeof(float), cudaMemcpyDeviceToDevice, st);
    return check_launch();
}

TMM_API tmm_status tmm_surrogate_layer(const tmm_surrogate *s, int32_t i, tmm_surrogate_layer_view *out)
{
    if (!s || !out || i < 0 || i > s->depth) return TMM_ERR_INVALID_ARG;
    const Layer &l = s->layers[i];
    out->N = l.N;
    out->K = l.K;
    out->Kvalid = l.Kvalid;
    out->W = l.W;
    out->b = l.b;
    out->dW = l.dW;
    out->db = l.db;
    return TMM_OK;
}

TMM_API tmm_status tmm_surrogate_status(tmm_surrogate *s, void *stream)
{
    if (!s) return TMM_ERR_INVALID_ARG;
    return gemm::flag_status(s->err, static_cast<cudaStream_t>(stream));
}

TMM_API tmm_status tmm_surrogate_save(tmm_surrogate *s, const char *path)
{
    if (!s || !path) return TMM_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e);
    FILE *f = std::fopen(path, "wb");
    if (!f) return TMM_ERR_INVALID_ARG;
    const char magic[8] = {'T', 'M', 'M', 'S', 'U', 'R', '1', 0};
    int32_t hdr[4] = {s->L, s->O, s->hidden, s->depth};
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              std::fwrite(&s->step, sizeof(s->step), 1, f) == 1;
    for (auto &l : s->layers) {
        const size_t nw = (size_t)l.N * l.K;
        float *bufs[6] = {l.W, l.mW, l.vW, l.b, l.mb, l.vb};
        const size_t cnt[6] = {nw, nw, nw, (size_t)l.N, (size_t)l.N, (size_t)l.N};
        for (int k = 0; k < 6 && ok; ++k) {
            std::vector<float> h(cnt[k]);
            ok = cudaMemcpy(h.data(), bufs[k], cnt[k] * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess &&
                 std::fwrite(h.data(), sizeof(float), cnt[k], f) == cnt[k];
        }
    }
    std::fclose(f);
    return ok ? TMM_OK : TMM_ERR_CUDA;
}

TMM_API tmm_status tmm_surrogate_load(tmm_surrogate *s, const char *path)
{
    if (!s || !path) return TMM_ERR_INVALID_ARG;
    FILE *f = std::fopen(path, "rb");
    if (!f) return TMM_ERR_INVALID_ARG;
    char magic[8];
    int32_t hdr[4];
    long long step = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "TMMSUR1", 8) == 0 &&
              std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == s->L && hdr[1] == s->O && hdr[2] == s->hidden &&
              hdr[3] == s->depth && std::fread(&step, sizeof(step), 1, f) == 1;
    for (auto &l : s->layers) {
        const size_t nw = (size_t)l.N * l.K;
        float *bufs[6] = {l.W, l.mW, l.vW, l.b, l.mb, l.vb};
        const size_t cnt[6] = {nw, nw, nw, (size_t)l.N, (size_t)l.N, (size_t)l.N};
        for (int k = 0; k < 6 && ok; ++k) {
            std::vector<float> h(cnt[k]);
            ok = std::fread(h.data(), sizeof(float), cnt[k], f) == cnt[k] &&
                 cudaMemcpy(bufs[k], h.data(), cnt[k] * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
        }
    }
    std::fclose(f);
    if (!ok) return TMM_ERR_INVALID_ARG;
    s->step = step;
    return refresh_bf16(s, nullptr);
}

}  // extern "C"
