// gemm.cu -- host side of the tcgen05 bf16 GEMM: TMA tensor maps, tile and
// pipeline-depth choice, launch, and the exported test entry point.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <tuple>
#include <vector>

#include "tcgen05_gemm.cuh"
#include "tmm_internal.h"

namespace tmm {
namespace gemm {

// Device-side error flag of the GEMM pipeline waits (one per device).
static __device__ int g_gemm_err;

// cuTensorMapEncodeTiled, resolved through the runtime so that the library
// itself does not link the driver (it must load on machines without one).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

static tmm_status make_tmap(CUtensorMap *map, const void *base, int rows, int K, int ld, int box_rows)
{
    if (reinterpret_cast<uintptr_t>(base) % 16 != 0 || (ld * 2) % 16 != 0) return TMM_ERR_INVALID_ARG;
    EncodeTiledFn cuTensorMapEncodeTiled = encode_tiled();
    if (!cuTensorMapEncodeTiled) return TMM_ERR_UNSUPPORTED;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = cuTensorMapEncodeTiled(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims,
                                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? TMM_OK : TMM_ERR_INVALID_ARG;
}

template <int BN, int STAGES>
static tmm_status launch_bn(const CUtensorMap &ta, const CUtensorMap &tb, int M, int N, int K, const EpiArgs &ep,
                            cudaStream_t st)
{
    auto k = ep.epi == EPI_GELU || ep.epi == EPI_DGELU ? gemm_bf16_kernel<BN, STAGES, FAM_GELU>
                                                       : gemm_bf16_kernel<BN, STAGES, FAM_F32>;
    constexpr size_t smem = GemmSmem<BN, STAGES>::total;
    tmm_status s = ensure_dynamic_smem(reinterpret_cast<const void *>(k), smem);
    if (s != TMM_OK) return s;
    DeviceInfo di;
    s = device_info(&di);
    if (s != TMM_OK) return s;
    const long long tiles = (long long)((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    const int grid = (int)std::min<long long>(tiles, di.sms);
    k<<<grid, kGemmThreads, smem, st>>>(ta, tb, M, N, K, ep);
    return check_launch();
}

// Two-CTA clusters of kernel fn that fit on the current device at once, asked
// once per (kernel, device): the query costs more than a launch.
static int resident_clusters(const void *fn, const cudaLaunchConfig_t &cfg, int fallback)
{
    static std::mutex mu;
    static std::vector<std::tuple<const void *, int, int>> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return fallback;
    }
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const auto &e : cache)
            if (std::get<0>(e) == fn && std::get<1>(e) == dev) return std::get<2>(e);
    }
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess || clusters < 1) {
        (void)cudaGetLastError();
        clusters = fallback;
    }
    std::lock_guard<std::mutex> lock(mu);
    cache.emplace_back(fn, dev, clusters);
    return clusters;
}

// Pair form: clusters of two CTAs, one cluster per two SMs (or as many as
// can be resident), each cluster a persistent worker over 256 x 256 tiles.
template <int STAGES, int EPI_WARPS>
static tmm_status launch_pair(const CUtensorMap &ta, const CUtensorMap &tb, int M, int N, int K, const EpiArgs &ep,
                              cudaStream_t st)
{
    auto k = ep.epi == EPI_GELU || ep.epi == EPI_DGELU ? gemm_bf16_pair_kernel<STAGES, EPI_WARPS, FAM_GELU>
                                                       : gemm_bf16_pair_kernel<STAGES, EPI_WARPS, FAM_F32>;
    constexpr size_t smem = PairSmem<STAGES, EPI_WARPS>::total;
    tmm_status s = ensure_dynamic_smem(reinterpret_cast<const void *>(k), smem);
    if (s != TMM_OK) return s;
    DeviceInfo di;
    s = device_info(&di);
    if (s != TMM_OK) return s;
    const long long tiles = (long long)((M + BM2 - 1) / BM2) * ((N + BN2 - 1) / BN2);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(PairSmem<STAGES, EPI_WARPS>::threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(2 * std::max(1, di.sms / 2));
    const int clusters = resident_clusters(reinterpret_cast<const void *>(k), cfg, std::max(1, di.sms / 2));
    const int pairs = (int)std::min<long long>(tiles, std::min(clusters, std::max(1, di.sms / 2)));
    cfg.gridDim = dim3(2 * pairs);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k, ta, tb, M, N, K, ep);
    if (e != cudaSuccess) return cuda_fail(e);
    return check_launch();
}

// Which kernel.  The pair form streams the main loop faster (1726 against 1585
// TFLOP/s at K = 4096 without an epilogue, M = 65536, N = 1024) and its
// eight epilogue warps store fp32 faster; the one-CTA form's sixteen epilogue
// warps run the GELU epilogues faster, which decides at K = 1024 (119.8 us
// against 124.0).  So: the pair form for N >= 256 past one row block when the
// epilogue stores fp32, K >= 2048 or N >= 2048; TMM_GEMM_FORM=single or =pair
// forces one (tests compare the two on the same shapes).
static bool use_pair(int M, int N, int K, int epi)
{
    const char *f = std::getenv("TMM_GEMM_FORM");
    if (f && std::strcmp(f, "single") == 0) return false;
    if (f && std::strcmp(f, "pair") == 0) return N >= 256;
    const bool f32 = epi == EPI_F32 || epi == EPI_F32_CLAMP;
    return N >= 256 && M > BM && (f32 || K >= 2048 || N >= 2048);
}

int *error_flag()
{
    int *p = nullptr;
    cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_gemm_err);
    return p;
}

// D[M][N] = A[M][K] . B[N][K]^T with the requested epilogue.  A, B row-major
// bf16 with leading dimensions lda, ldb (elements, multiples of 8).
tmm_status gemm(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M, int N, int K, EpiArgs ep,
                cudaStream_t st)
{
    if (M <= 0 || N <= 0 || K <= 0) return TMM_OK;
    if (lda < K || ldb < K || (lda % 8) || (ldb % 8) || ep.ldo < N) return TMM_ERR_INVALID_ARG;
    if (!ep.err) {
        ep.err = error_flag();
        if (!ep.err) return TMM_ERR_CUDA;
    }
    const int BN = N >= 256 ? 256 : (N >= 128 ? 128 : 64);  // >= 32 columns per epilogue warp slice
    auto al16 = [](const void *p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
    const bool f32 = ep.epi == EPI_F32 || ep.epi == EPI_F32_CLAMP;
    ep.vec = (f32 ? (ep.ldo % 4 == 0 && al16(ep.out_f32)) : (ep.ldo % 8 == 0 && al16(ep.out_bf))) && al16(ep.bias) &&
             al16(ep.aux) && (!ep.out_bfT || (ep.ldoT % 8 == 0 && al16(ep.out_bfT)));
    CUtensorMap ta, tb;
    tmm_status s = make_tmap(&ta, A, M, K, lda, BM);
    if (s != TMM_OK) return s;
    if (use_pair(M, N, K, ep.epi)) {
        s = make_tmap(&tb, B, N, K, ldb, BN2 / 2);
        if (s != TMM_OK) return s;
        return launch_pair<6, 8>(ta, tb, M, N, K, ep, st);
    }
    s = make_tmap(&tb, B, N, K, ldb, BN);
    if (s != TMM_OK) return s;
    if (BN == 256) return launch_bn<256, 3>(ta, tb, M, N, K, ep, st);
    if (BN == 128) return launch_bn<128, 4>(ta, tb, M, N, K, ep, st);
    return launch_bn<64, 6>(ta, tb, M, N, K, ep, st);
}

tmm_status flag_status(const int *flag, cudaStream_t st);

// Clear the wait-error flag (a set flag makes every later wait give up).
tmm_status clear_error(cudaStream_t st)
{
    int *p = error_flag();
    if (!p) return TMM_ERR_CUDA;
    cudaError_t e = cudaMemsetAsync(p, 0, sizeof(int), st);
    return e == cudaSuccess ? TMM_OK : cuda_fail(e);
}

tmm_status gemm_status(cudaStream_t st) { return flag_status(error_flag(), st); }

// TMM_ERR_TIMEOUT if the device flag `flag` is set (synchronises st).
tmm_status flag_status(const int *flag, cudaStream_t st)
{
    if (!flag) return TMM_ERR_CUDA;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    return h ? TMM_ERR_TIMEOUT : TMM_OK;
}

}  // namespace gemm
}  // namespace tmm

using namespace tmm;

static tmm_status gemm_entry(const void *A, const void *B, const float *bias, int32_t M, int32_t N, int32_t K,
                             int32_t epilogue, void *out, void *aux, void *outT, int32_t ldoT, void *stream)
{
    if (!A || !B || !out || M < 0 || N < 0 || K < 0 || epilogue < 0 || epilogue > 3) return TMM_ERR_INVALID_ARG;
    if ((epilogue == gemm::EPI_DGELU) && !aux) return TMM_ERR_INVALID_ARG;
    gemm::EpiArgs ep{};
    ep.epi = epilogue;
    ep.bias = bias;
    ep.ldo = N;
    if (epilogue == gemm::EPI_F32 || epilogue == gemm::EPI_F32_CLAMP) ep.out_f32 = static_cast<float *>(out);
    else ep.out_bf = static_cast<__nv_bfloat16 *>(out);
    ep.aux = static_cast<__nv_bfloat16 *>(aux);
    ep.out_bfT = static_cast<__nv_bfloat16 *>(outT);
    ep.ldoT = ldoT;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    tmm_status s = gemm::clear_error(st);
    if (s != TMM_OK) return s;
    s = gemm::gemm(static_cast<const __nv_bfloat16 *>(A), K, static_cast<const __nv_bfloat16 *>(B), K, M, N, K, ep,
                   st);
    if (s != TMM_OK) return s;
    return gemm::gemm_status(st);
}

extern "C" TMM_API tmm_status tmm_gemm_bf16(const void *A, const void *B, const float *bias, int32_t M, int32_t N,
                                            int32_t K, int32_t epilogue, void *out, void *aux, void *stream)
{
    TraceRange trace("tmm_gemm_bf16");
    return gemm_entry(A, B, bias, M, N, K, epilogue, out, aux, nullptr, 0, stream);
}

extern "C" TMM_API tmm_status tmm_gemm_bf16_t(const void *A, const void *B, const float *bias, int32_t M, int32_t N,
                                              int32_t K, int32_t epilogue, void *out, void *aux, void *outT,
                                              int32_t ldoT, void *stream)
{
    TraceRange trace("tmm_gemm_bf16_t");
    if (!outT || (epilogue != gemm::EPI_GELU && epilogue != gemm::EPI_DGELU) || ldoT < M) return TMM_ERR_INVALID_ARG;
    return gemm_entry(A, B, bias, M, N, K, epilogue, out, aux, outT, ldoT, stream);
}
