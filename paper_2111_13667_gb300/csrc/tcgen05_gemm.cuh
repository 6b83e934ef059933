// tcgen05_gemm.cuh -- bf16 x bf16 -> fp32 GEMM on the 5th-generation tensor
// cores of sm_103a, with fused epilogues, for the learned surrogate.
//
//   D[M][N] = sum_k A[M][K] * B[N][K]          (both operands K-major, bf16)
//
// One CTA of 128 threads computes a 128 x BN tile:
//   * warp 0 / lane 0 loads K-blocks of 64 (128-byte rows, 128-byte swizzle)
//     of A and B with TMA into an S-stage shared-memory ring (mbarrier
//     transaction counts);
//   * warp 1 / lane 0 issues tcgen05.mma (M = 128, N = BN, K = 16) into an
//     fp32 accumulator in tensor memory and frees each stage with
//     tcgen05.commit;
//   * all four warps read their 32 TMEM lanes back with tcgen05.ld and apply
//     the epilogue (bias, GELU, GELU derivative, clamp) before storing.
// Every wait is bounded by %globaltimer: on expiry the CTA records an error,
// drains what it issued (again bounded), frees its tensor memory and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace tmm {
namespace gemm {

constexpr int BM = 128;
constexpr int BK = 64;  // 64 bf16 = 128 bytes: one swizzle row
constexpr int UMMA_K = 16;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

enum Epilogue : int {
    EPI_F32 = 0,        // out_f32 = acc (+ bias)
    EPI_GELU = 1,       // aux = bf16(acc + bias); out_bf16 = gelu(acc + bias)
    EPI_DGELU = 2,      // out_bf16 = acc * gelu'(aux)
    EPI_F32_CLAMP = 3,  // out_f32 = clamp(acc + bias, 0, 1)
};

struct EpiArgs {
    int epi;
    const float *bias;      // [N] or null
    float *out_f32;         // [M][ldo]
    __nv_bfloat16 *out_bf;  // [M][ldo]
    __nv_bfloat16 *aux;     // [M][ldo] pre-activation (written by GELU, read by DGELU)
    __nv_bfloat16 *out_bfT; // [N][ldoT] transposed copy of out_bf, or null
    int ldo, ldoT;
    int *err;               // error flag (device)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait: false if the phase did not complete within kWaitNs or another
// thread of the grid already reported an error.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, const int *err)
{
    const unsigned long long t0 = globaltimer();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u) {
            if (*(volatile const int *)err != 0) return false;
            if (globaltimer() - t0 > kWaitNs) return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (stage buffers 1024-byte aligned).
__device__ __forceinline__ uint64_t smem_desc_sw128(const void *p)
{
    const uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;        // start address
    d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;              // descriptor version (sm_100 family)
    d |= (uint64_t)2 << 61;              // layout: 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: bf16 A and B, fp32 D, both K-major.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N)
{
    return (1u << 4)                     // D: fp32
           | (1u << 7)                   // A: bf16
           | (1u << 10)                  // B: bf16
           | ((uint32_t)(N >> 3) << 17)  // N / 8
           | ((uint32_t)(M >> 4) << 24); // M / 16
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32])
{
    tmem_ld16(taddr, v);
    tmem_ld16(taddr + 16, v + 16);
}

// GELU, erf form (CUDA's erff), and its derivative.
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z)
{
    const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * __expf(-0.5f * z * z);
    return cdf + z * pdf;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

constexpr int kEpiWarps = 16;                      // epilogue warps (four per TMEM lane quarter)
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;  // producer warp, MMA warp, epilogue warps

template <int BN, int STAGES>
struct GemmSmem {
    static constexpr size_t a_bytes = (size_t)BM * BK * 2;
    static constexpr size_t b_bytes = (size_t)BN * BK * 2;
    static constexpr size_t ring = STAGES * (a_bytes + b_bytes);
    static constexpr size_t stage = (size_t)kEpiWarps * 32 * 33 * 4;  // per-warp 32 x 33 floats
    static constexpr size_t bars = (2 * STAGES + 5) * 8 + 16;
    static constexpr size_t total = 1024 + ring + stage + bars;  // + alignment slack
};

// Apply the epilogue to one 32-column chunk of one warp's 32 rows: stage the
// values in shared memory, then write them back row by row (coalesced).
__device__ __forceinline__ void epilogue_chunk(const EpiArgs &ep, const float (&v)[32], float *stg, int row0, int n0c,
                                               int M, int N, int lane)
{
    const int row = row0 + lane;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int col = n0c + i;
        const bool in = row < M && col < N;
        const float z = v[i] + ((ep.bias && col < N) ? ep.bias[col] : 0.0f);
        float y;
        if (ep.epi == EPI_F32) {
            y = z;
        } else if (ep.epi == EPI_F32_CLAMP) {
            y = fminf(fmaxf(z, 0.0f), 1.0f);
        } else if (ep.epi == EPI_GELU) {
            const __nv_bfloat16 zb = __float2bfloat16(z);
            if (ep.aux && in) ep.aux[(long long)row * ep.ldo + col] = zb;
            y = gelu(__bfloat162float(zb));
        } else {  // EPI_DGELU
            y = in ? v[i] * gelu_grad(__bfloat162float(ep.aux[(long long)row * ep.ldo + col])) : 0.0f;
        }
        if (ep.out_bfT && in)  // lanes hold consecutive rows: coalesced
            ep.out_bfT[(long long)col * ep.ldoT + row] = __float2bfloat16(y);
        stg[lane * 33 + i] = y;
    }
    __syncwarp();
    const int col = n0c + lane;
    if (col < N) {
        for (int r = 0; r < 32; ++r) {
            const int rr = row0 + r;
            if (rr >= M) break;
            const float y = stg[r * 33 + lane];
            const long long o = (long long)rr * ep.ldo + col;
            if (ep.epi == EPI_F32 || ep.epi == EPI_F32_CLAMP) ep.out_f32[o] = y;
            else ep.out_bf[o] = __float2bfloat16(y);
        }
    }
    __syncwarp();
}

// Persistent, warp-specialised kernel.  Tiles (128 x BN) are dealt round-robin
// to the CTAs (one per SM); the accumulator is double-buffered in tensor
// memory (2 x BN columns) so the epilogue of one tile overlaps the MMAs of the
// next.  Barriers: full/empty per ring stage (TMA <-> MMA), acc_full/acc_empty
// per accumulator (MMA <-> epilogue), done (MMA drain before teardown).
template <int BN, int STAGES>
__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
                     int K, EpiArgs ep)
{
    using L = GemmSmem<BN, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * L::a_bytes;
    float *stg_all = reinterpret_cast<float *>(smem + L::ring);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::ring + L::stage);
    uint64_t *empty = full + STAGES;
    uint64_t *acc_full = empty + STAGES;
    uint64_t *acc_empty = acc_full + 2;
    uint64_t *done = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    int *s_fail = reinterpret_cast<int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = (N + BN - 1) / BN;
    const int tiles = ((M + BM - 1) / BM) * n_tiles;
    const int nkb = (K + BK - 1) / BK;
    constexpr uint32_t kCols = 2 * BN;  // power of two, <= 512

    if (threadIdx.x == 0) {
        *s_fail = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kEpiWarps);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // producer: TMA into the ring, across all tiles of this CTA
            long long it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
                const int m0 = (tile / n_tiles) * BM, n0 = (tile % n_tiles) * BN;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = (int)(it % STAGES);
                    if (it >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((it / STAGES) - 1) & 1), ep.err)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[s], (uint32_t)(L::a_bytes + L::b_bytes));
                    tma_load_2d(sA + s * L::a_bytes, &tmA, &full[s], kb * BK, m0);
                    tma_load_2d(sB + s * L::b_bytes, &tmB, &full[s], kb * BK, n0);
                }
            }
            // every issued load must land before the CTA may exit
            for (long long j = (it > STAGES ? it - STAGES : 0); j < it; ++j)
                if (!mbar_wait(&full[j % STAGES], (uint32_t)((j / STAGES) & 1), ep.err)) ok = false;
            if (!ok) *s_fail = 1;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            constexpr uint32_t idesc = instr_desc_bf16(BM, BN);
            long long it = 0;
            int t = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++t) {
                const int buf = t & 1, use = t >> 1;
                if (t >= 2 && !mbar_wait(&acc_empty[buf], (uint32_t)((use - 1) & 1), ep.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * BN);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = (int)(it % STAGES);
                    if (!mbar_wait(&full[s], (uint32_t)((it / STAGES) & 1), ep.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int k = 0; k < BK / UMMA_K; ++k) {
                        const uint64_t ad = smem_desc_sw128(sA + s * L::a_bytes + k * UMMA_K * 2);
                        const uint64_t bd = smem_desc_sw128(sB + s * L::b_bytes + k * UMMA_K * 2);
                        umma_bf16(d, ad, bd, idesc, (kb | k) != 0 ? 1u : 0u);
                    }
                    umma_commit(&empty[s]);
                }
                if (ok) umma_commit(&acc_full[buf]);
            }
            // drain: every MMA issued above completes before teardown
            umma_commit(done);
            if (!mbar_wait(done, 0, ep.err)) ok = false;
            if (!ok) *s_fail = 1;
        }
    } else {
        // epilogue warps: lane quarter q of TMEM, one of kEpiWarps / 4 column slices
        constexpr int kSlices = (kEpiWarps / 4) < (BN / 32) ? (kEpiWarps / 4) : (BN / 32);
        constexpr int kSliceCols = BN / kSlices;  // warps with half >= kSlices have no columns
        static_assert(kSliceCols % 32 == 0, "column slice must hold whole 32-column chunks");
        const int ew = warp - 2, q = warp & 3, half = ew >> 2;
        float *stg = stg_all + ew * (32 * 33);
        int t = 0;
        for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++t) {
            const int buf = t & 1, use = t >> 1;
            const bool have = __all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (uint32_t)(use & 1), ep.err));
            if (!have) {
                if (lane == 0) *s_fail = 1;
                break;
            }
            tc_fence_after();
            const int m0 = (tile / n_tiles) * BM, n0 = (tile % n_tiles) * BN;
            const int row0 = m0 + q * 32;
            for (int c = half * kSliceCols; half < kSlices && c < (half + 1) * kSliceCols; c += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + c), v);
                epilogue_chunk(ep, v, stg, row0, n0 + c, M, N, lane);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && *s_fail) atomicExch(ep.err, 1);
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();  // lanes 1..31 waited while lane 0 issued: reconverge for the aligned dealloc
        tmem_dealloc(tmem, kCols);
    }
}

}  // namespace gemm
}  // namespace tmm
