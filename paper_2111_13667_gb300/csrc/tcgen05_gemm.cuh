// tcgen05_gemm.cuh -- bf16 x bf16 -> fp32 GEMM on the 5th-generation tensor
// cores of sm_103a, with fused epilogues, for the learned surrogate.
//
//   D[M][N] = sum_k A[M][K] * B[N][K]          (both operands K-major, bf16)
//
// One persistent CTA per SM (576 threads) computes 128 x BN tiles:
//   * warp 0 / lane 0 loads K-blocks of 64 (128-byte rows, 128-byte swizzle)
//     of A and B with TMA into an S-stage shared-memory ring (mbarrier
//     transaction counts);
//   * warp 1 / lane 0 issues tcgen05.mma (M = 128, N = BN, K = 16) into one of
//     two fp32 accumulators in tensor memory and frees each stage with
//     tcgen05.commit;
//   * sixteen epilogue warps (four per 32-lane TMEM quarter, each a column
//     slice) read the other accumulator back with tcgen05.ld, apply the
//     epilogue (bias, GELU, GELU derivative, clamp) and store through a
//     per-warp staging buffer with 16-byte stores.
// Every wait is bounded by %globaltimer: on expiry the CTA records an error,
// drains what it issued (again bounded), frees its tensor memory and returns.
//
// The pair form (gemm_bf16_pair_kernel) runs the same roles on a cluster of
// two CTAs that share one 256 x 256 tile: each CTA loads its own 128 rows of A
// and its own 128 rows of B, and the even CTA issues tcgen05.mma.cta_group::2
// (M = 256, N = 256), which reads both CTAs' shared memory and writes rows
// 0-127 of the accumulator into its own tensor memory and rows 128-255 into
// its peer's.  Per SM this halves the B bytes through shared memory per flop.
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
    int vec;                // 1: pointers 16-byte aligned and ldo, ldoT multiples of 16 bytes
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
// thread of the grid already reported an error.  The clock is read only once
// the first test has failed (most waits of the pipeline find the phase done).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, const int *err)
{
    if (mbar_try_wait(bar, parity)) return true;
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

// 16 consecutive fp32 columns of this thread's TMEM lane (load, then a wait that
// names the loaded registers, so no use of them is scheduled before it).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive fp32 columns of this thread's TMEM lane: one load, one wait.
// The wait names the loaded registers as operands, so no use of them can be
// scheduled before it.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// GELU, erf form: gelu(z) = z Phi(z) = 0.5 z (1 + erf(z / sqrt 2)) = relu(z) -
// (a / sqrt 2) erfc(a) with a = |z| / sqrt 2; its derivative Phi(z) + z phi(z),
// Phi(z) = 1 - erfc(a) / 2 for z >= 0 and erfc(a) / 2 below, phi(z) =
// exp(-a^2) / sqrt(2 pi).  erfc(a) is the Chebyshev-fitted form of Press et
// al. (Numerical Recipes, 2nd ed., Sec. 6.2):
//   erfc(a) = t exp(-a^2 + P(t)),  t = 1 / (1 + a / 2),  P of degree 9,
// whose relative error is below 1.1e-7 for every a >= 0 (8e-6 evaluated in
// FP32 up to a = 9, where exp(-a^2) is near FP32's range end): far below the
// bf16 rounding of the outputs, in both tails.  Two lanes at a time on the
// paired FP32 pipes; rcp and ex2 are the MUFU approximations.
__device__ __forceinline__ float rcp_mufu(float v)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float ex2_mufu(float v)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float2 g2(float a) { return make_float2(a, a); }

// a >= 0 on both lanes: (erfc(a), exp(-a^2)) per lane; the second only when wanted
template <bool WANT_G>
__device__ __forceinline__ float2 erfc_pair(float2 a, float2 *g)
{
    constexpr float kL2e = 1.4426950408889634f;
    const float2 t = make_float2(rcp_mufu(fmaf(0.5f, a.x, 1.0f)), rcp_mufu(fmaf(0.5f, a.y, 1.0f)));
    float2 p = __ffma2_rn(t, g2(0.17087277f), g2(-0.82215223f));
    p = __ffma2_rn(t, p, g2(1.48851587f));
    p = __ffma2_rn(t, p, g2(-1.13520398f));
    p = __ffma2_rn(t, p, g2(0.27886807f));
    p = __ffma2_rn(t, p, g2(-0.18628806f));
    p = __ffma2_rn(t, p, g2(0.09678418f));
    p = __ffma2_rn(t, p, g2(0.37409196f));
    p = __ffma2_rn(t, p, g2(1.00002368f));
    p = __ffma2_rn(t, p, g2(-1.26551223f));
    const float2 na = __fmul2_rn(a, g2(-kL2e));           // -a log2(e)
    const float2 x = __ffma2_rn(na, a, __fmul2_rn(p, g2(kL2e)));  // (-a^2 + P) log2(e)
    if (WANT_G) {
        const float2 y = __fmul2_rn(na, a);
        *g = make_float2(ex2_mufu(y.x), ex2_mufu(y.y));
    }
    return __fmul2_rn(t, make_float2(ex2_mufu(x.x), ex2_mufu(x.y)));
}

__device__ __forceinline__ float2 gelu2(float2 z)
{
    const float2 a = __fmul2_rn(make_float2(fabsf(z.x), fabsf(z.y)), g2(0.70710678118654752f));
    const float2 h = __fmul2_rn(__fmul2_rn(a, g2(0.70710678118654752f)), erfc_pair<false>(a, nullptr));
    return make_float2(fmaxf(z.x, 0.0f) - h.x, fmaxf(z.y, 0.0f) - h.y);
}

__device__ __forceinline__ float2 gelu_grad2(float2 z)
{
    const float2 a = __fmul2_rn(make_float2(fabsf(z.x), fabsf(z.y)), g2(0.70710678118654752f));
    float2 g;
    const float2 E = erfc_pair<true>(a, &g);
    const float2 half = __fmul2_rn(E, g2(0.5f));
    const float2 cdf = make_float2(z.x >= 0.0f ? 1.0f - half.x : half.x, z.y >= 0.0f ? 1.0f - half.y : half.y);
    return __ffma2_rn(__fmul2_rn(z, g2(0.39894228040143268f)), g, cdf);
}

__device__ __forceinline__ float gelu(float z) { return gelu2(make_float2(z, z)).x; }
__device__ __forceinline__ float gelu_grad(float z) { return gelu_grad2(make_float2(z, z)).x; }

// Two floats to one word of two bf16 (round to nearest even), a in the low half.
__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

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
    static constexpr size_t stage = (size_t)kEpiWarps * 32 * 32 * 4;  // per warp 32 x 32 floats
    static constexpr size_t bars = (2 * STAGES + 5) * 8 + 16;
    static constexpr size_t total = 1024 + ring + stage + bars;  // + alignment slack
};

// ---- epilogue -------------------------------------------------------------
// Each epilogue warp owns 32 accumulator rows (its TMEM lane quarter); after a
// 32x32b tcgen05.ld lane i holds 32 consecutive columns of row row0 + i.  The
// warp's staging buffer (32 rows of 128 bytes) turns these per-row registers
// into 16-byte stores that are contiguous across lanes, and into the
// transposed copy.  Rows are stored as 16-byte groups at a row-dependent XOR
// position so that row-wise 16-byte accesses and the column-wise 4-byte reads
// of the transpose meet no bank conflicts.

// word offset of group g (0..7) of fp32 row r; of group g (0..3) of bf16 row r
__device__ __forceinline__ int stg_f32(int r, int g) { return r * 32 + 4 * (g ^ (r & 7)); }
__device__ __forceinline__ int stg_bf(int r, int g) { return r * 16 + 4 * (g ^ ((r >> 1) & 3)); }

// staged bf16 rows -> out[row0 + r][col0 ...]: four lanes per 64-byte row
__device__ __forceinline__ void store_rows_bf(const uint32_t *stg, __nv_bfloat16 *out, int ldo, int row0, int col0,
                                              int M, int lane)
{
    const int g = lane & 3;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = 8 * k + (lane >> 2);
        if (row0 + r < M)
            *reinterpret_cast<uint4 *>(out + (long long)(row0 + r) * ldo + col0 + 8 * g) =
                *reinterpret_cast<const uint4 *>(stg + stg_bf(r, g));
    }
}

// staged bf16 rows -> outT[col0 + c][row0 ... row0 + 31] (all 32 rows valid).
// Lane (cp, h) reads word cp (columns 2cp, 2cp+1) of rows 16h .. 16h+15 and
// splits each pair of rows into one word per column with a byte permute;
// lanes with h = 1 visit the rows in swapped pairs so that both halves of the
// warp read different banks.
__device__ __forceinline__ void store_cols_bf(const uint32_t *stg, __nv_bfloat16 *outT, int ldoT, int row0, int col0,
                                              int lane)
{
    const int cp = lane & 15, h = lane >> 4;
    uint32_t w[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int r = 16 * h + (j ^ h);
        w[j] = stg[r * 16 + 4 * ((cp >> 2) ^ ((r >> 1) & 3)) + (cp & 3)];
    }
    const uint32_t sel0 = h ? 0x1054u : 0x5410u;  // low halves of the two rows, in row order
    const uint32_t sel1 = h ? 0x3276u : 0x7632u;  // high halves
#pragma unroll
    for (int k = 0; k < 8; ++k) {  // w[2k]: column 2cp, w[2k+1]: column 2cp+1, rows 2k and 2k+1
        const uint32_t a = w[2 * k], b = w[2 * k + 1];
        w[2 * k] = __byte_perm(a, b, sel0);
        w[2 * k + 1] = __byte_perm(a, b, sel1);
    }
    uint4 *p0 = reinterpret_cast<uint4 *>(outT + (long long)(col0 + 2 * cp) * ldoT + row0 + 16 * h);
    uint4 *p1 = reinterpret_cast<uint4 *>(outT + (long long)(col0 + 2 * cp + 1) * ldoT + row0 + 16 * h);
    p0[0] = make_uint4(w[0], w[2], w[4], w[6]);
    p0[1] = make_uint4(w[8], w[10], w[12], w[14]);
    p1[0] = make_uint4(w[1], w[3], w[5], w[7]);
    p1[1] = make_uint4(w[9], w[11], w[13], w[15]);
}

// transposed copy of a partial row block (rows past M skipped): each lane
// takes its own staged row back and stores it one element at a time (lanes
// hold consecutive rows, so each warp store covers 64 contiguous bytes)
__device__ __forceinline__ void store_cols_bf_tail(const uint32_t *stg, __nv_bfloat16 *outT, int ldoT, int row0,
                                                   int col0, int M, int lane)
{
    const int row = row0 + lane;
    if (row >= M) return;
    uint32_t w[16];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const uint4 t = *reinterpret_cast<const uint4 *>(stg + stg_bf(lane, g));
        w[4 * g] = t.x, w[4 * g + 1] = t.y, w[4 * g + 2] = t.z, w[4 * g + 3] = t.w;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        outT[(long long)(col0 + 2 * i) * ldoT + row] = __ushort_as_bfloat16((unsigned short)(w[i] & 0xFFFFu));
        outT[(long long)(col0 + 2 * i + 1) * ldoT + row] = __ushort_as_bfloat16((unsigned short)(w[i] >> 16));
    }
}

// bias[col0 + 4j .. col0 + 4j + 3] (zeros without a bias); the address is the
// same in every lane, so the load is a broadcast
__device__ __forceinline__ float4 bias4(const float *bias, int col0, int j)
{
    return bias ? __ldg(reinterpret_cast<const float4 *>(bias + col0) + j) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// Full 32-column chunk, 16-byte aligned outputs, fp32 epilogues.
template <int EPI>
__device__ __forceinline__ void epilogue_chunk_vec(const EpiArgs &ep, const float (&v)[32], uint32_t *stg, int row0,
                                                   int col0, int M, int lane)
{
    if (EPI == EPI_F32 || EPI == EPI_F32_CLAMP) {
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            float4 t = bias4(ep.bias, col0, g);
            t.x += v[4 * g], t.y += v[4 * g + 1], t.z += v[4 * g + 2], t.w += v[4 * g + 3];
            if (EPI == EPI_F32_CLAMP) {
                t.x = fminf(fmaxf(t.x, 0.0f), 1.0f), t.y = fminf(fmaxf(t.y, 0.0f), 1.0f);
                t.z = fminf(fmaxf(t.z, 0.0f), 1.0f), t.w = fminf(fmaxf(t.w, 0.0f), 1.0f);
            }
            *reinterpret_cast<float4 *>(stg + stg_f32(lane, g)) = t;
        }
        __syncwarp();
        const int g = lane & 7;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int r = 4 * k + (lane >> 3);
            if (row0 + r < M)
                *reinterpret_cast<float4 *>(ep.out_f32 + (long long)(row0 + r) * ep.ldo + col0 + 4 * g) =
                    *reinterpret_cast<const float4 *>(stg + stg_f32(r, g));
        }
        __syncwarp();
    }
}

// Any chunk (ragged columns, unaligned outputs): element by element, staged
// through shared memory (rows of 32 floats, element i of row r at i ^ r, so
// that row writes and column reads meet no bank conflicts) for row-wise stores.
__device__ __forceinline__ void epilogue_chunk_scalar(const EpiArgs &ep, const float (&v)[32], float *stg, int row0,
                                                      int n0c, int M, int N, int lane)
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
        stg[lane * 32 + (i ^ lane)] = y;
    }
    __syncwarp();
    const int col = n0c + lane;
    if (col < N) {
        for (int r = 0; r < 32; ++r) {
            const int rr = row0 + r;
            if (rr >= M) break;
            const float y = stg[r * 32 + (lane ^ r)];
            const long long o = (long long)rr * ep.ldo + col;
            if (ep.epi == EPI_F32 || ep.epi == EPI_F32_CLAMP) ep.out_f32[o] = y;
            else ep.out_bf[o] = __float2bfloat16(y);
        }
    }
    __syncwarp();
}

// this lane's 8 words (16 bf16 columns, half h of a 32-column chunk) into its staged row
__device__ __forceinline__ void stage_half_bf(uint32_t *stg, const uint32_t (&w)[8], int lane, int h)
{
    *reinterpret_cast<uint4 *>(stg + stg_bf(lane, 2 * h)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4 *>(stg + stg_bf(lane, 2 * h + 1)) = make_uint4(w[4], w[5], w[6], w[7]);
}

// GELU and GELU' epilogues of a full 32-column chunk with 16-byte aligned
// outputs, in two halves of 16 columns read from TMEM one after the other, so
// that only half a chunk's values and activations are live at a time.  The
// warp's 4 KB staging buffer holds two 32-row bf16 tiles: the pre-activations
// (aux) and the outputs.
template <int EPI>
__device__ __forceinline__ void epilogue_chunk_halves(const EpiArgs &ep, uint32_t taddr, uint32_t *stg, int row0,
                                                      int col0, int M, int lane)
{
    uint32_t *stA = stg, *stO = stg + 32 * 16;
    if (EPI == EPI_DGELU) {  // rows of aux through the staging buffer (coalesced loads)
        const int g = lane & 3;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int r = 8 * k + (lane >> 2);
            uint4 t = make_uint4(0u, 0u, 0u, 0u);
            if (row0 + r < M)
                t = __ldg(reinterpret_cast<const uint4 *>(ep.aux + (long long)(row0 + r) * ep.ldo + col0 + 8 * g));
            *reinterpret_cast<uint4 *>(stA + stg_bf(r, g)) = t;
        }
        __syncwarp();
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float v[16];
        tmem_ld16(taddr + 16 * h, v);
        uint32_t w[8];
        if (EPI == EPI_GELU) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 b = bias4(ep.bias, col0 + 16 * h, j);
                w[2 * j] = pack_bf16(v[4 * j] + b.x, v[4 * j + 1] + b.y);
                w[2 * j + 1] = pack_bf16(v[4 * j + 2] + b.z, v[4 * j + 3] + b.w);
            }
            if (ep.aux) stage_half_bf(stA, w, lane, h);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float2 y = gelu2(make_float2(bf_lo(w[i]), bf_hi(w[i])));
                w[i] = pack_bf16(y.x, y.y);
            }
        } else {
            const uint4 t0 = *reinterpret_cast<const uint4 *>(stA + stg_bf(lane, 2 * h));
            const uint4 t1 = *reinterpret_cast<const uint4 *>(stA + stg_bf(lane, 2 * h + 1));
            const uint32_t z[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float2 d = __fmul2_rn(make_float2(v[2 * i], v[2 * i + 1]),
                                            gelu_grad2(make_float2(bf_lo(z[i]), bf_hi(z[i]))));
                w[i] = pack_bf16(d.x, d.y);
            }
        }
        stage_half_bf(stO, w, lane, h);
    }
    __syncwarp();
    if (EPI == EPI_GELU && ep.aux) store_rows_bf(stA, ep.aux, ep.ldo, row0, col0, M, lane);
    store_rows_bf(stO, ep.out_bf, ep.ldo, row0, col0, M, lane);
    if (ep.out_bfT) {
        if (row0 + 32 <= M) store_cols_bf(stO, ep.out_bfT, ep.ldoT, row0, col0, lane);
        else store_cols_bf_tail(stO, ep.out_bfT, ep.ldoT, row0, col0, M, lane);
    }
    __syncwarp();
}

// Epilogue families: the kernels are instantiated per family so that each
// carries only its own epilogue code (and register pressure).
enum EpiFamily : int {
    FAM_F32 = 0,   // EPI_F32, EPI_F32_CLAMP
    FAM_GELU = 1,  // EPI_GELU, EPI_DGELU
};
__host__ __device__ constexpr int family_of(int epi) { return (epi == EPI_GELU || epi == EPI_DGELU) ? FAM_GELU : FAM_F32; }

// One 32-column chunk of the accumulator at TMEM address taddr.
template <int FAM>
__device__ __forceinline__ void epilogue_chunk_tmem(const EpiArgs &ep, uint32_t taddr, float *stg, int row0, int n0c,
                                                    int M, int N, int lane)
{
    if (FAM == FAM_GELU && ep.vec && n0c + 32 <= N) {
        uint32_t *sw = reinterpret_cast<uint32_t *>(stg);
        if (ep.epi == EPI_GELU) epilogue_chunk_halves<EPI_GELU>(ep, taddr, sw, row0, n0c, M, lane);
        else epilogue_chunk_halves<EPI_DGELU>(ep, taddr, sw, row0, n0c, M, lane);
        return;
    }
    float v[32];
    tmem_ld32(taddr, v);
    if (FAM == FAM_F32 && ep.vec && n0c + 32 <= N) {
        uint32_t *sw = reinterpret_cast<uint32_t *>(stg);
        if (ep.epi == EPI_F32) epilogue_chunk_vec<EPI_F32>(ep, v, sw, row0, n0c, M, lane);
        else epilogue_chunk_vec<EPI_F32_CLAMP>(ep, v, sw, row0, n0c, M, lane);
        return;
    }
    epilogue_chunk_scalar(ep, v, stg, row0, n0c, M, N, lane);
}

// Persistent, warp-specialised kernel.  Tiles (128 x BN) are dealt round-robin
// to the CTAs (one per SM); the accumulator is double-buffered in tensor
// memory (2 x BN columns) so the epilogue of one tile overlaps the MMAs of the
// next.  Barriers: full/empty per ring stage (TMA <-> MMA), acc_full/acc_empty
// per accumulator (MMA <-> epilogue), done (MMA drain before teardown).
template <int BN, int STAGES, int FAM>
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
            // MMA issuer; stage descriptors are the ring's base descriptor plus the
            // offset / 16 (the start-address field; shared memory is below 256 KB)
            constexpr uint32_t idesc = instr_desc_bf16(BM, BN);
            const uint64_t a_desc0 = smem_desc_sw128(sA), b_desc0 = smem_desc_sw128(sB);
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
                        const uint64_t ad = a_desc0 + (uint64_t)((s * L::a_bytes + k * UMMA_K * 2) >> 4);
                        const uint64_t bd = b_desc0 + (uint64_t)((s * L::b_bytes + k * UMMA_K * 2) >> 4);
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
        float *stg = stg_all + ew * (32 * 32);
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
#pragma unroll 1
            for (int c = half * kSliceCols; half < kSlices && c < (half + 1) * kSliceCols; c += 32) {
                epilogue_chunk_tmem<FAM>(ep, tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + c), stg, row0,
                                    n0 + c, M, N, lane);
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

// ---- pair-CTA form ---------------------------------------------------------

constexpr int BM2 = 2 * BM;  // rows of a pair tile, 128 per CTA
constexpr int BN2 = 256;     // columns of a pair tile; B rows 128 per CTA

__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id_x()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count_x()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}

// The shared::cluster address of this CTA's shared variable at addr in CTA rank.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// Every thread of both CTAs (not .aligned: warps may arrive diverged).
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// Arrive on an mbarrier given by its shared::cluster address (own or peer CTA).
// Default (CTA-scope release) semantics: the arrival only has to follow the
// arriving warp's tcgen05.ld reads, which tcgen05.wait::ld and
// tcgen05.fence::before_thread_sync order; a cluster-scope release would also
// wait for the warp's global stores in flight.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}

// TMA load into this CTA's shared memory whose completion is counted on the
// mbarrier at the shared::cluster address bar (the even CTA's).
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, uint32_t bar, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void umma_bf16_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Completion of this thread's MMAs arrives once on the mbarrier at the same
// offset in both CTAs of the pair.
__device__ __forceinline__ void umma_commit_pair_both(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

// ... on this CTA's mbarrier only.
__device__ __forceinline__ void umma_commit_pair_own(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// One warp of each CTA of the pair, collectively: the same columns in both.
__device__ __forceinline__ void tmem_alloc_pair(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

template <int STAGES, int EPI_WARPS>
struct PairSmem {
    static constexpr int threads = 64 + 32 * EPI_WARPS;            // producer warp, MMA warp, epilogue warps
    static constexpr size_t a_bytes = (size_t)BM * BK * 2;         // this CTA's 128 rows of A
    static constexpr size_t b_bytes = (size_t)(BN2 / 2) * BK * 2;  // this CTA's 128 rows of B
    static constexpr size_t ring = STAGES * (a_bytes + b_bytes);
    static constexpr size_t stage = (size_t)EPI_WARPS * 32 * 32 * 4;
    static constexpr size_t bars = (2 * STAGES + 5) * 8 + 16;
    static constexpr size_t total = 1024 + ring + stage + bars;
};

// Persistent pair kernel: clusters of two CTAs (ranks 0 and 1); pair tiles of
// 256 x 256 dealt round-robin to the clusters.  Roles as in gemm_bf16_kernel;
// in addition:
//   full[s]      even CTA only: its producer's arrive with the byte count of
//                both CTAs' loads, which all complete on it;
//   empty[s]     both CTAs: the MMA's commit, multicast;
//   acc_full[b]  both CTAs: the MMA's commit, multicast;
//   acc_empty[b] even CTA only: one arrival per epilogue warp of either CTA;
//   done         even CTA: the MMA drain.
// All waits are CTA-scope acquires: what crosses CTAs is ordered by TMA
// completion, tcgen05.commit and the tcgen05 fences, not by memory ordering.
// A cluster barrier after set-up (barriers initialised, tensor memory
// allocated) and one before teardown (no CTA leaves while its peer may still
// read its shared memory, write its tensor memory or signal its barriers).
template <int STAGES, int EPI_WARPS, int FAM>
__global__ void __launch_bounds__(PairSmem<STAGES, EPI_WARPS>::threads, 1)
    gemm_bf16_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M,
                          int N, int K, EpiArgs ep)
{
    using L = PairSmem<STAGES, EPI_WARPS>;
    static_assert(EPI_WARPS % 4 == 0, "whole TMEM lane quarters");
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
    const uint32_t rank = cluster_ctarank();
    const bool even = rank == 0;
    const int pair = (int)cluster_id_x(), n_pairs = (int)cluster_count_x();
    const int n_tiles = (N + BN2 - 1) / BN2;
    const int tiles = ((M + BM2 - 1) / BM2) * n_tiles;
    const int nkb = (K + BK - 1) / BK;
    constexpr uint32_t kCols = 2 * BN2;  // two accumulators of 256 columns: all 512

    if (threadIdx.x == 0) {
        *s_fail = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 2 * EPI_WARPS);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc_pair(tmem_slot, kCols);
    tc_fence_before();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    auto fail = [&]() {
        *s_fail = 1;
        atomicExch(ep.err, 1);  // the peer's waits give up at once
    };

    if (warp == 0) {
        if (lane == 0) {
            // producer: this CTA's halves of A and B; completion on the even CTA's full[s]
            const uint32_t full_even = mapa_shared(smem_u32(full), 0);
            long long it = 0;
            bool ok = true;
            for (int tile = pair; tile < tiles && ok; tile += n_pairs) {
                const int m0 = (tile / n_tiles) * BM2 + (int)rank * BM;
                const int n0 = (tile % n_tiles) * BN2 + (int)rank * (BN2 / 2);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = (int)(it % STAGES);
                    if (it >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((it / STAGES) - 1) & 1), ep.err)) {
                        ok = false;
                        break;
                    }
                    if (even) mbar_expect_tx(&full[s], (uint32_t)(2 * (L::a_bytes + L::b_bytes)));
                    tma_load_2d_pair(sA + s * L::a_bytes, &tmA, full_even + 8u * s, kb * BK, m0);
                    tma_load_2d_pair(sB + s * L::b_bytes, &tmB, full_even + 8u * s, kb * BK, n0);
                }
            }
            // the even CTA sees both CTAs' loads land: none is in flight at teardown
            if (even)
                for (long long j = (it > STAGES ? it - STAGES : 0); j < it; ++j)
                    if (!mbar_wait(&full[j % STAGES], (uint32_t)((j / STAGES) & 1), ep.err)) ok = false;
            if (!ok) fail();
        }
    } else if (warp == 1) {
        if (even && lane == 0) {
            // MMA issuer for the pair (descriptors as in gemm_bf16_kernel)
            constexpr uint32_t idesc = instr_desc_bf16(BM2, BN2);
            const uint64_t a_desc0 = smem_desc_sw128(sA), b_desc0 = smem_desc_sw128(sB);
            long long it = 0;
            int t = 0;
            bool ok = true;
            for (int tile = pair; tile < tiles && ok; tile += n_pairs, ++t) {
                const int buf = t & 1, use = t >> 1;
                if (t >= 2 && !mbar_wait(&acc_empty[buf], (uint32_t)((use - 1) & 1), ep.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * BN2);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = (int)(it % STAGES);
                    if (!mbar_wait(&full[s], (uint32_t)((it / STAGES) & 1), ep.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int k = 0; k < BK / UMMA_K; ++k) {
                        const uint64_t ad = a_desc0 + (uint64_t)((s * L::a_bytes + k * UMMA_K * 2) >> 4);
                        const uint64_t bd = b_desc0 + (uint64_t)((s * L::b_bytes + k * UMMA_K * 2) >> 4);
                        umma_bf16_pair(d, ad, bd, idesc, (kb | k) != 0 ? 1u : 0u);
                    }
                    umma_commit_pair_both(&empty[s]);
                }
                if (ok) umma_commit_pair_both(&acc_full[buf]);
            }
            umma_commit_pair_own(done);
            if (!mbar_wait(done, 0, ep.err)) ok = false;
            if (!ok) fail();
        }
    } else {
        // epilogue warps: this CTA's 128 rows of the pair tile
        constexpr int kSlices = (EPI_WARPS / 4) < (BN2 / 32) ? (EPI_WARPS / 4) : (BN2 / 32);
        constexpr int kSliceCols = BN2 / kSlices;
        static_assert(kSliceCols % 32 == 0, "column slice must hold whole 32-column chunks");
        const int ew = warp - 2, q = warp & 3, half = ew >> 2;
        float *stg = stg_all + ew * (32 * 32);
        const uint32_t acc_empty_even = mapa_shared(smem_u32(acc_empty), 0);
        int t = 0;
        for (int tile = pair; tile < tiles; tile += n_pairs, ++t) {
            const int buf = t & 1, use = t >> 1;
            const bool have =
                __all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (uint32_t)(use & 1), ep.err));
            if (!have) {
                if (lane == 0) fail();
                break;
            }
            tc_fence_after();
            const int m0 = (tile / n_tiles) * BM2 + (int)rank * BM, n0 = (tile % n_tiles) * BN2;
            const int row0 = m0 + q * 32;
#pragma unroll 1
            for (int c = half * kSliceCols; half < kSlices && c < (half + 1) * kSliceCols; c += 32) {
                epilogue_chunk_tmem<FAM>(ep, tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN2 + c), stg, row0,
                                    n0 + c, M, N, lane);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(acc_empty_even + 8u * buf);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && *s_fail) atomicExch(ep.err, 1);
    tc_fence_before();
    cluster_sync();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        tmem_dealloc_pair(tmem, kCols);
    }
}

}  // namespace gemm
}  // namespace tmm
