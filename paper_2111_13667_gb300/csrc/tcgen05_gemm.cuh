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

// GELU, erf form: gelu(z) = z Phi(z) = 0.5 z (1 + erf(z / sqrt 2)), with CUDA's
// erff; its derivative Phi(z) + z phi(z), phi(z) = exp(-z^2 / 2) / sqrt(2 pi).
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z)
{
    const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * __expf(-0.5f * z * z);
    return fmaf(z, pdf, cdf);
}

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
    static constexpr size_t stage = (size_t)kEpiWarps * 32 * 33 * 4;  // per warp 32 x 33 floats (16-byte multiple)
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

// this lane's row of 16 bf16 pairs into the staging buffer
__device__ __forceinline__ void stage_row_bf(uint32_t *stg, const uint32_t (&w)[16], int lane)
{
#pragma unroll
    for (int g = 0; g < 4; ++g)
        *reinterpret_cast<uint4 *>(stg + stg_bf(lane, g)) = make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
}

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

// bf16 packed outputs of a full 32-column chunk: row-major out, optional transposed copy
__device__ __forceinline__ void write_bf_chunk(const EpiArgs &ep, const uint32_t (&y)[16], uint32_t *stg, int row0,
                                               int col0, int M, int lane)
{
    stage_row_bf(stg, y, lane);
    __syncwarp();
    store_rows_bf(stg, ep.out_bf, ep.ldo, row0, col0, M, lane);
    if (ep.out_bfT) {
        if (row0 + 32 <= M) store_cols_bf(stg, ep.out_bfT, ep.ldoT, row0, col0, lane);
        else store_cols_bf_tail(stg, ep.out_bfT, ep.ldoT, row0, col0, M, lane);
    }
    __syncwarp();
}

// Full 32-column chunk, 16-byte aligned outputs.
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
    } else if (EPI == EPI_GELU) {
        uint32_t w[16];  // bf16 pre-activations, then activations
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 b = bias4(ep.bias, col0, j);
            w[2 * j] = pack_bf16(v[4 * j] + b.x, v[4 * j + 1] + b.y);
            w[2 * j + 1] = pack_bf16(v[4 * j + 2] + b.z, v[4 * j + 3] + b.w);
        }
        if (ep.aux) {
            stage_row_bf(stg, w, lane);
            __syncwarp();
            store_rows_bf(stg, ep.aux, ep.ldo, row0, col0, M, lane);
            __syncwarp();
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) w[i] = pack_bf16(gelu(bf_lo(w[i])), gelu(bf_hi(w[i])));
        write_bf_chunk(ep, w, stg, row0, col0, M, lane);
    } else {  // EPI_DGELU: y = acc * gelu'(aux); rows of aux read through the staging buffer
        {
            const int g = lane & 3;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int r = 8 * k + (lane >> 2);
                uint4 t = make_uint4(0u, 0u, 0u, 0u);
                if (row0 + r < M)
                    t = __ldg(reinterpret_cast<const uint4 *>(ep.aux + (long long)(row0 + r) * ep.ldo + col0 + 8 * g));
                *reinterpret_cast<uint4 *>(stg + stg_bf(r, g)) = t;
            }
        }
        __syncwarp();
        uint32_t zw[16];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const uint4 t = *reinterpret_cast<const uint4 *>(stg + stg_bf(lane, g));
            zw[4 * g] = t.x, zw[4 * g + 1] = t.y, zw[4 * g + 2] = t.z, zw[4 * g + 3] = t.w;
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 16; ++i)
            zw[i] = pack_bf16(v[2 * i] * gelu_grad(bf_lo(zw[i])), v[2 * i + 1] * gelu_grad(bf_hi(zw[i])));
        write_bf_chunk(ep, zw, stg, row0, col0, M, lane);
    }
}

// Any chunk (ragged columns, unaligned outputs): element by element, staged
// through shared memory (stride 33 floats) for row-wise stores.
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

__device__ __forceinline__ void epilogue_chunk(const EpiArgs &ep, const float (&v)[32], float *stg, int row0, int n0c,
                                               int M, int N, int lane)
{
    if (ep.vec && n0c + 32 <= N) {
        uint32_t *sw = reinterpret_cast<uint32_t *>(stg);
        switch (ep.epi) {
        case EPI_F32: epilogue_chunk_vec<EPI_F32>(ep, v, sw, row0, n0c, M, lane); return;
        case EPI_F32_CLAMP: epilogue_chunk_vec<EPI_F32_CLAMP>(ep, v, sw, row0, n0c, M, lane); return;
        case EPI_GELU: epilogue_chunk_vec<EPI_GELU>(ep, v, sw, row0, n0c, M, lane); return;
        default: epilogue_chunk_vec<EPI_DGELU>(ep, v, sw, row0, n0c, M, lane); return;
        }
    }
    epilogue_chunk_scalar(ep, v, stg, row0, n0c, M, N, lane);
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
#pragma unroll 1
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
