// tmm_fwd.cu -- forward transfer-matrix kernels: R and T for every
// (stack, lambda, theta, polarisation) of a batch (arXiv 2111.13667, Sec. 2).
//
// Design (sm_103a):
//   * one thread per (stack, lambda, theta) -- in FP32 per (stack, lambda,
//     pair of angles), the two angles on the lanes of the paired FP32
//     instructions; it carries both polarisations, which share Snell's law
//     and the layer phase;
//   * the layer loop runs right to left in registers on the 2-vector
//     x_j = M_j x_{j+1}, x_{L+1} = (1, 0) -- the first column of the product of
//     Eq. 4, which is all Eqs. 5-6 need;
//   * each interface matrix is kept unnormalised, (1/t)[[1,r],[r,1]] times
//     2a (a = q_j for s, q_j / n_j^2 for p, q = n cos(theta)), so no layer needs
//     a complex division; the dropped scale factors only enter |t|^2 and are
//     carried as a product of |q_j|^2 (and |1/n_j^2|^2 for p);
//   * all running products are rescaled by exact powers of two every few
//     layers (two in FP32, eight in FP64), which keeps the FP32 path finite
//     through opaque layers;
//   * per-(medium, wavelength) data (n^2, 1/n^2, d/lambda) are staged once per
//     block in shared memory and reused by every angle of the block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "tmm_df64.cuh"
#include "tmm_device.cuh"
#include "tmm_internal.h"

namespace tmm {

// Largest block of the forward kernels (threads); keeps 128 registers per thread.
constexpr int kMaxThreads = 512;
// Paired-lane (two angles per thread) instances: at most 256 threads, compiled
// for three resident blocks per SM (<= 85 registers, 24 warps).
constexpr int kPairThreads = 256;
constexpr int kPairBlocks = 3;

// One (lambda, theta) point of one stack, both polarisations as requested:
// out = {R_s, T_s, R_p, T_p}.
//
// Each layer's phase matrix is applied divided by its real factor
// e^{Im delta}: diag(e^{-i Re delta}, e^{-2 Im delta} e^{i Re delta}).  R does
// not see the factor; for T the product of all factors enters |t|^2 as
// 2^{-2 K Y}, Y = sum of Im(delta) / (2 pi), K = 2 pi log2(e).  The p
// interfaces are kept unnormalised by 1/n_j^2 products; T_p takes back
// prod_{j=1..L+1} |1/n_j^2|^2, accumulated along the sweep.

// Running state of one point's right-to-left sweep.
template <typename R> struct Sweep {
    Cx<R> q_nx, g_nx;        // q and q / n^2 of the medium to the right
    Cx<R> s0, s1, p0, p1;    // s and p amplitude pairs (scaled)
    R Ps, Y;                 // prod |q_j|^2 (scaled), sum of Im delta_j / (2 pi)
    R Pp;                    // prod |1/n_j^2|^2 (scaled)
};

// Layer j (1..L): its interface with medium j+1, then its phase (Eq. 3).
template <typename R, int POL>
__device__ __forceinline__ void layer_step(const StageA<R> *__restrict__ sa, const StageB<R> *__restrict__ sb, int TL,
                                           int tl, int j, R q0sq, R yi_max, Sweep<R> &w)
{
    const StageA<R> A = sa[j * TL + tl];
    const StageB<R> B = sb[j * TL + tl];
    R absz;
    const Cx<R> q = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
    w.Ps *= absz;
    // layer phase in turns: delta / (2 pi) = (d / lambda) q, Im clamped
    const R yr = B.dl * q.x;
    const R yi = fmin(B.dl * q.y, yi_max);
    w.Y += yi;
    R sn, cs;
    sincos_turn(yr - rint_w(yr), &sn, &cs);
    const R E2 = exp_m2_turn(yi);
    // Both components turn, by conjugate factors: dropping the common phase
    // e^{-i Re delta} (R and T do not see it) would leave the rounding of
    // |(cs, sn)| on x1 alone, a spurious gain or loss per layer that high-Q
    // guided modes under total internal reflection amplify (in FP32 emulation
    // of a reflectivity map: |R - 1| from 7e-6 to 2e-3).
    const Cx<R> emi = {cs, -sn};            // e^{-i delta} / e^{Im delta}
    const Cx<R> epi = {E2 * cs, E2 * sn};   // e^{+i delta} / e^{Im delta}
    if (POL & 1) {
        interface_pair(q, w.q_nx, w.s0, w.s1);
        w.s0 = cmul(emi, w.s0);
        w.s1 = cmul(epi, w.s1);
    }
    if (POL & 2) {
        w.Pp *= B.ain2;
        const Cx<R> g = cmul(q, Cx<R>{A.in2x, A.in2y});
        interface_pair(g, w.g_nx, w.p0, w.p1);
        w.p0 = cmul(emi, w.p0);
        w.p1 = cmul(epi, w.p1);
        w.g_nx = g;
    }
    w.q_nx = q;
}

// Interface 0 | 1 and Eqs. 5-6 for one point, from the sweep's state after
// layer 1: scaled pairs, |q|^2 product Ps0 (exponent eP), sum Y of Im delta /
// (2 pi), p index product Pp (exponent ePp), pair exponents es, ep.
template <typename R, int POL>
__device__ __forceinline__ void finish_point(const StageA<R> &A, Cx<R> q_out, Cx<R> n2_out, Cx<R> q_nx, Cx<R> g_nx,
                                             Cx<R> s0, Cx<R> s1, Cx<R> p0, Cx<R> p1, R Ps0, R Y, R Pp, int eP,
                                             int ePp, int es, int ep, int L, R n0, R beta, R c0, R out[4])
{
    // interface 0 -> 1; the injection medium is real, so q_0 = n_0 cos(theta)
    // (computed directly: n_0^2 - beta^2 cancels near grazing incidence)
    const bool grazing = beta >= n0;  // false for a NaN (complex, rejected) n_0
    const Cx<R> q0 = {c0, R(0)};
    const R Ps = Ps0 * (q0.x * q0.x);
    const int e4 = 2 * (L + 1);  // the factors 2 of every 2a
    // 2^{-2 K Y} = 2^{yf} 2^{yn}, yn integer
    R u = R(-2.0 * kTwoPi * kLog2e) * Y;
    u = fmax(u, R(-1.0e6));
    const R un = floor_w(u);
    const R yscale = exp2_w(u - un);
    const int yn = (int)un;
    if (POL & 1) {
        Cx<R> x0 = s0, x1 = s1;
        interface_pair(q0, q_nx, x0, x1);
        const R ax0 = abs2(x0);
        R Rv = abs2(x1) / ax0;
        R Tv = q_out.x / q0.x * ldexp_w(Ps * yscale / ax0, e4 + eP + yn - 2 * es);
        if (grazing) { Rv = R(1); Tv = R(0); }
        out[0] = Rv;
        out[1] = Tv;
    }
    if (POL & 2) {
        const Cx<R> g0 = cmul(q0, Cx<R>{A.in2x, A.in2y});
        Cx<R> x0 = p0, x1 = p1;
        interface_pair(g0, g_nx, x0, x1);
        const R ax0 = abs2(x0);
        R Rv = abs2(x1) / ax0;
        const R num = cmul(n2_out, conj(q_out)).x;
        const R den = n0 * n0 * q0.x;
        R Tv = num / den * ldexp_w(Ps * Pp * yscale / ax0, e4 + eP + ePp + yn - 2 * ep);
        if (grazing) { Rv = R(1); Tv = R(0); }
        out[2] = Rv;
        out[3] = Tv;
    }
}

// Evaluate one (lambda, theta) point: right-to-left product (Eq. 4) applied to
// the vector (1, 0) of the exit medium, then r, t (Eqs. 5-6) and R, T.
template <typename R, int POL>
__device__ __forceinline__ void eval_point(const StageA<R> *__restrict__ sa, const StageB<R> *__restrict__ sb,
                                           int TL, int tl, int L, R n0, R sin_theta, R cos_theta, R out[4])
{
    constexpr int RN = RenormEvery<R>::value;
    const R beta = n0 * sin_theta;
    const R c0 = n0 * cos_theta;
    const R q0sq = c0 * c0;  // n_j^2 - beta^2 = (n_j^2 - n_0^2) + q0sq
    const R yi_max = R(kImDeltaMax / kTwoPi);

    StageA<R> A = sa[(L + 1) * TL + tl];
    R absz;
    Sweep<R> w;
    w.q_nx = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
    const Cx<R> q_out = w.q_nx, n2_out = {A.d2x + n0 * n0, A.n2y};
    w.g_nx = cmul(w.q_nx, Cx<R>{A.in2x, A.in2y});
    w.Ps = R(1), w.Y = R(0);
    int eP = 0;
    w.Pp = (POL & 2) ? sb[(L + 1) * TL + tl].ain2 : R(1);
    int ePp = 0;
    w.s0 = {R(1), R(0)}, w.s1 = {R(0), R(0)}, w.p0 = {R(1), R(0)}, w.p1 = {R(0), R(0)};
    int es = 0, ep = 0;

    // groups of RN layers, each followed by a power-of-two rescale of the
    // pairs; the |q|^2 product every second group
    int j = L;
    for (; j >= 2 * RN; j -= 2 * RN) {
#pragma unroll
        for (int k = 0; k < RN; ++k) layer_step<R, POL>(sa, sb, TL, tl, j - k, q0sq, yi_max, w);
        if (POL & 1) renorm_pair(w.s0, w.s1, es);
        if (POL & 2) renorm_pair(w.p0, w.p1, ep);
#pragma unroll
        for (int k = RN; k < 2 * RN; ++k) layer_step<R, POL>(sa, sb, TL, tl, j - k, q0sq, yi_max, w);
        renorm_scalar(w.Ps, eP);
        if (POL & 2) renorm_scalar(w.Pp, ePp);
        if (POL & 1) renorm_pair(w.s0, w.s1, es);
        if (POL & 2) renorm_pair(w.p0, w.p1, ep);
    }
    for (; j >= RN; j -= RN) {
#pragma unroll
        for (int k = 0; k < RN; ++k) layer_step<R, POL>(sa, sb, TL, tl, j - k, q0sq, yi_max, w);
        renorm_scalar(w.Ps, eP);
        if (POL & 2) renorm_scalar(w.Pp, ePp);
        if (POL & 1) renorm_pair(w.s0, w.s1, es);
        if (POL & 2) renorm_pair(w.p0, w.p1, ep);
    }
    for (; j >= 1; --j) layer_step<R, POL>(sa, sb, TL, tl, j, q0sq, yi_max, w);
    finish_point<R, POL>(sa[tl], q_out, n2_out, w.q_nx, w.g_nx, w.s0, w.s1, w.p0, w.p1, w.Ps, w.Y, w.Pp, eP, ePp, es,
                         ep, L, n0, beta, c0, out);
}

// Reduction mode (tmm_coh_reward): with Rt set, a work item writes no R, T
// but the sum over its points and output planes of |R_target - R| into
// partial[s * n_tiles + tile] (fixed-order block reduction).
template <typename R> struct Reduce {
    const R *Rt;  // [P][n_theta][n_lambda] or null (plain R, T output)
    R *partial;   // [S][n_tiles]
    int n_tiles;
};

// Stage one work item and evaluate it.  Every thread of the block calls this;
// it contains one barrier (more in reduction mode).
template <typename R, int POL, bool WITH_T, bool RED>
__device__ __forceinline__ void run_item(const tmm_problem &p, int s, int lt, int tt, int n_tt, int TL, int TT,
                                         unsigned char *smem, R *__restrict__ Rout, R *__restrict__ Tout,
                                         const Reduce<R> &red)
{
    StageA<R> *sa = reinterpret_cast<StageA<R> *>(smem);
    StageB<R> *sb = reinterpret_cast<StageB<R> *>(sa + (size_t)(p.L_max + 2) * TL);
    R *n0s = reinterpret_cast<R *>(sb + (size_t)(p.L_max + 2) * TL);

    const int tid = threadIdx.y * TL + threadIdx.x;
    const int nthr = TL * TT;
    const int L = layers_of(p, s);
    const int l0 = lt * TL, t0 = tt * TT;
    if (L >= 0) fill_stage<R>(p, s, L, l0, TL, sa, sb, n0s, tid, nthr);
    __syncthreads();

    const int tl = threadIdx.x, l = l0 + tl, a = t0 + threadIdx.y;
    R contrib = R(0);
    if (l < p.n_lambda && a < p.n_theta) {
        R out[4];
        if (L >= 0) {
            R sth, cth;
            sincos_w(((const R *)p.theta)[a], &sth, &cth);
            eval_point<R, POL>(sa, sb, TL, tl, L, n0s[tl], sth, cth, out);
        } else {
            out[0] = out[1] = out[2] = out[3] = nan_w<R>();
        }
        if (RED) {
            const long long tplane = (long long)p.n_theta * p.n_lambda, ot = (long long)a * p.n_lambda + l;
            if (POL & 4) {
                contrib = fabs(red.Rt[ot] - R(0.5) * (out[0] + out[2]));
            } else {
                int pi = 0;
                if (POL & 1) contrib += fabs(red.Rt[ot] - out[0]), ++pi;
                if (POL & 2) contrib += fabs(red.Rt[pi * tplane + ot] - out[2]);
            }
        } else {
            const long long plane = (long long)p.S * p.n_theta * p.n_lambda;
            const long long o = ((long long)s * p.n_theta + a) * p.n_lambda + l;
            int pi = 0;
            if (POL & 4) {  // unpolarised: the mean of s and p in one plane
                Rout[o] = R(0.5) * (out[0] + out[2]);
                if (WITH_T) Tout[o] = R(0.5) * (out[1] + out[3]);
            } else if (POL & 1) {
                Rout[o] = out[0];
                if (WITH_T) Tout[o] = out[1];
                ++pi;
            }
            if ((POL & 2) && !(POL & 4)) {
                Rout[pi * plane + o] = out[2];
                if (WITH_T) Tout[pi * plane + o] = out[3];
            }
        }
    }
    if (RED) {
        // fixed-order tree sum over the block (the stage is no longer read)
        __syncthreads();
        R *buf = reinterpret_cast<R *>(smem);
        buf[tid] = contrib;
        __syncthreads();
        int half = 1;
        while (half < nthr) half <<= 1;
        for (half >>= 1; half > 0; half >>= 1) {
            if (tid < half && tid + half < nthr) buf[tid] += buf[tid + half];
            __syncthreads();
        }
        if (tid == 0) red.partial[(long long)s * red.n_tiles + lt * n_tt + tt] = buf[0];
    }
    __syncthreads();
}

// ---------------------------------------------------------------- FP32 stage and layer phase
// The FP32 kernels stage, per (medium j, wavelength), 28 bytes:
//   StageQ  {n_j^2 - n_0^2 (rounded once from double-float arithmetic on the
//           inputs), d_j / lambda, f_j, Re m_j} with m_j = +-n_j (below) and
//           f_j the fraction of (d_j / lambda) Re m_j from a double-float
//           product;
//   1 / n_j^2 (complex) and Im m_j;
// per wavelength the injection index n_0 and per angle of the tile sin and
// cos of theta, each as a float pair.  Im n_j^2 = 2 Re m_j Im m_j and
// |1/n_j^2|^2 are formed where they are used, which keeps a 120-layer stage
// of 32 wavelengths within half of an SM's shared memory.  Inputs are float
// (TMM_F32) or double (TMM_F32D, split into float pairs by integer
// operations).
//
// Layer phase.  A float product (d/lambda) Re q carries the roundings of
// d/lambda, of q and of the product on the whole phase -- several turns in a
// thick high-index layer, which near grazing incidence a resonant stack turns
// into errors of 1e-4 in R.  The kernels instead split the phase in turns as
//   (d/lambda) Re q = f + (d/lambda) Re(q - m),
//   Re(q - m) = Re((q^2 - m^2) / (q + m)) = -beta^2 Re(1 / (q + m)),
// using q^2 = n^2 - beta^2 (Snell's law, beta = n_0 sin theta), where m = +-n
// is the root of n^2 that the interior root of q reaches at normal incidence
// (Im m >= 0; Re m >= 0 for a real index) and f the fraction of
// (d/lambda) Re m.  As beta grows, z = n^2 - beta^2 moves parallel to the real
// axis and q stays in m's quadrant, so |q + m| >= |m|.  f is staged exactly;
// the second term, computed in float, is small wherever the phase is large:
// the float roundings act only on the part of the phase that depends on the
// angle.  Where the wave in the layer is (nearly) evanescent, |Re q| < |Re m|/2,
// the two terms would cancel, and the plain product (d/lambda) Re q, then
// small, is used instead (exactly 0 for a lossless evanescent layer).
struct __align__(16) StageQ {
    float d2x, dl, fr, mx;
};

// Shared-memory layout of an FP32 work item: byte offsets of its arrays.
struct Stage32Layout {
    size_t in2, my, n0, th, total;
};
__host__ __device__ __forceinline__ size_t align16(size_t v) { return (v + 15) / 16 * 16; }
__host__ __device__ __forceinline__ Stage32Layout stage32_layout(int L_max, int TL, int TT)
{
    const size_t m = (size_t)(L_max + 2) * TL;
    Stage32Layout g;
    g.in2 = m * sizeof(float4);
    g.my = g.in2 + m * sizeof(float2);
    g.n0 = align16(g.my + m * sizeof(float));
    g.th = align16(g.n0 + (size_t)TL * sizeof(float2));
    g.total = g.th + (size_t)TT * sizeof(float4);
    return g;
}

struct Stage32 {
    StageQ *q;
    float2 *in2;  // 1 / n^2
    float *my;    // Im m
    float2 *n0;   // (hi, lo); NaN if the injection medium is complex
    float4 *th;   // {sin hi, sin lo, cos hi, cos lo} of the tile's angles
};

__device__ __forceinline__ Stage32 stage32_at(unsigned char *smem, int L_max, int TL, int TT)
{
    const Stage32Layout g = stage32_layout(L_max, TL, TT);
    return Stage32{reinterpret_cast<StageQ *>(smem), reinterpret_cast<float2 *>(smem + g.in2),
                   reinterpret_cast<float *>(smem + g.my), reinterpret_cast<float2 *>(smem + g.n0),
                   reinterpret_cast<float4 *>(smem + g.th)};
}

// One medium's staged data as the sweep uses it.
struct Medium32 {
    float d2x, n2y, dl, fr, mx, my;
    Cx<float> in2;
};
__device__ __forceinline__ Medium32 medium_at(const Stage32 &g, int idx)
{
    const StageQ Q = g.q[idx];
    const float2 i2 = g.in2[idx];
    const float my = g.my[idx];
    return Medium32{Q.d2x, 2.f * Q.mx * my, Q.dl, Q.fr, Q.mx, my, Cx<float>{i2.x, i2.y}};
}

template <typename In> __device__ __forceinline__ df::dd in_dd(In v);
template <> __device__ __forceinline__ df::dd in_dd<float>(float v) { return df::dd{v, 0.f}; }
template <> __device__ __forceinline__ df::dd in_dd<double>(double v)
{
    const df::dd t = split_f64(v);
    return df::fast_two_sum(t.hi, t.lo);  // hi = v rounded to float
}

// Fill the FP32 stage for media 0..L+1 of stack s, wavelengths l0..l0+TL-1 and
// angles t0..t0+TT-1.  Only the phase reference needs more than float
// precision: d/lambda as q1 + q2 (float quotient plus the exact remainder
// divided once more) and its product with Re m by a two-product.
template <typename In>
__device__ __forceinline__ void fill_stage32(const tmm_problem &p, int s, int L, int l0, int TL, int t0, int TT,
                                             const float4 *tab, const Stage32 &g, int tid, int nthr)
{
    const In *lam = (const In *)p.lambda;
    const In *d = (const In *)p.d;
    const int total = (L + 2) * TL;
    for (int idx = tid; idx < total; idx += nthr) {
        const int j = idx / TL, tl = idx - j * TL;
        const int l = min(l0 + tl, p.n_lambda - 1);
        const Cx<In> n = index_of<In>(p, s, j, l);
        const In n0v = j == 0 ? n.x : index_of<In>(p, s, 0, l).x;
        const df::dd nx = in_dd<In>(n.x), ny = in_dd<In>(n.y), n0 = in_dd<In>(n0v);
        // n^2 - n_0^2 = (n' - n_0)(n' + n_0) - n''^2, rounded once: both factors
        // and n''^2 as exact float pairs (TwoSum, two-product), then one
        // rounding of the leading difference plus the collected low parts
        df::dd a = df::two_sum(nx.hi, -n0.hi), b = df::two_sum(nx.hi, n0.hi);
        float yl2 = 0.f;
        if constexpr (std::is_same<In, double>::value) {
            a.lo = __fadd_rn(a.lo, __fsub_rn(nx.lo, n0.lo));
            b.lo = __fadd_rn(b.lo, __fadd_rn(nx.lo, n0.lo));
            yl2 = __fmul_rn(2.f * ny.hi, ny.lo);
        }
        const df::dd pab = df::two_prod(a.hi, b.hi), y2 = df::two_prod(ny.hi, ny.hi);
        const float lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, __fsub_rn(pab.lo, __fadd_rn(y2.lo, yl2))));
        const float d2 = __fadd_rn(__fsub_rn(pab.hi, y2.hi), lo);
        const Cx<float> nf = {nx.hi, ny.hi};
        const Cx<float> n2 = {fmaf(nf.x, nf.x, -nf.y * nf.y), 2.f * nf.x * nf.y};
        const float ia = 1.f / abs2(n2);
        // m = +-n, the interior root of n^2 (Im m >= 0, Re m >= 0 if Im m = 0);
        // Im m is stored as +0 for a real index, so that Im n^2 = 2 Re m Im m
        // is +0 and the interior root takes Re q >= 0 there too
        const bool flip = nf.y < 0.f || (nf.y == 0.f && nf.x < 0.f);
        const float mh = flip ? -nx.hi : nx.hi, ml = flip ? -nx.lo : nx.lo;
        StageQ Q;
        Q.d2x = d2;
        Q.dl = 0.f;
        Q.fr = 0.f;
        if (j >= 1 && j <= L) {
            const df::dd dv = in_dd<In>(d[(long long)s * p.L_max + (j - 1)]), lv = in_dd<In>(lam[l]);
            const float q1 = dv.hi / lv.hi;
            float r = fmaf(-q1, lv.hi, dv.hi);  // exact remainder of the float quotient
            if constexpr (std::is_same<In, double>::value) r += fmaf(-q1, lv.lo, dv.lo);
            const float q2 = r / lv.hi;
            // (q1 + q2) (mh + ml) = ph + e, ph = q1 mh rounded, e its error and the cross terms
            const float ph = __fmul_rn(q1, mh);
            float e = fmaf(q1, mh, -ph);
            e = fmaf(q1, ml, e);
            e = fmaf(q2, mh, e);
            const float k = rintf(ph);
            Q.dl = q1;
            Q.fr = __fadd_rn(__fsub_rn(ph, k), e);
        }
        Q.mx = mh;
        const float my = flip ? -nf.y : nf.y;
        g.q[idx] = Q;
        g.in2[idx] = make_float2(n2.x * ia, -n2.y * ia);
        g.my[idx] = my == 0.f ? 0.f : my;
        if (j == 0) g.n0[tl] = (n.y == In(0)) ? make_float2(n0.hi, n0.lo) : make_float2(nan_w<float>(), 0.f);
    }
    const In *th = (const In *)p.theta;
    for (int i = tid; i < TT; i += nthr) {
        const int a = min(t0 + i, p.n_theta - 1);
        const df::dd f = df::mul(in_dd<In>(th[a]), dconst(1.0 / (2.0 * kPi)));
        df::dd sv, cv;
        sincos_turn_dd(df::add_f(f, -rintf(f.hi)), tab, &sv, &cv);
        g.th[i] = make_float4(sv.hi, sv.lo, cv.hi, cv.lo);
    }
}

// The injection medium's 1 / n_0^2 in the StageA form finish_point takes.
__device__ __forceinline__ StageA<float> in2_stage(const Stage32 &g, int tl)
{
    const float2 i2 = g.in2[tl];
    return StageA<float>{0.f, 0.f, i2.x, i2.y};
}

// Per-angle terms of one point from the staged sin, cos (float pairs) and n_0:
// beta = n_0 sin theta, c0 = n_0 cos theta, q0sq = c0^2, nb2 = -beta^2.
struct Angle32 {
    float beta, c0, q0sq, nb2;
};
__device__ __forceinline__ Angle32 angle_terms(float4 t, float2 n0v)
{
    const df::dd n0{n0v.x, n0v.y};
    const df::dd b = df::mul(df::dd{t.x, t.y}, n0);
    const df::dd c = df::mul(df::dd{t.z, t.w}, n0);
    return Angle32{b.hi, c.hi, df::sqr(c).hi, -df::sqr(b).hi};
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Layer phase Re(delta) / (2 pi) reduced to [-1/2, 1/2] (see above).
__device__ __forceinline__ float phase_turns(Cx<float> q, const Medium32 &P, float nb2)
{
    const float sx = q.x + P.mx, sy = q.y + P.my;
    const float rs = rcp_approx(fmaf(sx, sx, sy * sy));
    const float fm = fmaf(P.dl, nb2 * sx * rs, P.fr);
    const float f = fabsf(q.x) >= 0.5f * fabsf(P.mx) ? fm : P.dl * q.x;
    return f - rintf(f);
}

// phase_turns for the two lanes of a thread (paired instructions).
__device__ __forceinline__ float2 phase_turns2(Cx<float> qa, Cx<float> qb, const Medium32 &P, float2 nb2)
{
    const float2 qx = f2(qa.x, qb.x);
    const float2 sx = add2(qx, bc2(P.mx)), sy = add2(f2(qa.y, qb.y), bc2(P.my));
    const float2 s2 = fma2(sx, sx, mul2(sy, sy));
    const float2 rs = f2(rcp_approx(s2.x), rcp_approx(s2.y));
    const float2 fm = fma2(bc2(P.dl), mul2(mul2(nb2, sx), rs), bc2(P.fr));
    const float2 fd = mul2(bc2(P.dl), qx);
    const float h = 0.5f * fabsf(P.mx);
    const float2 f = f2(fabsf(qa.x) >= h ? fm.x : fd.x, fabsf(qb.x) >= h ? fm.y : fd.y);
    return f2(f.x - rintf(f.x), f.y - rintf(f.y));
}

// ---------------------------------------------------------------- FP32: one angle per thread
template <int POL>
__device__ __forceinline__ void layer_step_f(const Stage32 &g, int TL, int tl, int j, float q0sq, float nb2,
                                             float yi_max, Sweep<float> &w)
{
    const Medium32 P = medium_at(g, j * TL + tl);
    float absz;
    const Cx<float> q = inner_root(Cx<float>{P.d2x + q0sq, P.n2y}, &absz);
    w.Ps *= absz;
    const float yi = fminf(P.dl * q.y, yi_max);
    w.Y += yi;
    float sn, cs;
    sincos_turn(phase_turns(q, P, nb2), &sn, &cs);
    const float E2 = exp_m2_turn(yi);
    const Cx<float> emi = {cs, -sn};
    const Cx<float> epi = {E2 * cs, E2 * sn};
    if (POL & 1) {
        interface_pair(q, w.q_nx, w.s0, w.s1);
        w.s0 = cmul(emi, w.s0);
        w.s1 = cmul(epi, w.s1);
    }
    if (POL & 2) {
        w.Pp *= abs2(P.in2);
        const Cx<float> gq = cmul(q, P.in2);
        interface_pair(gq, w.g_nx, w.p0, w.p1);
        w.p0 = cmul(emi, w.p0);
        w.p1 = cmul(epi, w.p1);
        w.g_nx = gq;
    }
    w.q_nx = q;
}

template <int POL>
__device__ __forceinline__ void eval_point_f(const Stage32 &g, int TL, int tl, int L, float n0, const Angle32 &an,
                                             float out[4])
{
    constexpr int RN = RenormEvery<float>::value;
    const float yi_max = float(kImDeltaMax / kTwoPi);
    const Medium32 A = medium_at(g, (L + 1) * TL + tl);
    float absz;
    Sweep<float> w;
    w.q_nx = forward_root(Cx<float>{A.d2x + an.q0sq, A.n2y}, &absz);
    const Cx<float> q_out = w.q_nx, n2_out = {A.d2x + n0 * n0, A.n2y};
    w.g_nx = cmul(w.q_nx, A.in2);
    w.Ps = 1.f, w.Y = 0.f;
    int eP = 0;
    w.Pp = (POL & 2) ? abs2(A.in2) : 1.f;
    int ePp = 0;
    w.s0 = {1.f, 0.f}, w.s1 = {0.f, 0.f}, w.p0 = {1.f, 0.f}, w.p1 = {0.f, 0.f};
    int es = 0, ep = 0;
    int j = L;
    for (; j >= 2 * RN; j -= 2 * RN) {
#pragma unroll
        for (int k = 0; k < RN; ++k) layer_step_f<POL>(g, TL, tl, j - k, an.q0sq, an.nb2, yi_max, w);
        if (POL & 1) renorm_pair(w.s0, w.s1, es);
        if (POL & 2) renorm_pair(w.p0, w.p1, ep);
#pragma unroll
        for (int k = RN; k < 2 * RN; ++k) layer_step_f<POL>(g, TL, tl, j - k, an.q0sq, an.nb2, yi_max, w);
        renorm_scalar(w.Ps, eP);
        if (POL & 2) renorm_scalar(w.Pp, ePp);
        if (POL & 1) renorm_pair(w.s0, w.s1, es);
        if (POL & 2) renorm_pair(w.p0, w.p1, ep);
    }
    for (; j >= RN; j -= RN) {
#pragma unroll
        for (int k = 0; k < RN; ++k) layer_step_f<POL>(g, TL, tl, j - k, an.q0sq, an.nb2, yi_max, w);
        renorm_scalar(w.Ps, eP);
        if (POL & 2) renorm_scalar(w.Pp, ePp);
        if (POL & 1) renorm_pair(w.s0, w.s1, es);
        if (POL & 2) renorm_pair(w.p0, w.p1, ep);
    }
    for (; j >= 1; --j) layer_step_f<POL>(g, TL, tl, j, an.q0sq, an.nb2, yi_max, w);
    finish_point<float, POL>(in2_stage(g, tl), q_out, n2_out, w.q_nx, w.g_nx, w.s0, w.s1, w.p0, w.p1, w.Ps, w.Y,
                             w.Pp, eP, ePp, es, ep, L, n0, an.beta, an.c0, out);
}

// ---------------------------------------------------------------- FP32: two angles per thread
// An FP32 thread carries two angles of one wavelength on the two lanes of the
// paired instructions: the amplitude pairs, |q|^2 products and phase sums are
// float2 per component; the stage (per medium and wavelength) and the p index
// product are shared.  Roots, sin/cos and exp2 stay per lane (one MUFU each).
// The arithmetic is the one-angle path's up to the order of two additions per
// interface and the branch of q inside the stack, which R and T do not see.
struct Sweep2 {
    C2 q_nx, g_nx;        // q and q / n^2 of the medium to the right
    float2 nqy_nx, ngy_nx;  // minus their imaginary parts
    C2 s0, s1, p0, p1;
    float2 Ps, Y;
    float Pp;
};

template <int POL>
__device__ __forceinline__ void layer_step2(const Stage32 &g, int TL, int tl, int j, float2 q0sq, float2 nb2,
                                            float yi_max, Sweep2 &w)
{
    const Medium32 P = medium_at(g, j * TL + tl);
    float absa, absb;
    const Cx<float> qa = inner_root(Cx<float>{P.d2x + q0sq.x, P.n2y}, &absa);
    const Cx<float> qb = inner_root(Cx<float>{P.d2x + q0sq.y, P.n2y}, &absb);
    w.Ps = mul2(w.Ps, f2(absa, absb));
    const float2 yi = f2(fminf(P.dl * qa.y, yi_max), fminf(P.dl * qb.y, yi_max));
    w.Y = add2(w.Y, yi);
    const float2 f = phase_turns2(qa, qb, P, nb2);
    float2 sn, cs;
    sincos_turn(f.x, &sn.x, &cs.x);
    sincos_turn(f.y, &sn.y, &cs.y);
    const float2 E2 = f2(exp_m2_turn(yi.x), exp_m2_turn(yi.y));
    const float2 nsn = neg2(sn), ec = mul2(E2, cs), es = mul2(E2, sn), nes = neg2(es);
    if (POL & 1) {
        const C2 q = pack2(qa, qb);
        const float2 nqy = neg2(q.y);
        interface_pair2(q, nqy, w.q_nx, w.nqy_nx, w.s0, w.s1);
        phase2(cs, sn, nsn, ec, es, nes, w.s0, w.s1);
        w.q_nx = q;
        w.nqy_nx = nqy;
    }
    if (POL & 2) {
        w.Pp *= abs2(P.in2);
        const C2 gq = pack2(cmul(qa, P.in2), cmul(qb, P.in2));
        const float2 ngy = neg2(gq.y);
        interface_pair2(gq, ngy, w.g_nx, w.ngy_nx, w.p0, w.p1);
        phase2(cs, sn, nsn, ec, es, nes, w.p0, w.p1);
        w.g_nx = gq;
        w.ngy_nx = ngy;
    }
}

// eval_point_f for the angles of the two lanes: out[i] = {R_s, T_s, R_p, T_p}
// of lane i.
template <int POL>
__device__ __forceinline__ void eval_point2(const Stage32 &g, int TL, int tl, int L, float n0, const Angle32 an[2],
                                            float out[2][4])
{
    constexpr int RN = RenormEvery<float>::value;
    const float2 q0sq = f2(an[0].q0sq, an[1].q0sq), nb2 = f2(an[0].nb2, an[1].nb2);
    const float yi_max = float(kImDeltaMax / kTwoPi);

    const Medium32 A = medium_at(g, (L + 1) * TL + tl);
    float absz;
    const Cx<float> qoa = forward_root(Cx<float>{A.d2x + q0sq.x, A.n2y}, &absz);
    const Cx<float> qob = forward_root(Cx<float>{A.d2x + q0sq.y, A.n2y}, &absz);
    const Cx<float> n2_out = {A.d2x + n0 * n0, A.n2y};
    const Cx<float> in2 = A.in2;
    Sweep2 w;
    w.q_nx = pack2(qoa, qob);
    w.nqy_nx = neg2(w.q_nx.y);
    w.g_nx = pack2(cmul(qoa, in2), cmul(qob, in2));
    w.ngy_nx = neg2(w.g_nx.y);
    w.Ps = bc2(1.f);
    w.Y = bc2(0.f);
    w.Pp = (POL & 2) ? abs2(in2) : 1.f;
    int ePa = 0, ePb = 0, ePp = 0;
    w.s0 = C2{bc2(1.f), bc2(0.f)};
    w.s1 = C2{bc2(0.f), bc2(0.f)};
    w.p0 = w.s0;
    w.p1 = w.s1;
    int esa = 0, esb = 0, epa = 0, epb = 0;

    // the one-angle kernel's grouping: RN layers, rescale the pairs, RN more,
    // rescale the products and the pairs
    int j = L;
    for (; j >= 2 * RN; j -= 2 * RN) {
#pragma unroll
        for (int k = 0; k < RN; ++k) layer_step2<POL>(g, TL, tl, j - k, q0sq, nb2, yi_max, w);
        if (POL & 1) renorm_pair2(w.s0, w.s1, esa, esb);
        if (POL & 2) renorm_pair2(w.p0, w.p1, epa, epb);
#pragma unroll
        for (int k = RN; k < 2 * RN; ++k) layer_step2<POL>(g, TL, tl, j - k, q0sq, nb2, yi_max, w);
        renorm_scalar(w.Ps.x, ePa);
        renorm_scalar(w.Ps.y, ePb);
        if (POL & 2) renorm_scalar(w.Pp, ePp);
        if (POL & 1) renorm_pair2(w.s0, w.s1, esa, esb);
        if (POL & 2) renorm_pair2(w.p0, w.p1, epa, epb);
    }
    for (; j >= RN; j -= RN) {
#pragma unroll
        for (int k = 0; k < RN; ++k) layer_step2<POL>(g, TL, tl, j - k, q0sq, nb2, yi_max, w);
        renorm_scalar(w.Ps.x, ePa);
        renorm_scalar(w.Ps.y, ePb);
        if (POL & 2) renorm_scalar(w.Pp, ePp);
        if (POL & 1) renorm_pair2(w.s0, w.s1, esa, esb);
        if (POL & 2) renorm_pair2(w.p0, w.p1, epa, epb);
    }
    for (; j >= 1; --j) layer_step2<POL>(g, TL, tl, j, q0sq, nb2, yi_max, w);
    const StageA<float> A0 = in2_stage(g, tl);
    finish_point<float, POL>(A0, qoa, n2_out, lane(w.q_nx, 0), lane(w.g_nx, 0), lane(w.s0, 0), lane(w.s1, 0),
                             lane(w.p0, 0), lane(w.p1, 0), w.Ps.x, w.Y.x, w.Pp, ePa, ePp, esa, epa, L, n0, an[0].beta,
                             an[0].c0, out[0]);
    finish_point<float, POL>(A0, qob, n2_out, lane(w.q_nx, 1), lane(w.g_nx, 1), lane(w.s0, 1), lane(w.s1, 1),
                             lane(w.p0, 1), lane(w.p1, 1), w.Ps.y, w.Y.y, w.Pp, ePb, ePp, esb, epb, L, n0, an[1].beta,
                             an[1].c0, out[1]);
}

// One FP32 work item: PAIR blocks are TL x ceil(TT / 2) threads, thread
// (x, y) taking angles t0 + 2y and t0 + 2y + 1; otherwise TL x TT threads of
// one angle each.  Inputs of type In (float, or double for TMM_F32D).
template <typename In, int POL, bool WITH_T, bool RED, bool PAIR>
__device__ __forceinline__ void run_item_f32(const tmm_problem &p, const float4 *tab, int s, int lt, int tt, int n_tt,
                                             int TL, int TT, unsigned char *smem, float *__restrict__ Rout,
                                             float *__restrict__ Tout, const Reduce<float> &red)
{
    const Stage32 g = stage32_at(smem, p.L_max, TL, TT);
    const int tid = threadIdx.y * TL + threadIdx.x;
    const int nthr = TL * (int)blockDim.y;
    const int L = layers_of(p, s);
    const int l0 = lt * TL, t0 = tt * TT;
    if (L >= 0) fill_stage32<In>(p, s, L, l0, TL, t0, TT, tab, g, tid, nthr);
    __syncthreads();

    constexpr int NP = PAIR ? 2 : 1;
    const int tl = threadIdx.x, l = l0 + tl;
    const int a0 = t0 + NP * (int)threadIdx.y, t_end = min(t0 + TT, p.n_theta);
    const int np = (PAIR && a0 + 1 < t_end) ? 2 : 1;
    float contrib = 0.f;
    if (l < p.n_lambda && a0 < t_end) {
        float out[2][4];
        if (L >= 0) {
            const float2 n0 = g.n0[tl];
            Angle32 an[2];
            an[0] = angle_terms(g.th[a0 - t0], n0);
            an[1] = PAIR ? angle_terms(g.th[a0 - t0 + np - 1], n0) : an[0];
            if constexpr (PAIR)
                eval_point2<POL>(g, TL, tl, L, n0.x, an, out);
            else
                eval_point_f<POL>(g, TL, tl, L, n0.x, an[0], out[0]);
        } else {
#pragma unroll
            for (int i = 0; i < 2; ++i) out[i][0] = out[i][1] = out[i][2] = out[i][3] = nan_w<float>();
        }
        const long long tplane = (long long)p.n_theta * p.n_lambda;
        const long long plane = (long long)p.S * tplane;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            if (i == 1 && np < 2) break;
            const int a = a0 + i;
            if (RED) {
                const long long ot = (long long)a * p.n_lambda + l;
                if (POL & 4) {
                    contrib += fabsf(red.Rt[ot] - 0.5f * (out[i][0] + out[i][2]));
                } else {
                    int pi = 0;
                    if (POL & 1) contrib += fabsf(red.Rt[ot] - out[i][0]), ++pi;
                    if (POL & 2) contrib += fabsf(red.Rt[pi * tplane + ot] - out[i][2]);
                }
            } else {
                const long long o = ((long long)s * p.n_theta + a) * p.n_lambda + l;
                int pi = 0;
                if (POL & 4) {
                    Rout[o] = 0.5f * (out[i][0] + out[i][2]);
                    if (WITH_T) Tout[o] = 0.5f * (out[i][1] + out[i][3]);
                } else if (POL & 1) {
                    Rout[o] = out[i][0];
                    if (WITH_T) Tout[o] = out[i][1];
                    ++pi;
                }
                if ((POL & 2) && !(POL & 4)) {
                    Rout[pi * plane + o] = out[i][2];
                    if (WITH_T) Tout[pi * plane + o] = out[i][3];
                }
            }
        }
    }
    if (RED) {
        // fixed-order tree sum over the block (the stage is no longer read)
        __syncthreads();
        float *buf = reinterpret_cast<float *>(smem);
        buf[tid] = contrib;
        __syncthreads();
        int half = 1;
        while (half < nthr) half <<= 1;
        for (half >>= 1; half > 0; half >>= 1) {
            if (tid < half && tid + half < nthr) buf[tid] += buf[tid + half];
            __syncthreads();
        }
        if (tid == 0) red.partial[(long long)s * red.n_tiles + lt * n_tt + tt] = buf[0];
    }
    __syncthreads();
}

// The item evaluator of a kernel instance: FP32 (float or double inputs,
// paired lanes or one angle per thread) or FP64.
template <typename R, typename In, int POL, bool WITH_T, bool RED, bool PAIR>
__device__ __forceinline__ void run_any(const tmm_problem &p, const SinCosTable &tab, int s, int lt, int tt, int n_tt,
                                        int TL, int TT, unsigned char *smem, R *__restrict__ Rout,
                                        R *__restrict__ Tout, const Reduce<R> &red)
{
    if constexpr (std::is_same<R, float>::value)
        run_item_f32<In, POL, WITH_T, RED, PAIR>(p, tab.sc, s, lt, tt, n_tt, TL, TT, smem, Rout, Tout, red);
    else
        run_item<R, POL, WITH_T, RED>(p, s, lt, tt, n_tt, TL, TT, smem, Rout, Tout, red);
}

template <typename R, typename In, int POL, bool WITH_T, bool RED, bool PAIR>
__global__ void __launch_bounds__(PAIR ? kPairThreads : kMaxThreads, PAIR ? kPairBlocks : 1)
    tmm_fwd_kernel(const tmm_problem p, const __grid_constant__ SinCosTable tab, int TL, int TT, int n_lt, int n_tt,
                   R *__restrict__ Rout, R *__restrict__ Tout, const Reduce<R> red)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const long long item = blockIdx.x;
    const int per_stack = n_lt * n_tt;
    const int s = (int)(item / per_stack);
    const int r = (int)(item - (long long)s * per_stack);
    run_any<R, In, POL, WITH_T, RED, PAIR>(p, tab, s, r / n_tt, r % n_tt, n_tt, TL, TT, smem, Rout, Tout, red);
}

// Persistent variant: blocks pull work items from `counter`; item k belongs to
// stack order[k / per_stack] (longest stacks first), tile k % per_stack.  The
// host keeps n_items + grid below 2^32, so the one increment past n_items that
// each block makes before it leaves cannot wrap the counter.
template <typename R, typename In, int POL, bool WITH_T, bool RED, bool PAIR>
__global__ void __launch_bounds__(PAIR ? kPairThreads : kMaxThreads, PAIR ? kPairBlocks : 1)
    tmm_fwd_persistent(const tmm_problem p, const __grid_constant__ SinCosTable tab, int TL, int TT, int n_lt,
                       int n_tt, const int *__restrict__ order, unsigned int *counter, int *err, unsigned int n_items,
                       int max_items, R *__restrict__ Rout, R *__restrict__ Tout, const Reduce<R> red)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned int item_sh;
    const int per_stack = n_lt * n_tt;
    int taken = 0;
    for (;;) {
        if (threadIdx.x == 0 && threadIdx.y == 0) item_sh = atomicAdd(counter, 1u);
        __syncthreads();
        const unsigned int item = item_sh;
        __syncthreads();  // item_sh is rewritten on the next pass
        if (item >= n_items) break;
        if (max_items > 0 && ++taken > max_items) {
            if (threadIdx.x == 0 && threadIdx.y == 0) atomicExch(err, 1);
            break;
        }
        const int k = (int)(item / per_stack);
        const int r = (int)(item - (unsigned int)k * per_stack);
        run_any<R, In, POL, WITH_T, RED, PAIR>(p, tab, order[k], r / n_tt, r % n_tt, n_tt, TL, TT, smem, Rout, Tout,
                                               red);
    }
}

// ---------------------------------------------------------------- longest-first ordering
// Counting sort of the stacks by layer count, descending; a bad count goes last.
__global__ void count_lengths(const int *__restrict__ Ls, int S, int L_max, int *counts)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int L = Ls[s];
    const int bucket = (L < 0 || L > L_max) ? L_max + 1 : L_max - L;
    atomicAdd(&counts[bucket], 1);
}

__global__ void scan_lengths(const int *__restrict__ counts, int n_buckets, int *offsets)
{
    if (threadIdx.x != 0) return;
    int acc = 0;
    for (int b = 0; b < n_buckets; ++b) {
        offsets[b] = acc;
        acc += counts[b];
    }
}

__global__ void scatter_lengths(const int *__restrict__ Ls, int S, int L_max, int *offsets, int *order)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int L = Ls[s];
    const int bucket = (L < 0 || L > L_max) ? L_max + 1 : L_max - L;
    order[atomicAdd(&offsets[bucket], 1)] = s;
}

__global__ void iota_order(int S, int *order)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) order[s] = s;
}

// ---------------------------------------------------------------- host side
static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

PersistentWs persistent_ws_layout(const tmm_problem *p)
{
    PersistentWs w;
    w.counter = 0;
    w.err = 4;
    w.counts = 256;
    w.offsets = align_up(w.counts + sizeof(int) * (size_t)(p->L_max + 2), 256);
    w.order = align_up(w.offsets + sizeof(int) * (size_t)(p->L_max + 2), 256);
    w.total = align_up(w.order + sizeof(int) * (size_t)p->S, 256);
    return w;
}

static bool fp32_family(const tmm_problem *p) { return p->prec == TMM_F32 || p->prec == TMM_F32D; }

static size_t stage_bytes(const tmm_problem *p, int TL, int TT)
{
    if (fp32_family(p)) return stage32_layout(p->L_max, TL, TT).total;
    const size_t r = real_size(p->prec);
    return (size_t)(p->L_max + 2) * TL * (6 * r) + (size_t)TL * r;
}

// FP32 tiles of two or more angles run two angles per thread (paired lanes).
static bool paired(const tmm_problem *p, int TT) { return fp32_family(p) && TT >= 2; }

const SinCosTable &sincos_table()
{
    static SinCosTable t;
    static std::once_flag once;
    std::call_once(once, [] {
        for (int k = 0; k < 64; ++k) {
            const double a = 2.0 * kPi * k / 256.0;
            const double sv = std::sin(a), cv = std::cos(a);
            const float sh = (float)sv, ch = (float)cv;
            t.sc[k] = make_float4(sh, (float)(sv - sh), ch, (float)(cv - ch));
        }
    });
    return t;
}

static int tile_threads(const tmm_problem *p, int TL, int TT) { return TL * (paired(p, TT) ? (TT + 1) / 2 : TT); }
static int max_threads(const tmm_problem *p, int TT) { return paired(p, TT) ? kPairThreads : kMaxThreads; }

tmm_status choose_tile(const tmm_problem *p, const tmm_launch_cfg *cfg, Tile *t)
{
    DeviceInfo di;
    tmm_status st = device_info(&di);
    if (st != TMM_OK) return st;
    int TT = cfg && cfg->tile_theta > 0 ? cfg->tile_theta : std::min(p->n_theta, 32);
    int TL = cfg && cfg->tile_lambda > 0 ? cfg->tile_lambda : 0;
    if (TT < 1 || TL < 0) return TMM_ERR_INVALID_ARG;
    if (TL == 0) {
        TL = 1;
        while (tile_threads(p, TL, TT) < 256 && tile_threads(p, 2 * TL, TT) <= max_threads(p, TT)) TL *= 2;
        while (TL > 1 && TL / 2 >= p->n_lambda) TL /= 2;
        while (TL > 1 && stage_bytes(p, TL, TT) > (size_t)di.max_smem_optin) TL /= 2;
    }
    if (TL < 1 || tile_threads(p, TL, TT) > max_threads(p, TT)) return TMM_ERR_INVALID_ARG;
    t->TL = TL;
    t->TT = TT;
    t->n_lt = (p->n_lambda + TL - 1) / TL;
    t->n_tt = (p->n_theta + TT - 1) / TT;
    t->n_items = (long long)p->S * t->n_lt * t->n_tt;
    t->smem = stage_bytes(p, TL, TT);
    if (t->smem > (size_t)di.max_smem_optin) return TMM_ERR_UNSUPPORTED;
    return TMM_OK;
}

// Per-(kernel, device) host-side facts, cached so that repeated launches (and
// launches recorded into a CUDA graph) make no attribute or occupancy calls.
struct KernelFacts {
    const void *fn;
    int dev, threads;
    size_t smem;
    int per_sm;
};
static std::mutex g_facts_mu;
static std::vector<KernelFacts> g_facts;

static KernelFacts *facts_for(const void *fn, int dev, int threads, size_t smem)
{
    for (auto &f : g_facts)
        if (f.fn == fn && f.dev == dev && f.threads == threads && f.smem == smem) return &f;
    g_facts.push_back(KernelFacts{fn, dev, threads, smem, 0});
    return &g_facts.back();
}

template <typename Kernel>
static tmm_status prepare_kernel(Kernel k, int threads, size_t smem, bool need_occupancy, int *per_sm)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    std::lock_guard<std::mutex> lk(g_facts_mu);
    KernelFacts *f = facts_for(reinterpret_cast<const void *>(k), dev, threads, smem);
    // the limit is granted per kernel (the largest size so far), not per entry:
    // setting it per size could lower it below an entry that was already set
    const tmm_status ss = ensure_dynamic_smem(reinterpret_cast<const void *>(k), smem);
    if (ss != TMM_OK) return ss;
    if (need_occupancy && f->per_sm == 0) {
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem);
        if (e != cudaSuccess) return cuda_fail(e);
        f->per_sm = std::max(n, 1);
    }
    if (per_sm) *per_sm = f->per_sm;
    return TMM_OK;
}

template <typename R, typename In, int POL, bool WITH_T, bool RED, bool PAIR>
static tmm_status launch_shaped(const tmm_problem *p, const tmm_launch_cfg *cfg, const Tile &t, void *ws,
                                R *Rout, R *Tout, const Reduce<R> &red, cudaStream_t st)
{
    const dim3 block(t.TL, PAIR ? (t.TT + 1) / 2 : t.TT);
    const int threads = (int)(block.x * block.y);
    const bool persistent = cfg && cfg->persistent;
    if (!persistent) {
        auto k = tmm_fwd_kernel<R, In, POL, WITH_T, RED, PAIR>;
        tmm_status s = prepare_kernel(k, threads, t.smem, false, nullptr);
        if (s != TMM_OK) return s;
        if (t.n_items > 0x7fffffffLL) return TMM_ERR_UNSUPPORTED;
        if (t.n_items == 0) return TMM_OK;
        k<<<(unsigned)t.n_items, block, t.smem, st>>>(*p, sincos_table(), t.TL, t.TT, t.n_lt, t.n_tt, Rout, Tout,
                                                     red);
        return check_launch();
    }
    auto k = tmm_fwd_persistent<R, In, POL, WITH_T, RED, PAIR>;
    int occ = 0;
    tmm_status s = prepare_kernel(k, threads, t.smem, true, &occ);
    if (s != TMM_OK) return s;
    DeviceInfo di;
    s = device_info(&di);
    if (s != TMM_OK) return s;
    const int per_sm = cfg->blocks_per_sm > 0 ? cfg->blocks_per_sm : occ;
    const long long grid = std::min((long long)per_sm * di.sms, t.n_items);
    // each block takes one item number past n_items before it leaves: keep the
    // 32-bit counter from wrapping
    if (t.n_items + grid > 0xffffffffLL) return TMM_ERR_UNSUPPORTED;
    const PersistentWs w = persistent_ws_layout(p);
    unsigned char *base = static_cast<unsigned char *>(ws);
    cudaError_t e = cudaMemsetAsync(base, 0, w.order, st);  // counter, err, counts, offsets
    if (e != cudaSuccess) return cuda_fail(e);
    int *order = reinterpret_cast<int *>(base + w.order);
    const int nb = (p->S + 255) / 256;
    if (p->S > 0) {
        if (p->L_per_stack) {
            int *counts = reinterpret_cast<int *>(base + w.counts);
            int *offsets = reinterpret_cast<int *>(base + w.offsets);
            count_lengths<<<nb, 256, 0, st>>>(p->L_per_stack, p->S, p->L_max, counts);
            scan_lengths<<<1, 32, 0, st>>>(counts, p->L_max + 2, offsets);
            scatter_lengths<<<nb, 256, 0, st>>>(p->L_per_stack, p->S, p->L_max, offsets, order);
        } else {
            iota_order<<<nb, 256, 0, st>>>(p->S, order);
        }
        tmm_status cs = check_launch();
        if (cs != TMM_OK) return cs;
    }
    if (t.n_items == 0) return TMM_OK;
    k<<<(unsigned)grid, block, t.smem, st>>>(*p, sincos_table(), t.TL, t.TT, t.n_lt, t.n_tt, order,
                                             reinterpret_cast<unsigned int *>(base + w.counter),
                                             reinterpret_cast<int *>(base + w.err), (unsigned)t.n_items,
                                             cfg->max_items_per_block, Rout, Tout, red);
    return check_launch();
}

template <typename R, typename In, int POL, bool WITH_T, bool RED>
static tmm_status launch_typed(const tmm_problem *p, const tmm_launch_cfg *cfg, const Tile &t, void *ws,
                               R *Rout, R *Tout, const Reduce<R> &red, cudaStream_t st)
{
    if constexpr (std::is_same<R, float>::value) {
        if (paired(p, t.TT))
            return launch_shaped<R, In, POL, WITH_T, RED, true>(p, cfg, t, ws, Rout, Tout, red, st);
    }
    return launch_shaped<R, In, POL, WITH_T, RED, false>(p, cfg, t, ws, Rout, Tout, red, st);
}

template <typename R, typename In>
static tmm_status launch_prec(const tmm_problem *p, const tmm_launch_cfg *cfg, const Tile &t, void *ws, void *R_,
                              void *T_, const Reduce<R> &red, cudaStream_t st)
{
    R *Ro = static_cast<R *>(R_);
    R *To = static_cast<R *>(T_);
    if (red.Rt) {  // reduction mode: no R, T output (inputs of the working type only)
        if constexpr (std::is_same<R, In>::value) {
            switch (p->pol_mask) {
            case 1: return launch_typed<R, In, 1, false, true>(p, cfg, t, ws, Ro, To, red, st);
            case 2: return launch_typed<R, In, 2, false, true>(p, cfg, t, ws, Ro, To, red, st);
            case 3: return launch_typed<R, In, 3, false, true>(p, cfg, t, ws, Ro, To, red, st);
            case 7: return launch_typed<R, In, 7, false, true>(p, cfg, t, ws, Ro, To, red, st);
            default: return TMM_ERR_INVALID_ARG;
            }
        } else {
            return TMM_ERR_UNSUPPORTED;
        }
    }
    const bool wt = To != nullptr;
    switch (p->pol_mask) {
    case 1: return wt ? launch_typed<R, In, 1, true, false>(p, cfg, t, ws, Ro, To, red, st) : launch_typed<R, In, 1, false, false>(p, cfg, t, ws, Ro, To, red, st);
    case 2: return wt ? launch_typed<R, In, 2, true, false>(p, cfg, t, ws, Ro, To, red, st) : launch_typed<R, In, 2, false, false>(p, cfg, t, ws, Ro, To, red, st);
    case 3: return wt ? launch_typed<R, In, 3, true, false>(p, cfg, t, ws, Ro, To, red, st) : launch_typed<R, In, 3, false, false>(p, cfg, t, ws, Ro, To, red, st);
    case 7: return wt ? launch_typed<R, In, 7, true, false>(p, cfg, t, ws, Ro, To, red, st) : launch_typed<R, In, 7, false, false>(p, cfg, t, ws, Ro, To, red, st);
    default: return TMM_ERR_INVALID_ARG;
    }
}

tmm_status launch_forward(const tmm_problem *p, const tmm_launch_cfg *cfg, void *ws, size_t ws_bytes, void *R,
                          void *T, cudaStream_t st)
{
    if (p->prec == TMM_F64X) return launch_forward_df64(p, cfg, R, T, st);
    Tile t;
    tmm_status s = choose_tile(p, cfg, &t);
    if (s != TMM_OK) return s;
    if (cfg && cfg->persistent) {
        if (!ws) return TMM_ERR_INVALID_ARG;
        if (ws_bytes < persistent_ws_layout(p).total) return TMM_ERR_NOMEM;
        if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return TMM_ERR_INVALID_ARG;
    }
    if (p->prec == TMM_F64)
        return launch_prec<double, double>(p, cfg, t, ws, R, T, Reduce<double>{nullptr, nullptr, 0}, st);
    if (p->prec == TMM_F32D)
        return launch_prec<float, double>(p, cfg, t, ws, R, T, Reduce<float>{nullptr, nullptr, 0}, st);
    return launch_prec<float, float>(p, cfg, t, ws, R, T, Reduce<float>{nullptr, nullptr, 0}, st);
}

// ---------------------------------------------------------------- reward
// reward[s] = -sum_k partial[s][k], k in tile order (deterministic).
template <typename R>
__global__ void reward_finalize(int S, int n_tiles, const R *__restrict__ partial, R *__restrict__ reward)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    R acc = R(0);
    for (int k = 0; k < n_tiles; ++k) acc += partial[(long long)s * n_tiles + k];
    reward[s] = -acc;
}

tmm_status reward_layout(const tmm_problem *p, const tmm_launch_cfg *cfg, Tile *t, size_t *partial_bytes,
                         size_t *total)
{
    tmm_status s = choose_tile(p, cfg, t);
    if (s != TMM_OK) return s;
    // the block's tree sum reuses the stage memory: one real per thread
    t->smem = std::max(t->smem, (size_t)t->TL * t->TT * real_size(p->prec));
    DeviceInfo di;
    s = device_info(&di);
    if (s != TMM_OK) return s;
    if (t->smem > (size_t)di.max_smem_optin) return TMM_ERR_UNSUPPORTED;
    *partial_bytes = align_up((size_t)p->S * t->n_lt * t->n_tt * real_size(p->prec), 256);
    *total = *partial_bytes + ((cfg && cfg->persistent) ? persistent_ws_layout(p).total : 0);
    return TMM_OK;
}

tmm_status launch_reward(const tmm_problem *p, const tmm_launch_cfg *cfg, const void *R_target, void *reward,
                         void *ws, size_t ws_bytes, cudaStream_t st)
{
    Tile t;
    size_t part = 0, total = 0;
    tmm_status s = reward_layout(p, cfg, &t, &part, &total);
    if (s != TMM_OK) return s;
    if (!ws || ws_bytes < total) return TMM_ERR_NOMEM;
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return TMM_ERR_INVALID_ARG;
    unsigned char *base = static_cast<unsigned char *>(ws);
    const int n_tiles = t.n_lt * t.n_tt;
    if (p->prec == TMM_F64) {
        s = launch_prec<double, double>(p, cfg, t, base + part, nullptr, nullptr,
                                Reduce<double>{static_cast<const double *>(R_target), reinterpret_cast<double *>(base), n_tiles}, st);
        if (s != TMM_OK) return s;
        reward_finalize<double><<<(p->S + 255) / 256, 256, 0, st>>>(p->S, n_tiles, reinterpret_cast<const double *>(base),
                                                                   static_cast<double *>(reward));
    } else {
        s = launch_prec<float, float>(p, cfg, t, base + part, nullptr, nullptr,
                               Reduce<float>{static_cast<const float *>(R_target), reinterpret_cast<float *>(base), n_tiles}, st);
        if (s != TMM_OK) return s;
        reward_finalize<float><<<(p->S + 255) / 256, 256, 0, st>>>(p->S, n_tiles, reinterpret_cast<const float *>(base),
                                                                  static_cast<float *>(reward));
    }
    return check_launch();
}

}  // namespace tmm
