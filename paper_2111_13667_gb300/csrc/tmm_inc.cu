// tmm_inc.cu -- stacks with incoherent (thick) layers.
//
// The media 0 and L_s+1 and every flagged finite layer are incoherent; the
// coherent blocks between consecutive incoherent media a < b are evaluated
// as amplitude products (Eqs. 1-4, the forward kernel's scaled right-to-left
// sweep, here with both columns of the block matrix M), and the blocks are
// combined by intensities.  Per block and polarisation:
//   R_f = |M10 / M00|^2 (light from a),  R_b = |M01 / M00|^2 (light from b),
//   T_f from M00 and the carried scales exactly as the forward kernel's T
//   (Eqs. 5-6 with the Poynting factors), and T_b = T_f (transmittance of a
//   stack between non-absorbing media is reciprocal).
// With (P, M) the forward and backward intensities on the left of the blocks
// done so far, scaled by the product t of their T_f,
//   P' = P - R_b M,   M' = R_f P' + T_f T_b M,   t' = t T_f
// from (1, 0, 1) in the exit medium; R = M / P and T = t / P in medium 0.
// Incoherent layers must be non-absorbing (else the point's outputs are NaN);
// the first incoherent layer in which the wave is evanescent ends the stack:
// it is the exit medium and T = 0.
#include <cuda_runtime.h>

#include <algorithm>

#include "tmm_device.cuh"
#include "tmm_internal.h"

namespace tmm {

namespace {

constexpr int kIncThreads = 256;

// Both columns of one block's scaled matrix for one polarisation.
template <typename R> struct Cols {
    Cx<R> x0, x1, y0, y1;
};

template <typename R> __device__ __forceinline__ void renorm_cols(Cols<R> &c, int &e)
{
    const R m = fmax(fmax(fmax(fabs(c.x0.x), fabs(c.x0.y)), fmax(fabs(c.x1.x), fabs(c.x1.y))),
                     fmax(fmax(fabs(c.y0.x), fabs(c.y0.y)), fmax(fabs(c.y1.x), fabs(c.y1.y))));
    const int k = exponent_of(m);
    const R s = pow2_neg<R>(k);
    c.x0 = scale(s, c.x0), c.x1 = scale(s, c.x1), c.y0 = scale(s, c.y0), c.y1 = scale(s, c.y1);
    e += k;
}

template <typename R> __device__ __forceinline__ void phase_cols(Cols<R> &c, Cx<R> emi, Cx<R> epi)
{
    c.x0 = cmul(emi, c.x0), c.x1 = cmul(epi, c.x1);
    c.y0 = cmul(emi, c.y0), c.y1 = cmul(epi, c.y1);
}

// R_f, R_b, T_f of the coherent block between incoherent media a < b, for the
// polarisations in POL ([0] s, [1] p).  q_a (> 0) and n_a^2 are real; a = 0
// takes q_0 = n_0 cos(theta) directly.
template <typename R, int POL>
__device__ __forceinline__ void block_coeffs(const StageA<R> *__restrict__ sa, const StageB<R> *__restrict__ sb,
                                             int TL, int tl, int a, int b, R q0sq, R qa, R n0, R Rf[2], R Rb[2],
                                             R Tf[2])
{
    constexpr int RN = RenormEvery<R>::value;
    const R yi_max = R(kImDeltaMax / kTwoPi);
    StageA<R> A = sa[b * TL + tl];
    R absz;
    Cx<R> q_nx = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
    const Cx<R> q_b = q_nx, n2_b = {A.d2x + n0 * n0, A.n2y};
    Cx<R> g_nx = cmul(q_nx, Cx<R>{A.in2x, A.in2y});
    R Pp = sb[b * TL + tl].ain2;
    int ePp = 0;
    R Ps = R(1), Y = R(0);
    int eP = 0, es = 0, ep = 0;
    const Cx<R> one = {R(1), R(0)}, zero = {R(0), R(0)};
    Cols<R> cs{one, zero, zero, one}, cp{one, zero, zero, one};
    int cnt = 0;
    for (int j = b - 1; j > a; --j) {
        A = sa[j * TL + tl];
        const StageB<R> B = sb[j * TL + tl];
        const Cx<R> q = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
        Ps *= absz;
        const R yr = B.dl * q.x;
        const R yi = fmin(B.dl * q.y, yi_max);
        Y += yi;
        R sn, cs_;
        sincos_turn(yr - rint_w(yr), &sn, &cs_);
        const R E2 = exp_m2_turn(yi);
        const Cx<R> emi = {cs_, -sn}, epi = {E2 * cs_, E2 * sn};
        if (POL & 1) {
            interface_pair(q, q_nx, cs.x0, cs.x1);
            interface_pair(q, q_nx, cs.y0, cs.y1);
            phase_cols(cs, emi, epi);
        }
        if (POL & 2) {
            Pp *= B.ain2;
            const Cx<R> g = cmul(q, Cx<R>{A.in2x, A.in2y});
            interface_pair(g, g_nx, cp.x0, cp.x1);
            interface_pair(g, g_nx, cp.y0, cp.y1);
            phase_cols(cp, emi, epi);
            g_nx = g;
        }
        q_nx = q;
        if (++cnt == RN) {
            cnt = 0;
            renorm_scalar(Ps, eP);
            if (POL & 2) renorm_scalar(Pp, ePp);
            if (POL & 1) renorm_cols(cs, es);
            if (POL & 2) renorm_cols(cp, ep);
        }
    }
    // interface a | a+1; medium a is real
    A = sa[a * TL + tl];
    const Cx<R> q_a = {qa, R(0)};
    Ps *= qa * qa;
    const int e4 = 2 * (b - a);
    R u = R(-2.0 * kTwoPi * kLog2e) * Y;
    u = fmax(u, R(-1.0e6));
    const R un = floor_w(u);
    const R yscale = exp2_w(u - un);
    const int yn = (int)un;
    if (POL & 1) {
        interface_pair(q_a, q_nx, cs.x0, cs.x1);
        interface_pair(q_a, q_nx, cs.y0, cs.y1);
        const R ax0 = abs2(cs.x0);
        Rf[0] = abs2(cs.x1) / ax0;
        Rb[0] = abs2(cs.y0) / ax0;
        Tf[0] = q_b.x / qa * ldexp_w(Ps * yscale / ax0, e4 + eP + yn - 2 * es);
    }
    if (POL & 2) {
        const R na2 = A.d2x + n0 * n0;
        const Cx<R> g_a = cmul(q_a, Cx<R>{A.in2x, A.in2y});
        interface_pair(g_a, g_nx, cp.x0, cp.x1);
        interface_pair(g_a, g_nx, cp.y0, cp.y1);
        const R ax0 = abs2(cp.x0);
        Rf[1] = abs2(cp.x1) / ax0;
        Rb[1] = abs2(cp.y0) / ax0;
        const R num = cmul(n2_b, conj(q_b)).x;
        Tf[1] = num / (na2 * qa) * ldexp_w(Ps * Pp * yscale / ax0, e4 + eP + ePp + yn - 2 * ep);
    }
}

template <typename R, int POL, bool WITH_T>
__global__ void __launch_bounds__(kIncThreads) tmm_inc_kernel(const tmm_problem p, const uint8_t *__restrict__ inc,
                                                              int TL, int TT, int n_lt, int n_tt,
                                                              R *__restrict__ Rout, R *__restrict__ Tout)
{
    extern __shared__ __align__(16) unsigned char smem[];
    StageA<R> *sa = reinterpret_cast<StageA<R> *>(smem);
    StageB<R> *sb = reinterpret_cast<StageB<R> *>(sa + (size_t)(p.L_max + 2) * TL);
    R *n0s = reinterpret_cast<R *>(sb + (size_t)(p.L_max + 2) * TL);
    unsigned char *flg = reinterpret_cast<unsigned char *>(n0s + TL);  // [L_max + 2]

    const long long item = blockIdx.x;
    const int per_stack = n_lt * n_tt;
    const int s = (int)(item / per_stack);
    const int rr = (int)(item - (long long)s * per_stack);
    const int lt = rr / n_tt, ttile = rr % n_tt;
    const int tid = threadIdx.y * TL + threadIdx.x, nthr = TL * TT;
    const int L = layers_of(p, s);
    const int l0 = lt * TL;
    if (L >= 0) {
        fill_stage<R>(p, s, L, l0, TL, sa, sb, n0s, tid, nthr);
        for (int j = tid; j < L + 2; j += nthr)
            flg[j] = (j == 0 || j == L + 1) ? 1 : (inc && inc[(long long)s * p.L_max + (j - 1)] ? 1 : 0);
    }
    __syncthreads();

    const int tl = threadIdx.x, l = l0 + tl, a_ = ttile * TT + threadIdx.y;
    if (l >= p.n_lambda || a_ >= p.n_theta) return;  // no barrier follows
    R Rv[2] = {nan_w<R>(), nan_w<R>()}, Tv[2] = {nan_w<R>(), nan_w<R>()};
    bool ok = L >= 0;
    if (ok)
        for (int j = 1; j <= L; ++j)
            if (flg[j] && sa[j * TL + tl].n2y != R(0)) ok = false;  // absorbing incoherent layer
    if (ok) {
        R sth, cth;
        sincos_w(((const R *)p.theta)[a_], &sth, &cth);
        const R n0 = n0s[tl];
        const R beta = n0 * sth, c0 = n0 * cth, q0sq = c0 * c0;
        if (beta >= n0) {  // grazing (false for a NaN n_0)
            Rv[0] = Rv[1] = R(1);
            Tv[0] = Tv[1] = R(0);
        } else if (n0 == n0) {
            // the first evanescent incoherent layer ends the stack
            int e = L + 1;
            bool cut = false;
            for (int j = 1; j <= L; ++j)
                if (flg[j] && sa[j * TL + tl].d2x + q0sq <= R(0)) {
                    e = j;
                    cut = true;
                    break;
                }
            R P[2] = {R(1), R(1)}, M[2] = {R(0), R(0)}, t[2] = {R(1), R(1)};
            int b = e;
            while (b > 0) {
                int a = b - 1;
                while (a > 0 && !flg[a]) --a;
                const R qa = a == 0 ? c0 : sqrt(sa[a * TL + tl].d2x + q0sq);
                R Rf[2] = {R(0), R(0)}, Rb[2] = {R(0), R(0)}, Tf[2] = {R(0), R(0)};
                block_coeffs<R, POL>(sa, sb, TL, tl, a, b, q0sq, qa, n0, Rf, Rb, Tf);
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (!(POL & (1 << k))) continue;
                    const R P1 = P[k] - Rb[k] * M[k];
                    const R M1 = Rf[k] * P1 + Tf[k] * Tf[k] * M[k];
                    const R inv = R(1) / P1;  // keep P = 1
                    P[k] = R(1);
                    M[k] = M1 * inv;
                    t[k] = t[k] * Tf[k] * inv;
                }
                b = a;
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                Rv[k] = M[k];
                Tv[k] = cut ? R(0) : t[k];
            }
        }
    }
    const long long plane = (long long)p.S * p.n_theta * p.n_lambda;
    const long long o = ((long long)s * p.n_theta + a_) * p.n_lambda + l;
    if (POL & 4) {
        Rout[o] = R(0.5) * (Rv[0] + Rv[1]);
        if (WITH_T) Tout[o] = R(0.5) * (Tv[0] + Tv[1]);
    } else {
        int pi = 0;
        if (POL & 1) {
            Rout[o] = Rv[0];
            if (WITH_T) Tout[o] = Tv[0];
            ++pi;
        }
        if (POL & 2) {
            Rout[pi * plane + o] = Rv[1];
            if (WITH_T) Tout[pi * plane + o] = Tv[1];
        }
    }
}

size_t inc_smem(const tmm_problem *p, int TL)
{
    const size_t r = real_size(p->prec);
    return (size_t)(p->L_max + 2) * TL * (6 * r) + (size_t)TL * r + (size_t)(p->L_max + 2) + 16;
}

template <typename R, int POL, bool WITH_T>
tmm_status launch_inc_typed(const tmm_problem *p, const uint8_t *inc, int TL, int TT, int n_lt, int n_tt,
                            long long items, size_t smem, R *Ro, R *To, cudaStream_t st)
{
    auto k = tmm_inc_kernel<R, POL, WITH_T>;
    if (smem > 48 * 1024) {
        // once per (instantiation, device) and size: repeated launches and graph
        // capture stay free of attribute calls
        static int set_bytes[64] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_fail(e);
        if (dev < 0 || dev >= 64) return TMM_ERR_UNSUPPORTED;
        if (set_bytes[dev] < (int)smem) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return cuda_fail(e);
            set_bytes[dev] = (int)smem;
        }
    }
    k<<<(unsigned)items, dim3(TL, TT), smem, st>>>(*p, inc, TL, TT, n_lt, n_tt, Ro, To);
    return check_launch();
}

template <typename R>
tmm_status launch_inc_prec(const tmm_problem *p, const uint8_t *inc, int TL, int TT, int n_lt, int n_tt,
                           long long items, size_t smem, void *R_, void *T_, cudaStream_t st)
{
    R *Ro = static_cast<R *>(R_), *To = static_cast<R *>(T_);
    const bool wt = To != nullptr;
#define TMM_INC_CASE(P_)                                                                                   \
    case P_:                                                                                               \
        return wt ? launch_inc_typed<R, P_, true>(p, inc, TL, TT, n_lt, n_tt, items, smem, Ro, To, st)    \
                  : launch_inc_typed<R, P_, false>(p, inc, TL, TT, n_lt, n_tt, items, smem, Ro, To, st);
    switch (p->pol_mask) {
        TMM_INC_CASE(1)
        TMM_INC_CASE(2)
        TMM_INC_CASE(3)
        TMM_INC_CASE(7)
    default: return TMM_ERR_INVALID_ARG;
    }
#undef TMM_INC_CASE
}

}  // namespace

}  // namespace tmm

using namespace tmm;

extern "C" TMM_API tmm_status tmm_inc_batched(const tmm_problem *p, const uint8_t *incoherent, void *R, void *T,
                                              void *stream)
{
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if (p->prec == TMM_F64X) return TMM_ERR_UNSUPPORTED;
    const long long pts = (long long)p->S * p->n_lambda * p->n_theta;
    if (pts == 0) return TMM_OK;
    if (!R) return TMM_ERR_INVALID_ARG;
    DeviceInfo di;
    s = device_info(&di);
    if (s != TMM_OK) return s;
    const int TT = std::min(p->n_theta, 32);
    int TL = 1;
    while (TL * TT * 2 <= kIncThreads) TL *= 2;
    while (TL > 1 && TL / 2 >= p->n_lambda) TL /= 2;
    while (TL > 1 && inc_smem(p, TL) > (size_t)di.max_smem_optin) TL /= 2;
    const size_t smem = inc_smem(p, TL);
    if (smem > (size_t)di.max_smem_optin) return TMM_ERR_UNSUPPORTED;
    const int n_lt = (p->n_lambda + TL - 1) / TL, n_tt = (p->n_theta + TT - 1) / TT;
    const long long items = (long long)p->S * n_lt * n_tt;
    if (items > 0x7fffffffLL) return TMM_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return p->prec == TMM_F64 ? launch_inc_prec<double>(p, incoherent, TL, TT, n_lt, n_tt, items, smem, R, T, st)
                              : launch_inc_prec<float>(p, incoherent, TL, TT, n_lt, n_tt, items, smem, R, T, st);
}
