// tmm_abs.cu -- absorbed fraction of the incident power in every layer.
//
// The right-to-left sweep of the forward kernel (Eqs. 1-4, unnormalised
// interfaces, phase divided by e^{Im delta}) passes the left boundary of every
// layer j; there the scaled amplitude pair x (s: E_y amplitudes; p: H_y
// amplitudes, interface admittance k = q / n^2) gives the Poynting flux
//   f_j = Re(k_j (x0 - x1) conj(x0 + x1))
// up to the squared modulus of the scalars dropped so far:
//   |true / scaled|^2 = 2^{LY} / D,  D = prod_{i >= j} 4 |k_i|^2 * 4^{-E},
// LY = sum_{i >= j} 2 Im(delta_i) log2(e), E the power-of-two rescalings.
// With x_0 and D_0, LY_0 after the last interface, the flux normalised by
// the incident flux k_0 |x_0[0]|^2 is
//   F_j = f_j 2^{LY_j - LY_0} (D_0 / D_j) / (k_0 |x_0[0]|^2),
// F_{L+1} = T, F_1 = 1 - R, and the absorbed fraction of layer j is
//   A_j = F_j - F_{j+1}   (flux is continuous across interfaces).
// Each thread keeps its layers' (f_j / mantissa(D_j) with 2^{frac(LY_j)},
// floor(LY_j) - exponent(D_j)) in local memory until the end of the sweep.
#include <cuda_runtime.h>

#include <algorithm>

#include "tmm_device.cuh"
#include "tmm_internal.h"

namespace tmm {

namespace {

constexpr int kAbsThreads = 256;
constexpr int kAbsMaxLayers = 127;

// f_j / mantissa(D_j) 2^{frac(LY_j)} for s and p, and floor(LY_j) - exponent(D_j)
// for s (low 16 bits) and p (high 16 bits).  |LY_j| <= 101 per layer (the
// Im delta clamp) and the exponent of D moves by at most about 60 per layer,
// so with L_max <= 127 both fit 16 bits.  (Records of 3 reals and 2 ints
// made the kernel memory-bound on them.)
template <typename R> struct AbsRec {
    R hs, hp;
    int k;
};

__device__ __forceinline__ int pack_k(int ks, int kp) { return (ks & 0xffff) | (kp << 16); }
__device__ __forceinline__ int k_s(int k) { return (int)(short)(k & 0xffff); }
__device__ __forceinline__ int k_p(int k) { return k >> 16; }

template <typename R> __device__ __forceinline__ R flux(Cx<R> k, Cx<R> x0, Cx<R> x1)
{
    return cmul(k, cmul(x0 - x1, conj(x0 + x1))).x;
}

// D <- D * v (v > 0) kept as mantissa in [1, 2) and exponent
template <typename R> __device__ __forceinline__ void dmul(R &m, int &e, R v)
{
    m *= v;
    renorm_scalar(m, e);
}

template <typename R, int POL, bool WITH_RT, int KMAX>
__global__ void __launch_bounds__(kAbsThreads) tmm_abs_kernel(const tmm_problem p, int TL, int TT, int n_lt, int n_tt,
                                                              R *__restrict__ Aout, R *__restrict__ Rout,
                                                              R *__restrict__ Tout)
{
    extern __shared__ __align__(16) unsigned char smem[];
    StageA<R> *sa = reinterpret_cast<StageA<R> *>(smem);
    StageB<R> *sb = reinterpret_cast<StageB<R> *>(sa + (size_t)(p.L_max + 2) * TL);
    R *n0s = reinterpret_cast<R *>(sb + (size_t)(p.L_max + 2) * TL);

    const long long item = blockIdx.x;
    const int per_stack = n_lt * n_tt;
    const int s = (int)(item / per_stack);
    const int rr = (int)(item - (long long)s * per_stack);
    const int lt = rr / n_tt, ttile = rr % n_tt;
    const int tid = threadIdx.y * TL + threadIdx.x, nthr = TL * TT;
    const int L = layers_of(p, s);
    const int l0 = lt * TL;
    if (L >= 0) fill_stage<R>(p, s, L, l0, TL, sa, sb, n0s, tid, nthr);
    __syncthreads();
    const int tl = threadIdx.x, l = l0 + tl, a_ = ttile * TT + threadIdx.y;
    if (l >= p.n_lambda || a_ >= p.n_theta) return;  // no barrier follows

    const long long tplane = (long long)p.n_theta * p.n_lambda;
    const long long pt = (long long)a_ * p.n_lambda + l;
    const long long lplane = (long long)p.L_max * tplane;        // one (pol, stack) block of A
    const long long Apol = (long long)p.S * lplane;
    const long long RTplane = (long long)p.S * tplane;
    const int nplanes = (POL & 4) ? 1 : ((POL & 1) + ((POL >> 1) & 1));
    auto store_A = [&](int pi, int j, R v) { Aout[pi * Apol + (long long)s * lplane + (long long)j * tplane + pt] = v; };

    R Rv[2] = {nan_w<R>(), nan_w<R>()}, Tv[2] = {nan_w<R>(), nan_w<R>()};
    const R n0 = L >= 0 ? n0s[tl] : nan_w<R>();
    R sth, cth;
    sincos_w(((const R *)p.theta)[a_], &sth, &cth);
    const R beta = n0 * sth, c0 = n0 * cth, q0sq = c0 * c0;
    const bool grazing = beta >= n0;
    if (L < 0 || !(n0 == n0) || grazing) {
        const R fill = grazing ? R(0) : nan_w<R>();
        for (int pi = 0; pi < nplanes; ++pi)
            for (int j = 0; j < p.L_max; ++j) store_A(pi, j, (j < L || L < 0) ? fill : R(0));
        if (grazing) Rv[0] = Rv[1] = R(1), Tv[0] = Tv[1] = R(0);
    } else {
        constexpr int RN = RenormEvery<R>::value;
        const R yi_max = R(kImDeltaMax / kTwoPi);
        const R kLY = R(2.0 * kTwoPi * kLog2e);  // 2 Im(delta) log2(e) per unit of yi
        AbsRec<R> rec[KMAX];
        StageA<R> A = sa[(L + 1) * TL + tl];
        R absz;
        Cx<R> q_nx = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
        Cx<R> g_nx = cmul(q_nx, Cx<R>{A.in2x, A.in2y});
        // exit medium: x = (1, 0), D = 1, LY = 0
        rec[L + 1] = AbsRec<R>{q_nx.x, g_nx.x, 0};
        Cx<R> s0 = {R(1), R(0)}, s1 = {R(0), R(0)}, p0 = s0, p1 = s1;
        R Dsm = R(1), Dpm = R(1), LY = R(0);
        int Dse = 0, Dpe = 0, cnt = 0;
        for (int j = L; j >= 1; --j) {
            A = sa[j * TL + tl];
            const StageB<R> B = sb[j * TL + tl];
            const Cx<R> q = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
            const R yr = B.dl * q.x;
            const R yi = fmin(B.dl * q.y, yi_max);
            LY += kLY * yi;
            R sn, cs;
            sincos_turn(yr - rint_w(yr), &sn, &cs);
            const R E2 = exp_m2_turn(yi);
            const Cx<R> emi = {cs, -sn}, epi = {E2 * cs, E2 * sn};
            const Cx<R> g = cmul(q, Cx<R>{A.in2x, A.in2y});
            if (POL & 1) {
                interface_pair(q, q_nx, s0, s1);
                s0 = cmul(emi, s0);
                s1 = cmul(epi, s1);
                dmul(Dsm, Dse, R(4) * absz);
            }
            if (POL & 2) {
                interface_pair(g, g_nx, p0, p1);
                p0 = cmul(emi, p0);
                p1 = cmul(epi, p1);
                dmul(Dpm, Dpe, R(4) * absz * B.ain2);
            }
            if (++cnt == RN) {
                cnt = 0;
                if (POL & 1) {
                    int k = 0;
                    renorm_pair(s0, s1, k);
                    Dse -= 2 * k;
                }
                if (POL & 2) {
                    int k = 0;
                    renorm_pair(p0, p1, k);
                    Dpe -= 2 * k;
                }
            }
            const R lyf = floor_w(LY);
            const R fr = exp2_w(LY - lyf);
            AbsRec<R> rj;
            rj.hs = (POL & 1) ? flux(q, s0, s1) / Dsm * fr : R(0);
            rj.hp = (POL & 2) ? flux(g, p0, p1) / Dpm * fr : R(0);
            rj.k = pack_k((int)lyf - Dse, (int)lyf - Dpe);
            rec[j] = rj;
            q_nx = q;
            g_nx = g;
        }
        // interface 0 | 1
        A = sa[tl];
        const Cx<R> q0 = {c0, R(0)};
        const Cx<R> g0 = cmul(q0, Cx<R>{A.in2x, A.in2y});
        R pre[2] = {R(0), R(0)};
        int e0[2] = {0, 0};
        if (POL & 1) {
            interface_pair(q0, q_nx, s0, s1);
            dmul(Dsm, Dse, R(4) * c0 * c0);
            const R ax0 = abs2(s0);
            Rv[0] = abs2(s1) / ax0;
            pre[0] = Dsm / (ax0 * q0.x);
            e0[0] = Dse;
        }
        if (POL & 2) {
            interface_pair(g0, g_nx, p0, p1);
            dmul(Dpm, Dpe, R(4) * abs2(g0));
            const R ax0 = abs2(p0);
            Rv[1] = abs2(p1) / ax0;
            pre[1] = Dpm / (ax0 * g0.x);
            e0[1] = Dpe;
        }
        // F_j from the records, then A_j = F_j - F_{j+1} (j = L .. 1):
        // F_j = h_j pre 2^{-LY_0} 2^{floor(LY_j) - e_j + e0}
        const R LYf = floor_w(LY);
        const R sc = exp2_w(LYf - LY);  // 2^{-frac(LY_0)}
        const int kb = -(int)LYf;
        R Fn[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) Fn[k] = R(0);
        for (int j = L + 1; j >= 1; --j) {
            const AbsRec<R> rj = rec[j];
            R F[2] = {R(0), R(0)};
            if (POL & 1) F[0] = ldexp_w(rj.hs * pre[0] * sc, e0[0] + k_s(rj.k) + kb);
            if (POL & 2) F[1] = ldexp_w(rj.hp * pre[1] * sc, e0[1] + k_p(rj.k) + kb);
            if (j == L + 1) {
                Tv[0] = F[0], Tv[1] = F[1];
            } else {
                const R As = F[0] - Fn[0], Ap = F[1] - Fn[1];
                if (POL & 4) {
                    store_A(0, j - 1, R(0.5) * (As + Ap));
                } else {
                    int pi = 0;
                    if (POL & 1) store_A(pi++, j - 1, As);
                    if (POL & 2) store_A(pi, j - 1, Ap);
                }
            }
            Fn[0] = F[0], Fn[1] = F[1];
        }
        for (int pi = 0; pi < nplanes; ++pi)
            for (int j = L; j < p.L_max; ++j) store_A(pi, j, R(0));
    }
    if (WITH_RT) {
        const long long o = (long long)s * tplane + pt;
        if (POL & 4) {
            Rout[o] = R(0.5) * (Rv[0] + Rv[1]);
            if (Tout) Tout[o] = R(0.5) * (Tv[0] + Tv[1]);
        } else {
            int pi = 0;
            if (POL & 1) {
                Rout[pi * RTplane + o] = Rv[0];
                if (Tout) Tout[pi * RTplane + o] = Tv[0];
                ++pi;
            }
            if (POL & 2) {
                Rout[pi * RTplane + o] = Rv[1];
                if (Tout) Tout[pi * RTplane + o] = Tv[1];
            }
        }
    }
}

size_t abs_smem(const tmm_problem *p, int TL)
{
    const size_t r = real_size(p->prec);
    return (size_t)(p->L_max + 2) * TL * (6 * r) + (size_t)TL * r;
}

template <typename R, int POL, bool WITH_RT, int KMAX>
tmm_status launch_abs_k(const tmm_problem *p, int TL, int TT, int n_lt, int n_tt, long long items, size_t smem,
                        R *A, R *Ro, R *To, cudaStream_t st)
{
    auto k = tmm_abs_kernel<R, POL, WITH_RT, KMAX>;
    {
        const tmm_status ss = ensure_dynamic_smem(reinterpret_cast<const void *>(k), smem);
        if (ss != TMM_OK) return ss;
    }
    k<<<(unsigned)items, dim3(TL, TT), smem, st>>>(*p, TL, TT, n_lt, n_tt, A, Ro, To);
    return check_launch();
}

template <typename R, int POL, bool WITH_RT>
tmm_status launch_abs_km(const tmm_problem *p, int TL, int TT, int n_lt, int n_tt, long long items, size_t smem,
                         R *A, R *Ro, R *To, cudaStream_t st)
{
    const int need = p->L_max + 2;
    if (need <= 18) return launch_abs_k<R, POL, WITH_RT, 18>(p, TL, TT, n_lt, n_tt, items, smem, A, Ro, To, st);
    if (need <= 34) return launch_abs_k<R, POL, WITH_RT, 34>(p, TL, TT, n_lt, n_tt, items, smem, A, Ro, To, st);
    if (need <= 66) return launch_abs_k<R, POL, WITH_RT, 66>(p, TL, TT, n_lt, n_tt, items, smem, A, Ro, To, st);
    return launch_abs_k<R, POL, WITH_RT, kAbsMaxLayers + 2>(p, TL, TT, n_lt, n_tt, items, smem, A, Ro, To, st);
}

template <typename R>
tmm_status launch_abs_prec(const tmm_problem *p, int TL, int TT, int n_lt, int n_tt, long long items, size_t smem,
                           void *A_, void *R_, void *T_, cudaStream_t st)
{
    R *A = static_cast<R *>(A_), *Ro = static_cast<R *>(R_), *To = static_cast<R *>(T_);
    const bool rt = Ro != nullptr;
#define TMM_ABS_CASE(P_)                                                                            \
    case P_:                                                                                        \
        return rt ? launch_abs_km<R, P_, true>(p, TL, TT, n_lt, n_tt, items, smem, A, Ro, To, st)   \
                  : launch_abs_km<R, P_, false>(p, TL, TT, n_lt, n_tt, items, smem, A, Ro, To, st);
    switch (p->pol_mask) {
        TMM_ABS_CASE(1)
        TMM_ABS_CASE(2)
        TMM_ABS_CASE(3)
        TMM_ABS_CASE(7)
    default: return TMM_ERR_INVALID_ARG;
    }
#undef TMM_ABS_CASE
}

}  // namespace

}  // namespace tmm

using namespace tmm;

extern "C" TMM_API tmm_status tmm_absorption_batched(const tmm_problem *p, void *A, void *R, void *T, void *stream)
{
    TraceRange trace("tmm_absorption_batched");
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if (p->prec != TMM_F64 && p->prec != TMM_F32) return TMM_ERR_UNSUPPORTED;
    if (p->L_max > kAbsMaxLayers) return TMM_ERR_UNSUPPORTED;
    const long long pts = (long long)p->S * p->n_lambda * p->n_theta;
    if (pts == 0) return TMM_OK;
    if (!A || (T && !R)) return TMM_ERR_INVALID_ARG;
    DeviceInfo di;
    s = device_info(&di);
    if (s != TMM_OK) return s;
    const int TT = std::min(p->n_theta, 32);
    int TL = 1;
    while (TL * TT * 2 <= kAbsThreads) TL *= 2;
    while (TL > 1 && TL / 2 >= p->n_lambda) TL /= 2;
    while (TL > 1 && abs_smem(p, TL) > (size_t)di.max_smem_optin) TL /= 2;
    const size_t smem = abs_smem(p, TL);
    if (smem > (size_t)di.max_smem_optin) return TMM_ERR_UNSUPPORTED;
    const int n_lt = (p->n_lambda + TL - 1) / TL, n_tt = (p->n_theta + TT - 1) / TT;
    const long long items = (long long)p->S * n_lt * n_tt;
    if (items > 0x7fffffffLL) return TMM_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return p->prec == TMM_F64 ? launch_abs_prec<double>(p, TL, TT, n_lt, n_tt, items, smem, A, R, T, st)
                              : launch_abs_prec<float>(p, TL, TT, n_lt, n_tt, items, smem, A, R, T, st);
}
