// tmm_grad.cu -- adjoint (reverse-sweep) gradient of the per-stack merit
//   m_s = mean over (pol, theta, lambda) of (R - R_target)^2
// with respect to every thickness d_j and a real index offset Delta n_j.
// It replaces the autograd route of the paper's TMM-Torch (Sec. 4).
//
// Per (stack, lambda, theta) thread, both polarisations:
//   1. the forward sweep of the forward kernel (right to left,
//      x_j = P_j F_j x_{j+1}), keeping every x_j (rescaled, with its power-of-two
//      exponent) in thread-local storage;
//   2. the cotangent of R at x_0, weighted by 2 (R - R_t) / N:
//      dR = 2 Re(g . dx_0), g = (-R / x_0[0], conj(x_0[1]) / |x_0[0]|^2);
//   3. a left-to-right sweep of the row cotangent w_{j+1} = w_j P_j F_j.  For
//      layer j it adds
//        d_j:       2 Re(D_j d(delta_j)/d(d_j)),  D_j = i (w_j[1] x_j[1] - w_j[0] x_j[0])
//        n_j:       2 Re(D_j d(delta_j)/d(n_j))
//                 + 2 Re((w_j P_j)[0] + (w_j P_j)[1]) (x_{j+1}[0] + x_{j+1}[1]) da_j/dn_j)
//                 + 2 Re(((w_{j-1} P_{j-1})[0] - (w_{j-1} P_{j-1})[1]) (x_j[0] - x_j[1]) da_j/dn_j)
//      where F_j = [[a_j + a_{j+1}, a_j - a_{j+1}], [a_j - a_{j+1}, a_j + a_{j+1}]],
//      a = q = n cos(theta) for s and a = q / n^2 for p.  (R does not depend
//      on the dropped interface scale factors, so they need no derivative.)
//   4. per layer, a warp-shuffle sum over the warp's 32 points, added by lane 0
//      into a per-warp row of shared memory; rows are summed in a fixed order
//      at the end, so results are bit-reproducible.
// With a workspace the (lambda, theta) tiles of a stack are split over G blocks
// whose partial sums a second kernel adds in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>

#include "tmm_device.cuh"
#include "tmm_internal.h"

namespace tmm {

constexpr int kGradThreads = 256;
constexpr int kGradMaxLayers = 127;  // L_max + 2 <= 129 media

// Stored right-sweep state of one layer (both polarisations).
// The pairs' exponents share one int, s in the low and p in the high 16
// bits: they move by the rescalings only (at most about 63 per two layers),
// so L_max <= 127 keeps them within 16 bits; 36 bytes per layer in FP32.
template <typename R> struct XState {
    Cx<R> s0, s1, p0, p1;
    int e;
    __device__ int es() const { return (int)(short)(e & 0xffff); }
    __device__ int ep() const { return e >> 16; }
};
__device__ __forceinline__ int pack_e(int es, int ep) { return (es & 0xffff) | (ep << 16); }

template <typename R> __device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 2^e built from the exponent bits (0 below the normal range, which only
// happens for the masked lanes whose contributions are discarded).
__device__ __forceinline__ float pow2_bits(int e, float)
{
    return e < -126 ? 0.0f : __int_as_float(min(e, 127) + 127 << 23);
}
__device__ __forceinline__ double pow2_bits(int e, double)
{
    return e < -1022 ? 0.0 : __longlong_as_double((long long)(min(e, 1023) + 1023) << 52);
}
template <typename R> __device__ __forceinline__ R pow2_w(int e) { return pow2_bits(e, R(0)); }

// Per-medium quantities of one point: root q, a_s = q, a_p = q / n^2 and
// their derivatives with respect to n (dq/dn = n / q, da_p/dn = (1/n)(1/q - 2 q / n^2)).
template <typename R> struct Medium {
    Cx<R> q, ap, dq, dap;
    R absz;
};

template <typename R>
__device__ __forceinline__ Medium<R> medium_at(const StageA<R> &A, Cx<R> n, R q0sq, bool derivs)
{
    Medium<R> m;
    m.q = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &m.absz);
    const Cx<R> in2 = {A.in2x, A.in2y};
    m.ap = cmul(m.q, in2);
    if (derivs) {
        const R iz = R(1) / m.absz;
        const Cx<R> iq = {m.q.x * iz, -m.q.y * iz};  // 1 / q
        m.dq = cmul(n, iq);
        const Cx<R> inv_n = cmul(n, in2);              // 1 / n
        m.dap = cmul(inv_n, iq - scale(R(2), cmul(m.q, in2)));
    } else {
        m.dq = m.dap = Cx<R>{R(0), R(0)};
    }
    return m;
}

// Fill the grad stage (forward stage plus n itself) for one tile.
template <typename R>
__device__ __forceinline__ void fill_stage_grad(const tmm_problem &p, int s, int L, int l0, int TL, StageA<R> *sa,
                                                StageB<R> *sb, Cx<R> *sn, R *n0, int tid, int nthr)
{
    fill_stage<R>(p, s, L, l0, TL, sa, sb, n0, tid, nthr);
    const int total = (L + 2) * TL;
    for (int idx = tid; idx < total; idx += nthr) {
        const int j = idx / TL, tl = idx - j * TL;
        const int l = min(l0 + tl, p.n_lambda - 1);
        sn[idx] = index_of<R>(p, s, j, l);
    }
}

// Resident blocks per SM the FP32 instance is compiled for: the kernel is
// latency-bound (thread-local states, two warp sums per layer), and capping
// registers at 64 for four 256-thread blocks per SM beats two blocks at 111
// registers (measured 18 % faster, same results); the FP64 instance is held to
// two blocks (128 registers).
template <typename R> struct GradMinBlocks { static constexpr int value = 2; };
template <> struct GradMinBlocks<float> { static constexpr int value = 4; };

// WITH_DN = false (dm_dn not requested, as in the thickness optimiser) leaves
// out the index terms: the root derivatives, three products per polarisation
// and one warp sum per layer.
template <typename R, int KMAX, bool WITH_DN>
__global__ void __launch_bounds__(kGradThreads, GradMinBlocks<R>::value) tmm_grad_kernel(const tmm_problem p, const R *__restrict__ Rt,
                                                                int TL, int TT, int n_lt, int n_tt, int G, R inv_N,
                                                                R *__restrict__ merit, R *__restrict__ dm_dd,
                                                                R *__restrict__ dm_dn, R *__restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int Lm2 = p.L_max + 2;
    StageA<R> *sa = reinterpret_cast<StageA<R> *>(smem);
    StageB<R> *sb = reinterpret_cast<StageB<R> *>(sa + (size_t)Lm2 * TL);
    Cx<R> *sn = reinterpret_cast<Cx<R> *>(sb + (size_t)Lm2 * TL);
    R *n0s = reinterpret_cast<R *>(sn + (size_t)Lm2 * TL);
    R *acc = n0s + TL;  // [nwarps][NP]

    const int NP = 2 * p.L_max + 1;  // dd_1..dd_L, dn_1..dn_L, merit
    const int s = blockIdx.x / G, gidx = blockIdx.x - s * G;
    const int nthr = TL * TT, tid = threadIdx.x;
    const int nwarps = nthr >> 5, warp = tid >> 5, lane = tid & 31;
    const int tl = tid % TL, tt = tid / TL;
    const int L = layers_of(p, s);
    const bool do_s = p.pol_mask & 1u, do_p = p.pol_mask & 2u;
    const int P = (do_s ? 1 : 0) + (do_p ? 1 : 0);
    const R yi_max = R(kImDeltaMax / kTwoPi);
    const R *lam = (const R *)p.lambda;
    const R *th = (const R *)p.theta;

    for (int i = tid; i < nwarps * NP; i += nthr) acc[i] = R(0);

    XState<R> X[KMAX];

    for (int t = gidx; t < n_lt * n_tt && L >= 0; t += G) {
        const int lt = t / n_tt, ttile = t - lt * n_tt;
        __syncthreads();  // the previous tile's stage is no longer read
        fill_stage_grad<R>(p, s, L, lt * TL, TL, sa, sb, sn, n0s, tid, nthr);
        __syncthreads();

        const int l = lt * TL + tl, a = ttile * TT + tt;
        const bool active = l < p.n_lambda && a < p.n_theta;
        const int lc = min(l, p.n_lambda - 1), ac = min(a, p.n_theta - 1);
        R sth, cth;
        sincos_w(th[ac], &sth, &cth);
        const R beta = n0s[tl] * sth;
        const R q0sq = (n0s[tl] * cth) * (n0s[tl] * cth);
        const R two_pi_inv_lam = R(kTwoPi) / lam[lc];

        // ---- 1. right-to-left sweep, storing x_j (j = L+1 .. 1)
        Medium<R> nx = medium_at(sa[(L + 1) * TL + tl], sn[(L + 1) * TL + tl], q0sq, false);
        Cx<R> s0 = {R(1), R(0)}, s1 = {R(0), R(0)}, p0 = s0, p1 = s1;
        int es = 0, ep = 0;
        X[L + 1] = XState<R>{s0, s1, p0, p1, 0};
        // The phase matrix is applied divided by its real factor e^{Im delta}
        // (one exponential per layer).  Stored states and, below, the row
        // cotangents then carry inverse scales, so every gradient term --
        // always a cotangent times a state -- is unchanged.
        for (int j = L; j >= 1; --j) {
            const StageA<R> A = sa[j * TL + tl];
            const StageB<R> B = sb[j * TL + tl];
            const Medium<R> m = medium_at(A, sn[j * TL + tl], q0sq, false);
            const R yr = B.dl * m.q.x, yi = fmin(B.dl * m.q.y, yi_max);
            R sn_, cs;
            sincos_turn(yr - rint_w(yr), &sn_, &cs);
            const R E2 = exp_m2_turn(yi);
            const Cx<R> emi = {cs, -sn_}, epi = {E2 * cs, E2 * sn_};
            const bool rn = ((L - j) & 1) == 1;
            if (do_s) {
                interface_pair(m.q, nx.q, s0, s1);
                s0 = cmul(emi, s0);
                s1 = cmul(epi, s1);
                if (rn) renorm_pair(s0, s1, es);
            }
            if (do_p) {
                interface_pair(m.ap, nx.ap, p0, p1);
                p0 = cmul(emi, p0);
                p1 = cmul(epi, p1);
                if (rn) renorm_pair(p0, p1, ep);
            }
            X[j] = XState<R>{s0, s1, p0, p1, pack_e(es, ep)};
            nx = m;
        }
        // interface 0 -> 1 and the cotangent of R at x_0
        // injection medium (real n_0): q_0 = n_0 cos(theta), computed directly
        Medium<R> cur;
        cur.q = Cx<R>{n0s[tl] * cth, R(0)};
        cur.ap = cmul(cur.q, Cx<R>{sa[tl].in2x, sa[tl].in2y});
        cur.dq = cur.dap = Cx<R>{R(0), R(0)};
        cur.absz = cur.q.x * cur.q.x;
        const bool grazing = beta >= n0s[tl];
        const int pbase = 0;
        R mer = R(0);
        Cx<R> ws0 = {R(0), R(0)}, ws1 = ws0, wp0 = ws0, wp1 = ws0;
        int ews = 0, ewp = 0;
        {
            int pi = 0;
            if (do_s) {
                Cx<R> x0 = s0, x1 = s1;
                interface_pair(cur.q, nx.q, x0, x1);
                const R ia = R(1) / abs2(x0);
                const R Rv = grazing ? R(1) : abs2(x1) * ia;
                const R e = Rv - Rt[((long long)pi * p.n_theta + ac) * p.n_lambda + lc];
                mer += e * e;
                const R c = (active && !grazing) ? R(2) * e * inv_N : R(0);
                ws0 = scale(-c * Rv * ia, conj(x0));
                ws1 = scale(c * ia, conj(x1));
                ews = -es;
                renorm_pair(ws0, ws1, ews);
                ++pi;
            }
            if (do_p) {
                Cx<R> x0 = p0, x1 = p1;
                interface_pair(cur.ap, nx.ap, x0, x1);
                const R ia = R(1) / abs2(x0);
                const R Rv = grazing ? R(1) : abs2(x1) * ia;
                const R e = Rv - Rt[((long long)pi * p.n_theta + ac) * p.n_lambda + lc];
                mer += e * e;
                const R c = (active && !grazing) ? R(2) * e * inv_N : R(0);
                wp0 = scale(-c * Rv * ia, conj(x0));
                wp1 = scale(c * ia, conj(x1));
                ewp = -ep;
                renorm_pair(wp0, wp1, ewp);
            }
        }
        (void)pbase;
        mer = active ? mer * inv_N : R(0);
        mer = warp_sum(mer);
        if (lane == 0) acc[warp * NP + NP - 1] += mer;

        // ---- 3. left-to-right cotangent sweep
        // cur = medium j, nx = medium j+1 (with n-derivatives when it is a layer)
        nx = medium_at(sa[1 * TL + tl], sn[1 * TL + tl], q0sq, WITH_DN && L >= 1);
        R dn_carry = R(0);  // right-side F term for layer j+1, from step j
        XState<R> Xc = X[1];  // the state of the current layer (x_j); unused at j = 0
        for (int j = 0; j <= L; ++j) {
            const XState<R> Xn = X[j + 1];
            R dd = R(0), dn = dn_carry;
            dn_carry = R(0);
            Cx<R> emi = {R(1), R(0)}, epi = {R(1), R(0)};
            Cx<R> ddel_d = {R(0), R(0)}, ddel_n = {R(0), R(0)};
            if (j >= 1) {
                const StageB<R> B = sb[j * TL + tl];
                const R yr = B.dl * cur.q.x, yi_raw = B.dl * cur.q.y;
                const bool clamped = yi_raw > yi_max;
                R sn_, cs;
                sincos_turn(yr - rint_w(yr), &sn_, &cs);
                const R E2 = exp_m2_turn(fmin(yi_raw, yi_max));
                emi = Cx<R>{cs, -sn_};
                epi = Cx<R>{E2 * cs, E2 * sn_};
                // d delta / d d = 2 pi q / lambda; d delta / d n = 2 pi (d/lambda) n / q
                ddel_d = scale(two_pi_inv_lam, cur.q);
                if (WITH_DN) ddel_n = scale(R(kTwoPi) * B.dl, cur.dq);
                if (clamped) {
                    ddel_d.y = R(0);
                    ddel_n.y = R(0);
                }
            }
            const bool rn = (j & 1) == 1;
            // s polarisation
            if (do_s) {
                const Cx<R> v0 = cmul(ws0, emi), v1 = cmul(ws1, epi);
                const R sc_b = pow2_w<R>(ews + Xn.es());
                if (j >= 1) {
                    const R sc_a = pow2_w<R>(ews + Xc.es());
                    const Cx<R> D = mul_i(cmul(ws1, Xc.s1) - cmul(ws0, Xc.s0));
                    dd += R(2) * cmul(D, ddel_d).x * sc_a;
                    if (WITH_DN) {
                        dn += R(2) * cmul(D, ddel_n).x * sc_a;
                        dn += R(2) * cmul(cmul(v0 + v1, Xn.s0 + Xn.s1), cur.dq).x * sc_b;
                    }
                }
                if (WITH_DN && j + 1 <= L)
                    dn_carry += R(2) * cmul(cmul(v0 - v1, Xn.s0 - Xn.s1), nx.dq).x * sc_b;
                // (ws0, ws1) <- (v0 a + v1 b, v0 b + v1 a), a, b = q_j +- q_{j+1}
                ws0 = v0, ws1 = v1;
                interface_pair(cur.q, nx.q, ws0, ws1);
                if (rn) renorm_pair(ws0, ws1, ews);
            }
            if (do_p) {
                const Cx<R> v0 = cmul(wp0, emi), v1 = cmul(wp1, epi);
                const R sc_b = pow2_w<R>(ewp + Xn.ep());
                if (j >= 1) {
                    const R sc_a = pow2_w<R>(ewp + Xc.ep());
                    const Cx<R> D = mul_i(cmul(wp1, Xc.p1) - cmul(wp0, Xc.p0));
                    dd += R(2) * cmul(D, ddel_d).x * sc_a;
                    if (WITH_DN) {
                        dn += R(2) * cmul(D, ddel_n).x * sc_a;
                        dn += R(2) * cmul(cmul(v0 + v1, Xn.p0 + Xn.p1), cur.dap).x * sc_b;
                    }
                }
                if (WITH_DN && j + 1 <= L)
                    dn_carry += R(2) * cmul(cmul(v0 - v1, Xn.p0 - Xn.p1), nx.dap).x * sc_b;
                wp0 = v0, wp1 = v1;
                interface_pair(cur.ap, nx.ap, wp0, wp1);
                if (rn) renorm_pair(wp0, wp1, ewp);
            }
            if (j >= 1) {
                dd = warp_sum(active ? dd : R(0));
                if (WITH_DN) dn = warp_sum(active ? dn : R(0));
                if (lane == 0) {
                    acc[warp * NP + (j - 1)] += dd;
                    if (WITH_DN) acc[warp * NP + p.L_max + (j - 1)] += dn;
                }
            }
            if (j + 1 <= L) {
                cur = nx;
                const int jn = j + 2;
                nx = medium_at(sa[jn * TL + tl], sn[jn * TL + tl], q0sq, WITH_DN && jn <= L);
            }
            Xc = Xn;
        }
        (void)P;
    }
    __syncthreads();

    // fixed-order sum of the warp rows
    for (int k = tid; k < NP; k += nthr) {
        R v = R(0);
        if (L < 0) {
            v = nan_w<R>();
        } else {
            for (int w = 0; w < nwarps; ++w) v += acc[w * NP + k];
        }
        if (G > 1) {
            partial[((long long)s * G + gidx) * NP + k] = v;
        } else {
            const bool beyond = L >= 0 && k < NP - 1 && (k % p.L_max) >= L;
            if (k == NP - 1) merit[s] = v;
            else if (k < p.L_max) dm_dd[(long long)s * p.L_max + k] = beyond ? R(0) : v;
            else if (dm_dn) dm_dn[(long long)s * p.L_max + (k - p.L_max)] = beyond ? R(0) : v;
        }
    }
}

template <typename R>
__global__ void grad_finalize(const tmm_problem p, int G, const R *__restrict__ partial, R *__restrict__ merit,
                              R *__restrict__ dm_dd, R *__restrict__ dm_dn)
{
    const int NP = 2 * p.L_max + 1;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)p.S * NP) return;
    const int s = (int)(i / NP), k = (int)(i - (long long)s * NP);
    R v = R(0);
    for (int g = 0; g < G; ++g) v += partial[((long long)s * G + g) * NP + k];
    const int L = layers_of(p, s);
    const bool beyond = L >= 0 && k < NP - 1 && (k % p.L_max) >= L;
    if (k == NP - 1) merit[s] = v;
    else if (k < p.L_max) dm_dd[(long long)s * p.L_max + k] = beyond ? R(0) : v;
    else if (dm_dn) dm_dn[(long long)s * p.L_max + (k - p.L_max)] = beyond ? R(0) : v;
}

// ---------------------------------------------------------------- host side
struct GradPlan {
    int TL, TT, n_lt, n_tt, G;
    size_t smem;
};

static size_t grad_smem(const tmm_problem *p, int TL, int TT)
{
    const size_t r = real_size(p->prec);
    const size_t Lm2 = (size_t)p->L_max + 2;
    return Lm2 * TL * (8 * r) + (size_t)TL * r + (size_t)(TL * TT / 32) * (2 * p->L_max + 1) * r;
}

static tmm_status grad_plan(const tmm_problem *p, bool with_ws, GradPlan *g)
{
    DeviceInfo di;
    tmm_status st = device_info(&di);
    if (st != TMM_OK) return st;
    g->TT = std::min(p->n_theta, 8);
    while (kGradThreads % g->TT) --g->TT;
    g->TL = kGradThreads / g->TT;
    while (g->TL > 32 && g->TL / 2 >= p->n_lambda && (g->TL / 2) * g->TT >= 32) g->TL /= 2;
    while (g->TL * g->TT > 32 && grad_smem(p, g->TL, g->TT) > (size_t)di.max_smem_optin) g->TL /= 2;
    g->n_lt = (p->n_lambda + g->TL - 1) / g->TL;
    g->n_tt = (p->n_theta + g->TT - 1) / g->TT;
    g->smem = grad_smem(p, g->TL, g->TT);
    if (g->smem > (size_t)di.max_smem_optin) return TMM_ERR_UNSUPPORTED;
    const int tiles = g->n_lt * g->n_tt;
    const long long want = 4LL * di.sms;
    g->G = with_ws ? (int)std::min<long long>(tiles, std::max<long long>(1, (want + p->S - 1) / p->S)) : 1;
    return TMM_OK;
}

size_t grad_ws_bytes(const tmm_problem *p)
{
    GradPlan g;
    if (p->S == 0 || p->n_lambda == 0 || p->n_theta == 0 || grad_plan(p, true, &g) != TMM_OK) return 0;
    if (g.G <= 1) return 0;
    return (size_t)p->S * g.G * (2 * p->L_max + 1) * real_size(p->prec);
}

template <typename R, int KMAX, bool WITH_DN>
static tmm_status launch_grad_typed(const tmm_problem *p, const GradPlan &g, const void *Rt, void *merit,
                                    void *dm_dd, void *dm_dn, void *ws, cudaStream_t st)
{
    auto k = tmm_grad_kernel<R, KMAX, WITH_DN>;
    {
        const tmm_status ss = ensure_dynamic_smem(reinterpret_cast<const void *>(k), g.smem);
        if (ss != TMM_OK) return ss;
    }
    const long long blocks = (long long)p->S * g.G;
    if (blocks > 0x7fffffffLL) return TMM_ERR_UNSUPPORTED;
    const R inv_N = R(1) / (R(npol(p->pol_mask)) * R(p->n_theta) * R(p->n_lambda));
    k<<<(unsigned)blocks, g.TL * g.TT, g.smem, st>>>(*p, (const R *)Rt, g.TL, g.TT, g.n_lt, g.n_tt, g.G, inv_N,
                                                    (R *)merit, (R *)dm_dd, (R *)dm_dn, (R *)ws);
    tmm_status s = check_launch();
    if (s != TMM_OK || g.G <= 1) return s;
    const long long n = (long long)p->S * (2 * p->L_max + 1);
    grad_finalize<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(*p, g.G, (const R *)ws, (R *)merit, (R *)dm_dd,
                                                                   (R *)dm_dn);
    return check_launch();
}

template <typename R>
static tmm_status launch_grad_prec(const tmm_problem *p, const GradPlan &g, const void *Rt, void *merit, void *dm_dd,
                                   void *dm_dn, void *ws, cudaStream_t st)
{
    const int need = p->L_max + 2;
    if (dm_dn) {
        if (need <= 18) return launch_grad_typed<R, 18, true>(p, g, Rt, merit, dm_dd, dm_dn, ws, st);
        if (need <= 34) return launch_grad_typed<R, 34, true>(p, g, Rt, merit, dm_dd, dm_dn, ws, st);
        if (need <= 66) return launch_grad_typed<R, 66, true>(p, g, Rt, merit, dm_dd, dm_dn, ws, st);
        return launch_grad_typed<R, kGradMaxLayers + 2, true>(p, g, Rt, merit, dm_dd, dm_dn, ws, st);
    }
    if (need <= 18) return launch_grad_typed<R, 18, false>(p, g, Rt, merit, dm_dd, dm_dn, ws, st);
    if (need <= 34) return launch_grad_typed<R, 34, false>(p, g, Rt, merit, dm_dd, dm_dn, ws, st);
    if (need <= 66) return launch_grad_typed<R, 66, false>(p, g, Rt, merit, dm_dd, dm_dn, ws, st);
    return launch_grad_typed<R, kGradMaxLayers + 2, false>(p, g, Rt, merit, dm_dd, dm_dn, ws, st);
}

tmm_status launch_grad(const tmm_problem *p, const void *R_target, void *merit, void *dm_dd, void *dm_dn, void *ws,
                       size_t ws_bytes, cudaStream_t st)
{
    if (p->L_max > kGradMaxLayers) return TMM_ERR_UNSUPPORTED;
    GradPlan g;
    const bool with_ws = ws != nullptr && ws_bytes > 0;
    tmm_status s = grad_plan(p, with_ws, &g);
    if (s != TMM_OK) return s;
    if (g.G > 1) {
        const size_t need = (size_t)p->S * g.G * (2 * p->L_max + 1) * real_size(p->prec);
        if (ws_bytes < need) return TMM_ERR_NOMEM;
        if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return TMM_ERR_INVALID_ARG;
    }
    return p->prec == TMM_F64 ? launch_grad_prec<double>(p, g, R_target, merit, dm_dd, dm_dn, ws, st)
                              : launch_grad_prec<float>(p, g, R_target, merit, dm_dd, dm_dn, ws, st);
}

}  // namespace tmm
