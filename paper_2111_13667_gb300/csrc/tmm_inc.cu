// tmm_inc.cu -- stacks with incoherent (thick) layers.
//
// The media 0 and L_s+1 and every flagged finite layer are incoherent; the
// coherent blocks between consecutive incoherent media a < b are evaluated
// as amplitude products (Eqs. 1-4, the forward kernel's scaled right-to-left
// sweep, here with both columns of the block matrix M), and the blocks are
// combined by intensities.  Per block and polarisation:
//   R_f = |M10 / M00|^2 (light from a),  R_b = |M01 / M00|^2 (light from b),
//   T_f from M00 and the carried scales exactly as the forward kernel's T
//   (Eqs. 5-6 with the Poynting factors Re k, k = q for s, q / n^2 for p), and
//   T_b = T_f (Re k_a / |k_a|)^2 / (Re k_b / |k_b|)^2: the amplitude
//   transmissions from either side differ by det M = k_b / k_a (1 between
//   non-absorbing media).
// An absorbing incoherent layer j attenuates every single pass by
// p_j = exp(-4 pi Im(q_j) d_j / lambda).  With (P, M) the forward and backward
// intensities on the left of the blocks done so far, scaled by the product t
// of their T_f and single-pass factors, crossing layer b from its right
// boundary to its left takes (P, M, t) to (P, p_b^2 M, p_b t), and a block
//   P' = P - R_b M,   M' = R_f P' + T_f T_b M,   t' = t T_f
// from (1, 0, 1) in the exit medium; R = M / P and T = t / P in medium 0.
// The first incoherent layer with Re(n_j^2 - n_0^2 sin^2 theta) <= 0 (for a
// real index: the wave is evanescent) ends the stack: it is the exit medium
// and T = 0.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "tmm_device.cuh"
#include "tmm_pair.cuh"
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

// (Re k_a / |k_a|)^2 / (Re k_b / |k_b|)^2, exactly 1 for real k_a, k_b; 0 when
// medium b carries no flux (Re k_b = 0: evanescent), where nothing returns.
template <typename R> __device__ __forceinline__ R back_ratio(Cx<R> ka, Cx<R> kb)
{
    if (ka.y == R(0) && kb.y == R(0)) return R(1);
    const R den = kb.x * kb.x * abs2(ka);
    return den > R(0) ? (ka.x * ka.x * abs2(kb)) / den : R(0);
}

// R_f, R_b, T_f, T_b of the coherent block between incoherent media a < b,
// for the polarisations in POL ([0] s, [1] p).  q_a is medium a's root (a = 0:
// q_0 = n_0 cos(theta), computed directly).
template <typename R, int POL>
__device__ __forceinline__ void block_coeffs(const StageA<R> *__restrict__ sa, const StageB<R> *__restrict__ sb,
                                             int TL, int tl, int a, int b, R q0sq, Cx<R> q_a, R n0, R Rf[2], R Rb[2],
                                             R Tf[2], R Tb[2])
{
    constexpr int RN = RenormEvery<R>::value;
    const R yi_max = R(kImDeltaMax / kTwoPi);
    StageA<R> A = sa[b * TL + tl];
    R absz;
    Cx<R> q_nx = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
    const Cx<R> q_b = q_nx, n2_b = {A.d2x + n0 * n0, A.n2y};
    Cx<R> g_nx = cmul(q_nx, Cx<R>{A.in2x, A.in2y});
    const Cx<R> g_b = g_nx;
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
    // interface a | a+1
    A = sa[a * TL + tl];
    Ps *= abs2(q_a);
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
        Tf[0] = q_b.x / q_a.x * ldexp_w(Ps * yscale / ax0, e4 + eP + yn - 2 * es);
        Tb[0] = Tf[0] * back_ratio(q_a, q_b);
    }
    if (POL & 2) {
        const Cx<R> n2_a = {A.d2x + n0 * n0, A.n2y};
        const Cx<R> g_a = cmul(q_a, Cx<R>{A.in2x, A.in2y});
        interface_pair(g_a, g_nx, cp.x0, cp.x1);
        interface_pair(g_a, g_nx, cp.y0, cp.y1);
        const R ax0 = abs2(cp.x0);
        Rf[1] = abs2(cp.x1) / ax0;
        Rb[1] = abs2(cp.y0) / ax0;
        const R num = cmul(n2_b, conj(q_b)).x, den = cmul(n2_a, conj(q_a)).x;
        Tf[1] = num / den * ldexp_w(Ps * Pp * yscale / ax0, e4 + eP + ePp + yn - 2 * ep);
        Tb[1] = Tf[1] * back_ratio(g_a, g_b);
    }
}

// Single-pass power factor exp(-4 pi Im(q_j) d_j / lambda) of finite layer j.
template <typename R>
__device__ __forceinline__ R pass_factor(const StageA<R> &A, const StageB<R> &B, R q0sq)
{
    R absz;
    const Cx<R> q = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
    return exp_m2_turn(B.dl * q.y);
}

// One point (one angle), both polarisations: Rv, Tv = {s, p}.
template <typename R, int POL>
__device__ __forceinline__ void inc_point(const StageA<R> *__restrict__ sa, const StageB<R> *__restrict__ sb,
                                          const unsigned char *flg, int TL, int tl, int L, R n0, R sth, R cth,
                                          R Rv[2], R Tv[2])
{
    const R beta = n0 * sth, c0 = n0 * cth, q0sq = c0 * c0;
    if (beta >= n0) {  // grazing (false for a NaN n_0)
        Rv[0] = Rv[1] = R(1);
        Tv[0] = Tv[1] = R(0);
        return;
    }
    if (!(n0 == n0)) return;
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
        if (b != e) {  // across incoherent layer b, right boundary to left
            const R pb = pass_factor(sa[b * TL + tl], sb[b * TL + tl], q0sq);
#pragma unroll
            for (int k = 0; k < 2; ++k) M[k] *= pb * pb, t[k] *= pb;
        }
        int a = b - 1;
        while (a > 0 && !flg[a]) --a;
        R absa;
        const Cx<R> qa = a == 0 ? Cx<R>{c0, R(0)}
                                : forward_root(Cx<R>{sa[a * TL + tl].d2x + q0sq, sa[a * TL + tl].n2y}, &absa);
        R Rf[2] = {R(0), R(0)}, Rb[2] = {R(0), R(0)}, Tf[2] = {R(0), R(0)}, Tb[2] = {R(0), R(0)};
        block_coeffs<R, POL>(sa, sb, TL, tl, a, b, q0sq, qa, n0, Rf, Rb, Tf, Tb);
        if (b == e) Rb[0] = Rb[1] = Tb[0] = Tb[1] = R(0);  // nothing returns from the exit medium
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!(POL & (1 << k))) continue;
            const R P1 = P[k] - Rb[k] * M[k];
            const R M1 = Rf[k] * P1 + Tf[k] * Tb[k] * M[k];
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

// ---------------------------------------------------------------- FP32: two angles per thread
// block_coeffs for the two angles in the lanes of q0sq (qa: the root of
// medium a per lane); outputs [lane][pol].
template <int POL>
__device__ __forceinline__ void block_coeffs2(const StageA<float> *__restrict__ sa,
                                              const StageB<float> *__restrict__ sb, int TL, int tl, int a, int b,
                                              float2 q0sq, const Cx<float> qa[2], float n0, float Rf[2][2],
                                              float Rb[2][2], float Tf[2][2], float Tb[2][2])
{
    constexpr int RN = RenormEvery<float>::value;
    const float yi_max = float(kImDeltaMax / kTwoPi);
    StageA<float> A = sa[b * TL + tl];
    float absz;
    const Cx<float> qba = forward_root(Cx<float>{A.d2x + q0sq.x, A.n2y}, &absz);
    const Cx<float> qbb = forward_root(Cx<float>{A.d2x + q0sq.y, A.n2y}, &absz);
    const Cx<float> n2_b = {A.d2x + n0 * n0, A.n2y}, in2b = {A.in2x, A.in2y};
    C2 q_nx = pack2(qba, qbb), g_nx = pack2(cmul(qba, in2b), cmul(qbb, in2b));
    float2 nqy_nx = neg2(q_nx.y), ngy_nx = neg2(g_nx.y);
    float Pp = sb[b * TL + tl].ain2;
    int ePp = 0;
    float2 Ps = bc2(1.f), Y = bc2(0.f);
    int ePa = 0, ePb = 0, esa = 0, esb = 0, epa = 0, epb = 0;
    const C2 one = {bc2(1.f), bc2(0.f)}, zero = {bc2(0.f), bc2(0.f)};
    Cols2 cs{one, zero, zero, one}, cp{one, zero, zero, one};
    int cnt = 0;
    for (int j = b - 1; j > a; --j) {
        A = sa[j * TL + tl];
        const StageB<float> B = sb[j * TL + tl];
        float absa, absb;
        // a layer inside the block: the branch of q does not reach R and T
        const Cx<float> qla = inner_root(Cx<float>{A.d2x + q0sq.x, A.n2y}, &absa);
        const Cx<float> qlb = inner_root(Cx<float>{A.d2x + q0sq.y, A.n2y}, &absb);
        Ps = mul2(Ps, f2(absa, absb));
        const float yra = B.dl * qla.x, yrb = B.dl * qlb.x;
        const float2 yi = f2(fminf(B.dl * qla.y, yi_max), fminf(B.dl * qlb.y, yi_max));
        Y = add2(Y, yi);
        float2 sn, cs_;
        sincos_turn(yra - rintf(yra), &sn.x, &cs_.x);
        sincos_turn(yrb - rintf(yrb), &sn.y, &cs_.y);
        const float2 E2 = f2(exp_m2_turn(yi.x), exp_m2_turn(yi.y));
        const float2 nsn = neg2(sn), ec = mul2(E2, cs_), es = mul2(E2, sn), nes = neg2(es);
        const C2 q = pack2(qla, qlb);
        if (POL & 1) {
            const float2 nqy = neg2(q.y);
            interface_pair2(q, nqy, q_nx, nqy_nx, cs.x0, cs.x1);
            interface_pair2(q, nqy, q_nx, nqy_nx, cs.y0, cs.y1);
            phase2(cs_, sn, nsn, ec, es, nes, cs.x0, cs.x1);
            phase2(cs_, sn, nsn, ec, es, nes, cs.y0, cs.y1);
            nqy_nx = nqy;
        }
        if (POL & 2) {
            Pp *= B.ain2;
            const Cx<float> in2 = {A.in2x, A.in2y};
            const C2 g = pack2(cmul(qla, in2), cmul(qlb, in2));
            const float2 ngy = neg2(g.y);
            interface_pair2(g, ngy, g_nx, ngy_nx, cp.x0, cp.x1);
            interface_pair2(g, ngy, g_nx, ngy_nx, cp.y0, cp.y1);
            phase2(cs_, sn, nsn, ec, es, nes, cp.x0, cp.x1);
            phase2(cs_, sn, nsn, ec, es, nes, cp.y0, cp.y1);
            g_nx = g;
            ngy_nx = ngy;
        }
        q_nx = q;
        if (++cnt == RN) {
            cnt = 0;
            renorm_scalar(Ps.x, ePa);
            renorm_scalar(Ps.y, ePb);
            if (POL & 2) renorm_scalar(Pp, ePp);
            if (POL & 1) renorm_cols2(cs, esa, esb);
            if (POL & 2) renorm_cols2(cp, epa, epb);
        }
    }
    // interface a | a+1 per lane
    A = sa[a * TL + tl];
    const int e4 = 2 * (b - a);
    const Cx<float> n2_a = {A.d2x + n0 * n0, A.n2y};
    const Cx<float> in2a = {A.in2x, A.in2y};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const Cx<float> q_a = qa[i], q_b = i ? qbb : qba;
        const float Psi = (i ? Ps.y : Ps.x) * abs2(q_a), Yi = i ? Y.y : Y.x;
        const int ePi = i ? ePb : ePa;
        float u = float(-2.0 * kTwoPi * kLog2e) * Yi;
        u = fmaxf(u, -1.0e6f);
        const float un = floorf(u);
        const float yscale = exp2f(u - un);
        const int yn = (int)un;
        if (POL & 1) {
            Cx<float> x0 = lane(cs.x0, i), x1 = lane(cs.x1, i), y0 = lane(cs.y0, i), y1 = lane(cs.y1, i);
            const Cx<float> qn = lane(q_nx, i);
            interface_pair(q_a, qn, x0, x1);
            interface_pair(q_a, qn, y0, y1);
            const float ax0 = abs2(x0);
            Rf[i][0] = abs2(x1) / ax0;
            Rb[i][0] = abs2(y0) / ax0;
            Tf[i][0] = q_b.x / q_a.x * ldexpf(Psi * yscale / ax0, e4 + ePi + yn - 2 * (i ? esb : esa));
            Tb[i][0] = Tf[i][0] * back_ratio(q_a, q_b);
        }
        if (POL & 2) {
            const Cx<float> g_a = cmul(q_a, in2a), gn = lane(g_nx, i);
            Cx<float> x0 = lane(cp.x0, i), x1 = lane(cp.x1, i), y0 = lane(cp.y0, i), y1 = lane(cp.y1, i);
            interface_pair(g_a, gn, x0, x1);
            interface_pair(g_a, gn, y0, y1);
            const float ax0 = abs2(x0);
            Rf[i][1] = abs2(x1) / ax0;
            Rb[i][1] = abs2(y0) / ax0;
            const float num = cmul(n2_b, conj(q_b)).x, den = cmul(n2_a, conj(q_a)).x;
            Tf[i][1] = num / den * ldexpf(Psi * Pp * yscale / ax0, e4 + ePi + ePp + yn - 2 * (i ? epb : epa));
            Tb[i][1] = Tf[i][1] * back_ratio(g_a, cmul(q_b, in2b));
        }
    }
}

// inc_point for the two angles (sin, cos in the lanes of st, ct): Rv, Tv
// [lane][pol].  Lanes whose stacks end at different incoherent layers (an
// evanescent one for one angle only), or at grazing incidence, take the
// one-angle path each.
template <int POL>
__device__ __forceinline__ void inc_point2(const StageA<float> *__restrict__ sa,
                                           const StageB<float> *__restrict__ sb, const unsigned char *flg, int TL,
                                           int tl, int L, float n0, float2 st, float2 ct, float Rv[2][2],
                                           float Tv[2][2])
{
    const float2 c0 = f2(n0 * ct.x, n0 * ct.y), q0sq = f2(c0.x * c0.x, c0.y * c0.y);
    int e[2] = {L + 1, L + 1};
#pragma unroll
    for (int i = 0; i < 2; ++i)
        for (int j = 1; j <= L; ++j)
            if (flg[j] && sa[j * TL + tl].d2x + (i ? q0sq.y : q0sq.x) <= 0.f) {
                e[i] = j;
                break;
            }
    const bool graze = n0 * st.x >= n0 || n0 * st.y >= n0;
    if (e[0] != e[1] || graze || !(n0 == n0)) {
        inc_point<float, POL>(sa, sb, flg, TL, tl, L, n0, st.x, ct.x, Rv[0], Tv[0]);
        inc_point<float, POL>(sa, sb, flg, TL, tl, L, n0, st.y, ct.y, Rv[1], Tv[1]);
        return;
    }
    const bool cut = e[0] <= L;
    float P[2][2] = {{1.f, 1.f}, {1.f, 1.f}}, M[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, t[2][2] = {{1.f, 1.f}, {1.f, 1.f}};
    int b = e[0];
    while (b > 0) {
        if (b != e[0]) {  // across incoherent layer b, right boundary to left
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const float pb = pass_factor(sa[b * TL + tl], sb[b * TL + tl], i ? q0sq.y : q0sq.x);
#pragma unroll
                for (int k = 0; k < 2; ++k) M[i][k] *= pb * pb, t[i][k] *= pb;
            }
        }
        int a = b - 1;
        while (a > 0 && !flg[a]) --a;
        Cx<float> qa[2];
        if (a == 0) {
            qa[0] = Cx<float>{c0.x, 0.f};
            qa[1] = Cx<float>{c0.y, 0.f};
        } else {
            const StageA<float> Aa = sa[a * TL + tl];
            float absa;
            qa[0] = forward_root(Cx<float>{Aa.d2x + q0sq.x, Aa.n2y}, &absa);
            qa[1] = forward_root(Cx<float>{Aa.d2x + q0sq.y, Aa.n2y}, &absa);
        }
        float Rf[2][2] = {}, Rb[2][2] = {}, Tf[2][2] = {}, Tb[2][2] = {};
        block_coeffs2<POL>(sa, sb, TL, tl, a, b, q0sq, qa, n0, Rf, Rb, Tf, Tb);
        if (b == e[0])  // nothing returns from the exit medium
#pragma unroll
            for (int i = 0; i < 2; ++i) Rb[i][0] = Rb[i][1] = Tb[i][0] = Tb[i][1] = 0.f;
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!(POL & (1 << k))) continue;
                const float P1 = P[i][k] - Rb[i][k] * M[i][k];
                const float M1 = Rf[i][k] * P1 + Tf[i][k] * Tb[i][k] * M[i][k];
                const float inv = 1.f / P1;
                P[i][k] = 1.f;
                M[i][k] = M1 * inv;
                t[i][k] = t[i][k] * Tf[i][k] * inv;
            }
        b = a;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            Rv[i][k] = M[i][k];
            Tv[i][k] = cut ? 0.f : t[i][k];
        }
}

// One block per (stack, tile of TL lambda x TT theta); PAIR: FP32 with two
// angles per thread, TL x ceil(TT / 2) threads.
template <typename R, int POL, bool WITH_T, bool PAIR>
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
    const int tid = threadIdx.y * TL + threadIdx.x, nthr = TL * (int)blockDim.y;
    const int L = layers_of(p, s);
    const int l0 = lt * TL;
    if (L >= 0) {
        fill_stage<R>(p, s, L, l0, TL, sa, sb, n0s, tid, nthr);
        for (int j = tid; j < L + 2; j += nthr)
            flg[j] = (j == 0 || j == L + 1) ? 1 : (inc && inc[(long long)s * p.L_max + (j - 1)] ? 1 : 0);
    }
    __syncthreads();

    const int tl = threadIdx.x, l = l0 + tl;
    const int t0 = ttile * TT, t_end = min(t0 + TT, p.n_theta);
    const int a0 = PAIR ? t0 + 2 * (int)threadIdx.y : t0 + (int)threadIdx.y;
    if (l >= p.n_lambda || a0 >= t_end) return;  // no barrier follows
    const int np = PAIR && a0 + 1 < t_end ? 2 : 1;
    R Rv[2][2], Tv[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i) Rv[i][0] = Rv[i][1] = Tv[i][0] = Tv[i][1] = nan_w<R>();
    if (L >= 0) {
        const R *th = (const R *)p.theta;
        const R n0 = n0s[tl];
        if constexpr (PAIR) {
            float2 st, ct;
            sincos_w(th[a0], &st.x, &ct.x);
            sincos_w(th[np == 2 ? a0 + 1 : a0], &st.y, &ct.y);
            inc_point2<POL>(sa, sb, flg, TL, tl, L, n0, st, ct, Rv, Tv);
        } else {
            R sth, cth;
            sincos_w(th[a0], &sth, &cth);
            inc_point<R, POL>(sa, sb, flg, TL, tl, L, n0, sth, cth, Rv[0], Tv[0]);
        }
    }
    const long long plane = (long long)p.S * p.n_theta * p.n_lambda;
    for (int i = 0; i < np; ++i) {
        const long long o = ((long long)s * p.n_theta + a0 + i) * p.n_lambda + l;
        if (POL & 4) {
            Rout[o] = R(0.5) * (Rv[i][0] + Rv[i][1]);
            if (WITH_T) Tout[o] = R(0.5) * (Tv[i][0] + Tv[i][1]);
        } else {
            int pi = 0;
            if (POL & 1) {
                Rout[o] = Rv[i][0];
                if (WITH_T) Tout[o] = Tv[i][0];
                ++pi;
            }
            if (POL & 2) {
                Rout[pi * plane + o] = Rv[i][1];
                if (WITH_T) Tout[pi * plane + o] = Tv[i][1];
            }
        }
    }
}

size_t inc_smem(const tmm_problem *p, int TL)
{
    const size_t r = real_size(p->prec);
    return (size_t)(p->L_max + 2) * TL * (6 * r) + (size_t)TL * r + (size_t)(p->L_max + 2) + 16;
}

template <typename R, int POL, bool WITH_T, bool PAIR>
tmm_status launch_inc_shaped(const tmm_problem *p, const uint8_t *inc, int TL, int TT, int n_lt, int n_tt,
                             long long items, size_t smem, R *Ro, R *To, cudaStream_t st)
{
    auto k = tmm_inc_kernel<R, POL, WITH_T, PAIR>;
    {
        const tmm_status ss = ensure_dynamic_smem(reinterpret_cast<const void *>(k), smem);
        if (ss != TMM_OK) return ss;
    }
    k<<<(unsigned)items, dim3(TL, PAIR ? (TT + 1) / 2 : TT), smem, st>>>(*p, inc, TL, TT, n_lt, n_tt, Ro, To);
    return check_launch();
}

// FP32 tiles of two or more angles run two angles per thread.
template <typename R, int POL, bool WITH_T>
tmm_status launch_inc_typed(const tmm_problem *p, const uint8_t *inc, int TL, int TT, int n_lt, int n_tt,
                            long long items, size_t smem, R *Ro, R *To, cudaStream_t st)
{
    if constexpr (std::is_same<R, float>::value) {
        if (TT >= 2) return launch_inc_shaped<R, POL, WITH_T, true>(p, inc, TL, TT, n_lt, n_tt, items, smem, Ro, To, st);
    }
    return launch_inc_shaped<R, POL, WITH_T, false>(p, inc, TL, TT, n_lt, n_tt, items, smem, Ro, To, st);
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
    TraceRange trace("tmm_inc_batched");
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if (p->prec != TMM_F64 && p->prec != TMM_F32) return TMM_ERR_UNSUPPORTED;
    const long long pts = (long long)p->S * p->n_lambda * p->n_theta;
    if (pts == 0) return TMM_OK;
    if (!R) return TMM_ERR_INVALID_ARG;
    DeviceInfo di;
    s = device_info(&di);
    if (s != TMM_OK) return s;
    const int TT = std::min(p->n_theta, 32);
    const int rows = (p->prec == TMM_F32 && TT >= 2) ? (TT + 1) / 2 : TT;  // thread rows per block
    int TL = 1;
    while (TL * rows * 2 <= kIncThreads) TL *= 2;
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
