// tmm_pcoh.cu -- stacks with one partially coherent layer.
//
// Finite layer j = layer[s] of stack s has the thickness d_j + D with
// D ~ N(0, sigma_s^2); R and T are the expectations of the coherent R, T
// (Eqs. 1-6) over D, by the Gauss-Hermite rule
//   E[f] = sum_k (w_k / sqrt(pi)) f(sqrt(2) sigma x_k)
// (a reading: the paper treats coherent stacks only).  Only layer j's phase
// depends on D, so one thread per (stack, lambda, theta) -- in FP32 per pair
// of angles on paired lanes -- evaluates, for both polarisations:
//   y  = F_j x_{j+1}: the forward kernel's right-to-left sweep from the exit
//        medium through interface j | j+1 (scaled, unnormalised interfaces);
//   ML = F_0 P_1 F_1 ... P_{j-1} F_{j-1}: the block left of layer j, both
//        columns carried through the same sweep from the identity;
//   per node: x_0 = ML P_j(d_j + D_k) y, R_k = |x_0[1] / x_0[0]|^2 and T_k
//        from the dropped scales exactly as the forward kernel's T.  The
//        products ML_ab y_b are formed once and reduced to quadratic forms
//        of |x_0[a]|^2 in the node's (cos 2 Re delta, sin 2 Re delta,
//        e^{-2 Im delta}); T's scale factor does not depend on the node and is
//        applied to the node sum once; node pairs +-D_k share one sincos.
// The nodes come from a Sturm-sequence bisection of the Hermite Jacobi matrix
// on the host; they are symmetric, so the kernel takes the non-negative half.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "tmm_device.cuh"
#include "tmm_pair.cuh"
#include "tmm_internal.h"

namespace tmm {

namespace {

constexpr int kPcThreads = 256;
constexpr int kPcMaxNodes = 256;
constexpr int kPcHalf = kPcMaxNodes / 2;

// The non-negative Gauss-Hermite nodes h_i (descending) of an n_nodes rule
// as sqrt(2) x, with their weights w / sqrt(pi); an odd rule's node 0 is the
// last entry and is taken once.
template <typename R> struct Nodes {
    int n_half;   // entries
    int odd;      // the last entry is the node 0
    R off[kPcHalf + 1];
    R w[kPcHalf + 1];
};

// Gauss-Hermite rule: the nodes are the eigenvalues of the symmetric
// tridiagonal Jacobi matrix of the Hermite polynomials (zero diagonal,
// off-diagonal sqrt(i / 2)), found by bisection on the Sturm count; the
// weights are 1 / (K psi_{K-1}(x)^2) with psi the orthonormal Hermite
// polynomials (psi_0 = pi^{-1/4}), here divided by sqrt(pi).
static int eigen_below(const double *b2, int K, double x)
{
    double q = -x;
    if (q == 0.0) q = -1e-300;
    int c = q < 0.0 ? 1 : 0;
    for (int i = 1; i < K; ++i) {
        q = -x - b2[i - 1] / q;
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++c;
    }
    return c;
}

static void gauss_hermite(int K, double *x, double *w)
{
    double b2[kPcMaxNodes];
    for (int i = 1; i < K; ++i) b2[i - 1] = 0.5 * i;
    const double bound = std::sqrt(2.0 * K) + 1.0;
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < K; ++k) {
        double lo = -bound, hi = bound;
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid == lo || mid == hi) break;
            if (eigen_below(b2, K, mid) >= k + 1) hi = mid;
            else lo = mid;
        }
        const double xk = 0.5 * (lo + hi);
        double pm = std::pow(pi, -0.25), pc = std::sqrt(2.0) * xk * pm;
        double pk1 = pm;
        if (K > 1) {
            for (int n = 1; n < K - 1; ++n) {
                const double pn = std::sqrt(2.0 / (n + 1)) * xk * pc - std::sqrt(n / (n + 1.0)) * pm;
                pm = pc;
                pc = pn;
            }
            pk1 = pc;
        }
        x[k] = xk;
        w[k] = 1.0 / (K * pk1 * pk1) / std::sqrt(pi);
    }
}

template <typename R> static Nodes<R> make_nodes(int K)
{
    double x[kPcMaxNodes], w[kPcMaxNodes];
    gauss_hermite(K, x, w);
    Nodes<R> nd{};
    nd.odd = K & 1;
    nd.n_half = (K + 1) / 2;
    // x ascends: the non-negative half from the top down, symmetric weights
    // averaged with their mirror
    for (int i = 0; i < nd.n_half; ++i) {
        const int hi = K - 1 - i, lo = i;
        const double xh = hi == lo ? 0.0 : 0.5 * (x[hi] - x[lo]);
        nd.off[i] = R(std::sqrt(2.0) * xh);
        nd.w[i] = R(hi == lo ? w[hi] : 0.5 * (w[hi] + w[lo]));
    }
    return nd;
}

// The phase factors of one layer, e^{-i delta} and e^{+i delta} divided by
// e^{Im delta}, with the clamped Im(delta) / (2 pi): the forward kernel's.
template <typename R> struct Step {
    Cx<R> emi, epi;
    R yi;
};

template <typename R>
__device__ __forceinline__ Step<R> phase_of(R dl, Cx<R> q, R yi_max)
{
    Step<R> st;
    const R yr = dl * q.x;
    st.yi = fmin(dl * q.y, yi_max);
    R sn, cs;
    sincos_turn(yr - rint_w(yr), &sn, &cs);
    const R E2 = exp_m2_turn(st.yi);
    st.emi = Cx<R>{cs, -sn};
    st.epi = Cx<R>{E2 * cs, E2 * sn};
    return st;
}

// R and T of one point from x_0's pair and the scale bookkeeping (the
// forward kernel's Eqs. 5-6 with the dropped factors restored).
template <typename R>
__device__ __forceinline__ void rt_of(Cx<R> x0, Cx<R> x1, R scale, int e, R kappa_out, R kappa_in, R &Rv, R &Tv)
{
    const R ax0 = abs2(x0);
    Rv = abs2(x1) / ax0;
    Tv = kappa_out / kappa_in * ldexp_w(scale / ax0, e);
}

// A node's |x|^2 with x = A e^{-i t} + E B e^{+i t} (t = Re delta, E = e^{-2 Im delta}):
//   |x|^2 = |A|^2 + E^2 |B|^2 + 2 E Re(A conj(B) e^{-2 i t}) = a + E (E b + cx cos 2t + cy sin 2t),
// a quadratic form whose coefficients do not depend on the node.
template <typename R> struct Quad {
    R a, b, cx, cy;
};
template <typename R> __device__ __forceinline__ Quad<R> quad_of(Cx<R> A, Cx<R> B)
{
    return Quad<R>{abs2(A), abs2(B), R(2) * fma(A.x, B.x, A.y * B.y), R(2) * fma(A.y, B.x, -A.x * B.y)};
}
template <typename R> __device__ __forceinline__ R quad_at(const Quad<R> &q, R c2, R s2, R E)
{
    return fma(E, fma(E, q.b, fma(q.cx, c2, q.cy * s2)), q.a);
}

// cos 2t, sin 2t and E = e^{-2 Im delta} of layer jp at thickness / lambda = dl
// (Im delta / 2 pi clamped like every layer's).
template <typename R>
__device__ __forceinline__ void twice_phase(R dl, Cx<R> q, R yi_max, R &c2, R &s2, R &E)
{
    const R y2 = R(2) * dl * q.x;
    sincos_turn(y2 - rint_w(y2), &s2, &c2);
    E = exp_m2_turn(fmin(dl * q.y, yi_max));
}

template <typename R, int POL>
__device__ __forceinline__ void pc_point(const StageA<R> *__restrict__ sa, const StageB<R> *__restrict__ sb, int TL,
                                         int tl, int L, int jp, R sig, R inv_lam, R dj, R n0, R sth, R cth,
                                         const Nodes<R> &nd, R out[4])
{
    constexpr int RN = RenormEvery<R>::value;
    const R beta = n0 * sth, c0 = n0 * cth, q0sq = c0 * c0;
    const R yi_max = R(kImDeltaMax / kTwoPi);
    StageA<R> A = sa[(L + 1) * TL + tl];
    R absz;
    Cx<R> q_nx = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
    const Cx<R> q_out = q_nx, n2_out = {A.d2x + n0 * n0, A.n2y};
    Cx<R> g_nx = cmul(q_nx, Cx<R>{A.in2x, A.in2y});
    R Ps = R(1), Y = R(0), Pp = (POL & 2) ? sb[(L + 1) * TL + tl].ain2 : R(1);
    int eP = 0, ePp = 0, es = 0, ep = 0;
    Cx<R> s0 = {R(1), R(0)}, s1 = {R(0), R(0)}, p0 = s0, p1 = s1;
    int cnt = 0;
    auto rescale = [&]() {
        renorm_scalar(Ps, eP);
        if (POL & 2) renorm_scalar(Pp, ePp);
        if (POL & 1) renorm_pair(s0, s1, es);
        if (POL & 2) renorm_pair(p0, p1, ep);
    };
    // right of the partial layer (the whole stack when jp = 0)
    for (int j = L; j > jp; --j) {
        A = sa[j * TL + tl];
        const StageB<R> B = sb[j * TL + tl];
        const Cx<R> q = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
        Ps *= absz;
        const Step<R> st = phase_of(B.dl, q, yi_max);
        Y += st.yi;
        if (POL & 1) {
            interface_pair(q, q_nx, s0, s1);
            s0 = cmul(st.emi, s0);
            s1 = cmul(st.epi, s1);
        }
        if (POL & 2) {
            Pp *= B.ain2;
            const Cx<R> g = cmul(q, Cx<R>{A.in2x, A.in2y});
            interface_pair(g, g_nx, p0, p1);
            p0 = cmul(st.emi, p0);
            p1 = cmul(st.epi, p1);
            g_nx = g;
        }
        q_nx = q;
        if (++cnt == RN) {
            cnt = 0;
            rescale();
        }
    }
    const bool grazing = beta >= n0;
    const Cx<R> q0 = {c0, R(0)};
    const int e4 = 2 * (L + 1);
    const StageA<R> A0 = sa[tl];
    const Cx<R> g0 = cmul(q0, Cx<R>{A0.in2x, A0.in2y});
    const R kout_p = cmul(n2_out, conj(q_out)).x, kin_p = n0 * n0 * q0.x;
    auto finish = [&](Cx<R> xs0, Cx<R> xs1, Cx<R> xp0, Cx<R> xp1, R Yt, int esx, int epx, R res[4]) {
        R u = R(-2.0 * kTwoPi * kLog2e) * Yt;
        u = fmax(u, R(-1.0e6));
        const R un = floor_w(u);
        const R yscale = exp2_w(u - un);
        const int yn = (int)un;
        const R Pst = Ps * (q0.x * q0.x);
        if (POL & 1) rt_of(xs0, xs1, Pst * yscale, e4 + eP + yn - 2 * esx, q_out.x, q0.x, res[0], res[1]);
        if (POL & 2) rt_of(xp0, xp1, Pst * Pp * yscale, e4 + eP + ePp + yn - 2 * epx, kout_p, kin_p, res[2], res[3]);
        if (grazing) res[0] = res[2] = R(1), res[1] = res[3] = R(0);
    };
    if (jp == 0) {
        if (POL & 1) interface_pair(q0, q_nx, s0, s1);
        if (POL & 2) interface_pair(g0, g_nx, p0, p1);
        finish(s0, s1, p0, p1, Y, es, ep, out);
        return;
    }
    // layer jp: its root and interface jp | jp+1; its phase waits for the nodes
    A = sa[jp * TL + tl];
    const Cx<R> qj = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
    Ps *= absz;
    Cx<R> gj = {R(0), R(0)};
    if (POL & 1) interface_pair(qj, q_nx, s0, s1);
    if (POL & 2) {
        Pp *= sb[jp * TL + tl].ain2;
        gj = cmul(qj, Cx<R>{A.in2x, A.in2y});
        interface_pair(gj, g_nx, p0, p1);
    }
    rescale();
    // the block left of layer jp: both columns of ML, from the identity
    Cx<R> sc00 = {R(1), R(0)}, sc10 = {R(0), R(0)}, sc01 = sc10, sc11 = sc00;
    Cx<R> pc00 = sc00, pc10 = sc10, pc01 = sc01, pc11 = sc11;
    int els = 0, elp = 0;
    Cx<R> qr = qj, gr = gj;
    cnt = 0;
    for (int j = jp - 1; j >= 1; --j) {
        A = sa[j * TL + tl];
        const StageB<R> B = sb[j * TL + tl];
        const Cx<R> q = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
        Ps *= absz;
        const Step<R> st = phase_of(B.dl, q, yi_max);
        Y += st.yi;
        if (POL & 1) {
            interface_pair(q, qr, sc00, sc10);
            interface_pair(q, qr, sc01, sc11);
            sc00 = cmul(st.emi, sc00), sc10 = cmul(st.epi, sc10);
            sc01 = cmul(st.emi, sc01), sc11 = cmul(st.epi, sc11);
        }
        if (POL & 2) {
            Pp *= B.ain2;
            const Cx<R> g = cmul(q, Cx<R>{A.in2x, A.in2y});
            interface_pair(g, gr, pc00, pc10);
            interface_pair(g, gr, pc01, pc11);
            pc00 = cmul(st.emi, pc00), pc10 = cmul(st.epi, pc10);
            pc01 = cmul(st.emi, pc01), pc11 = cmul(st.epi, pc11);
            gr = g;
        }
        qr = q;
        if (++cnt == RN) {
            cnt = 0;
            renorm_scalar(Ps, eP);
            if (POL & 2) renorm_scalar(Pp, ePp);
            if (POL & 1) {
                // one exponent for the whole matrix: renorm both columns together
                int k0 = 0, k1 = 0;
                Cx<R> a = sc00, b = sc10, c = sc01, d = sc11;
                renorm_pair(a, b, k0);
                renorm_pair(c, d, k1);
                const int k = max(k0, k1);
                const R f = pow2_neg<R>(k);
                sc00 = scale(f, sc00), sc10 = scale(f, sc10), sc01 = scale(f, sc01), sc11 = scale(f, sc11);
                els += k;
            }
            if (POL & 2) {
                int k0 = 0, k1 = 0;
                Cx<R> a = pc00, b = pc10, c = pc01, d = pc11;
                renorm_pair(a, b, k0);
                renorm_pair(c, d, k1);
                const int k = max(k0, k1);
                const R f = pow2_neg<R>(k);
                pc00 = scale(f, pc00), pc10 = scale(f, pc10), pc01 = scale(f, pc01), pc11 = scale(f, pc11);
                elp += k;
            }
        }
    }
    // interface 0 | 1
    if (POL & 1) {
        interface_pair(q0, qr, sc00, sc10);
        interface_pair(q0, qr, sc01, sc11);
    }
    if (POL & 2) {
        interface_pair(g0, gr, pc00, pc10);
        interface_pair(g0, gr, pc01, pc11);
    }
    // node-independent products: x_0 = (ML00 y0) e^{-i delta} + (ML01 y1) e^{+i delta}
    // (row 0), likewise row 1, with e^{+-i delta} the node's phase factors
    Cx<R> sA = {R(0), R(0)}, sB = sA, sC = sA, sD = sA, pA = sA, pB = sA, pC = sA, pD = sA;
    if (POL & 1) sA = cmul(sc00, s0), sB = cmul(sc01, s1), sC = cmul(sc10, s0), sD = cmul(sc11, s1);
    if (POL & 2) pA = cmul(pc00, p0), pB = cmul(pc01, p1), pC = cmul(pc10, p0), pD = cmul(pc11, p1);
    const Quad<R> fs0 = quad_of(sA, sB), fs1 = quad_of(sC, sD), fp0 = quad_of(pA, pB), fp1 = quad_of(pC, pD);
    // the nodes: layer jp's phase at thickness d_jp +- sqrt(2) sigma x_k.  A node's
    // R is |x_0[1]|^2 / |x_0[0]|^2; its T is a node-independent factor times
    // E / |x_0[0]|^2, so the sums carry w E / |x_0[0]|^2 and the factor (with the
    // dropped scales) is applied once.
    R aRs = R(0), aTs = R(0), aRp = R(0), aTp = R(0);
    auto node = [&](R c2, R s2, R E, R w) {
        if (POL & 1) {
            const R wr = w / quad_at(fs0, c2, s2, E);
            aRs = fma(wr, quad_at(fs1, c2, s2, E), aRs);
            aTs = fma(wr, E, aTs);
        }
        if (POL & 2) {
            const R wr = w / quad_at(fp0, c2, s2, E);
            aRp = fma(wr, quad_at(fp1, c2, s2, E), aRp);
            aTp = fma(wr, E, aTp);
        }
    };
    // While no node's thickness or Im(delta) is clamped, delta is linear in the
    // thickness: the nodes d_jp +- D turn the base (cos 2t_0, sin 2t_0) by
    // +-2 dt (angle addition, one sincos per pair) and scale E_0 by
    // e^{-+2 Im d delta}; otherwise each node's phase is taken on its own.
    const R dl0 = dj * inv_lam, dmax = sig * nd.off[0] * inv_lam;
    const bool rotate = dj >= sig * nd.off[0] && (dl0 + dmax) * qj.y <= yi_max;
    R C0, S0, E0;
    twice_phase(dl0, qj, yi_max, C0, S0, E0);
    for (int i = 0; i < nd.n_half; ++i) {
        const bool both = !(nd.odd && i == nd.n_half - 1);
        const R D = sig * nd.off[i], w = nd.w[i];
        if (rotate) {
            const R dl = D * inv_lam, y2 = R(2) * dl * qj.x;
            R sd, cd;
            sincos_turn(y2 - rint_w(y2), &sd, &cd);
            const R a = C0 * cd, b = S0 * sd, c = S0 * cd, d = C0 * sd;
            R Ep = E0, Em = E0;
            if (qj.y != R(0)) Ep *= exp_m2_turn(dl * qj.y), Em *= exp_m2_turn(-dl * qj.y);
            node(a - b, c + d, Ep, w);
            if (both) node(a + b, c - d, Em, w);
        } else {
            for (int sg = 0; sg < (both ? 2 : 1); ++sg) {
                R c2, s2, E;
                twice_phase(fmax(dj + (sg ? -D : D), R(0)) * inv_lam, qj, yi_max, c2, s2, E);
                node(c2, s2, E, w);
            }
        }
    }
    // T's factor: Eqs. 5-6 with the dropped scales, exp(-2 Im) of the other layers
    R u = R(-2.0 * kTwoPi * kLog2e) * Y;
    u = fmax(u, R(-1.0e6));
    const R un = floor_w(u);
    const R ys = Ps * (q0.x * q0.x) * exp2_w(u - un);
    const int yn = (int)un;
    out[0] = aRs;
    out[1] = q_out.x / q0.x * ldexp_w(ys * aTs, e4 + eP + yn - 2 * (es + els));
    out[2] = aRp;
    out[3] = kout_p / kin_p * ldexp_w(ys * Pp * aTp, e4 + eP + ePp + yn - 2 * (ep + elp));
    if (grazing) out[0] = out[2] = R(1), out[1] = out[3] = R(0);
}

// ---------------------------------------------------------------- FP32: two angles per thread

// Quad on the two lanes.
struct Quad2 {
    float2 a, b, cx, cy;
};
__device__ __forceinline__ Quad2 quad_of2(const C2 &A, const C2 &B)
{
    const float2 two = bc2(2.f);
    return Quad2{fma2(A.x, A.x, mul2(A.y, A.y)), fma2(B.x, B.x, mul2(B.y, B.y)),
                 mul2(two, fma2(A.x, B.x, mul2(A.y, B.y))), mul2(two, sub2(mul2(A.y, B.x), mul2(A.x, B.y)))};
}
__device__ __forceinline__ float2 quad_at2(const Quad2 &q, float2 c2, float2 s2, float2 E)
{
    return fma2(E, fma2(E, q.b, fma2(q.cx, c2, mul2(q.cy, s2))), q.a);
}

// pc_point for the two angles in the lanes of st, ct (see tmm_fwd.cu): the
// sweeps and the node products on paired lanes; the nodes' thicknesses are
// the same for both lanes.  out[lane][{R_s, T_s, R_p, T_p}].
template <int POL>
__device__ __forceinline__ void pc_point2(const StageA<float> *__restrict__ sa,
                                          const StageB<float> *__restrict__ sb, int TL, int tl, int L, int jp,
                                          float sig, float inv_lam, float dj, float n0, float2 st, float2 ct,
                                          const Nodes<float> &nd, float out[2][4])
{
    constexpr int RN = RenormEvery<float>::value;
    const float2 c0 = f2(n0 * ct.x, n0 * ct.y), q0sq = f2(c0.x * c0.x, c0.y * c0.y);
    const float yi_max = float(kImDeltaMax / kTwoPi);
    StageA<float> A = sa[(L + 1) * TL + tl];
    float absz;
    const Cx<float> qoa = forward_root(Cx<float>{A.d2x + q0sq.x, A.n2y}, &absz);
    const Cx<float> qob = forward_root(Cx<float>{A.d2x + q0sq.y, A.n2y}, &absz);
    const Cx<float> n2_out = {A.d2x + n0 * n0, A.n2y}, in2o = {A.in2x, A.in2y};
    C2 q_nx = pack2(qoa, qob), g_nx = pack2(cmul(qoa, in2o), cmul(qob, in2o));
    float2 nqy_nx = neg2(q_nx.y), ngy_nx = neg2(g_nx.y);
    float2 Ps = bc2(1.f), Y = bc2(0.f);
    float Pp = (POL & 2) ? sb[(L + 1) * TL + tl].ain2 : 1.f;
    int ePa = 0, ePb = 0, ePp = 0, esa = 0, esb = 0, epa = 0, epb = 0;
    C2 s0 = {bc2(1.f), bc2(0.f)}, s1 = {bc2(0.f), bc2(0.f)}, p0 = s0, p1 = s1;
    int cnt = 0;
    auto rescale = [&]() {
        renorm_scalar(Ps.x, ePa);
        renorm_scalar(Ps.y, ePb);
        if (POL & 2) renorm_scalar(Pp, ePp);
        if (POL & 1) renorm_pair2(s0, s1, esa, esb);
        if (POL & 2) renorm_pair2(p0, p1, epa, epb);
    };
    // right of the partial layer (the whole stack when jp = 0)
    for (int j = L; j > jp; --j) {
        A = sa[j * TL + tl];
        const StageB<float> B = sb[j * TL + tl];
        float absa, absb;
        const Cx<float> qa = inner_root(Cx<float>{A.d2x + q0sq.x, A.n2y}, &absa);
        const Cx<float> qb = inner_root(Cx<float>{A.d2x + q0sq.y, A.n2y}, &absb);
        Ps = mul2(Ps, f2(absa, absb));
        const Phase2 f = phase_pair(B.dl, qa, qb, yi_max);
        Y = add2(Y, f.yi);
        const C2 q = pack2(qa, qb);
        if (POL & 1) {
            const float2 nqy = neg2(q.y);
            interface_pair2(q, nqy, q_nx, nqy_nx, s0, s1);
            phase2(f.cs, f.sn, f.nsn, f.ec, f.es, f.nes, s0, s1);
            nqy_nx = nqy;
        }
        if (POL & 2) {
            Pp *= B.ain2;
            const Cx<float> in2 = {A.in2x, A.in2y};
            const C2 g = pack2(cmul(qa, in2), cmul(qb, in2));
            const float2 ngy = neg2(g.y);
            interface_pair2(g, ngy, g_nx, ngy_nx, p0, p1);
            phase2(f.cs, f.sn, f.nsn, f.ec, f.es, f.nes, p0, p1);
            g_nx = g;
            ngy_nx = ngy;
        }
        q_nx = q;
        if (++cnt == RN) {
            cnt = 0;
            rescale();
        }
    }
    const int e4 = 2 * (L + 1);
    const StageA<float> A0 = sa[tl];
    const Cx<float> in20 = {A0.in2x, A0.in2y};
    auto finish = [&](int i, Cx<float> xs0, Cx<float> xs1, Cx<float> xp0, Cx<float> xp1, float Yt, int esx,
                      int epx, float res[4]) {
        const float c0i = i ? c0.y : c0.x;
        const Cx<float> q_out = i ? qob : qoa;
        float u = float(-2.0 * kTwoPi * kLog2e) * Yt;
        u = fmaxf(u, -1.0e6f);
        const float un = floorf(u);
        const float yscale = exp2f(u - un);
        const int yn = (int)un;
        const float Pst = (i ? Ps.y : Ps.x) * (c0i * c0i);
        const int ePi = i ? ePb : ePa;
        if (POL & 1) rt_of(xs0, xs1, Pst * yscale, e4 + ePi + yn - 2 * esx, q_out.x, c0i, res[0], res[1]);
        if (POL & 2)
            rt_of(xp0, xp1, Pst * Pp * yscale, e4 + ePi + ePp + yn - 2 * epx, cmul(n2_out, conj(q_out)).x,
                  n0 * n0 * c0i, res[2], res[3]);
        if (n0 * (i ? st.y : st.x) >= n0) res[0] = res[2] = 1.f, res[1] = res[3] = 0.f;  // grazing
    };
    if (jp == 0) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const Cx<float> q0 = {i ? c0.y : c0.x, 0.f}, g0 = cmul(q0, in20);
            Cx<float> xs0 = lane(s0, i), xs1 = lane(s1, i), xp0 = lane(p0, i), xp1 = lane(p1, i);
            if (POL & 1) interface_pair(q0, lane(q_nx, i), xs0, xs1);
            if (POL & 2) interface_pair(g0, lane(g_nx, i), xp0, xp1);
            finish(i, xs0, xs1, xp0, xp1, i ? Y.y : Y.x, i ? esb : esa, i ? epb : epa, out[i]);
        }
        return;
    }
    // layer jp: its roots and interface jp | jp+1; its phase waits for the nodes
    A = sa[jp * TL + tl];
    float absa, absb;
    const Cx<float> qja = inner_root(Cx<float>{A.d2x + q0sq.x, A.n2y}, &absa);
    const Cx<float> qjb = inner_root(Cx<float>{A.d2x + q0sq.y, A.n2y}, &absb);
    Ps = mul2(Ps, f2(absa, absb));
    const C2 qj = pack2(qja, qjb);
    const float2 nqjy = neg2(qj.y);
    C2 gj = {bc2(0.f), bc2(0.f)};
    float2 ngjy = bc2(0.f);
    if (POL & 1) interface_pair2(qj, nqjy, q_nx, nqy_nx, s0, s1);
    if (POL & 2) {
        Pp *= sb[jp * TL + tl].ain2;
        const Cx<float> in2 = {A.in2x, A.in2y};
        gj = pack2(cmul(qja, in2), cmul(qjb, in2));
        ngjy = neg2(gj.y);
        interface_pair2(gj, ngjy, g_nx, ngy_nx, p0, p1);
    }
    rescale();
    // the block left of layer jp: both columns of ML, from the identity
    const C2 one = {bc2(1.f), bc2(0.f)}, zero = {bc2(0.f), bc2(0.f)};
    Cols2 cs{one, zero, zero, one}, cp{one, zero, zero, one};
    int elsa = 0, elsb = 0, elpa = 0, elpb = 0;
    C2 qr = qj, gr = gj;
    float2 nqry = nqjy, ngry = ngjy;
    cnt = 0;
    for (int j = jp - 1; j >= 1; --j) {
        A = sa[j * TL + tl];
        const StageB<float> B = sb[j * TL + tl];
        float aa, ab;
        const Cx<float> qa = inner_root(Cx<float>{A.d2x + q0sq.x, A.n2y}, &aa);
        const Cx<float> qb = inner_root(Cx<float>{A.d2x + q0sq.y, A.n2y}, &ab);
        Ps = mul2(Ps, f2(aa, ab));
        const Phase2 f = phase_pair(B.dl, qa, qb, yi_max);
        Y = add2(Y, f.yi);
        const C2 q = pack2(qa, qb);
        const float2 nqy = neg2(q.y);
        if (POL & 1) cols_step2(cs, q, nqy, qr, nqry, f);
        if (POL & 2) {
            Pp *= B.ain2;
            const Cx<float> in2 = {A.in2x, A.in2y};
            const C2 g = pack2(cmul(qa, in2), cmul(qb, in2));
            const float2 ngy = neg2(g.y);
            cols_step2(cp, g, ngy, gr, ngry, f);
            gr = g;
            ngry = ngy;
        }
        qr = q;
        nqry = nqy;
        if (++cnt == RN) {
            cnt = 0;
            renorm_scalar(Ps.x, ePa);
            renorm_scalar(Ps.y, ePb);
            if (POL & 2) renorm_scalar(Pp, ePp);
            if (POL & 1) renorm_cols2(cs, elsa, elsb);
            if (POL & 2) renorm_cols2(cp, elpa, elpb);
        }
    }
    // interface 0 | 1 (q_0 = n_0 cos(theta) real per lane)
    const C2 Q0 = {c0, bc2(0.f)};
    if (POL & 1) {
        interface_pair2(Q0, bc2(0.f), qr, nqry, cs.x0, cs.x1);
        interface_pair2(Q0, bc2(0.f), qr, nqry, cs.y0, cs.y1);
    }
    if (POL & 2) {
        const C2 G0 = pack2(cmul(Cx<float>{c0.x, 0.f}, in20), cmul(Cx<float>{c0.y, 0.f}, in20));
        interface_pair2(G0, neg2(G0.y), gr, ngry, cp.x0, cp.x1);
        interface_pair2(G0, neg2(G0.y), gr, ngry, cp.y0, cp.y1);
    }
    // node-independent products: row a of x_0 = (ML_a0 y0) e^{-i delta} + (ML_a1 y1) e^{+i delta},
    // reduced to the quadratic forms of |x_0[a]|^2 (see Quad)
    Quad2 fs0{}, fs1{}, fp0{}, fp1{};
    if (POL & 1) {
        const float2 n0y = neg2(s0.y), n1y = neg2(s1.y);
        const C2 sA = cmul2(cs.x0, s0, n0y), sB = cmul2(cs.y0, s1, n1y);
        const C2 sC = cmul2(cs.x1, s0, n0y), sD = cmul2(cs.y1, s1, n1y);
        fs0 = quad_of2(sA, sB), fs1 = quad_of2(sC, sD);
    }
    if (POL & 2) {
        const float2 n0y = neg2(p0.y), n1y = neg2(p1.y);
        const C2 pA = cmul2(cp.x0, p0, n0y), pB = cmul2(cp.y0, p1, n1y);
        const C2 pC = cmul2(cp.x1, p0, n0y), pD = cmul2(cp.y1, p1, n1y);
        fp0 = quad_of2(pA, pB), fp1 = quad_of2(pC, pD);
    }
    // the nodes (see pc_point): sums of w |x_0[1]|^2 / |x_0[0]|^2 and w E / |x_0[0]|^2
    float2 aRs = bc2(0.f), aTs = bc2(0.f), aRp = bc2(0.f), aTp = bc2(0.f);
    auto node = [&](float2 c2, float2 s2, float2 E, float w) {
        if (POL & 1) {
            const float2 x0 = quad_at2(fs0, c2, s2, E);
            const float2 wr = f2(w / x0.x, w / x0.y);
            aRs = fma2(wr, quad_at2(fs1, c2, s2, E), aRs);
            aTs = fma2(wr, E, aTs);
        }
        if (POL & 2) {
            const float2 x0 = quad_at2(fp0, c2, s2, E);
            const float2 wr = f2(w / x0.x, w / x0.y);
            aRp = fma2(wr, quad_at2(fp1, c2, s2, E), aRp);
            aTp = fma2(wr, E, aTp);
        }
    };
    const float dl0 = dj * inv_lam, dmax = sig * nd.off[0] * inv_lam;
    const bool rotate = dj >= sig * nd.off[0] && (dl0 + dmax) * fmaxf(qja.y, qjb.y) <= yi_max;
    const bool lossy = qja.y != 0.f || qjb.y != 0.f;
    float2 C0, S0, E0;
    twice_phase(dl0, qja, yi_max, C0.x, S0.x, E0.x);
    twice_phase(dl0, qjb, yi_max, C0.y, S0.y, E0.y);
    for (int i = 0; i < nd.n_half; ++i) {
        const bool both = !(nd.odd && i == nd.n_half - 1);
        const float D = sig * nd.off[i], w = nd.w[i];
        if (rotate) {
            const float dl = D * inv_lam;
            const float ya = 2.f * dl * qja.x, yb = 2.f * dl * qjb.x;
            float2 sd, cd;
            sincos_turn(ya - rintf(ya), &sd.x, &cd.x);
            sincos_turn(yb - rintf(yb), &sd.y, &cd.y);
            const float2 a = mul2(C0, cd), b = mul2(S0, sd), c = mul2(S0, cd), d = mul2(C0, sd);
            float2 Ep = E0, Em = E0;
            if (lossy) {  // a lossless layer's E is E_0 at every node
                const float2 ei = f2(dl * qja.y, dl * qjb.y);
                Ep = mul2(E0, f2(exp_m2_turn(ei.x), exp_m2_turn(ei.y)));
                Em = mul2(E0, f2(exp_m2_turn(-ei.x), exp_m2_turn(-ei.y)));
            }
            node(sub2(a, b), add2(c, d), Ep, w);
            if (both) node(add2(a, b), sub2(c, d), Em, w);
        } else {
            for (int sg = 0; sg < (both ? 2 : 1); ++sg) {
                const float dl = fmaxf(dj + (sg ? -D : D), 0.f) * inv_lam;
                float2 c2, s2, E;
                twice_phase(dl, qja, yi_max, c2.x, s2.x, E.x);
                twice_phase(dl, qjb, yi_max, c2.y, s2.y, E.y);
                node(c2, s2, E, w);
            }
        }
    }
#pragma unroll
    for (int ln = 0; ln < 2; ++ln) {
        const float c0i = ln ? c0.y : c0.x;
        const Cx<float> q_out = ln ? qob : qoa;
        float u = float(-2.0 * kTwoPi * kLog2e) * (ln ? Y.y : Y.x);
        u = fmaxf(u, -1.0e6f);
        const float un = floorf(u);
        const float ys = (ln ? Ps.y : Ps.x) * (c0i * c0i) * exp2f(u - un);
        const int e = e4 + (ln ? ePb : ePa) + (int)un;
        out[ln][0] = ln ? aRs.y : aRs.x;
        out[ln][1] = q_out.x / c0i * ldexpf(ys * (ln ? aTs.y : aTs.x), e - 2 * (ln ? esb + elsb : esa + elsa));
        out[ln][2] = ln ? aRp.y : aRp.x;
        out[ln][3] = cmul(n2_out, conj(q_out)).x / (n0 * n0 * c0i) *
                     ldexpf(ys * Pp * (ln ? aTp.y : aTp.x), e + ePp - 2 * (ln ? epb + elpb : epa + elpa));
        if (n0 * (ln ? st.y : st.x) >= n0) out[ln][0] = out[ln][2] = 1.f, out[ln][1] = out[ln][3] = 0.f;  // grazing
    }
}

template <typename R, int POL, bool WITH_T, bool PAIR>
__global__ void __launch_bounds__(kPcThreads, 2) tmm_pcoh_kernel(const tmm_problem p, const int32_t *__restrict__ layer,
                                                               const R *__restrict__ sigma, const Nodes<R> nd, int TL,
                                                               int TT, int n_lt, int n_tt, R *__restrict__ Rout,
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
    const int tid = threadIdx.y * TL + threadIdx.x, nthr = TL * (int)blockDim.y;
    const int L = layers_of(p, s);
    const int l0 = lt * TL;
    if (L >= 0) fill_stage<R>(p, s, L, l0, TL, sa, sb, n0s, tid, nthr);
    __syncthreads();
    const int tl = threadIdx.x, l = l0 + tl;
    const int t0 = ttile * TT, t_end = min(t0 + TT, p.n_theta);
    const int a0 = PAIR ? t0 + 2 * (int)threadIdx.y : t0 + (int)threadIdx.y;
    if (l >= p.n_lambda || a0 >= t_end) return;  // no barrier follows
    const int np = PAIR && a0 + 1 < t_end ? 2 : 1;

    R out[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i) out[i][0] = out[i][1] = out[i][2] = out[i][3] = nan_w<R>();
    const int jp = layer[s];
    const R sig = sigma[s];
    const bool valid = L >= 0 && jp >= 0 && jp <= L && sig >= R(0) && sig <= R(1e30);  // false for NaN
    if (valid) {
        const R *th = (const R *)p.theta;
        const R inv_lam = R(1) / ((const R *)p.lambda)[l];
        const R dj = jp >= 1 ? ((const R *)p.d)[(long long)s * p.L_max + (jp - 1)] : R(0);
        if constexpr (PAIR) {
            float2 st, ct;
            sincos_w(th[a0], &st.x, &ct.x);
            sincos_w(th[np == 2 ? a0 + 1 : a0], &st.y, &ct.y);
            pc_point2<POL>(sa, sb, TL, tl, L, jp, sig, inv_lam, dj, n0s[tl], st, ct, nd, out);
        } else {
            R sth, cth;
            sincos_w(th[a0], &sth, &cth);
            pc_point<R, POL>(sa, sb, TL, tl, L, jp, sig, inv_lam, dj, n0s[tl], sth, cth, nd, out[0]);
        }
    }
    const long long plane = (long long)p.S * p.n_theta * p.n_lambda;
    for (int i = 0; i < np; ++i) {
        const long long o = ((long long)s * p.n_theta + a0 + i) * p.n_lambda + l;
        if (POL & 4) {
            Rout[o] = R(0.5) * (out[i][0] + out[i][2]);
            if (WITH_T) Tout[o] = R(0.5) * (out[i][1] + out[i][3]);
        } else {
            int pi = 0;
            if (POL & 1) {
                Rout[o] = out[i][0];
                if (WITH_T) Tout[o] = out[i][1];
                ++pi;
            }
            if (POL & 2) {
                Rout[pi * plane + o] = out[i][2];
                if (WITH_T) Tout[pi * plane + o] = out[i][3];
            }
        }
    }
}

size_t pcoh_smem(const tmm_problem *p, int TL)
{
    const size_t r = real_size(p->prec);
    return (size_t)(p->L_max + 2) * TL * (6 * r) + (size_t)TL * r;
}

template <typename R, int POL, bool WITH_T, bool PAIR>
tmm_status launch_pcoh_shaped(const tmm_problem *p, const int32_t *layer, const R *sigma, const Nodes<R> &nd,
                              int TL, int TT, int n_lt, int n_tt, long long items, size_t smem, R *Ro, R *To,
                              cudaStream_t st)
{
    auto k = tmm_pcoh_kernel<R, POL, WITH_T, PAIR>;
    {
        const tmm_status ss = ensure_dynamic_smem(reinterpret_cast<const void *>(k), smem);
        if (ss != TMM_OK) return ss;
    }
    k<<<(unsigned)items, dim3(TL, PAIR ? (TT + 1) / 2 : TT), smem, st>>>(*p, layer, sigma, nd, TL, TT, n_lt, n_tt,
                                                                       Ro, To);
    return check_launch();
}

// FP32 tiles of two or more angles run two angles per thread.
template <typename R, int POL, bool WITH_T>
tmm_status launch_pcoh_k(const tmm_problem *p, const int32_t *layer, const R *sigma, const Nodes<R> &nd, int TL,
                         int TT, int n_lt, int n_tt, long long items, size_t smem, R *Ro, R *To, cudaStream_t st)
{
    if constexpr (std::is_same<R, float>::value) {
        if (TT >= 2)
            return launch_pcoh_shaped<R, POL, WITH_T, true>(p, layer, sigma, nd, TL, TT, n_lt, n_tt, items, smem, Ro,
                                                             To, st);
    }
    return launch_pcoh_shaped<R, POL, WITH_T, false>(p, layer, sigma, nd, TL, TT, n_lt, n_tt, items, smem, Ro, To,
                                                      st);
}

template <typename R>
tmm_status launch_pcoh_prec(const tmm_problem *p, const int32_t *layer, const void *sigma_, int K, int TL, int TT,
                            int n_lt, int n_tt, long long items, size_t smem, void *R_, void *T_, cudaStream_t st)
{
    const Nodes<R> nd = make_nodes<R>(K);
    const R *sigma = static_cast<const R *>(sigma_);
    R *Ro = static_cast<R *>(R_), *To = static_cast<R *>(T_);
    const bool wt = To != nullptr;
#define TMM_PC_CASE(P_)                                                                                          \
    case P_:                                                                                                     \
        return wt ? launch_pcoh_k<R, P_, true>(p, layer, sigma, nd, TL, TT, n_lt, n_tt, items, smem, Ro, To, st)  \
                  : launch_pcoh_k<R, P_, false>(p, layer, sigma, nd, TL, TT, n_lt, n_tt, items, smem, Ro, To, st);
    switch (p->pol_mask) {
        TMM_PC_CASE(1)
        TMM_PC_CASE(2)
        TMM_PC_CASE(3)
        TMM_PC_CASE(7)
    default: return TMM_ERR_INVALID_ARG;
    }
#undef TMM_PC_CASE
}

}  // namespace

}  // namespace tmm

using namespace tmm;

extern "C" TMM_API tmm_status tmm_pcoh_batched(const tmm_problem *p, const int32_t *layer, const void *sigma,
                                               int32_t n_nodes, void *R, void *T, void *stream)
{
    TraceRange trace("tmm_pcoh_batched");
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if (p->prec != TMM_F64 && p->prec != TMM_F32) return TMM_ERR_UNSUPPORTED;
    if (n_nodes < 1 || n_nodes > kPcMaxNodes) return TMM_ERR_INVALID_ARG;
    const long long pts = (long long)p->S * p->n_lambda * p->n_theta;
    if (pts == 0) return TMM_OK;
    if (!layer || !sigma || !R) return TMM_ERR_INVALID_ARG;
    if (pcoh_smem(p, 1) > kSmemBlockCeiling) return TMM_ERR_UNSUPPORTED;
    DeviceInfo di;
    s = device_info(&di);
    if (s != TMM_OK) return s;
    const int TT = std::min(p->n_theta, 32);
    const int rows = (p->prec == TMM_F32 && TT >= 2) ? (TT + 1) / 2 : TT;  // thread rows per block
    int TL = 1;
    while (TL * rows * 2 <= kPcThreads) TL *= 2;
    while (TL > 1 && TL / 2 >= p->n_lambda) TL /= 2;
    while (TL > 1 && pcoh_smem(p, TL) > (size_t)di.max_smem_optin) TL /= 2;
    const size_t smem = pcoh_smem(p, TL);
    if (smem > (size_t)di.max_smem_optin) return TMM_ERR_UNSUPPORTED;
    const int n_lt = (p->n_lambda + TL - 1) / TL, n_tt = (p->n_theta + TT - 1) / TT;
    const long long items = (long long)p->S * n_lt * n_tt;
    if (items > 0x7fffffffLL) return TMM_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return p->prec == TMM_F64
               ? launch_pcoh_prec<double>(p, layer, sigma, n_nodes, TL, TT, n_lt, n_tt, items, smem, R, T, st)
               : launch_pcoh_prec<float>(p, layer, sigma, n_nodes, TL, TT, n_lt, n_tt, items, smem, R, T, st);
}
