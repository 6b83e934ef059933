// tmm_field.cu -- field intensity profile inside every layer.
//
// |E(z) / E_inc|^2 at the depths z_k = (k + 1/2) d_j / n_z of every layer j,
// from the right-to-left sweep of the forward kernel (Eqs. 1-4).  In layer j
// the field is a forward wave a(z) = a_L e^{i kappa z} and a backward wave
// b(z) = b_R e^{i kappa (d - z)} (kappa = 2 pi q_j / lambda), each written
// from the boundary it decays away from: a_L is the sweep's forward amplitude
// at the left boundary (after the layer's phase), b_R its backward amplitude
// at the right boundary (before the phase).  Both are scaled amplitudes; the
// scalars dropped by the sweep are complex but common to the pair at each
// step, so with the incident amplitude set to 1 only their moduli enter:
//   |rho|^2 = 2^{LY - LY_0} (D_0 / D) / |x_0[0]|^2
// (D = prod 4 |k_i|^2 with the power-of-two rescalings, LY = sum of
// 2 Im(delta_i) log2(e) over the layers passed, both at the point where the
// amplitude was taken).  s: |E|^2 = |a + b|^2; p (H_y amplitudes):
// |E|^2 = (|q|^2 |a - b|^2 + beta^2 |a + b|^2) / |n|^4, times n_0^2 for the
// incident E = H / n_0.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "tmm_device.cuh"
#include "tmm_pair.cuh"
#include "tmm_internal.h"

namespace tmm {

namespace {

constexpr int kFieldThreads = 256;

// One polarisation's running sweep: the scaled amplitude pair and D as
// mantissa and exponent.
template <typename R> struct Wave {
    Cx<R> x0, x1;
    R m;
    int e;
};

// Layer j's amplitudes as the sweep passes it: the backward one at the right
// boundary (after interface j|j+1, before the phase) and the forward one at
// the left boundary (after the phase and any rescaling), each with the
// exponent of D where it was taken (the mantissa is the same at both).
template <typename R> struct Taken {
    Cx<R> bR, aL;
    R m;
    int eR, eL;
};

template <typename R> __device__ __forceinline__ void dmul_f(R &m, int &e, R v)
{
    m *= v;
    renorm_scalar(m, e);
}

// The right-to-left sweep from the substrate through interface 1|2 (Eqs. 1-4),
// calling visit(j, q_j, B_j, s amplitudes, p amplitudes, LY at the right
// boundary, LY at the left boundary) after each layer j = L .. 1.  Leaves the
// pairs and D ready for interface 0|1 and q_nx, g_nx those of layer 1.
template <typename R, int POL, typename Visit>
__device__ __forceinline__ void sweep_layers(const StageA<R> *sa, const StageB<R> *sb, int TL, int tl, int L,
                                             R q0sq, Wave<R> &ws, Wave<R> &wp, R &LY, Cx<R> &q_nx, Cx<R> &g_nx,
                                             Visit visit)
{
    constexpr int RN = RenormEvery<R>::value;
    const R yi_max = R(kImDeltaMax / kTwoPi);
    const R kLY = R(2.0 * kTwoPi * kLog2e);
    R absz;
    StageA<R> A = sa[(L + 1) * TL + tl];
    q_nx = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
    g_nx = cmul(q_nx, Cx<R>{A.in2x, A.in2y});
    ws = Wave<R>{{R(1), R(0)}, {R(0), R(0)}, R(1), 0};
    wp = ws;
    LY = R(0);
    int cnt = 0;
    for (int j = L; j >= 1; --j) {
        A = sa[j * TL + tl];
        const StageB<R> B = sb[j * TL + tl];
        const Cx<R> q = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
        const R yr = B.dl * q.x;
        const R yi = fmin(B.dl * q.y, yi_max);
        R sn, cs;
        sincos_turn(yr - rint_w(yr), &sn, &cs);
        const R E2 = exp_m2_turn(yi);
        const Cx<R> emi = {cs, -sn}, epi = {E2 * cs, E2 * sn};
        const Cx<R> g = cmul(q, Cx<R>{A.in2x, A.in2y});
        Taken<R> ts{}, tp{};
        if (POL & 1) {
            interface_pair(q, q_nx, ws.x0, ws.x1);
            dmul_f(ws.m, ws.e, R(4) * absz);
            ts.bR = ws.x1, ts.m = ws.m, ts.eR = ws.e;
            ws.x0 = cmul(emi, ws.x0);
            ws.x1 = cmul(epi, ws.x1);
        }
        if (POL & 2) {
            interface_pair(g, g_nx, wp.x0, wp.x1);
            dmul_f(wp.m, wp.e, R(4) * absz * B.ain2);
            tp.bR = wp.x1, tp.m = wp.m, tp.eR = wp.e;
            wp.x0 = cmul(emi, wp.x0);
            wp.x1 = cmul(epi, wp.x1);
        }
        const R lyR = LY;
        LY += kLY * yi;
        if (++cnt == RN) {
            cnt = 0;
            if (POL & 1) {
                int k = 0;
                renorm_pair(ws.x0, ws.x1, k);
                ws.e -= 2 * k;
            }
            if (POL & 2) {
                int k = 0;
                renorm_pair(wp.x0, wp.x1, k);
                wp.e -= 2 * k;
            }
        }
        if (POL & 1) ts.aL = ws.x0, ts.eL = ws.e;
        if (POL & 2) tp.aL = wp.x0, tp.eL = wp.e;
        visit(j, q, B, ts, tp, lyR, LY);
        q_nx = q;
        g_nx = g;
    }
}

// Two sweeps per thread: the first only carries the chain to interface 0|1
// for the incident amplitude x_0[0] and the final D and LY; the second
// repeats the same arithmetic and writes each layer's profile as it passes
// it.  Keeping the amplitudes of every layer instead (40 bytes per layer and
// polarisation and thread) spills to DRAM at this occupancy and costs more
// than the repeated sweep.  store(pi, j, kz, v) writes plane pi, layer j,
// depth kz of the point.
template <typename R, int POL, typename Store>
__device__ __forceinline__ void field_point(const StageA<R> *__restrict__ sa, const StageB<R> *__restrict__ sb,
                                            int TL, int tl, int L, int L_max, int n_z, R n0, R sth, R cth,
                                            Store store)
{
    const int nplanes = (POL & 4) ? 1 : ((POL & 1) + ((POL >> 1) & 1));
    const R beta = n0 * sth, c0 = n0 * cth, q0sq = c0 * c0;
    const bool grazing = beta >= n0;
    if (L < 0 || !(n0 == n0) || grazing) {
        // exact grazing: no field enters the stack
        const R fill = grazing ? R(0) : nan_w<R>();
        for (int pi = 0; pi < nplanes; ++pi)
            for (int j = 0; j < L_max; ++j)
                for (int kz = 0; kz < n_z; ++kz) store(pi, j, kz, (j < L || L < 0) ? fill : R(0));
        return;
    }
    Wave<R> ws, wp;
    R LY;
    Cx<R> q_nx, g_nx;
    sweep_layers<R, POL>(sa, sb, TL, tl, L, q0sq, ws, wp, LY, q_nx, g_nx,
                         [](int, const Cx<R> &, const StageB<R> &, const Taken<R> &, const Taken<R> &, R, R) {});
    // interface 0 | 1: the incident amplitude x_0[0]
    const StageA<R> A0 = sa[tl];
    const Cx<R> q0 = {c0, R(0)};
    const Cx<R> g0 = cmul(q0, Cx<R>{A0.in2x, A0.in2y});
    R pre[2] = {R(0), R(0)};
    int e0[2] = {0, 0};
    if (POL & 1) {
        interface_pair(q0, q_nx, ws.x0, ws.x1);
        dmul_f(ws.m, ws.e, R(4) * c0 * c0);
        pre[0] = ws.m / abs2(ws.x0);
        e0[0] = ws.e;
    }
    if (POL & 2) {
        interface_pair(g0, g_nx, wp.x0, wp.x1);
        dmul_f(wp.m, wp.e, R(4) * abs2(g0));
        pre[1] = wp.m / abs2(wp.x0) * n0 * n0;  // the incident E = H / n_0
        e0[1] = wp.e;
    }
    const R LY0 = LY;
    // |rho| of an amplitude taken at (m, e, ly)
    auto rho = [&](int k, R m, int e, R ly) {
        const R w = ly - LY0;  // <= 0
        const R wn = floor_w(w);
        return sqrt(ldexp_w(pre[k] / m * exp2_w(w - wn), e0[k] - e + (int)wn));
    };
    auto emit = [&](int j, const Cx<R> &q, const StageB<R> &Bj, const Taken<R> &ts, const Taken<R> &tp, R lyR,
                    R lyL) {
        const R n4 = R(1) / Bj.ain2;  // |n_j|^4
        Cx<R> fa[2], fb[2];
        if (POL & 1) {
            fa[0] = scale(rho(0, ts.m, ts.eL, lyL), ts.aL);
            fb[0] = scale(rho(0, ts.m, ts.eR, lyR), ts.bR);
        }
        if (POL & 2) {
            fa[1] = scale(rho(1, tp.m, tp.eL, lyL), tp.aL);
            fb[1] = scale(rho(1, tp.m, tp.eR, lyR), tp.bR);
        }
        // e^{i kappa z_k} (z_k = (k + 1/2) d / n_z) from the layer phase in
        // turns: modulus e^{-2 pi Im(y) f}, angle 2 pi Re(y) f with f = z / d
        const R yr = Bj.dl * q.x, yi = Bj.dl * q.y;
        auto depth_factor = [&](int k) {
            const R f = (R(k) + R(0.5)) / R(n_z);
            const R y = yr * f;
            R sn, cs;
            sincos_turn(y - rint_w(y), &sn, &cs);
            const R m = exp_m2_turn(R(0.5) * yi * f);
            return Cx<R>{m * cs, m * sn};
        };
        auto put = [&](int kz, const Cx<R> &ez, const Cx<R> &edz) {
            R v[2] = {R(0), R(0)};
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!(POL & (1 << k))) continue;
                const Cx<R> af = cmul(fa[k], ez), bf = cmul(fb[k], edz);
                v[k] = k == 0 ? abs2(af + bf) : (abs2(q) * abs2(af - bf) + beta * beta * abs2(af + bf)) / n4;
            }
            if (POL & 4) {
                store(0, j - 1, kz, R(0.5) * (v[0] + v[1]));
            } else {
                int pi = 0;
                if (POL & 1) store(pi++, j - 1, kz, v[0]);
                if (POL & 2) store(pi, j - 1, kz, v[1]);
            }
        };
        // d - z_k = z_{n_z-1-k}: the backward wave's factor e^{i kappa (d - z)}
        // at depth k is the forward wave's at depth n_z - 1 - k, so each
        // factor is computed once and the depths are taken in mirrored pairs
        for (int k = 0, kb = n_z - 1; k <= kb; ++k, --kb) {
            const Cx<R> e1 = depth_factor(k);
            if (k == kb) {
                put(k, e1, e1);
            } else {
                const Cx<R> e2 = depth_factor(kb);
                put(k, e1, e2);
                put(kb, e2, e1);
            }
        }
    };
    sweep_layers<R, POL>(sa, sb, TL, tl, L, q0sq, ws, wp, LY, q_nx, g_nx, emit);
    for (int pi = 0; pi < nplanes; ++pi)
        for (int j = L; j < L_max; ++j)
            for (int kz = 0; kz < n_z; ++kz) store(pi, j, kz, R(0));
}

template <typename R, int POL>
__global__ void __launch_bounds__(kFieldThreads) tmm_field_kernel(const tmm_problem p, int n_z, int TL, int TT,
                                                                  int n_lt, int n_tt, R *__restrict__ Eout)
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
    const long long zplane = (long long)n_z * tplane;             // one layer
    const long long splane = (long long)p.L_max * zplane;          // one stack
    const long long Ppol = (long long)p.S * splane;
    auto store = [&](int pi, int j, int kz, R v) {
        Eout[pi * Ppol + (long long)s * splane + (long long)j * zplane + (long long)kz * tplane + pt] = v;
    };
    const R n0 = L >= 0 ? n0s[tl] : nan_w<R>();
    R sth, cth;
    sincos_w(((const R *)p.theta)[a_], &sth, &cth);
    field_point<R, POL>(sa, sb, TL, tl, L, p.L_max, n_z, n0, sth, cth, store);
}

// ---------------------------------------------------------------- FP32: two angles per thread
// The forward kernel's paired lanes (see tmm_fwd.cu): amplitude pairs, the
// scalars D and LY per lane; roots and phase factors per lane.
struct Wave2 {
    C2 x0, x1;
    float2 m;   // mantissa of D per lane
    int ea, eb; // exponent of D per lane
};

struct Taken2 {
    C2 bR, aL;
    float2 m;
    int eRa, eRb, eLa, eLb;
};

template <int POL, typename Visit>
__device__ __forceinline__ void sweep_layers2(const StageA<float> *sa, const StageB<float> *sb, int TL, int tl,
                                              int L, float2 q0sq, Wave2 &ws, Wave2 &wp, float2 &LY, C2 &q_nx,
                                              C2 &g_nx, Visit visit)
{
    constexpr int RN = RenormEvery<float>::value;
    const float yi_max = float(kImDeltaMax / kTwoPi);
    const float kLY = float(2.0 * kTwoPi * kLog2e);
    float absz;
    StageA<float> A = sa[(L + 1) * TL + tl];
    const Cx<float> qoa = forward_root(Cx<float>{A.d2x + q0sq.x, A.n2y}, &absz);
    const Cx<float> qob = forward_root(Cx<float>{A.d2x + q0sq.y, A.n2y}, &absz);
    const Cx<float> in2o = {A.in2x, A.in2y};
    q_nx = pack2(qoa, qob);
    g_nx = pack2(cmul(qoa, in2o), cmul(qob, in2o));
    float2 nqy_nx = neg2(q_nx.y), ngy_nx = neg2(g_nx.y);
    ws = Wave2{{bc2(1.f), bc2(0.f)}, {bc2(0.f), bc2(0.f)}, bc2(1.f), 0, 0};
    wp = ws;
    LY = bc2(0.f);
    int cnt = 0;
    for (int j = L; j >= 1; --j) {
        A = sa[j * TL + tl];
        const StageB<float> B = sb[j * TL + tl];
        float absa, absb;
        const Cx<float> qa = inner_root(Cx<float>{A.d2x + q0sq.x, A.n2y}, &absa);
        const Cx<float> qb = inner_root(Cx<float>{A.d2x + q0sq.y, A.n2y}, &absb);
        const Phase2 f = phase_pair(B.dl, qa, qb, yi_max);
        const C2 q = pack2(qa, qb);
        Taken2 ts{}, tp{};
        if (POL & 1) {
            const float2 nqy = neg2(q.y);
            interface_pair2(q, nqy, q_nx, nqy_nx, ws.x0, ws.x1);
            ws.m = mul2(ws.m, f2(4.f * absa, 4.f * absb));
            renorm_scalar(ws.m.x, ws.ea);
            renorm_scalar(ws.m.y, ws.eb);
            ts.bR = ws.x1, ts.m = ws.m, ts.eRa = ws.ea, ts.eRb = ws.eb;
            phase2(f.cs, f.sn, f.nsn, f.ec, f.es, f.nes, ws.x0, ws.x1);
            nqy_nx = nqy;
        }
        if (POL & 2) {
            const Cx<float> in2 = {A.in2x, A.in2y};
            const C2 g = pack2(cmul(qa, in2), cmul(qb, in2));
            const float2 ngy = neg2(g.y);
            interface_pair2(g, ngy, g_nx, ngy_nx, wp.x0, wp.x1);
            wp.m = mul2(wp.m, f2(4.f * absa * B.ain2, 4.f * absb * B.ain2));
            renorm_scalar(wp.m.x, wp.ea);
            renorm_scalar(wp.m.y, wp.eb);
            tp.bR = wp.x1, tp.m = wp.m, tp.eRa = wp.ea, tp.eRb = wp.eb;
            phase2(f.cs, f.sn, f.nsn, f.ec, f.es, f.nes, wp.x0, wp.x1);
            g_nx = g;
            ngy_nx = ngy;
        }
        const float2 lyR = LY;
        LY = fma2(bc2(kLY), f.yi, LY);
        if (++cnt == RN) {
            cnt = 0;
            if (POL & 1) {
                int ka = 0, kb = 0;
                renorm_pair2(ws.x0, ws.x1, ka, kb);
                ws.ea -= 2 * ka, ws.eb -= 2 * kb;
            }
            if (POL & 2) {
                int ka = 0, kb = 0;
                renorm_pair2(wp.x0, wp.x1, ka, kb);
                wp.ea -= 2 * ka, wp.eb -= 2 * kb;
            }
        }
        if (POL & 1) ts.aL = ws.x0, ts.eLa = ws.ea, ts.eLb = ws.eb;
        if (POL & 2) tp.aL = wp.x0, tp.eLa = wp.ea, tp.eLb = wp.eb;
        visit(j, q, B, ts, tp, lyR, LY);
        q_nx = q;
    }
}

// field_point for two angles (neither at grazing incidence) in the lanes of
// st, ct; store(lane, pi, j, kz, v).
template <int POL, typename Store>
__device__ __forceinline__ void field_point2(const StageA<float> *__restrict__ sa,
                                             const StageB<float> *__restrict__ sb, int TL, int tl, int L, int L_max,
                                             int n_z, float n0, float2 st, float2 ct, Store store)
{
    const int nplanes = (POL & 4) ? 1 : ((POL & 1) + ((POL >> 1) & 1));
    const float2 c0 = f2(n0 * ct.x, n0 * ct.y), q0sq = f2(c0.x * c0.x, c0.y * c0.y);
    const float2 beta2 = f2(n0 * st.x * (n0 * st.x), n0 * st.y * (n0 * st.y));
    Wave2 ws, wp;
    float2 LY;
    C2 q_nx, g_nx;
    sweep_layers2<POL>(sa, sb, TL, tl, L, q0sq, ws, wp, LY, q_nx, g_nx,
                       [](int, const C2 &, const StageB<float> &, const Taken2 &, const Taken2 &, float2, float2) {});
    // interface 0 | 1 per lane: the incident amplitudes
    const StageA<float> A0 = sa[tl];
    const Cx<float> in20 = {A0.in2x, A0.in2y};
    float pre[2][2] = {};
    int e0[2][2] = {};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float c0i = i ? c0.y : c0.x;
        const Cx<float> q0 = {c0i, 0.f}, g0 = cmul(q0, in20);
        if (POL & 1) {
            Cx<float> x0 = lane(ws.x0, i), x1 = lane(ws.x1, i);
            interface_pair(q0, lane(q_nx, i), x0, x1);
            float m = i ? ws.m.y : ws.m.x;
            int e = i ? ws.eb : ws.ea;
            dmul_f(m, e, 4.f * c0i * c0i);
            pre[i][0] = m / abs2(x0);
            e0[i][0] = e;
        }
        if (POL & 2) {
            Cx<float> x0 = lane(wp.x0, i), x1 = lane(wp.x1, i);
            interface_pair(g0, lane(g_nx, i), x0, x1);
            float m = i ? wp.m.y : wp.m.x;
            int e = i ? wp.eb : wp.ea;
            dmul_f(m, e, 4.f * abs2(g0));
            pre[i][1] = m / abs2(x0) * n0 * n0;  // the incident E = H / n_0
            e0[i][1] = e;
        }
    }
    const float2 LY0 = LY;
    auto rho = [&](int i, int k, float m, int e, float ly) {
        const float w = ly - (i ? LY0.y : LY0.x);  // <= 0
        const float wn = floorf(w);
        return sqrtf(ldexpf(pre[i][k] / m * exp2f(w - wn), e0[i][k] - e + (int)wn));
    };
    auto emit = [&](int j, const C2 &q, const StageB<float> &Bj, const Taken2 &ts, const Taken2 &tp, float2 lyR,
                    float2 lyL) {
        C2 fa[2], fb[2];
        auto scaled = [](float2 r, const C2 &a) { return C2{mul2(r, a.x), mul2(r, a.y)}; };
        // the two amplitudes of a layer share the mantissa of D; their scales
        // differ by the layer's phase division (lyL - lyR) and rescaling
        // (eR - eL, even): |rho_L| = |rho_R| 2^{((lyL - lyR) + (eR - eL)) / 2}
        const float2 dly = sub2(lyL, lyR);
        if (POL & 1) {
            const float2 rR = f2(rho(0, 0, ts.m.x, ts.eRa, lyR.x), rho(1, 0, ts.m.y, ts.eRb, lyR.y));
            const float2 rL = mul2(rR, f2(exp2f(0.5f * (dly.x + float(ts.eRa - ts.eLa))),
                                          exp2f(0.5f * (dly.y + float(ts.eRb - ts.eLb)))));
            fa[0] = scaled(rL, ts.aL);
            fb[0] = scaled(rR, ts.bR);
        }
        if (POL & 2) {
            const float2 rR = f2(rho(0, 1, tp.m.x, tp.eRa, lyR.x), rho(1, 1, tp.m.y, tp.eRb, lyR.y));
            const float2 rL = mul2(rR, f2(exp2f(0.5f * (dly.x + float(tp.eRa - tp.eLa))),
                                          exp2f(0.5f * (dly.y + float(tp.eRb - tp.eLb)))));
            fa[1] = scaled(rL, tp.aL);
            fb[1] = scaled(rR, tp.bR);
        }
        const float2 yr = mul2(bc2(Bj.dl), q.x), yi = mul2(bc2(Bj.dl), q.y);
        const float2 aq2 = fma2(q.x, q.x, mul2(q.y, q.y));
        auto depth_factor = [&](int k) {
            const float f = (float(k) + 0.5f) / float(n_z);
            const float2 y = mul2(yr, bc2(f));
            float2 sn, cs;
            sincos_turn(y.x - rintf(y.x), &sn.x, &cs.x);
            sincos_turn(y.y - rintf(y.y), &sn.y, &cs.y);
            const float2 h = mul2(mul2(bc2(0.5f), yi), bc2(f));
            const float2 m = f2(exp_m2_turn(h.x), exp_m2_turn(h.y));
            return C2{mul2(m, cs), mul2(m, sn)};
        };
        auto put = [&](int kz, const C2 &ez, const C2 &edz) {
            const float2 nezy = neg2(ez.y), nedzy = neg2(edz.y);
            float2 v[2] = {bc2(0.f), bc2(0.f)};
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!(POL & (1 << k))) continue;
                const C2 af = cmul2(fa[k], ez, nezy), bf = cmul2(fb[k], edz, nedzy);
                const C2 sm = {add2(af.x, bf.x), add2(af.y, bf.y)};
                const float2 as = fma2(sm.x, sm.x, mul2(sm.y, sm.y));
                if (k == 0) {
                    v[0] = as;
                } else {
                    const C2 df = {sub2(af.x, bf.x), sub2(af.y, bf.y)};
                    const float2 ad = fma2(df.x, df.x, mul2(df.y, df.y));
                    v[1] = mul2(fma2(aq2, ad, mul2(beta2, as)), bc2(Bj.ain2));  // / |n_j|^4
                }
            }
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const float vs = i ? v[0].y : v[0].x, vp = i ? v[1].y : v[1].x;
                if (POL & 4) {
                    store(i, 0, j - 1, kz, 0.5f * (vs + vp));
                } else {
                    int pi = 0;
                    if (POL & 1) store(i, pi++, j - 1, kz, vs);
                    if (POL & 2) store(i, pi, j - 1, kz, vp);
                }
            }
        };
        for (int k = 0, kb = n_z - 1; k <= kb; ++k, --kb) {
            const C2 e1 = depth_factor(k);
            if (k == kb) {
                put(k, e1, e1);
            } else {
                const C2 e2 = depth_factor(kb);
                put(k, e1, e2);
                put(kb, e2, e1);
            }
        }
    };
    sweep_layers2<POL>(sa, sb, TL, tl, L, q0sq, ws, wp, LY, q_nx, g_nx, emit);
#pragma unroll
    for (int i = 0; i < 2; ++i)
        for (int pi = 0; pi < nplanes; ++pi)
            for (int j = L; j < L_max; ++j)
                for (int kz = 0; kz < n_z; ++kz) store(i, pi, j, kz, 0.f);
}

// FP32 with two angles per thread: TL x ceil(TT / 2) threads; a thread whose
// angles meet grazing incidence, or whose stack is invalid, takes the
// one-angle path per lane.
template <int POL>
__global__ void __launch_bounds__(kFieldThreads) tmm_field_kernel2(const tmm_problem p, int n_z, int TL, int TT,
                                                                   int n_lt, int n_tt, float *__restrict__ Eout)
{
    extern __shared__ __align__(16) unsigned char smem[];
    StageA<float> *sa = reinterpret_cast<StageA<float> *>(smem);
    StageB<float> *sb = reinterpret_cast<StageB<float> *>(sa + (size_t)(p.L_max + 2) * TL);
    float *n0s = reinterpret_cast<float *>(sb + (size_t)(p.L_max + 2) * TL);

    const long long item = blockIdx.x;
    const int per_stack = n_lt * n_tt;
    const int s = (int)(item / per_stack);
    const int rr = (int)(item - (long long)s * per_stack);
    const int lt = rr / n_tt, ttile = rr % n_tt;
    const int tid = threadIdx.y * TL + threadIdx.x, nthr = TL * (int)blockDim.y;
    const int L = layers_of(p, s);
    const int l0 = lt * TL;
    if (L >= 0) fill_stage<float>(p, s, L, l0, TL, sa, sb, n0s, tid, nthr);
    __syncthreads();
    const int tl = threadIdx.x, l = l0 + tl;
    const int t0 = ttile * TT, t_end = min(t0 + TT, p.n_theta);
    const int a0 = t0 + 2 * (int)threadIdx.y;
    if (l >= p.n_lambda || a0 >= t_end) return;  // no barrier follows
    const int np = a0 + 1 < t_end ? 2 : 1;

    const long long tplane = (long long)p.n_theta * p.n_lambda;
    const long long zplane = (long long)n_z * tplane;
    const long long splane = (long long)p.L_max * zplane;
    const long long Ppol = (long long)p.S * splane;
    const long long pt0 = (long long)a0 * p.n_lambda + l;
    auto store2 = [&](int i, int pi, int j, int kz, float v) {
        if (i < np)
            Eout[pi * Ppol + (long long)s * splane + (long long)j * zplane + (long long)kz * tplane + pt0 +
                 (long long)i * p.n_lambda] = v;
    };
    const float n0 = L >= 0 ? n0s[tl] : nan_w<float>();
    const float *th = (const float *)p.theta;
    float2 st, ct;
    sincos_w(th[a0], &st.x, &ct.x);
    sincos_w(th[np == 2 ? a0 + 1 : a0], &st.y, &ct.y);
    if (L < 0 || !(n0 == n0) || n0 * st.x >= n0 || n0 * st.y >= n0) {
        for (int i = 0; i < np; ++i)
            field_point<float, POL>(sa, sb, TL, tl, L, p.L_max, n_z, n0, i ? st.y : st.x, i ? ct.y : ct.x,
                                    [&](int pi, int j, int kz, float v) { store2(i, pi, j, kz, v); });
        return;
    }
    field_point2<POL>(sa, sb, TL, tl, L, p.L_max, n_z, n0, st, ct, store2);
}

size_t field_smem(const tmm_problem *p, int TL)
{
    const size_t r = real_size(p->prec);
    return (size_t)(p->L_max + 2) * TL * (6 * r) + (size_t)TL * r;
}

// One instantiation per kernel, so that each keeps its own attribute cache.
template <typename Out, void (*k)(const tmm_problem, int, int, int, int, int, Out *)>
tmm_status launch_field_with(const tmm_problem *p, int n_z, int TL, int TT, int rows, int n_lt, int n_tt,
                             long long items, size_t smem, Out *E, cudaStream_t st)
{
    {
        const tmm_status ss = ensure_dynamic_smem(reinterpret_cast<const void *>(k), smem);
        if (ss != TMM_OK) return ss;
    }
    k<<<(unsigned)items, dim3(TL, rows), smem, st>>>(*p, n_z, TL, TT, n_lt, n_tt, E);
    return check_launch();
}

// FP32 tiles of two or more angles run two angles per thread.
template <typename R, int POL>
tmm_status launch_field_k(const tmm_problem *p, int n_z, int TL, int TT, int n_lt, int n_tt, long long items,
                          size_t smem, R *E, cudaStream_t st)
{
    if constexpr (std::is_same<R, float>::value) {
        if (TT >= 2)
            return launch_field_with<float, tmm_field_kernel2<POL>>(p, n_z, TL, TT, (TT + 1) / 2, n_lt, n_tt, items,
                                                                    smem, E, st);
    }
    return launch_field_with<R, tmm_field_kernel<R, POL>>(p, n_z, TL, TT, TT, n_lt, n_tt, items, smem, E, st);
}

template <typename R>
tmm_status launch_field_prec(const tmm_problem *p, int n_z, int TL, int TT, int n_lt, int n_tt, long long items,
                             size_t smem, void *E_, cudaStream_t st)
{
    R *E = static_cast<R *>(E_);
    switch (p->pol_mask) {
    case 1: return launch_field_k<R, 1>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st);
    case 2: return launch_field_k<R, 2>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st);
    case 3: return launch_field_k<R, 3>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st);
    case 7: return launch_field_k<R, 7>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st);
    default: return TMM_ERR_INVALID_ARG;
    }
}

}  // namespace

}  // namespace tmm

using namespace tmm;

extern "C" TMM_API tmm_status tmm_field_profile(const tmm_problem *p, int32_t n_z, void *E, void *stream)
{
    TraceRange trace("tmm_field_profile");
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if (p->prec != TMM_F64 && p->prec != TMM_F32) return TMM_ERR_UNSUPPORTED;
    if (n_z < 1) return TMM_ERR_INVALID_ARG;
    const long long pts = (long long)p->S * p->n_lambda * p->n_theta;
    if (pts == 0 || p->L_max == 0) return TMM_OK;
    if (!E) return TMM_ERR_INVALID_ARG;
    if (field_smem(p, 1) > kSmemBlockCeiling) return TMM_ERR_UNSUPPORTED;
    DeviceInfo di;
    s = device_info(&di);
    if (s != TMM_OK) return s;
    const int TT = std::min(p->n_theta, 32);
    const int rows = (p->prec == TMM_F32 && TT >= 2) ? (TT + 1) / 2 : TT;  // thread rows per block
    int TL = 1;
    while (TL * rows * 2 <= kFieldThreads) TL *= 2;
    while (TL > 1 && TL / 2 >= p->n_lambda) TL /= 2;
    while (TL > 1 && field_smem(p, TL) > (size_t)di.max_smem_optin) TL /= 2;
    const size_t smem = field_smem(p, TL);
    if (smem > (size_t)di.max_smem_optin) return TMM_ERR_UNSUPPORTED;
    const int n_lt = (p->n_lambda + TL - 1) / TL, n_tt = (p->n_theta + TT - 1) / TT;
    const long long items = (long long)p->S * n_lt * n_tt;
    if (items > 0x7fffffffLL) return TMM_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return p->prec == TMM_F64 ? launch_field_prec<double>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st)
                              : launch_field_prec<float>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st);
}
