// tmm_fwd_df64.cu -- the forward transfer-matrix kernel in double-float
// arithmetic (TMM_F64X): FP64 inputs and outputs, FP64-level accuracy, the
// arithmetic on the FP32 pipes (see tmm_df64.cuh).
//
// Same method and layout as tmm_fwd.cu (one thread per (stack, lambda,
// theta), or per pair of angles on paired FP32 lanes; both polarisations,
// right-to-left 2-vector sweep of Eq. 3 with unnormalised interfaces, phase
// applied divided by e^{Im delta}, power-of-two rescaling every two layers).  Transcendentals:
//   sin, cos of 2 pi f: f = j/256 + r, |r| <= 1/512; Taylor series of
//     sin, cos (2 pi r) to x^5 / x^6, recombined with a table of
//     sin, cos(2 pi k / 256) by the angle-addition formulas (the paired
//     sweep: j/1024, a whole-turn table, shorter series);
//   2^v: v = n + i/64 + s, |s| <= 1/128; Taylor series of e^{s ln 2} to s^5,
//     times a table of 2^{i/64}, times 2^n;
//   square roots: Karp-Markstein correction of the float reciprocal root.
// The tables are computed on the host in double precision and passed with
// the launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "tmm_device.cuh"
#include "tmm_df64.cuh"
#include "tmm_df64x2.cuh"
#include "tmm_internal.h"

namespace tmm {

using df::cdd;
using df::dd;

namespace {

constexpr int kDfMaxThreads = 512;
constexpr int kDfPairThreads = 256;

constexpr int kFine = 1024;  // entries of the whole-turn table of the paired sweep

struct DfTables {
    float4 sc[64];     // {sin hi, sin lo, cos hi, cos lo} of 2 pi k / 256, k < 64 (sincos_turn_dd)
    float4 sf[kFine];  // the same of 2 pi k / 1024 over the whole turn (sincos_turn_dd2)
    float2 e2[65];     // 2^{i/64}, i = -32 .. 32
};

// per (medium, wavelength): n^2 - n0^2, Im n^2, 1/n^2, d/lambda, |1/n^2|^2
struct __align__(16) DStage {
    float d2h, d2l, n2yh, n2yl;
    float in2xh, in2xl, in2yh, in2yl;
    float dlh, dll, ain2h, ain2l;
};

// 2^v as m * 2^n with m a dd in [2^-0.5, 2^0.5]
__device__ __forceinline__ dd exp2_dd(dd v, const float2 *tab, int *n_out)
{
    const float nf = rintf(v.hi);
    const dd r = df::add_f(v, -nf);
    const float i_f = rintf(__fmul_rn(r.hi, 64.0f));
    const dd s = df::add_f(r, -__fmul_rn(i_f, 1.0f / 64.0f));
    const dd t = df::mul(s, dconst(0.69314718055994530941723212145818));
    const dd t2 = df::sqr(t);
    const dd t3_6 = df::mul(t2, df::mul(t, dconst(1.0 / 6.0)));
    const float t4 = __fmul_rn(t2.hi, t2.hi);
    const float tail = __fadd_rn(__fmul_rn(t4, 1.0f / 24.0f), __fmul_rn(__fmul_rn(t4, t.hi), 1.0f / 120.0f));
    dd p = df::add(df::make(1.0f), t);
    p = df::add(p, df::scale2(t2, 0.5f));
    p = df::add(p, t3_6);
    p = df::add_f(p, tail);
    const float2 e = tab[(int)i_f + 32];
    *n_out = (int)nf;
    return df::mul(p, dd{e.x, e.y});
}

__device__ __forceinline__ bool dd_less(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ dd dd_abs(dd a) { return a.hi < 0.0f ? df::neg(a) : a; }

// forward root q = sqrt(z) (decaying / propagating choice) and |z|
__device__ __forceinline__ cdd root_dd(cdd z, dd *absz)
{
    const dd hyp = df::cabs2(z);
    cdd q{dd{0.0f, 0.0f}, dd{0.0f, 0.0f}};
    dd az{0.0f, 0.0f};
    if (!(hyp.hi <= 0.0f)) {
        dd rh;
        df::sqrt_rsqrt(hyp, &az, &rh);
        const dd u = df::scale2(df::add(az, dd_abs(z.x)), 0.5f);
        dd t, ru;
        df::sqrt_rsqrt(u, &t, &ru);
        const dd o = df::scale2(df::mul(z.y, ru), 0.5f);
        if (z.x.hi >= 0.0f) {
            q = cdd{t, o};
        } else {
            q = cdd{dd_abs(o), z.y.hi < 0.0f || (z.y.hi == 0.0f && signbit(z.y.hi)) ? df::neg(t) : t};
        }
        // decaying root unless Im q is zero to rounding (|Im q| <= 100 * 2^-46 |q|)
        const float tol = 100.0f * 1.4210855e-14f;
        if (q.y.hi < 0.0f && q.y.hi * q.y.hi > tol * tol * az.hi) q = cdd{df::neg(q.x), df::neg(q.y)};
    }
    *absz = az;
    return q;
}

__device__ __forceinline__ void renorm_dd_pair(cdd &a, cdd &b, int &e)
{
    const float m = fmaxf(fmaxf(fabsf(a.x.hi), fabsf(a.y.hi)), fmaxf(fabsf(b.x.hi), fabsf(b.y.hi)));
    const int k = exponent_of(m);
    const float s = pow2_neg<float>(k);
    a = cdd{df::scale2(a.x, s), df::scale2(a.y, s)};
    b = cdd{df::scale2(b.x, s), df::scale2(b.y, s)};
    e += k;
}

__device__ __forceinline__ void renorm_dd(dd &m, int &e)
{
    const int k = exponent_of(m.hi);
    m = df::scale2(m, pow2_neg<float>(k));
    e += k;
}

__device__ __forceinline__ cdd ld_c(float h1, float l1, float h2, float l2) { return cdd{dd{h1, l1}, dd{h2, l2}}; }

// Interface 0 | 1 and Eqs. 5-6 for one point from the sweep's state after
// layer 1 (the dd form of tmm_fwd.cu's finish_point).
template <int POL>
__device__ __forceinline__ void finish_dd(const DStage &A, const float2 *e2, const cdd &q_out, const cdd &n2_out,
                                          const cdd &q_nx, const cdd &g_nx, const cdd &s0, const cdd &s1,
                                          const cdd &p0, const cdd &p1, dd Ps, int eP, dd Y, int es, int ep, int L,
                                          dd n0, dd cth, dd beta, dd c0, dd q0sq, dd Pp, int Pp_e, double out[4])
{
    // grazing: cos(theta) <= 0 or beta >= n_0 (both false for a NaN n_0)
    const bool grazing = cth.hi <= 0.0f || (!dd_less(beta, n0) && beta.hi == beta.hi);
    const cdd q0{c0, df::make(0.0f)};
    Ps = df::mul(Ps, q0sq);
    const int e4 = 2 * (L + 1);
    // 2^{-2 K Y} split as m * 2^n
    int yn;
    const dd ym = exp2_dd(df::mul(Y, dconst(-4.0 * kPi * 1.4426950408889634073599246810019)), e2, &yn);
    const double ys = df::to_double(ym);
    if (POL & 1) {
        cdd x0 = s0, x1 = s1;
        df::interface_pair(q0, q_nx, x0, x1);
        const dd ax0 = df::cabs2(x0);
        double Rv = df::to_double(df::div(df::cabs2(x1), ax0));
        double Tv = df::to_double(df::div(df::mul(q_out.x, Ps), df::mul(q0.x, ax0)));
        Tv = ldexp(Tv * ys, e4 + eP + yn - 2 * es);
        if (grazing) { Rv = 1.0; Tv = 0.0; }
        out[0] = Rv;
        out[1] = Tv;
    }
    if (POL & 2) {
        const cdd g0 = df::cmul(q0, ld_c(A.in2xh, A.in2xl, A.in2yh, A.in2yl));
        cdd x0 = p0, x1 = p1;
        df::interface_pair(g0, g_nx, x0, x1);
        const dd ax0 = df::cabs2(x0);
        double Rv = df::to_double(df::div(df::cabs2(x1), ax0));
        // Re(n_out^2 conj(q_out)) / (n_0^2 q_0)
        const dd num = df::dot2(n2_out.x, q_out.x, n2_out.y, q_out.y, 1.0f);
        const dd den = df::mul(df::sqr(n0), q0.x);
        double Tv = df::to_double(df::div(df::mul(num, df::mul(Ps, Pp)), df::mul(den, ax0)));
        Tv = ldexp(Tv * ys, e4 + eP + Pp_e + yn - 2 * ep);
        if (grazing) { Rv = 1.0; Tv = 0.0; }
        out[2] = Rv;
        out[3] = Tv;
    }
}

template <int POL>
__device__ __forceinline__ void eval_point_dd(const DStage *__restrict__ st, const float4 *sc, const float2 *e2, int TL,
                                              int tl, int L, dd n0, dd sth, dd cth, dd Pp, int Pp_e, double out[4])
{
    const dd beta = df::mul(n0, sth);
    const dd c0 = df::mul(n0, cth);
    const dd q0sq = df::sqr(c0);
    const dd yi_max = dconst(35.0 / (2.0 * kPi));

    DStage A = st[(L + 1) * TL + tl];
    dd absz;
    cdd q_nx = root_dd(cdd{df::add(dd{A.d2h, A.d2l}, q0sq), dd{A.n2yh, A.n2yl}}, &absz);
    const cdd q_out = q_nx;
    const cdd n2_out{df::add(dd{A.d2h, A.d2l}, df::sqr(n0)), dd{A.n2yh, A.n2yl}};
    cdd g_nx = df::cmul(q_nx, ld_c(A.in2xh, A.in2xl, A.in2yh, A.in2yl));
    dd Ps = df::make(1.0f), Y = df::make(0.0f);
    int eP = 0;
    const cdd one{df::make(1.0f), df::make(0.0f)}, zero{df::make(0.0f), df::make(0.0f)};
    cdd s0 = one, s1 = zero, p0 = one, p1 = zero;
    int es = 0, ep = 0;

    for (int j = L; j >= 1; --j) {
        A = st[j * TL + tl];
        const cdd q = root_dd(cdd{df::add(dd{A.d2h, A.d2l}, q0sq), dd{A.n2yh, A.n2yl}}, &absz);
        Ps = df::mul(Ps, absz);
        const dd dl{A.dlh, A.dll};
        const dd yr = df::mul(dl, q.x);
        dd yi = df::mul(dl, q.y);
        if (dd_less(yi_max, yi)) yi = yi_max;
        Y = df::add(Y, yi);
        dd sn, cs;
        sincos_turn_dd(df::add_f(yr, -rintf(yr.hi)), sc, &sn, &cs);
        int n2;
        const dd m2 = exp2_dd(df::mul(yi, dconst(-4.0 * kPi * 1.4426950408889634073599246810019)), e2, &n2);
        const dd E2 = df::scale2(m2, ldexpf(1.0f, n2));
        const cdd emi{cs, df::neg(sn)};
        const cdd epi{df::mul(E2, cs), df::mul(E2, sn)};
        if (POL & 1) {
            df::interface_pair(q, q_nx, s0, s1);
            s0 = df::cmul(emi, s0);
            s1 = df::cmul(epi, s1);
        }
        if (POL & 2) {
            const cdd g = df::cmul(q, ld_c(A.in2xh, A.in2xl, A.in2yh, A.in2yl));
            df::interface_pair(g, g_nx, p0, p1);
            p0 = df::cmul(emi, p0);
            p1 = df::cmul(epi, p1);
            g_nx = g;
        }
        q_nx = q;
        if (((L - j) & 1) == 1) {
            renorm_dd(Ps, eP);
            if (POL & 1) renorm_dd_pair(s0, s1, es);
            if (POL & 2) renorm_dd_pair(p0, p1, ep);
        }
    }
    finish_dd<POL>(st[tl], e2, q_out, n2_out, q_nx, g_nx, s0, s1, p0, p1, Ps, eP, Y, es, ep, L, n0, cth, beta, c0,
                   q0sq, Pp, Pp_e, out);
}

// ---------------------------------------------------------------- two angles per thread
// eval_point_dd for two angles of one wavelength on the lanes of the paired
// FP32 instructions (tmm_df64x2.cuh): the sweep, roots, phase factors and
// renormalisation per lane in dd2 arithmetic; table lookups and branch
// choices per lane by selects; interface 0 | 1 and R, T per lane in dd.
using df2::cdd2;
using df2::dd2;

// sin and cos of 2 pi y per lane for a phase y in turns: y = n + m/1024 + r
// with n = rint(y.hi), m = rint(1024 (y.hi - n)) and r = ((y.hi - n) - m/1024)
// + y.lo.  Both float differences are exact (Sterbenz: the operands lie within
// a factor of two of each other, or the subtrahend is 0), so the reduction
// takes no error-free transformation; |r.hi| <= 1/2048 and r is an
// unnormalised pair.  With x = 2 pi r, |x| <= pi/1024:
//   sin x = x - x e, e = x^2/6 - x^4/120 < 1.6e-6, so e and x e are formed in
//     float (their roundings move sin x by less than 2^-50);
//   cos x = 1 - x^2/2 + x^4/24 with x^2 as a float pair and x^4/24 < 3.7e-12
//     in float (the next term, x^6/720, is below 2^-60);
// then the angle-addition formulas with the table entry of m mod 1024.
__device__ __forceinline__ void sincos_turn_dd2(const dd2 &y, const float4 *tab, dd2 *s, dd2 *c)
{
    const float2 c0 = df2::psub(y.hi, df2::p2(rintf(y.hi.x), rintf(y.hi.y)));
    const float2 jf = df2::p2(rintf(__fmul_rn(c0.x, (float)kFine)), rintf(__fmul_rn(c0.y, (float)kFine)));
    const dd2 r{df2::pfma(jf, df2::b2(-1.0f / kFine), c0), y.lo};
    const dd2 x = df2::mul(r, df2::bcast(dconst(2.0 * kPi)));
    const dd2 x2 = df2::sqr(x);
    const float2 e = df2::pmul(x2.hi, df2::pfma(x2.hi, df2::b2(-1.0f / 120.0f), df2::b2(1.0f / 6.0f)));
    const dd2 sx = df2::add_u(x, dd2{df2::pneg(df2::pmul(x.hi, e)), df2::b2(0.0f)});
    dd2 cx = df2::sub_u(df2::make(1.0f), df2::scale2(x2, df2::b2(0.5f)));
    cx.lo = df2::pfma(df2::pmul(x2.hi, x2.hi), df2::b2(1.0f / 24.0f), cx.lo);
    const float4 ea = tab[(int)jf.x & (kFine - 1)], eb = tab[(int)jf.y & (kFine - 1)];
    const dd2 S{df2::p2(ea.x, eb.x), df2::p2(ea.y, eb.y)}, C{df2::p2(ea.z, eb.z), df2::p2(ea.w, eb.w)};
    // cos + i sin of the sum: (C + i S)(cx + i sx)
    const cdd2 w = df2::cmul_t<true, false>(cdd2{C, S}, cdd2{cx, sx});
    *c = w.x;
    *s = w.y;
}

// 2^v as m * 2^n per lane, m in [2^-0.5, 2^0.5]: v = k/64 + s with
// k = rint(64 v.hi) and s = (v.hi - k/64) + v.lo (the float difference exact,
// as in sincos_turn_dd2), k = 64 n + i with |i| <= 32; e^{s ln 2} = 1 + t +
// t^2/2 + t^3 (1/6 + t/24 + t^2/120) with t = s ln 2, |t| <= ln 2 / 128, so the
// terms from t^3 on (below 2.7e-8) are summed in float; times the table entry
// 2^{i/64}.
__device__ __forceinline__ dd2 exp2_dd2(const dd2 &v, const float2 *tab, int n_out[2])
{
    const float2 kf = df2::p2(rintf(__fmul_rn(v.hi.x, 64.0f)), rintf(__fmul_rn(v.hi.y, 64.0f)));
    const dd2 s{df2::pfma(kf, df2::b2(-1.0f / 64.0f), v.hi), v.lo};
    const float2 nf = df2::p2(rintf(__fmul_rn(kf.x, 1.0f / 64.0f)), rintf(__fmul_rn(kf.y, 1.0f / 64.0f)));
    const float2 i_f = df2::pfma(nf, df2::b2(-64.0f), kf);
    const dd2 t = df2::mul(s, df2::bcast(dconst(0.69314718055994530941723212145818)));
    const dd2 t2 = df2::sqr(t);
    const float2 tail = df2::pmul(df2::pmul(t2.hi, t.hi),
                                  df2::pfma(t.hi, df2::pfma(t.hi, df2::b2(1.0f / 120.0f), df2::b2(1.0f / 24.0f)),
                                            df2::b2(1.0f / 6.0f)));
    dd2 p = df2::add_u(df2::make(1.0f), t);
    p = df2::add_u(p, df2::scale2(t2, df2::b2(0.5f)));
    p = df2::add_f(p, tail);
    const float2 ea = tab[(int)i_f.x + 32], eb = tab[(int)i_f.y + 32];
    n_out[0] = (int)nf.x;
    n_out[1] = (int)nf.y;
    return df2::mul(p, dd2{df2::p2(ea.x, eb.x), df2::p2(ea.y, eb.y)});
}

__device__ __forceinline__ bool dd_less_lane(const dd2 &a, const dd2 &b, int i)
{
    return dd_less(df2::lane(a, i), df2::lane(b, i));
}

// root_dd per lane
__device__ __forceinline__ cdd2 root_dd2(const cdd2 &z, dd2 *absz)
{
    const dd2 hyp = df2::cabs2(z);
    const bool v0 = !(hyp.hi.x <= 0.0f), v1 = !(hyp.hi.y <= 0.0f);
    dd2 az, rh;
    df2::sqrt_rsqrt(df2::sel(v0, v1, hyp, df2::make(1.0f)), &az, &rh);
    const float2 sgx = df2::p2(z.x.hi.x < 0.0f ? -1.0f : 1.0f, z.x.hi.y < 0.0f ? -1.0f : 1.0f);
    const dd2 u = df2::scale2(df2::add(az, df2::scale2(z.x, sgx)), df2::b2(0.5f));
    dd2 t, ru;
    df2::sqrt_rsqrt(u, &t, &ru);
    const dd2 o = df2::scale2(df2::mul(z.y, ru), df2::b2(0.5f));
    const float2 sgo = df2::p2(o.hi.x < 0.0f ? -1.0f : 1.0f, o.hi.y < 0.0f ? -1.0f : 1.0f);
    const dd2 ao = df2::scale2(o, sgo);
    auto yneg = [](float h) { return h < 0.0f || (h == 0.0f && signbit(h)); };
    const float2 sgt = df2::p2(yneg(z.y.hi.x) ? -1.0f : 1.0f, yneg(z.y.hi.y) ? -1.0f : 1.0f);
    const bool rp0 = z.x.hi.x >= 0.0f, rp1 = z.x.hi.y >= 0.0f;
    cdd2 q{df2::sel(rp0, rp1, t, ao), df2::sel(rp0, rp1, o, df2::scale2(t, sgt))};
    // decaying root unless Im q is zero to rounding (|Im q| <= 100 * 2^-46 |q|)
    const float tol = 100.0f * 1.4210855e-14f;
    const bool f0 = q.y.hi.x < 0.0f && q.y.hi.x * q.y.hi.x > tol * tol * az.hi.x;
    const bool f1 = q.y.hi.y < 0.0f && q.y.hi.y * q.y.hi.y > tol * tol * az.hi.y;
    const float2 sgf = df2::p2(f0 ? -1.0f : 1.0f, f1 ? -1.0f : 1.0f);
    q = cdd2{df2::scale2(q.x, sgf), df2::scale2(q.y, sgf)};
    const dd2 zero = df2::make(0.0f);
    q = cdd2{df2::sel(v0, v1, q.x, zero), df2::sel(v0, v1, q.y, zero)};
    *absz = df2::sel(v0, v1, az, zero);
    return q;
}

// |x| and x with the sign of another value, on a float pair by its sign bits
// (integer instructions, off the FMA pipe): both floats of a pair share the
// sign of the high part's value.
__device__ __forceinline__ unsigned sign_of(float h) { return __float_as_uint(h) & 0x80000000u; }
__device__ __forceinline__ dd xor_sign(dd a, unsigned sb)
{
    return dd{__uint_as_float(__float_as_uint(a.hi) ^ sb), __uint_as_float(__float_as_uint(a.lo) ^ sb)};
}

// Root of z = n^2 - beta^2 inside the stack, per lane: R and T do not depend
// on which of the two roots an interior layer takes (the sign flips cancel;
// an oracle test pins it), so Im q >= 0 is taken by the sign of Im z alone, without the
// bounding media's tolerance band: q = sgn(Im z) sqrt(z) from the principal
// root, i.e. (sgn(Im z) t, |o|) for Re z >= 0 and (sgn(Im z) |o|, t) otherwise,
// with t = sqrt((|z| + |Re z|) / 2), o = Im z / (2 t).
__device__ __forceinline__ cdd2 root_inner_dd2(const cdd2 &z, dd2 *absz)
{
    const dd2 hyp = df2::cabs2(z);
    const bool v0 = !(hyp.hi.x <= 0.0f), v1 = !(hyp.hi.y <= 0.0f);
    dd2 az, rh;
    df2::sqrt_rsqrt(df2::sel(v0, v1, hyp, df2::make(1.0f)), &az, &rh);
    const dd zx0 = df2::lane(z.x, 0), zx1 = df2::lane(z.x, 1);
    const dd ax0 = xor_sign(zx0, sign_of(zx0.hi)), ax1 = xor_sign(zx1, sign_of(zx1.hi));
    const dd2 u = df2::scale2(df2::add(az, df2::pack(ax0, ax1)), df2::b2(0.5f));
    dd2 t, ru;
    df2::sqrt_rsqrt(u, &t, &ru);
    const dd2 o = df2::scale2(df2::mul(z.y, ru), df2::b2(0.5f));
    dd qx[2], qy[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const dd zi = df2::lane(z.y, i), ti = df2::lane(t, i), oi = df2::lane(o, i);
        const unsigned sy = sign_of(zi.hi);
        const dd ao = xor_sign(oi, sign_of(oi.hi));
        const bool rp = (i ? z.x.hi.y : z.x.hi.x) >= 0.0f;
        qx[i] = xor_sign(rp ? ti : ao, sy);
        qy[i] = rp ? ao : ti;
    }
    const dd2 zero = df2::make(0.0f);
    *absz = df2::sel(v0, v1, az, zero);
    return cdd2{df2::sel(v0, v1, df2::pack(qx[0], qx[1]), zero), df2::sel(v0, v1, df2::pack(qy[0], qy[1]), zero)};
}

__device__ __forceinline__ void renorm_dd_pair2(cdd2 &a, cdd2 &b, int e[2])
{
    int k[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float m = fmaxf(fmaxf(fabsf(i ? a.x.hi.y : a.x.hi.x), fabsf(i ? a.y.hi.y : a.y.hi.x)),
                              fmaxf(fabsf(i ? b.x.hi.y : b.x.hi.x), fabsf(i ? b.y.hi.y : b.y.hi.x)));
        k[i] = exponent_of(m);
        e[i] += k[i];
    }
    const float2 f = df2::p2(pow2_neg<float>(k[0]), pow2_neg<float>(k[1]));
    a = cdd2{df2::scale2(a.x, f), df2::scale2(a.y, f)};
    b = cdd2{df2::scale2(b.x, f), df2::scale2(b.y, f)};
}

__device__ __forceinline__ void renorm_dd2(dd2 &m, int e[2])
{
    const int k0 = exponent_of(m.hi.x), k1 = exponent_of(m.hi.y);
    m = df2::scale2(m, df2::p2(pow2_neg<float>(k0), pow2_neg<float>(k1)));
    e[0] += k0;
    e[1] += k1;
}

__device__ __forceinline__ cdd2 bc_c(float h1, float l1, float h2, float l2)
{
    return cdd2{dd2{df2::b2(h1), df2::b2(l1)}, dd2{df2::b2(h2), df2::b2(l2)}};
}

template <int POL>
__device__ __forceinline__ void eval_point_dd2(const DStage *__restrict__ st, const float4 *sc, const float2 *e2,
                                               int TL, int tl, int L, dd n0, const dd sth[2], const dd cth[2], dd Pp,
                                               int Pp_e, double out[2][4])
{
    dd beta[2], c0[2], q0sq[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        beta[i] = df::mul(n0, sth[i]);
        c0[i] = df::mul(n0, cth[i]);
        q0sq[i] = df::sqr(c0[i]);
    }
    const dd2 Q0SQ = df2::pack(q0sq[0], q0sq[1]);
    const dd2 yi_max = df2::bcast(dconst(35.0 / (2.0 * kPi)));
    const dd2 kE = df2::bcast(dconst(-4.0 * kPi * 1.4426950408889634073599246810019));

    DStage A = st[(L + 1) * TL + tl];
    dd2 absz;
    cdd2 q_nx = root_dd2(cdd2{df2::add(df2::bcast(dd{A.d2h, A.d2l}), Q0SQ), df2::bcast(dd{A.n2yh, A.n2yl})}, &absz);
    const cdd2 q_out = q_nx;
    const cdd n2_out{df::add(dd{A.d2h, A.d2l}, df::sqr(n0)), dd{A.n2yh, A.n2yl}};
    cdd2 g_nx = df2::cmul(q_nx, bc_c(A.in2xh, A.in2xl, A.in2yh, A.in2yl));
    dd2 Ps = df2::make(1.0f), Y = df2::make(0.0f);
    int eP[2] = {0, 0};
    const cdd2 one{df2::make(1.0f), df2::make(0.0f)}, zero{df2::make(0.0f), df2::make(0.0f)};
    cdd2 s0 = one, s1 = zero, p0 = one, p1 = zero;
    int es[2] = {0, 0}, ep[2] = {0, 0};

    for (int j = L; j >= 1; --j) {
        A = st[j * TL + tl];
        const cdd2 q = root_inner_dd2(
            cdd2{df2::add(df2::bcast(dd{A.d2h, A.d2l}), Q0SQ), df2::bcast(dd{A.n2yh, A.n2yl})}, &absz);
        Ps = df2::mul(Ps, absz);
        const dd2 dl = df2::bcast(dd{A.dlh, A.dll});
        const dd2 yr = df2::mul(dl, q.x);
        dd2 yi = df2::mul(dl, q.y);
        yi = df2::sel(dd_less_lane(yi_max, yi, 0), dd_less_lane(yi_max, yi, 1), yi_max, yi);
        Y = df2::add(Y, yi);
        dd2 sn, cs;
        sincos_turn_dd2(yr, sc, &sn, &cs);
        int n2[2];
        const dd2 m2 = exp2_dd2(df2::mul(yi, kE), e2, n2);
        const dd2 E2 = df2::scale2(m2, df2::p2(ldexpf(1.0f, n2[0]), ldexpf(1.0f, n2[1])));
        // phase factors e^{-i Re delta} = conj(w) and e^{i delta} / e^{Im delta} = E2 w
        const cdd2 w{cs, sn};
        const cdd2 epi{df2::mul(E2, cs), df2::mul(E2, sn)};
        if (POL & 1) {
            df2::interface_pair_u(q, q_nx, s0, s1);
            s0 = df2::cmul_t<true, true>(w, s0);
            s1 = df2::cmul_t<true, false>(epi, s1);
        }
        if (POL & 2) {
            const cdd2 g = df2::cmul_t<true, false>(q, bc_c(A.in2xh, A.in2xl, A.in2yh, A.in2yl));
            df2::interface_pair_u(g, g_nx, p0, p1);
            p0 = df2::cmul_t<true, true>(w, p0);
            p1 = df2::cmul_t<true, false>(epi, p1);
            g_nx = g;
        }
        q_nx = q;
        if (((L - j) & 1) == 1) {
            renorm_dd2(Ps, eP);
            if (POL & 1) renorm_dd_pair2(s0, s1, es);
            if (POL & 2) renorm_dd_pair2(p0, p1, ep);
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
        finish_dd<POL>(st[tl], e2, df2::lane(q_out, i), n2_out, df2::lane(q_nx, i), df2::lane(g_nx, i),
                       df2::lane(s0, i), df2::lane(s1, i), df2::lane(p0, i), df2::lane(p1, i), df2::lane(Ps, i), eP[i],
                       df2::lane(Y, i), es[i], ep[i], L, n0, cth[i], beta[i], c0[i], q0sq[i], Pp, Pp_e, out[i]);
}

// PAIR: two angles per thread, TL x ceil(TT / 2) threads (at most 256),
// compiled for two resident blocks per SM.  The dd chains are long and
// dependent, so the kernel is latency-bound: the paired lanes halve its issue
// slots but not its latency, and their doubled state costs occupancy
// (measured on the dispersive workload: 214 ms one angle per thread, 236 ms
// paired at one block per SM, 203 ms paired at two).
template <int POL, bool WITH_T, bool PAIR>
__global__ void __launch_bounds__(PAIR ? kDfPairThreads : kDfMaxThreads, PAIR ? 2 : 1) tmm_fwd_df64_kernel(const tmm_problem p, const __grid_constant__ DfTables tabs,
                                                                     int TL, int TT, int n_lt, int n_tt,
                                                                     double *__restrict__ Rout, double *__restrict__ Tout)
{
    extern __shared__ __align__(16) unsigned char smem[];
    DStage *st = reinterpret_cast<DStage *>(smem);
    float4 *sc = reinterpret_cast<float4 *>(st + (size_t)(p.L_max + 2) * TL);
    float4 *sf = sc + 64;
    float2 *e2 = reinterpret_cast<float2 *>(sf + kFine);
    float2 *n0s = e2 + 65;         // [TL] dd n_0 (NaN if complex)
    float2 *ppm = n0s + TL;        // [TL] dd prod |1/n^2|^2
    int *ppe = reinterpret_cast<int *>(ppm + TL);

    const long long item = blockIdx.x;
    const int per_stack = n_lt * n_tt;
    const int s = (int)(item / per_stack);
    const int rr = (int)(item - (long long)s * per_stack);
    const int lt = rr / n_tt, ttile = rr % n_tt;
    const int tid = threadIdx.y * TL + threadIdx.x, nthr = TL * (int)blockDim.y;
    const int L = layers_of(p, s);
    const int l0 = lt * TL;
    const double *lam = (const double *)p.lambda;
    const double *d = (const double *)p.d;

    for (int i = tid; i < 64; i += nthr) sc[i] = tabs.sc[i];
    if (PAIR)
        for (int i = tid; i < kFine; i += nthr) sf[i] = tabs.sf[i];
    for (int i = tid; i < 65; i += nthr) e2[i] = tabs.e2[i];
    if (L >= 0) {
        const int total = (L + 2) * TL;
        for (int idx = tid; idx < total; idx += nthr) {
            const int j = idx / TL, tl = idx - j * TL;
            const int l = min(l0 + tl, p.n_lambda - 1);
            // inputs split into float pairs once; the rest in dd arithmetic on the
            // FP32 pipes (the FP64 pipe would dominate when few angles share it)
            const Cx<double> n = index_of<double>(p, s, j, l);
            const dd nx = df::from_double(n.x), ny = df::from_double(n.y);
            const dd n0d = j == 0 ? nx : df::from_double(index_of<double>(p, s, 0, l).x);
            const dd n2x = df::sub(df::sqr(nx), df::sqr(ny)), n2y = df::scale2(df::mul(nx, ny), 2.0f);
            const dd ia = df::div(df::make(1.0f), df::dot2(n2x, n2x, n2y, n2y, 1.0f));
            const dd d2 = df::sub(df::mul(df::sub(nx, n0d), df::add(nx, n0d)), df::sqr(ny));
            const dd ix = df::mul(n2x, ia), iy = df::neg(df::mul(n2y, ia));
            const dd dld = (j >= 1 && j <= L)
                               ? df::div(df::from_double(d[(long long)s * p.L_max + (j - 1)]), df::from_double(lam[l]))
                               : df::make(0.0f);
            st[idx] = DStage{d2.hi, d2.lo, n2y.hi, n2y.lo, ix.hi, ix.lo, iy.hi, iy.lo, dld.hi, dld.lo, ia.hi, ia.lo};
            if (j == 0) {
                const dd nd = df::from_double(n.y == 0.0 ? n.x : __longlong_as_double(0x7ff8000000000000LL));
                n0s[tl] = make_float2(nd.hi, nd.lo);
            }
        }
    }
    __syncthreads();
    if ((POL & 2) && L >= 0 && tid < TL) {
        dd m = df::make(1.0f);
        int e = 0;
        for (int j = 1; j <= L + 1; ++j) {
            const DStage &X = st[j * TL + tid];
            m = df::mul(m, dd{X.ain2h, X.ain2l});
            renorm_dd(m, e);
        }
        ppm[tid] = make_float2(m.hi, m.lo);
        ppe[tid] = e;
    }
    __syncthreads();

    const int tl = threadIdx.x, l = l0 + tl;
    const int t0 = ttile * TT, t_end = min(t0 + TT, p.n_theta);
    const int a0 = PAIR ? t0 + 2 * (int)threadIdx.y : t0 + (int)threadIdx.y;
    if (l < p.n_lambda && a0 < t_end) {
        const int np = PAIR && a0 + 1 < t_end ? 2 : 1;
        double out[2][4];
        if (L >= 0) {
            // sin, cos of theta through the same turn-based routine: f = theta / (2 pi)
            dd sth[2], cth[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int a = i < np ? a0 + i : a0;
                const dd f = df::mul(df::from_double(((const double *)p.theta)[a]), dconst(1.0 / (2.0 * kPi)));
                sincos_turn_dd(df::add_f(f, -rintf(f.hi)), sc, &sth[i], &cth[i]);
            }
            const float2 n0 = n0s[tl];
            const dd Ppd = (POL & 2) ? dd{ppm[tl].x, ppm[tl].y} : df::make(1.0f);
            const int Ppe = (POL & 2) ? ppe[tl] : 0;
            if constexpr (PAIR)
                eval_point_dd2<POL>(st, sf, e2, TL, tl, L, dd{n0.x, n0.y}, sth, cth, Ppd, Ppe, out);
            else
                eval_point_dd<POL>(st, sc, e2, TL, tl, L, dd{n0.x, n0.y}, sth[0], cth[0], Ppd, Ppe, out[0]);
        } else {
#pragma unroll
            for (int i = 0; i < 2; ++i) out[i][0] = out[i][1] = out[i][2] = out[i][3] = __longlong_as_double(0x7ff8000000000000LL);
        }
        const long long plane = (long long)p.S * p.n_theta * p.n_lambda;
        for (int i = 0; i < np; ++i) {
            const long long o = ((long long)s * p.n_theta + a0 + i) * p.n_lambda + l;
            int pi = 0;
            if (POL & 4) {  // unpolarised: the mean of s and p in one plane
                Rout[o] = 0.5 * (out[i][0] + out[i][2]);
                if (WITH_T) Tout[o] = 0.5 * (out[i][1] + out[i][3]);
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

const DfTables &host_tables()
{
    static DfTables t;
    static std::once_flag once;
    std::call_once(once, [] {
        const SinCosTable &q = sincos_table();
        for (int k = 0; k < 64; ++k) t.sc[k] = q.sc[k];
        for (int k = 0; k < kFine; ++k) {
            const double a = 2.0 * kPi * k / kFine;
            const double sv = std::sin(a), cv = std::cos(a);
            const float sh = (float)sv, ch = (float)cv;
            t.sf[k] = make_float4(sh, (float)(sv - sh), ch, (float)(cv - ch));
        }
        for (int i = -32; i <= 32; ++i) {
            const double v = std::exp2(i / 64.0);
            const float h = (float)v;
            t.e2[i + 32] = make_float2(h, (float)(v - h));
        }
    });
    return t;
}

size_t df_stage_bytes(const tmm_problem *p, int TL)
{
    return (size_t)(p->L_max + 2) * TL * sizeof(DStage) + (64 + kFine) * sizeof(float4) + 65 * sizeof(float2) +
           (size_t)TL * (2 * sizeof(float2) + sizeof(int));
}

template <int POL, bool WITH_T, bool PAIR>
tmm_status launch_df_shaped(const tmm_problem *p, int TL, int TT, int n_lt, int n_tt, long long n_items, size_t smem,
                            double *R, double *T, cudaStream_t st)
{
    auto k = tmm_fwd_df64_kernel<POL, WITH_T, PAIR>;
    const tmm_status ss = ensure_dynamic_smem(reinterpret_cast<const void *>(k), smem);
    if (ss != TMM_OK) return ss;
    if (n_items > 0x7fffffffLL) return TMM_ERR_UNSUPPORTED;
    k<<<(unsigned)n_items, dim3(TL, PAIR ? (TT + 1) / 2 : TT), smem, st>>>(*p, host_tables(), TL, TT, n_lt, n_tt, R,
                                                                          T);
    return check_launch();
}

// tiles of two or more angles run two angles per thread
template <int POL, bool WITH_T>
tmm_status launch_df_typed(const tmm_problem *p, int TL, int TT, int n_lt, int n_tt, long long n_items, size_t smem,
                           double *R, double *T, cudaStream_t st)
{
    if (TT >= 2) return launch_df_shaped<POL, WITH_T, true>(p, TL, TT, n_lt, n_tt, n_items, smem, R, T, st);
    return launch_df_shaped<POL, WITH_T, false>(p, TL, TT, n_lt, n_tt, n_items, smem, R, T, st);
}

}  // namespace

tmm_status launch_forward_df64(const tmm_problem *p, const tmm_launch_cfg *cfg, void *R, void *T, cudaStream_t st)
{
    if (cfg && cfg->persistent) return TMM_ERR_UNSUPPORTED;
    DeviceInfo di;
    tmm_status s = device_info(&di);
    if (s != TMM_OK) return s;
    int TT = cfg && cfg->tile_theta > 0 ? cfg->tile_theta : std::min(p->n_theta, 32);
    int TL = cfg && cfg->tile_lambda > 0 ? cfg->tile_lambda : 0;
    if (TT < 1 || TL < 0) return TMM_ERR_INVALID_ARG;
    const int rows = TT >= 2 ? (TT + 1) / 2 : TT;  // thread rows: two angles per thread
    const int max_threads = TT >= 2 ? kDfPairThreads : kDfMaxThreads;
    if (TL == 0) {
        TL = 1;
        while (TL * rows < 256 && TL * 2 * rows <= max_threads) TL *= 2;
        while (TL > 1 && TL / 2 >= p->n_lambda) TL /= 2;
        while (TL > 1 && df_stage_bytes(p, TL) > (size_t)di.max_smem_optin) TL /= 2;
    }
    if (TL < 1 || TL * rows > max_threads) return TMM_ERR_INVALID_ARG;
    const size_t smem = df_stage_bytes(p, TL);
    if (smem > (size_t)di.max_smem_optin) return TMM_ERR_UNSUPPORTED;
    const int n_lt = (p->n_lambda + TL - 1) / TL, n_tt = (p->n_theta + TT - 1) / TT;
    const long long n_items = (long long)p->S * n_lt * n_tt;
    if (n_items == 0) return TMM_OK;
    double *Ro = static_cast<double *>(R);
    double *To = static_cast<double *>(T);
    const bool wt = To != nullptr;
    switch (p->pol_mask) {
    case 1: return wt ? launch_df_typed<1, true>(p, TL, TT, n_lt, n_tt, n_items, smem, Ro, To, st)
                      : launch_df_typed<1, false>(p, TL, TT, n_lt, n_tt, n_items, smem, Ro, To, st);
    case 2: return wt ? launch_df_typed<2, true>(p, TL, TT, n_lt, n_tt, n_items, smem, Ro, To, st)
                      : launch_df_typed<2, false>(p, TL, TT, n_lt, n_tt, n_items, smem, Ro, To, st);
    case 3: return wt ? launch_df_typed<3, true>(p, TL, TT, n_lt, n_tt, n_items, smem, Ro, To, st)
                      : launch_df_typed<3, false>(p, TL, TT, n_lt, n_tt, n_items, smem, Ro, To, st);
    case 7: return wt ? launch_df_typed<7, true>(p, TL, TT, n_lt, n_tt, n_items, smem, Ro, To, st)
                      : launch_df_typed<7, false>(p, TL, TT, n_lt, n_tt, n_items, smem, Ro, To, st);
    default: return TMM_ERR_INVALID_ARG;
    }
}

}  // namespace tmm
