// tmm_df64x2.cuh -- double-float arithmetic (tmm_df64.cuh) on the two lanes
// of the paired FP32 instructions: a value per lane is dd2 = (hi, lo) with
// hi, lo float2.  __fadd2_rn, __fmul2_rn and __ffma2_rn round each lane
// exactly as __fadd_rn, __fmul_rn and __fmaf_rn do, and are never
// contracted, so every error-free transformation holds lane by lane; a - b is
// written as the single rounding fma(b, -1, a).
#pragma once

#include <cuda_runtime.h>

#include "tmm_df64.cuh"

namespace tmm {
namespace df2 {

struct dd2 {
    float2 hi, lo;
};
struct cdd2 {
    dd2 x, y;
};

__device__ __forceinline__ float2 p2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 b2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, b2(-1.f), a); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pneg(float2 a) { return __fmul2_rn(a, b2(-1.f)); }

__device__ __forceinline__ dd2 make(float h) { return dd2{b2(h), b2(0.f)}; }
__device__ __forceinline__ dd2 bcast(df::dd a) { return dd2{b2(a.hi), b2(a.lo)}; }
__device__ __forceinline__ dd2 pack(df::dd a, df::dd b) { return dd2{p2(a.hi, b.hi), p2(a.lo, b.lo)}; }
__device__ __forceinline__ df::dd lane(const dd2 &a, int i)
{
    return i ? df::dd{a.hi.y, a.lo.y} : df::dd{a.hi.x, a.lo.x};
}
__device__ __forceinline__ df::cdd lane(const cdd2 &a, int i) { return df::cdd{lane(a.x, i), lane(a.y, i)}; }

__device__ __forceinline__ dd2 fast_two_sum(float2 a, float2 b)
{
    const float2 s = padd(a, b);
    return dd2{s, psub(b, psub(s, a))};
}

__device__ __forceinline__ dd2 two_sum(float2 a, float2 b)
{
    const float2 s = padd(a, b);
    const float2 bb = psub(s, a);
    return dd2{s, padd(psub(a, psub(s, bb)), psub(b, bb))};
}

__device__ __forceinline__ dd2 neg(const dd2 &a) { return dd2{pneg(a.hi), pneg(a.lo)}; }

__device__ __forceinline__ dd2 add(const dd2 &a, const dd2 &b)
{
    dd2 s = two_sum(a.hi, b.hi);
    s.lo = padd(s.lo, padd(a.lo, b.lo));
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd2 sub(const dd2 &a, const dd2 &b)
{
    // a + (-b) with the negation folded into single roundings
    const float2 s = psub(a.hi, b.hi);
    const float2 bb = psub(s, a.hi);  // the part of -b.hi in s
    const float2 e = psub(psub(a.hi, psub(s, bb)), padd(b.hi, bb));
    return fast_two_sum(s, padd(e, psub(a.lo, b.lo)));
}

__device__ __forceinline__ dd2 add_f(const dd2 &a, float2 b)
{
    dd2 s = two_sum(a.hi, b);
    s.lo = padd(s.lo, a.lo);
    return fast_two_sum(s.hi, s.lo);
}

// p + e = a b exactly; -p formed as (-a) b so that e = fma(a, b, -p) is one rounding
__device__ __forceinline__ dd2 mul(const dd2 &a, const dd2 &b)
{
    const float2 np = pmul(pneg(a.hi), b.hi);
    float2 e = pfma(a.hi, b.hi, np);
    e = pfma(a.hi, b.lo, e);
    e = pfma(a.lo, b.hi, e);
    // fast_two_sum(p, e) with p = -np
    const float2 s = psub(e, np);
    return dd2{s, psub(e, padd(s, np))};
}

__device__ __forceinline__ dd2 mul_f(const dd2 &a, float2 b)
{
    const float2 np = pmul(pneg(a.hi), b);
    float2 e = pfma(a.hi, b, np);
    e = pfma(a.lo, b, e);
    const float2 s = psub(e, np);
    return dd2{s, psub(e, padd(s, np))};
}

__device__ __forceinline__ dd2 sqr(const dd2 &a)
{
    const float2 np = pmul(pneg(a.hi), a.hi);
    float2 e = pfma(a.hi, a.hi, np);
    e = pfma(pmul(b2(2.f), a.hi), a.lo, e);
    const float2 s = psub(e, np);
    return dd2{s, psub(e, padd(s, np))};
}

// exact scaling by powers of two (per lane)
__device__ __forceinline__ dd2 scale2(const dd2 &a, float2 s) { return dd2{pmul(a.hi, s), pmul(a.lo, s)}; }

// a b + sgn c d (sgn = +-1) with the two high products taken exactly
__device__ __forceinline__ dd2 dot2(const dd2 &a, const dd2 &b, const dd2 &c, const dd2 &d, float sgn)
{
    const float2 sc = pmul(b2(sgn), c.hi), sl = pmul(b2(sgn), c.lo);
    const float2 np1 = pmul(pneg(a.hi), b.hi);
    const float2 e1 = pfma(a.hi, b.hi, np1);
    const float2 np2 = pmul(pneg(sc), d.hi);
    const float2 e2 = pfma(sc, d.hi, np2);
    // two_sum(p1, p2) with p1 = -np1, p2 = -np2: s = -(np1 + np2) exactly as
    // the rounding of p1 + p2 (the rounding is symmetric)
    const dd2 t = two_sum(np1, np2);  // np1 + np2 = -(p1 + p2)
    float2 e = padd(pneg(t.lo), padd(e1, e2));
    e = pfma(a.hi, b.lo, e);
    e = pfma(a.lo, b.hi, e);
    e = pfma(sc, d.lo, e);
    e = pfma(sl, d.hi, e);
    // fast_two_sum(-t.hi, e)
    const float2 s = psub(e, t.hi);
    return dd2{s, psub(e, padd(s, t.hi))};
}

// sqrt and 1/sqrt (Karp-Markstein), a.hi > 0 in both lanes
__device__ __forceinline__ void sqrt_rsqrt(const dd2 &a, dd2 *s, dd2 *r)
{
    const float2 r0 = p2(rsqrtf(a.hi.x), rsqrtf(a.hi.y));
    const float2 s0 = pmul(a.hi, r0);
    const float2 np = pmul(pneg(s0), s0);
    const float2 pe = pfma(s0, s0, np);  // s0^2 = -np + pe exactly
    // a - s0^2 = (a.hi + np) - pe + a.lo
    const float2 e = padd(psub(padd(a.hi, np), pe), a.lo);
    *s = fast_two_sum(s0, pmul(pmul(e, b2(0.5f)), r0));
    const dd2 q = mul(*s, dd2{r0, b2(0.f)});  // ~ 1
    const float2 c = psub(psub(b2(1.f), q.hi), q.lo);
    *r = fast_two_sum(r0, pmul(r0, c));
}

// per-lane select: lane i of a where m_i, else of b
__device__ __forceinline__ float2 sel(bool m0, bool m1, float2 a, float2 b)
{
    return p2(m0 ? a.x : b.x, m1 ? a.y : b.y);
}
__device__ __forceinline__ dd2 sel(bool m0, bool m1, const dd2 &a, const dd2 &b)
{
    return dd2{sel(m0, m1, a.hi, b.hi), sel(m0, m1, a.lo, b.lo)};
}

// ---------------------------------------------------------------- complex
__device__ __forceinline__ cdd2 cadd(const cdd2 &a, const cdd2 &b) { return cdd2{add(a.x, b.x), add(a.y, b.y)}; }
__device__ __forceinline__ cdd2 csub(const cdd2 &a, const cdd2 &b) { return cdd2{sub(a.x, b.x), sub(a.y, b.y)}; }
__device__ __forceinline__ cdd2 cmul(const cdd2 &a, const cdd2 &b)
{
    return cdd2{dot2(a.x, b.x, a.y, b.y, -1.0f), dot2(a.x, b.y, a.y, b.x, 1.0f)};
}
__device__ __forceinline__ dd2 cabs2(const cdd2 &a) { return dot2(a.x, a.x, a.y, a.y, 1.0f); }

__device__ __forceinline__ void interface_pair(const cdd2 &k, const cdd2 &kn, cdd2 &x0, cdd2 &x1)
{
    const cdd2 X = cmul(k, cadd(x0, x1));
    const cdd2 Z = cmul(kn, csub(x0, x1));
    x0 = cadd(X, Z);
    x1 = csub(X, Z);
}

// ---------------------------------------------------------------- unnormalised intermediates
// Sums and products without their closing fast_two_sum: hi + lo is the value
// to the same order of accuracy, with |lo| up to a few ulp(hi) instead of
// ulp(hi) / 2.  Every consumer takes lo into account (two_sum of the high
// parts plus the low parts; products with both cross terms), so a following
// operation's error grows by a small factor only.  The paired sweep keeps
// these values inside one interface step and normalises the state in the
// phase product that follows: 202.5 -> 191.7 ms on the 16384 x 24 dispersive
// launch, the largest error against the oracle unchanged (1.2e-11 on the
// paper's timing stack near grazing incidence, 8.4e-12 on 97 layers).
__device__ __forceinline__ dd2 add_u(const dd2 &a, const dd2 &b)
{
    dd2 s = two_sum(a.hi, b.hi);
    s.lo = padd(s.lo, padd(a.lo, b.lo));
    return s;
}

__device__ __forceinline__ dd2 sub_u(const dd2 &a, const dd2 &b)
{
    const float2 s = psub(a.hi, b.hi);
    const float2 bb = psub(s, a.hi);
    const float2 e = psub(psub(a.hi, psub(s, bb)), padd(b.hi, bb));
    return dd2{s, padd(e, psub(a.lo, b.lo))};
}

// ---------------------------------------------------------------- complex product, few negations
// Paired instructions take no sign modifiers, so every negation is an
// instruction of its own.  cmul_t forms a b (CONJ: conj(a) b) with the four
// high products taken exactly from -a.x.hi, -a.y.hi and -a.y.lo only, each
// used twice: a product term t = x y is rounded as q = fl(x y) and its exact
// error carried negated, q - x y = fma(-x, y, q); a term t = -x y likewise as
// q = fl((-x) y) with q + x y = fma(x, y, q).  Each part is then
// two_sum(q1, q2) minus the two carried errors plus the cross terms with the
// low parts, the same roundings as dot2.  NORM: close with fast_two_sum.
template <bool NORM>
__device__ __forceinline__ dd2 close_dd2(const dd2 &s, float2 e)
{
    if constexpr (NORM) {
        return fast_two_sum(s.hi, e);
    } else {
        return dd2{s.hi, e};
    }
}

template <bool NORM, bool CONJ>
__device__ __forceinline__ cdd2 cmul_t(const cdd2 &a, const cdd2 &b)
{
    const float2 nax = pneg(a.x.hi), nay = pneg(a.y.hi), nayl = pneg(a.y.lo);
    // real part: a.x b.x -+ a.y b.y
    const float2 q1 = pmul(a.x.hi, b.x.hi);
    const float2 c1 = pfma(nax, b.x.hi, q1);  // q1 - a.x.hi b.x.hi
    const float2 q2 = CONJ ? pmul(a.y.hi, b.y.hi) : pmul(nay, b.y.hi);
    const float2 c2 = CONJ ? pfma(nay, b.y.hi, q2) : pfma(a.y.hi, b.y.hi, q2);
    const dd2 sr = two_sum(q1, q2);
    float2 er = psub(psub(sr.lo, c1), c2);
    er = pfma(a.x.hi, b.x.lo, er);
    er = pfma(a.x.lo, b.x.hi, er);
    er = pfma(CONJ ? a.y.hi : nay, b.y.lo, er);
    er = pfma(CONJ ? a.y.lo : nayl, b.y.hi, er);
    // imaginary part: a.x b.y +- a.y b.x
    const float2 q3 = pmul(a.x.hi, b.y.hi);
    const float2 c3 = pfma(nax, b.y.hi, q3);
    const float2 q4 = CONJ ? pmul(nay, b.x.hi) : pmul(a.y.hi, b.x.hi);
    const float2 c4 = CONJ ? pfma(a.y.hi, b.x.hi, q4) : pfma(nay, b.x.hi, q4);
    const dd2 si = two_sum(q3, q4);
    float2 ei = psub(psub(si.lo, c3), c4);
    ei = pfma(a.x.hi, b.y.lo, ei);
    ei = pfma(a.x.lo, b.y.hi, ei);
    ei = pfma(CONJ ? nay : a.y.hi, b.x.lo, ei);
    ei = pfma(CONJ ? nayl : a.y.lo, b.x.hi, ei);
    return cdd2{close_dd2<NORM>(sr, er), close_dd2<NORM>(si, ei)};
}

// interface_pair with unnormalised intermediates and outputs (see above)
__device__ __forceinline__ void interface_pair_u(const cdd2 &k, const cdd2 &kn, cdd2 &x0, cdd2 &x1)
{
    const cdd2 u{add_u(x0.x, x1.x), add_u(x0.y, x1.y)};
    const cdd2 v{sub_u(x0.x, x1.x), sub_u(x0.y, x1.y)};
    const cdd2 X = cmul_t<false, false>(k, u);
    const cdd2 Z = cmul_t<false, false>(kn, v);
    x0 = cdd2{add_u(X.x, Z.x), add_u(X.y, Z.y)};
    x1 = cdd2{sub_u(X.x, Z.x), sub_u(X.y, Z.y)};
}

}  // namespace df2
}  // namespace tmm
