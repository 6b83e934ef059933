// tmm_df64.cuh -- double-float ("dd") arithmetic: a value is the unevaluated
// sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about 48 significant
// bits.  GB300's FP64 pipe executes ~2 operations per clock per SM while its
// FP32 pipes execute 128, so FP64-accurate transfer matrices run faster as
// dd arithmetic on the FP32 pipes.
//
// Building blocks (error-free transformations):
//   two_sum       Knuth: s + e = a + b exactly (6 additions)
//   fast_two_sum  Dekker: the same when |a| >= |b| (3 additions)
//   two_prod      p + e = a b exactly, using one FMA
// Every rounding step is written with __fadd_rn / __fsub_rn / __fmul_rn, which
// the compiler never contracts into FMAs (a contraction would break the
// error-free transformations).
// Sums use the "sloppy" dd addition (one two_sum of the high parts plus the
// low parts): its absolute error is O(2^-46 (|a| + |b|)), which is what an
// FP64-accurate absolute tolerance needs.  Products accumulate the exact
// errors of the high-part products and the cross terms with FMAs.
#pragma once

#include <cuda_runtime.h>

namespace tmm {
namespace df {

struct dd {
    float hi, lo;
};
struct cdd {
    dd x, y;
};

__device__ __forceinline__ dd make(float h) { return dd{h, 0.0f}; }

__device__ __forceinline__ dd from_double(double v)
{
    const float h = (float)v;
    return dd{h, (float)(v - (double)h)};
}
__device__ __forceinline__ double to_double(dd a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ dd fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return dd{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dd two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return dd{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ dd two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return dd{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ dd neg(dd a) { return dd{-a.hi, -a.lo}; }

__device__ __forceinline__ dd add(dd a, dd b)
{
    dd s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd sub(dd a, dd b) { return add(a, neg(b)); }

__device__ __forceinline__ dd add_f(dd a, float b)
{
    dd s = two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd mul(dd a, dd b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ dd mul_f(dd a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ dd sqr(dd a)
{
    const float p = __fmul_rn(a.hi, a.hi);
    float e = fmaf(a.hi, a.hi, -p);
    e = fmaf(2.0f * a.hi, a.lo, e);
    return fast_two_sum(p, e);
}

// exact scaling by a power of two
__device__ __forceinline__ dd scale2(dd a, float s) { return dd{__fmul_rn(a.hi, s), __fmul_rn(a.lo, s)}; }

// a b + sgn c d with the two high products taken exactly
__device__ __forceinline__ dd dot2(dd a, dd b, dd c, dd d, float sgn)
{
    const float sc = __fmul_rn(sgn, c.hi), sl = __fmul_rn(sgn, c.lo);
    const float p1 = __fmul_rn(a.hi, b.hi);
    const float e1 = fmaf(a.hi, b.hi, -p1);
    const float p2 = __fmul_rn(sc, d.hi);
    const float e2 = fmaf(sc, d.hi, -p2);
    dd s = two_sum(p1, p2);
    float e = __fadd_rn(s.lo, __fadd_rn(e1, e2));
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    e = fmaf(sc, d.lo, e);
    e = fmaf(sl, d.hi, e);
    return fast_two_sum(s.hi, e);
}

// sqrt and 1/sqrt (Karp and Markstein: one correction of the float estimate)
__device__ __forceinline__ void sqrt_rsqrt(dd a, dd *s, dd *r)
{
    const float r0 = rsqrtf(a.hi);
    const float s0 = __fmul_rn(a.hi, r0);
    const dd p = two_prod(s0, s0);
    const float e = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), a.lo);  // a - s0^2
    *s = fast_two_sum(s0, __fmul_rn(__fmul_rn(e, 0.5f), r0));
    // 1/sqrt(a) = r0 (1 + (1 - a r0^2) / 2): correction from the residual of s
    const dd q = mul(*s, make(r0));  // ~ 1
    const float c = __fsub_rn(__fsub_rn(1.0f, q.hi), q.lo);
    *r = fast_two_sum(r0, __fmul_rn(r0, c));
}

__device__ __forceinline__ dd div(dd a, dd b)
{
    const float q1 = a.hi / b.hi;
    const dd r = sub(a, mul_f(b, q1));
    const float q2 = r.hi / b.hi;
    return fast_two_sum(q1, q2);
}

// ---------------------------------------------------------------- complex
__device__ __forceinline__ cdd cadd(cdd a, cdd b) { return cdd{add(a.x, b.x), add(a.y, b.y)}; }
__device__ __forceinline__ cdd csub(cdd a, cdd b) { return cdd{sub(a.x, b.x), sub(a.y, b.y)}; }
__device__ __forceinline__ cdd cmul(cdd a, cdd b)
{
    return cdd{dot2(a.x, b.x, a.y, b.y, -1.0f), dot2(a.x, b.y, a.y, b.x, 1.0f)};
}
__device__ __forceinline__ dd cabs2(cdd a) { return dot2(a.x, a.x, a.y, a.y, 1.0f); }

// (x0, x1) <- (a x0 + b x1, b x0 + a x1) with a = k + k', b = k - k', in
// sum/difference form: X = k (x0 + x1), Z = k' (x0 - x1), (X + Z, X - Z).
__device__ __forceinline__ void interface_pair(cdd k, cdd kn, cdd &x0, cdd &x1)
{
    const cdd X = cmul(k, cadd(x0, x1));
    const cdd Z = cmul(kn, csub(x0, x1));
    x0 = cadd(X, Z);
    x1 = csub(X, Z);
}

}  // namespace df
}  // namespace tmm
