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

// ---------------------------------------------------------------- shared by the FP32 and double-float kernels
constexpr double kPi = 3.14159265358979323846264338327950288;

// A double constant as a float pair (the conversions fold at compile time).
__device__ __forceinline__ df::dd dconst(double v)
{
    const float h = (float)v;
    return df::dd{h, (float)(v - (double)h)};
}

// {sin hi, sin lo, cos hi, cos lo} of 2 pi k / 256, k = 0..63, built on the host
// in double precision and passed to the kernels by value.
struct SinCosTable {
    float4 sc[64];
};

// sin and cos of 2 pi f in double-float: f = j/256 + r, |r| <= 1/512; Taylor
// series of sin, cos (2 pi r) to x^5 / x^6 (remainder below 2^-56), combined
// with the table entry of j by the angle-addition formulas.
__device__ __forceinline__ void sincos_turn_dd(df::dd f, const float4 *tab, df::dd *s, df::dd *c)
{
    using df::dd;
    const float jf = rintf(__fmul_rn(f.hi, 256.0f));
    const int j = (int)jf;
    const dd r = df::add_f(f, -__fmul_rn(jf, 1.0f / 256.0f));
    const dd x = df::mul(r, dconst(2.0 * kPi));
    const dd x2 = df::sqr(x);
    // sin x = x (1 - x^2/6 + x^4/120), cos x = 1 - x^2/2 + (x^4/24 - x^6/720)
    const dd t = df::mul(x2, dconst(1.0 / 6.0));
    const float x4 = __fmul_rn(x2.hi, x2.hi);
    const dd p = df::add_f(df::sub(df::make(1.0f), t), __fmul_rn(x4, 1.0f / 120.0f));
    const dd sx = df::mul(x, p);
    const float h4 = __fsub_rn(__fmul_rn(x4, 1.0f / 24.0f), __fmul_rn(__fmul_rn(x4, x2.hi), 1.0f / 720.0f));
    const dd cx = df::add_f(df::sub(df::make(1.0f), df::scale2(x2, 0.5f)), h4);
    const int jj = j & 255, quad = jj >> 6, k = jj & 63;
    const float4 e = tab[k];
    const dd sk{e.x, e.y}, ck{e.z, e.w};
    dd sj, cj;
    if (quad == 0) { sj = sk; cj = ck; }
    else if (quad == 1) { sj = ck; cj = df::neg(sk); }
    else if (quad == 2) { sj = df::neg(sk); cj = df::neg(ck); }
    else { sj = df::neg(ck); cj = sk; }
    *s = df::dot2(sj, cx, cj, sx, 1.0f);
    *c = df::dot2(cj, cx, sj, sx, -1.0f);
}

// An FP64 value as a float pair hi + lo by integer operations only (no work on
// the FP64 pipe, which executes ~2 operations per clock per SM on this part):
// hi keeps the sign, the exponent and the leading 23 stored mantissa bits
// (truncated), lo the remaining 29 bits rounded to a float, so hi + lo equals
// x to about 2^-47 relative.  |x| below 2^-126 gives (+-0, 0); |x| at or above
// 2^128 gives +-inf; NaN stays NaN.  lo is dropped below |x| = 2^-74.
__host__ __device__ __forceinline__ df::dd split_f64(double x)
{
#ifdef __CUDA_ARCH__
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    __builtin_memcpy(&b, &x, sizeof b);
#endif
    const unsigned hi32 = (unsigned)(b >> 32);
    const unsigned sign = hi32 & 0x80000000u;
    const int e = (int)((hi32 >> 20) & 0x7ffu);
    const unsigned mtop = (unsigned)((b >> 29) & 0x7fffffu);
    const unsigned mlow = (unsigned)(b & 0x1fffffffu);
    unsigned hb, lb = 0u;
    if (e == 0x7ff) {  // inf or NaN
        hb = sign | 0x7f800000u | (((b & 0xfffffffffffffull) != 0ull) ? 0x00400000u : 0u);
    } else if (e - 896 >= 255) {
        hb = sign | 0x7f800000u;
    } else if (e - 896 <= 0) {
        hb = sign;
    } else {
        hb = sign | ((unsigned)(e - 896) << 23) | mtop;
        if (e >= 949 && mlow != 0u) {
            // mlow * 2^(e - 1075): the float of mlow times an exact power of two
            const float m = (float)mlow;
            const unsigned pb = (unsigned)(e - 948) << 23;
            float p2;
            __builtin_memcpy(&p2, &pb, sizeof p2);
            float l = m * p2;
            unsigned l_bits;
            __builtin_memcpy(&l_bits, &l, sizeof l_bits);
            lb = l_bits | sign;
        }
    }
    float h, l;
    __builtin_memcpy(&h, &hb, sizeof h);
    __builtin_memcpy(&l, &lb, sizeof l);
    return df::dd{h, l};
}

}  // namespace tmm
