// tmm_device.cuh -- device-side building blocks of the transfer-matrix kernels.
//
// Working-precision helpers (complex arithmetic, the forward root of
// cos(theta_j), the layer phase factors and exact power-of-two rescaling),
// the per-(medium, wavelength) shared-memory stage and the index assembly that
// fills it.  Everything here is written for sm_103a and shared by the forward,
// ragged and adjoint kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tmm.h"

namespace tmm {

// Largest Im(delta) of a layer phase (opaque-layer clamp), in turns: 35 / (2 pi).
constexpr double kImDeltaMax = 35.0;
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kLog2e = 1.4426950408889634073599246810019;

template <typename R> struct Cx { R x, y; };

template <typename R> __device__ __forceinline__ Cx<R> cx(R x, R y) { return Cx<R>{x, y}; }
template <typename R> __device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R> __device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <typename R> __device__ __forceinline__ Cx<R> operator-(Cx<R> a) { return {-a.x, -a.y}; }
template <typename R> __device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b)
{
    return {fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)};
}
// a * b + c
template <typename R> __device__ __forceinline__ Cx<R> cfma(Cx<R> a, Cx<R> b, Cx<R> c)
{
    return {fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
}
// c - a * b
template <typename R> __device__ __forceinline__ Cx<R> cfnma(Cx<R> a, Cx<R> b, Cx<R> c)
{
    return {fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y))};
}
template <typename R> __device__ __forceinline__ Cx<R> conj(Cx<R> a) { return {a.x, -a.y}; }
template <typename R> __device__ __forceinline__ R abs2(Cx<R> a) { return fma(a.x, a.x, a.y * a.y); }
template <typename R> __device__ __forceinline__ Cx<R> scale(R s, Cx<R> a) { return {s * a.x, s * a.y}; }
// i * a
template <typename R> __device__ __forceinline__ Cx<R> mul_i(Cx<R> a) { return {-a.y, a.x}; }

// Interface j | j+1 applied to the amplitude pair (x0, x1) carried from the
// right, in sum/difference form: with a = k + k', b = k - k' (k = q_j for s,
// q_j / n_j^2 for p; k' the same for medium j+1),
//   a x0 + b x1 = k (x0 + x1) + k' (x0 - x1),  b x0 + a x1 = k (x0 + x1) - k' (x0 - x1).
template <typename R>
__device__ __forceinline__ void interface_pair(Cx<R> k, Cx<R> kn, Cx<R> &x0, Cx<R> &x1)
{
    const Cx<R> sg = x0 + x1, df = x0 - x1;
    const Cx<R> X = cmul(k, sg);
    x0 = cfma(kn, df, X);
    x1 = cfnma(kn, df, X);
}

// ---------------------------------------------------------------- precision-specific math
__device__ __forceinline__ float rsqrt_w(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsqrt_w(double v) { return rsqrt(v); }
__device__ __forceinline__ float rint_w(float v) { return rintf(v); }
__device__ __forceinline__ double rint_w(double v) { return rint(v); }
// sin and cos of 2 pi f for |f| <= 1/2.
__device__ __forceinline__ void sincos_turn(float f, float *s, float *c) { __sincosf(6.2831853f * f, s, c); }
__device__ __forceinline__ void sincos_turn(double f, double *s, double *c) { sincospi(2.0 * f, s, c); }
// exp(2 pi y) and exp(-2 pi y).
__device__ __forceinline__ void exp_pm_turn(float y, float *ep, float *em)
{
    const float k = (float)(kTwoPi * kLog2e);
    *ep = exp2f(k * y);
    *em = exp2f(-k * y);
}
__device__ __forceinline__ void exp_pm_turn(double y, double *ep, double *em)
{
    *ep = exp(kTwoPi * y);
    *em = exp(-kTwoPi * y);
}
// exp(-4 pi y): the e^{+i delta} factor relative to e^{-i delta} for Im delta = 2 pi y.
__device__ __forceinline__ float exp_m2_turn(float y) { return exp2f((float)(-2.0 * kTwoPi * kLog2e) * y); }
__device__ __forceinline__ double exp_m2_turn(double y) { return exp(-2.0 * kTwoPi * y); }
__device__ __forceinline__ float exp2_w(float v) { return exp2f(v); }
__device__ __forceinline__ double exp2_w(double v) { return exp2(v); }
__device__ __forceinline__ float floor_w(float v) { return floorf(v); }
__device__ __forceinline__ double floor_w(double v) { return floor(v); }
__device__ __forceinline__ float sin_w(float v) { return sinf(v); }
__device__ __forceinline__ double sin_w(double v) { return sin(v); }
__device__ __forceinline__ void sincos_w(float v, float *s, float *c) { sincosf(v, s, c); }
__device__ __forceinline__ void sincos_w(double v, double *s, double *c) { sincos(v, s, c); }
// Layers between two rescalings of the amplitude pairs: the per-layer growth
// is below 2^63 (|n| <= 32 and the Im(delta) <= 35 clamp), so FP32 can take
// two layers and FP64 eight before the exponent range is at risk.  The scalar
// product of |q_j|^2 (a factor in [2^-31, 2^11] per layer unless it is 0) is
// rescaled every second interval.
template <typename R> struct RenormEvery;
template <> struct RenormEvery<float> { static constexpr int value = 2; };
template <> struct RenormEvery<double> { static constexpr int value = 8; };
template <typename R> __device__ __forceinline__ R eps_w();
template <> __device__ __forceinline__ float eps_w<float>() { return 1.1920929e-7f; }
template <> __device__ __forceinline__ double eps_w<double>() { return 2.220446049250313e-16; }
template <typename R> __device__ __forceinline__ R min_normal();
template <> __device__ __forceinline__ float min_normal<float>() { return 1.17549435e-38f; }
template <> __device__ __forceinline__ double min_normal<double>() { return 2.2250738585072014e-308; }
template <typename R> __device__ __forceinline__ R nan_w();
template <> __device__ __forceinline__ float nan_w<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double nan_w<double>() { return __longlong_as_double(0x7ff8000000000000LL); }

// Exact rescaling by powers of two.  `exponent_of(m)` is floor(log2 m) for a
// normal positive m (-127 / -1023 for zero and subnormals); `pow2_neg(e)` is
// 2^-e for e inside the normal range.
__device__ __forceinline__ int exponent_of(float m) { return ((__float_as_int(m) >> 23) & 0xff) - 127; }
__device__ __forceinline__ int exponent_of(double m) { return (int)((__double_as_longlong(m) >> 52) & 0x7ff) - 1023; }
template <typename R> __device__ __forceinline__ R pow2_neg(int e);
template <> __device__ __forceinline__ float pow2_neg<float>(int e) { return __int_as_float((127 - e) << 23); }
template <> __device__ __forceinline__ double pow2_neg<double>(int e) { return __longlong_as_double((long long)(1023 - e) << 52); }
__device__ __forceinline__ float ldexp_w(float v, int e) { return ldexpf(v, e); }
__device__ __forceinline__ double ldexp_w(double v, int e) { return ldexp(v, e); }

// Keep a positive running product m in [1, 2): m <- m 2^-k, e <- e + k.
template <typename R> __device__ __forceinline__ void renorm_scalar(R &m, int &e)
{
    const int k = exponent_of(m);
    m *= pow2_neg<R>(k);
    e += k;
}

// Rescale the amplitude pair (x0, x1) so its largest component is in [1, 2).
template <typename R> __device__ __forceinline__ void renorm_pair(Cx<R> &x0, Cx<R> &x1, int &e)
{
    const R m = fmax(fmax(fabs(x0.x), fabs(x0.y)), fmax(fabs(x1.x), fabs(x1.y)));
    const int k = exponent_of(m);
    const R s = pow2_neg<R>(k);
    x0 = scale(s, x0);
    x1 = scale(s, x1);
    e += k;
}

// q = n cos(theta) = sqrt(n^2 - beta^2), the forward root (see tmm.h); also
// returns |q|^2 = |z|.  z = 0 gives q = 0.
template <typename R> __device__ __forceinline__ Cx<R> forward_root(Cx<R> z, R *absz_out)
{
    // Branch-free: the reciprocal roots take max(., smallest normal), which
    // leaves every normal input unchanged and turns z = 0 into q = 0, |z| = 0
    // (no 0 * inf); a NaN z still reaches q and |z| through u and o.
    const R hyp = fma(z.x, z.x, z.y * z.y);
    const R tiny = min_normal<R>();
    const R absz = hyp * rsqrt_w(fmax(hyp, tiny));
    const R u = R(0.5) * (absz + fabs(z.x));
    const R ru = rsqrt_w(fmax(u, tiny));
    const R t = u * ru;             // sqrt(u)
    const R o = R(0.5) * z.y * ru;  // Im z / (2 sqrt(u))
    Cx<R> q = z.x >= R(0) ? Cx<R>{t, o} : Cx<R>{fabs(o), copysign(t, z.y)};
    // principal root has Re >= 0; take the decaying one unless Im q is zero to
    // rounding (|Im q| <= 100 eps |q|, compared squared)
    const R tol = R(100) * eps_w<R>();
    if (q.y < R(0) && q.y * q.y > tol * tol * absz) q = -q;
    *absz_out = absz;
    return q;
}

// ---------------------------------------------------------------- paired FP32 lanes
// sm_100+ issues two FP32 lanes per instruction (fma/mul/add .f32x2) at the
// scalar lane throughput: arithmetic that two points do alike costs half the
// issue slots.  A value per lane is a float2, a complex value per lane a C2.
struct C2 { float2 x, y; };

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return __fmul2_rn(a, bc2(-1.f)); }
// a - b, rounded once like the scalar subtraction: a + (-1) b
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bc2(-1.f), a); }
__device__ __forceinline__ C2 neg2(C2 a) { return C2{neg2(a.x), neg2(a.y)}; }
__device__ __forceinline__ Cx<float> lane(const C2 &a, int i) { return i ? Cx<float>{a.x.y, a.y.y} : Cx<float>{a.x.x, a.y.x}; }
__device__ __forceinline__ C2 pack2(Cx<float> a, Cx<float> b) { return C2{f2(a.x, b.x), f2(a.y, b.y)}; }

// interface_pair per lane: X = k (x0 + x1), Y = k' (x0 - x1), x0 = X + Y,
// x1 = X - Y.  Paired instructions take no sign modifiers, so the products
// use carried negatives of the imaginary parts, nky = -Im k, nkny = -Im k'.
__device__ __forceinline__ void interface_pair2(const C2 &k, float2 nky, const C2 &kn, float2 nkny, C2 &x0, C2 &x1)
{
    const C2 sg = {add2(x0.x, x1.x), add2(x0.y, x1.y)};
    const C2 df = {sub2(x0.x, x1.x), sub2(x0.y, x1.y)};
    const C2 X = {fma2(k.x, sg.x, mul2(nky, sg.y)), fma2(k.x, sg.y, mul2(k.y, sg.x))};
    const C2 Y = {fma2(kn.x, df.x, mul2(nkny, df.y)), fma2(kn.x, df.y, mul2(kn.y, df.x))};
    x0 = C2{add2(X.x, Y.x), add2(X.y, Y.y)};
    x1 = C2{sub2(X.x, Y.x), sub2(X.y, Y.y)};
}

// x0 <- (cs - i sn) x0, x1 <- (ec + i es) x1 per lane (the layer phase); nsn,
// nes the negatives
__device__ __forceinline__ void phase2(float2 cs, float2 sn, float2 nsn, float2 ec, float2 es, float2 nes, C2 &x0,
                                       C2 &x1)
{
    x0 = C2{fma2(cs, x0.x, mul2(sn, x0.y)), fma2(cs, x0.y, mul2(nsn, x0.x))};
    x1 = C2{fma2(ec, x1.x, mul2(nes, x1.y)), fma2(ec, x1.y, mul2(es, x1.x))};
}

// renorm_pair per lane
__device__ __forceinline__ void renorm_pair2(C2 &x0, C2 &x1, int &ea, int &eb)
{
    const float ma = fmaxf(fmaxf(fabsf(x0.x.x), fabsf(x0.y.x)), fmaxf(fabsf(x1.x.x), fabsf(x1.y.x)));
    const float mb = fmaxf(fmaxf(fabsf(x0.x.y), fabsf(x0.y.y)), fmaxf(fabsf(x1.x.y), fabsf(x1.y.y)));
    const int ka = exponent_of(ma), kb = exponent_of(mb);
    const float2 sc = f2(pow2_neg<float>(ka), pow2_neg<float>(kb));
    x0 = C2{mul2(sc, x0.x), mul2(sc, x0.y)};
    x1 = C2{mul2(sc, x1.x), mul2(sc, x1.y)};
    ea += ka;
    eb += kb;
}

// forward_root for a finite layer inside the stack.  R and T do not depend on
// the branch taken there (the sign flips cancel), so the tolerance band of the
// bounding media is not needed: the root with Im q >= 0 (Im q = 0: Re q of the
// sign of Im z) keeps the phase clamp and the rescaling bounds valid.  With
// t = sqrt(u), o = Im z / (2 sqrt(u)), u = (|z| + |Re z|) / 2, that root is
//   Re z >= 0: (sign(Im z) t, |o|);  Re z < 0: (sign(Im z) |o|, t).
__device__ __forceinline__ Cx<float> inner_root(Cx<float> z, float *absz_out)
{
    const float hyp = fmaf(z.x, z.x, z.y * z.y);
    const float tiny = min_normal<float>();
    const float absz = hyp * rsqrtf(fmaxf(hyp, tiny));
    const float u = 0.5f * (absz + fabsf(z.x));
    const float ru = rsqrtf(fmaxf(u, tiny));
    const float t = u * ru;
    const float ao = fabsf(0.5f * z.y * ru);
    const bool re_pos = z.x >= 0.f;
    *absz_out = absz;
    return Cx<float>{copysignf(re_pos ? t : ao, z.y), re_pos ? ao : t};
}

// ---------------------------------------------------------------- shared-memory stage
// Per (medium j, wavelength): n_j^2 - n_0^2 (real part; the imaginary part is
// that of n_j^2), 1 / n_j^2, |1 / n_j^2|^2 and d_j / lambda (0 for the two
// semi-infinite media).  A point then forms n_j^2 - beta^2 as
// (n_j^2 - n_0^2) + (n_0 cos theta)^2, which has no cancellation for media
// index-matched to the injection medium near grazing incidence.  Two arrays
// keep the loads vectorised.
template <typename R> struct StageA { R d2x, n2y, in2x, in2y; };
template <typename R> struct StageB { R ain2, dl; };

template <typename R> __device__ __forceinline__ Cx<R> load_cx(const R *p, long long i)
{
    return Cx<R>{p[2 * i], p[2 * i + 1]};
}

// Index n[s][j][l] of a problem (either source); poison = NaN on a bad index.
template <typename R>
__device__ __forceinline__ Cx<R> index_of(const tmm_problem &p, int s, int j, int l)
{
    if (p.n_direct) {
        const R *nd = (const R *)p.n_direct;
        const long long row = (long long)s * (p.L_max + 2) + j;
        return p.n_direct_per_lambda ? load_cx(nd, row * p.n_lambda + l) : load_cx(nd, row);
    }
    const int m = p.mat_idx[(long long)s * (p.L_max + 2) + j];
    if (m < 0 || m >= p.n_materials) return Cx<R>{nan_w<R>(), nan_w<R>()};
    return load_cx((const R *)p.mat_table, (long long)m * p.n_lambda + l);
}

// Layer count of stack s, or -1 if it is outside [0, L_max].
__device__ __forceinline__ int layers_of(const tmm_problem &p, int s)
{
    if (!p.L_per_stack) return p.L_max;
    const int L = p.L_per_stack[s];
    return (L < 0 || L > p.L_max) ? -1 : L;
}

// Fill the stage for media 0..L+1 of stack s and wavelengths l0..l0+TL-1.
// Row L+1 is the outcoupling medium (row L_s+1 of the stack's media).
// n0 receives the (real) injection index per wavelength, NaN if complex.
template <typename R>
__device__ __forceinline__ void fill_stage(const tmm_problem &p, int s, int L, int l0, int TL,
                                           StageA<R> *sa, StageB<R> *sb, R *n0, int tid, int nthr)
{
    const R *lam = (const R *)p.lambda;
    const R *d = (const R *)p.d;
    const int total = (L + 2) * TL;
    for (int idx = tid; idx < total; idx += nthr) {
        const int j = idx / TL, tl = idx - j * TL;
        const int l = min(l0 + tl, p.n_lambda - 1);
        Cx<R> n = index_of<R>(p, s, j, l);
        const R n0v = j == 0 ? n.x : index_of<R>(p, s, 0, l).x;
        const Cx<R> n2 = {fma(n.x, n.x, -n.y * n.y), R(2) * n.x * n.y};
        const R a = abs2(n2);
        const R ia = R(1) / a;
        StageA<R> A;
        A.d2x = (n.x - n0v) * (n.x + n0v) - n.y * n.y;
        A.n2y = n2.y;
        A.in2x = n2.x * ia;
        A.in2y = -n2.y * ia;
        StageB<R> B;
        B.ain2 = ia;  // |1/n^2|^2 = 1 / |n^2|^2
        B.dl = (j >= 1 && j <= L) ? d[(long long)s * p.L_max + (j - 1)] / lam[l] : R(0);
        sa[idx] = A;
        sb[idx] = B;
        if (j == 0) n0[tl] = (n.y == R(0)) ? n.x : nan_w<R>();
    }
}

}  // namespace tmm
