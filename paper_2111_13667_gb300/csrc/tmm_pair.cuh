// tmm_pair.cuh -- two angles per thread on paired FP32 lanes: the pieces
// shared by the incoherent-layer and partially coherent kernels (the forward
// kernel's are in tmm_fwd.cu).
#pragma once

#include "tmm_device.cuh"

namespace tmm {

// Both columns of a block's matrix for the two angles of a thread.
struct Cols2 {
    C2 x0, x1, y0, y1;
};

__device__ __forceinline__ void renorm_cols2(Cols2 &c, int &ea, int &eb)
{
    auto mx = [](const C2 &v, int i) {
        return i ? fmaxf(fabsf(v.x.y), fabsf(v.y.y)) : fmaxf(fabsf(v.x.x), fabsf(v.y.x));
    };
    const float ma = fmaxf(fmaxf(mx(c.x0, 0), mx(c.x1, 0)), fmaxf(mx(c.y0, 0), mx(c.y1, 0)));
    const float mb = fmaxf(fmaxf(mx(c.x0, 1), mx(c.x1, 1)), fmaxf(mx(c.y0, 1), mx(c.y1, 1)));
    const int ka = exponent_of(ma), kb = exponent_of(mb);
    const float2 f = f2(pow2_neg<float>(ka), pow2_neg<float>(kb));
    c.x0 = C2{mul2(f, c.x0.x), mul2(f, c.x0.y)}, c.x1 = C2{mul2(f, c.x1.x), mul2(f, c.x1.y)};
    c.y0 = C2{mul2(f, c.y0.x), mul2(f, c.y0.y)}, c.y1 = C2{mul2(f, c.y1.x), mul2(f, c.y1.y)};
    ea += ka;
    eb += kb;
}

// The phase factors of one layer for the two lanes: x0 turns by cs - i sn,
// x1 by ec + i es (= e^{-2 Im delta} (cs + i sn)); nsn, nes their negatives;
// yi the clamped Im(delta) / (2 pi) per lane.
struct Phase2 {
    float2 cs, sn, nsn, ec, es, nes, yi;
};

__device__ __forceinline__ Phase2 phase_pair(float dl, const Cx<float> &qa, const Cx<float> &qb, float yi_max)
{
    Phase2 f;
    const float yra = dl * qa.x, yrb = dl * qb.x;
    f.yi = f2(fminf(dl * qa.y, yi_max), fminf(dl * qb.y, yi_max));
    sincos_turn(yra - rintf(yra), &f.sn.x, &f.cs.x);
    sincos_turn(yrb - rintf(yrb), &f.sn.y, &f.cs.y);
    const float2 E2 = f2(exp_m2_turn(f.yi.x), exp_m2_turn(f.yi.y));
    f.nsn = neg2(f.sn);
    f.ec = mul2(E2, f.cs);
    f.es = mul2(E2, f.sn);
    f.nes = neg2(f.es);
    return f;
}

// a (cs - i sn) and a (ec + i es), lane by lane
__device__ __forceinline__ C2 turn_minus(const C2 &a, const Phase2 &f)
{
    return C2{fma2(f.cs, a.x, mul2(f.sn, a.y)), fma2(f.cs, a.y, mul2(f.nsn, a.x))};
}
__device__ __forceinline__ C2 turn_plus(const C2 &a, const Phase2 &f)
{
    return C2{fma2(f.ec, a.x, mul2(f.nes, a.y)), fma2(f.ec, a.y, mul2(f.es, a.x))};
}

// a * b lane by lane, nby = -Im b
__device__ __forceinline__ C2 cmul2(const C2 &a, const C2 &b, float2 nby)
{
    return C2{fma2(b.x, a.x, mul2(nby, a.y)), fma2(b.x, a.y, mul2(b.y, a.x))};
}

// One layer on both columns (interface with the medium to the right, then
// the phase): the block sweep of the incoherent and partially coherent kernels.
__device__ __forceinline__ void cols_step2(Cols2 &c, const C2 &k, float2 nky, const C2 &kn, float2 nkny,
                                           const Phase2 &f)
{
    interface_pair2(k, nky, kn, nkny, c.x0, c.x1);
    interface_pair2(k, nky, kn, nkny, c.y0, c.y1);
    phase2(f.cs, f.sn, f.nsn, f.ec, f.es, f.nes, c.x0, c.x1);
    phase2(f.cs, f.sn, f.nsn, f.ec, f.es, f.nes, c.y0, c.y1);
}

}  // namespace tmm
