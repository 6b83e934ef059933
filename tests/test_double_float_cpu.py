"""Error bounds of the double-float building blocks, on the CPU.

The double-float kernel keeps each value as an unevaluated pair of floats and
relies on a few exact-arithmetic facts and error bounds.  These tests restate
the float operations in plain Python (each rounding done once, an FMA as the
exact product-sum rounded once) and check the facts against exact rational or
200-bit arithmetic:

* the range reduction y -> (y - rint y) - m/1024 is exact in float
  (Sterbenz's lemma), for phases of any size;
* with |x| <= pi/1024, sin x = x - x e (e = x^2/6 - x^4/120 in float) and
  cos x = 1 - x^2/2 + x^4/24 (x^2 as a float pair) are within 2^-49 of the
  exact values;
* the complex product with three shared negations (each part: the two high
  products exact, their errors carried negated, two_sum, cross terms) is
  within a few 2^-48 of the exact product, in the plain and conjugate forms
  and with unnormalised outputs.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

f32 = np.float32


def rnd(v):
    """Round a rational (or float) to the nearest float32 (ties to even)."""
    return f32(float(v)) if not isinstance(v, Fr) else _round_fraction(v)


def _round_fraction(v):
    # float(Fraction) rounds correctly to double; double -> float32 can round
    # twice, so settle the tie cases exactly
    d = float(v)
    c = f32(d)
    if Fr(float(c)) == v:
        return c
    lo, hi = (c, np.nextafter(c, f32(np.inf))) if Fr(float(c)) < v else (np.nextafter(c, f32(-np.inf)), c)
    dl, dh = v - Fr(float(lo)), Fr(float(hi)) - v
    if dl < dh:
        return lo
    if dh < dl:
        return hi
    return lo if (np.frombuffer(lo.tobytes(), np.uint32)[0] & 1) == 0 else hi


def add(a, b):
    return rnd(Fr(float(a)) + Fr(float(b)))


def sub(a, b):
    return rnd(Fr(float(a)) - Fr(float(b)))


def mul(a, b):
    return rnd(Fr(float(a)) * Fr(float(b)))


def fma(a, b, c):
    return rnd(Fr(float(a)) * Fr(float(b)) + Fr(float(c)))


def two_sum(a, b):
    s = add(a, b)
    bb = sub(s, a)
    return s, add(sub(a, sub(s, bb)), sub(b, bb))


def fast_two_sum(a, b):
    s = add(a, b)
    return s, sub(b, sub(s, a))


def val(p):
    return Fr(float(p[0])) + Fr(float(p[1]))


def split(v):
    """A value as a float pair hi + lo."""
    h = f32(float(v))
    return h, f32(float(mp.mpf(v) - mp.mpf(float(h))))


def dd_mul(a, b):
    p = mul(a[0], b[0])
    e = fma(a[0], b[0], -p)
    e = fma(a[0], b[1], e)
    e = fma(a[1], b[0], e)
    return fast_two_sum(p, e)


def dd_sqr(a):
    p = mul(a[0], a[0])
    e = fma(a[0], a[0], -p)
    e = fma(mul(f32(2), a[0]), a[1], e)
    return fast_two_sum(p, e)


def test_range_reduction_is_exact():
    rng = np.random.default_rng(11)
    ys = np.concatenate([rng.uniform(-3, 3, 400), rng.uniform(-5e3, 5e3, 300), [0.0, 0.5, -0.5, 1 / 2048, 3e-8]])
    for y in ys.astype(np.float32):
        n = f32(np.rint(y))
        c0 = sub(y, n)
        assert Fr(float(c0)) == Fr(float(y)) - Fr(float(n))
        m = f32(np.rint(mul(c0, f32(1024))))
        r = fma(m, f32(-1.0 / 1024), c0)
        assert Fr(float(r)) == Fr(float(c0)) - Fr(float(m)) / 1024
        assert abs(float(r)) <= 1.0 / 2048


def test_short_series_sin_cos_within_2_to_minus_49():
    mp.mp.prec = 200
    rng = np.random.default_rng(12)
    two_pi = split(2 * mp.pi)
    worst = 0.0
    for r in rng.uniform(-1.0 / 2048, 1.0 / 2048, 3000):
        rd = split(mp.mpf(r) * (1 + mp.mpf(rng.standard_normal()) * 2 ** -30))
        x = dd_mul(rd, two_pi)
        x2 = dd_sqr(x)
        e = mul(x2[0], fma(x2[0], f32(-1.0 / 120), f32(1.0 / 6)))
        s_hi, s_lo = two_sum(x[0], -mul(x[0], e))
        sx = (s_hi, add(s_lo, x[1]))
        h = (mul(x2[0], f32(0.5)), mul(x2[1], f32(0.5)))
        c_hi, c_lo = two_sum(f32(1), -h[0])
        cx = (c_hi, fma(mul(x2[0], x2[0]), f32(1.0 / 24), add(c_lo, -h[1])))
        xv = mp.mpf(float(x[0])) + mp.mpf(float(x[1]))
        err = max(abs(mp.mpf(val(sx).numerator) / val(sx).denominator - mp.sin(xv)),
                  abs(mp.mpf(val(cx).numerator) / val(cx).denominator - mp.cos(xv)))
        worst = max(worst, float(err))
    assert worst <= 2.0 ** -49, worst


def cmul_t(a, b, norm, conj):
    """The complex product of the paired sweep, restated in float steps."""
    (axh, axl), (ayh, ayl) = a
    (bxh, bxl), (byh, byl) = b
    nax, nay, nayl = -axh, -ayh, -ayl
    q1 = mul(axh, bxh)
    c1 = fma(nax, bxh, q1)
    q2 = mul(ayh, byh) if conj else mul(nay, byh)
    c2 = fma(nay, byh, q2) if conj else fma(ayh, byh, q2)
    s, lo = two_sum(q1, q2)
    er = sub(sub(lo, c1), c2)
    er = fma(axh, bxl, er)
    er = fma(axl, bxh, er)
    er = fma(ayh if conj else nay, byl, er)
    er = fma(ayl if conj else nayl, byh, er)
    re = fast_two_sum(s, er) if norm else (s, er)
    q3 = mul(axh, byh)
    c3 = fma(nax, byh, q3)
    q4 = mul(nay, bxh) if conj else mul(ayh, bxh)
    c4 = fma(ayh, bxh, q4) if conj else fma(nay, bxh, q4)
    s, lo = two_sum(q3, q4)
    ei = sub(sub(lo, c3), c4)
    ei = fma(axh, byl, ei)
    ei = fma(axl, byh, ei)
    ei = fma(nay if conj else ayh, bxl, ei)
    ei = fma(nayl if conj else ayl, bxh, ei)
    im = fast_two_sum(s, ei) if norm else (s, ei)
    return re, im


@pytest.mark.parametrize("conj", [False, True])
@pytest.mark.parametrize("norm", [False, True])
def test_complex_product_with_shared_negations(conj, norm):
    mp.mp.prec = 200
    rng = np.random.default_rng(13 + 2 * conj + norm)

    def rdd():
        return split(mp.mpf(rng.standard_normal()) * mp.mpf(10) ** rng.uniform(-2, 2))

    worst = 0.0
    for _ in range(1500):
        a, b = (rdd(), rdd()), (rdd(), rdd())
        ax, ay, bx, by = (val(t) for t in (a[0], a[1], b[0], b[1]))
        if conj:
            ay = -ay
        re, im = cmul_t(a, b, norm, conj)
        scale = (abs(ax) + abs(ay)) * (abs(bx) + abs(by))
        err = max(abs(val(re) - (ax * bx - ay * by)), abs(val(im) - (ax * by + ay * bx))) / scale
        worst = max(worst, float(err))
    assert worst <= 8 * 2.0 ** -48, worst
