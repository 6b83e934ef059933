"""Pins of the incoherent-layer oracle (``oracle/incoherent.py``) on the CPU.

The strongest pin is independent of its combination rule: a lossless thick
layer treated incoherently must equal the coherent result averaged over one
full period of that layer's round-trip phase (the Airy response averaged over
phase is the incoherent sum); a uniform grid of thicknesses over the period
converges exponentially.  Several incoherent layers are pinned by invariances
(splitting a homogeneous thick region, reversal of a lossless stack); plus
closed forms (a bare slab: R = 2 R1 / (1 + R1)), the all-coherent limit,
energy conservation and the evanescent-layer reading.  Absorbing incoherent
layers: the block coefficients against the C oracle, the closed form of a
free-standing absorbing slab (Beer-Lambert single-pass factor, Fresnel
coefficients of complex index, multiple passes summed), the opaque and the
lossless limits, and the phase average of a weakly absorbing slab."""
import numpy as np
import pytest

import oracle
from oracle import incoherent as inc

LAM = np.array([600.0])


def media(*ns):
    return np.array([list(ns)], dtype=np.complex128)[:, :, None]


def phase_period(n_layer, beta, lam):
    cos_t = np.sqrt(1.0 - (beta / n_layer) ** 2)
    return lam / (2.0 * n_layer * cos_t)


@pytest.mark.parametrize("pol", ["s", "p"])
@pytest.mark.parametrize("theta_deg", [0.0, 40.0, 75.0])
@pytest.mark.parametrize("coating", [2.0, 2.0 + 0.15j])
def test_incoherent_slab_equals_phase_averaged_coherent(pol, theta_deg, coating):
    th = np.deg2rad(theta_deg)
    n = media(1.0, coating, 1.5, 1.0)
    N = 96
    d_slab = 1e6 + phase_period(1.5, np.sin(th), 600.0) * np.arange(N) / N
    d = np.stack([np.full(N, 100.0), d_slab], axis=1)
    Rc, Tc = oracle.coh_tmm(pol, np.repeat(n, N, axis=0), d, np.array([th]), LAM)
    Ri, Ti = inc.inc_tmm(pol, n, d[:1], np.array([[0, 1]]), np.array([th]), LAM)
    assert abs(Rc.mean() - Ri[0, 0, 0]) < 1e-12
    assert abs(Tc.mean() - Ti[0, 0, 0]) < 1e-12


def test_several_incoherent_layers_combine_consistently():
    # (a) a homogeneous thick region split into two incoherent layers (an
    # interface between equal media) is the same as one layer; (b) T of a
    # lossless stack does not depend on the side the light comes from.
    # With two or more incoherent layers the intensity method leaves out the
    # interference of paths that cross each layer equally often in another
    # order, so averaging over independent phases differs (3.4e-4 here): that
    # is the method, not an error.
    th = np.deg2rad(30.0)
    for pol in "sp":
        one = inc.inc_tmm(pol, media(1.0, 1.9, 1.45, 2.2, 1.33), np.array([[90.0, 3e5, 70.0]]),
                          np.array([[0, 1, 0]]), np.array([th]), LAM)
        two = inc.inc_tmm(pol, media(1.0, 1.9, 1.45, 1.45, 2.2, 1.33), np.array([[90.0, 1e5, 2e5, 70.0]]),
                          np.array([[0, 1, 1, 0]]), np.array([th]), LAM)
        assert abs(one[0][0, 0, 0] - two[0][0, 0, 0]) < 1e-15 and abs(one[1][0, 0, 0] - two[1][0, 0, 0]) < 1e-15
        # reversal: same beta, entering from the 1.33 side
        n_f = media(1.33, 1.9, 1.45, 2.2, 1.6, 1.33)
        n_r = media(1.33, 1.6, 2.2, 1.45, 1.9, 1.33)
        d_f = np.array([[90.0, 3e5, 70.0, 7e5]])
        f = inc.inc_tmm(pol, n_f, d_f, np.array([[0, 1, 0, 1]]), np.array([th]), LAM)
        r = inc.inc_tmm(pol, n_r, d_f[:, ::-1].copy(), np.array([[1, 0, 1, 0]]), np.array([th]), LAM)
        assert abs(f[1][0, 0, 0] - r[1][0, 0, 0]) < 1e-14


@pytest.mark.parametrize("pol", ["s", "p"])
def test_bare_thick_slab_closed_form(pol):
    th = np.deg2rad(50.0)
    n = media(1.0, 1.5, 1.0)
    Ri, Ti = inc.inc_tmm(pol, n, np.array([[5e5]]), np.array([[1]]), np.array([th]), LAM)
    R1, _ = oracle.coh_tmm(pol, media(1.0, 1.5), np.zeros((1, 0)), np.array([th]), LAM)
    R1 = R1[0, 0, 0]
    assert abs(Ri[0, 0, 0] - 2 * R1 / (1 + R1)) < 1e-14
    assert abs(Ri[0, 0, 0] + Ti[0, 0, 0] - 1.0) < 1e-14


def test_no_incoherent_layer_is_the_coherent_oracle():
    rng = np.random.default_rng(4)
    S, L = 3, 5
    lam = np.linspace(450.0, 700.0, 6)
    n = np.empty((S, L + 2, lam.size), dtype=np.complex128)
    n[:, 0] = 1.0
    n[:, 1:L + 1] = (rng.uniform(1.3, 2.4, (S, L)) + 1j * rng.uniform(0, 0.05, (S, L)))[:, :, None]
    n[:, L + 1] = 1.52
    d = rng.uniform(20, 300, (S, L))
    th = np.deg2rad([0.0, 35.0])
    for pol in "sp":
        Rc, Tc = oracle.coh_tmm(pol, n, d, th, lam)
        Ri, Ti = inc.inc_tmm(pol, n, d, np.zeros((S, L)), th, lam)
        # the incoherent oracle evaluates blocks with its own restatement of
        # the coherent method (block_RT): equal up to rounding order
        assert np.max(np.abs(Rc - Ri)) < 1e-13 and np.max(np.abs(Tc - Ti)) < 1e-13


def test_energy_balance():
    th = np.deg2rad([0.0, 20.0, 60.0])
    flags = np.array([[0, 1, 0, 1]])
    d = np.array([[80.0, 2e5, 120.0, 4e5]])
    lossless = media(1.0, 2.1, 1.5, 1.7, 1.45, 1.0)
    lossy = media(1.0, 2.1 + 0.2j, 1.5, 1.7, 1.45, 1.0)
    for pol in "sp":
        R, T = inc.inc_tmm(pol, lossless, d, flags, th, LAM)
        assert np.max(np.abs(R + T - 1.0)) < 1e-14
        R, T = inc.inc_tmm(pol, lossy, d, flags, th, LAM)
        assert np.all(R + T < 1.0 - 1e-3)


def test_evanescent_incoherent_layer_passes_no_power():
    # injection 1.8 at 70 deg: n sin(theta) = 1.69 > 1.5, the slab is evanescent
    th = np.deg2rad(70.0)
    n = media(1.8, 2.2, 1.5, 2.0, 1.0)
    d = np.array([[110.0, 1e6, 90.0]])
    for pol in "sp":
        R, T = inc.inc_tmm(pol, n, d, np.array([[0, 1, 0]]), np.array([th]), LAM)
        Rc, _ = oracle.coh_tmm(pol, media(1.8, 2.2, 1.5), d[:, :1], np.array([th]), LAM)
        assert T[0, 0, 0] == 0.0 and abs(R[0, 0, 0] - Rc[0, 0, 0]) < 1e-15


def _fresnel(pol, n1, n2, beta):
    """r, t of Eq. 1 and the Poynting factor k2 / k1 for interface n1 | n2."""
    q1, q2 = inc.forward_root(n1 * n1 - beta * beta), inc.forward_root(n2 * n2 - beta * beta)
    c1, c2 = q1 / n1, q2 / n2
    if pol == "s":
        a, b = n1 * c1, n2 * c2
        r, t = (a - b) / (a + b), 2 * a / (a + b)
        f = (n2 * c2).real / (n1 * c1).real
    else:
        a, b = n2 * c1, n1 * c2
        r, t = (a - b) / (a + b), 2 * n1 * c1 / (a + b)
        f = (n2 * np.conj(c2)).real / (n1 * np.conj(c1)).real
    return r, t, f, q2


@pytest.mark.parametrize("pol", ["s", "p"])
def test_block_coefficients_equal_the_c_oracle(pol):
    # block_RT (numpy, beta given) against oracle.coh_tmm (C, theta given) on
    # blocks between real media, with absorbing layers and an absorbing exit
    rng = np.random.default_rng(8)
    for trial in range(6):
        L = int(rng.integers(0, 6))
        nl = list(rng.uniform(1.3, 2.4, L) + 1j * rng.uniform(0, 0.1, L))
        n_blk = np.array([1.0 + 0.4 * (trial % 2)] + nl + [1.52 + 0.02j * (trial % 3)], dtype=np.complex128)
        d_blk = rng.uniform(20, 300, L)
        th = np.deg2rad(rng.uniform(0, 70))
        R, T = oracle.coh_tmm(pol, n_blk[None, :, None], d_blk[None], np.array([th]), LAM)
        Rb, Tb = inc.block_RT(pol, n_blk, d_blk, n_blk[0].real * np.sin(th), LAM[0])
        assert abs(R[0, 0, 0] - Rb) < 1e-13 and abs(T[0, 0, 0] - Tb) < 1e-13


@pytest.mark.parametrize("pol", ["s", "p"])
@pytest.mark.parametrize("theta_deg", [0.0, 35.0, 70.0])
def test_absorbing_slab_closed_form(pol, theta_deg):
    # free-standing slab n = 1.5 + i k in air, incoherent: every pass through
    # it is attenuated by P = exp(-4 pi Im(q) d / lambda) (Beer-Lambert along
    # the oblique path); front and back interfaces reflect R1 = |r|^2 from
    # either side, and the slab transmits T01 T10 of the power in and out:
    #   R = R1 + T01 T10 R1 P^2 / (1 - R1^2 P^2),  T = T01 T10 P / (1 - R1^2 P^2)
    beta = np.sin(np.deg2rad(theta_deg))
    for k in (1e-6, 3e-5, 2e-3):
        ns = 1.5 + 1j * k
        d = 2e5
        r01, t01, f01, q1 = _fresnel(pol, 1.0 + 0j, ns, beta)
        r10, t10, f10, _ = _fresnel(pol, ns, 1.0 + 0j, beta)
        R1 = abs(r01) ** 2
        assert abs(abs(r10) ** 2 - R1) < 1e-15
        T01, T10 = f01 * abs(t01) ** 2, f10 * abs(t10) ** 2
        P = np.exp(-4 * np.pi * q1.imag * d / LAM[0])
        R_cf = R1 + T01 * T10 * R1 * P * P / (1 - R1 * R1 * P * P)
        T_cf = T01 * T10 * P / (1 - R1 * R1 * P * P)
        R, T = inc.inc_tmm(pol, media(1.0, ns, 1.0), np.array([[d]]), np.array([[1]]),
                           np.array([np.deg2rad(theta_deg)]), LAM)
        assert abs(R[0, 0, 0] - R_cf) < 1e-14 and abs(T[0, 0, 0] - T_cf) < 1e-14
        assert 0.0 < P < 1.0 and R[0, 0, 0] + T[0, 0, 0] < 1.0


def test_opaque_and_lossless_limits():
    th = np.array([np.deg2rad(25.0)])
    for pol in "sp":
        # opaque incoherent absorber: R of the front structure with it as the
        # exit medium, T = 0
        n = media(1.0, 2.0, 1.5 + 0.05j, 1.0)
        R, T = inc.inc_tmm(pol, n, np.array([[90.0, 1e6]]), np.array([[0, 1]]), th, LAM)
        Rc, _ = oracle.coh_tmm(pol, media(1.0, 2.0, 1.5 + 0.05j), np.array([[90.0]]), th, LAM)
        assert abs(R[0, 0, 0] - Rc[0, 0, 0]) < 1e-14 and T[0, 0, 0] < 1e-300
        # a vanishing extinction coefficient gives the lossless result
        d = np.array([[90.0, 3e5, 60.0]])
        f = np.array([[0, 1, 0]])
        R0, T0 = inc.inc_tmm(pol, media(1.0, 2.0, 1.5, 1.8, 1.0), d, f, th, LAM)
        R1, T1 = inc.inc_tmm(pol, media(1.0, 2.0, 1.5 + 1e-13j, 1.8, 1.0), d, f, th, LAM)
        assert abs(R0[0, 0, 0] - R1[0, 0, 0]) < 1e-8 and abs(T0[0, 0, 0] - T1[0, 0, 0]) < 1e-8


@pytest.mark.parametrize("pol", ["s", "p"])
def test_weakly_absorbing_slab_is_the_phase_average(pol):
    # with k = 1e-7 the single-pass factor changes by 4e-7 over one phase
    # period, so the coherent average over the period equals the incoherent
    # result to that order
    th = np.deg2rad(30.0)
    ns = 1.5 + 1e-7j
    n = media(1.0, 2.0, ns, 1.0)
    N = 96
    d_slab = 1e5 + phase_period(1.5, np.sin(th), 600.0) * np.arange(N) / N
    d = np.stack([np.full(N, 100.0), d_slab], axis=1)
    Rc, Tc = oracle.coh_tmm(pol, np.repeat(n, N, axis=0), d, np.array([th]), LAM)
    Ri, Ti = inc.inc_tmm(pol, n, d[:1], np.array([[0, 1]]), np.array([th]), LAM)
    assert abs(Rc.mean() - Ri[0, 0, 0]) < 2e-6 and abs(Tc.mean() - Ti[0, 0, 0]) < 2e-6


def test_complex_injection_medium_is_rejected():
    n = media(1.0 + 0.01j, 1.5, 1.0)
    R, T = inc.inc_tmm("s", n, np.array([[1e5]]), np.array([[1]]), np.array([0.0]), LAM)
    assert np.isnan(R).all() and np.isnan(T).all()
