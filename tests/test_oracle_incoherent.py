"""Pins of the incoherent-layer oracle (``oracle/incoherent.py``) on the CPU.

The strongest pin is independent of its combination rule: a lossless thick
layer treated incoherently must equal the coherent result averaged over one
full period of that layer's round-trip phase (the Airy response averaged over
phase is the incoherent sum); a uniform grid of thicknesses over the period
converges exponentially.  Several incoherent layers are pinned by invariances
(splitting a homogeneous thick region, reversal of a lossless stack); plus
closed forms (a bare slab: R = 2 R1 / (1 + R1)), the all-coherent limit,
energy conservation, the evanescent-layer reading and the rejection of
absorbing incoherent layers."""
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
        assert np.max(np.abs(Rc - Ri)) < 1e-15 and np.max(np.abs(Tc - Ti)) < 1e-15


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


def test_absorbing_incoherent_layer_is_rejected():
    n = media(1.0, 1.5 + 0.01j, 1.0)
    R, T = inc.inc_tmm("s", n, np.array([[1e5]]), np.array([[1]]), np.array([0.0]), LAM)
    assert np.isnan(R).all() and np.isnan(T).all()
