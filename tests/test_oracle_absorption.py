"""Pins of the per-layer absorption oracle (``oracle/absorption.py``) on the CPU.

Its R and T come from the same amplitudes as its absorption integrals, so
they are checked against the paper-steps C oracle; the absorption integrals
are pinned by energy balance R + T + sum_j A_j = 1 (lossy layers and a lossy
substrate, both polarisations, oblique incidence), by exact zeros in lossless
layers, and by Beer-Lambert attenuation in an index-matched weak absorber."""
import numpy as np
import pytest

import oracle
from oracle import absorption as ab


def lossy_stacks(seed, S=3, L=5, n_lambda=7):
    rng = np.random.default_rng(seed)
    lam = np.linspace(400.0, 800.0, n_lambda)
    n = np.empty((S, L + 2, n_lambda), dtype=np.complex128)
    n[:, 0] = 1.0
    n[:, 1:L + 1] = (rng.uniform(1.3, 2.4, (S, L)) + 1j * rng.uniform(0.0, 0.3, (S, L)))[:, :, None]
    n[:, L + 1] = 1.52 + 0.05j
    d = rng.uniform(20.0, 300.0, (S, L))
    return n, d, lam


@pytest.mark.parametrize("pol", ["s", "p"])
def test_R_T_agree_with_the_paper_steps_oracle(pol):
    n, d, lam = lossy_stacks(1)
    th = np.deg2rad([0.0, 30.0, 70.0])
    A, R, T = ab.absorption(pol, n, d, th, lam)
    Ro, To = oracle.coh_tmm(pol, n, d, th, lam)
    assert np.max(np.abs(R - Ro)) < 1e-14 and np.max(np.abs(T - To)) < 1e-14


@pytest.mark.parametrize("pol", ["s", "p"])
def test_energy_balance(pol):
    n, d, lam = lossy_stacks(2)
    th = np.deg2rad([0.0, 25.0, 55.0, 80.0])
    A, R, T = ab.absorption(pol, n, d, th, lam)
    assert np.max(np.abs(R + T + A.sum(axis=1) - 1.0)) < 1e-13
    assert np.all(A >= 0.0) and np.all(A.sum(axis=1) > 1e-3)


def test_lossless_layers_absorb_nothing():
    n, d, lam = lossy_stacks(3)
    n[:, 2] = n[:, 2].real  # layer 2 lossless
    A, _, _ = ab.absorption("p", n, d, np.deg2rad([10.0, 40.0]), lam)
    assert np.all(A[:, 1] == 0.0)
    assert np.all(A[:, 0] > 0.0)


@pytest.mark.parametrize("theta_deg", [0.0, 35.0])
def test_beer_lambert_in_an_index_matched_absorber(theta_deg):
    # n = 1.5 + i kappa between n = 1.5 media: reflections are O(kappa^2) and
    # the absorbed fraction is 1 - exp(-2 Im(k0 q) d)
    kap, d, lam = 1e-3, 5e4, 600.0
    th = np.deg2rad(theta_deg)
    n = np.array([[[1.5], [1.5 + 1j * kap], [1.5]]])
    for pol in "sp":
        A, R, _ = ab.absorption(pol, n, np.array([[d]]), np.array([th]), np.array([lam]))
        q = np.sqrt((1.5 + 1j * kap) ** 2 - (1.5 * np.sin(th)) ** 2)
        expect = 1.0 - np.exp(-2 * (2 * np.pi / lam) * q.imag * d)
        assert abs(A[0, 0, 0, 0] - expect) < 1e-6 and R[0, 0, 0] < 1e-6


def test_layers_past_L_s_are_zero():
    n, d, lam = lossy_stacks(4, S=3, L=6)
    Ls = np.array([6, 2, 4], dtype=np.int32)
    for s in range(3):
        n[s, Ls[s] + 1:] = n[s, 7]
    A, R, T = ab.absorption("s", n, d, np.array([0.2]), lam, L_per_stack=Ls)
    for s in range(3):
        assert np.all(A[s, Ls[s]:] == 0.0)
    assert np.max(np.abs(R + T + A.sum(axis=1) - 1.0)) < 1e-13


@pytest.mark.parametrize("pol", ["s", "p"])
def test_field_profile_integrates_to_the_absorbed_fraction(pol):
    # k0 Im(n^2) |E / E_inc|^2 is the absorption density per incident flux
    # (times the flux of a unit incident wave); its midpoint-rule integral over
    # each layer converges to A_j
    n, d, lam = lossy_stacks(5, S=2, L=4, n_lambda=3)
    n0 = 1.3  # a denser injection medium pins the n_0^2 of the p normalisation
    n[:, 0] = n0
    th = np.deg2rad([0.0, 50.0])
    A, _, _ = ab.absorption(pol, n, d, th, lam)
    nz = 400
    E2 = ab.field_profile(pol, n, d, th, lam, nz)
    k0 = 2 * np.pi / lam
    flux_inc = np.cos(th)[:, None] * n0 if pol == "s" else np.cos(th)[:, None] / n0
    im_eps = (n[:, 1:5, :] ** 2).imag                       # [S][L][N_lambda]
    dens = k0 * im_eps[:, :, None, None, :] * E2            # [S][L][n_z][N_theta][N_lambda]
    if pol == "p":
        dens = dens / n0 ** 2
    integral = dens.mean(axis=2) * d[:, :, None, None] / flux_inc[None, None]
    assert np.max(np.abs(integral - A)) < 2e-5


def test_field_profile_of_a_bare_interface_region():
    # no layer reflects: an index-matched lossless layer carries the incident
    # wave unchanged, |E / E_inc|^2 = 1 (s) and, for p, the same
    n = np.array([[[1.5], [1.5], [1.5]]], dtype=np.complex128)
    for pol in "sp":
        E2 = ab.field_profile(pol, n, np.array([[300.0]]), np.deg2rad([30.0]), np.array([600.0]), 5)
        assert np.max(np.abs(E2 - 1.0)) < 1e-14
