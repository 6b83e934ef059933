"""Pins of the partially coherent oracle (``oracle/partial.py``) on the CPU.

* A single non-absorbing film: T(delta) = (1 - r01^2)(1 - r12^2) /
  |1 + r01 r12 e^{2 i delta}|^2 expands (Poisson kernel) into
  T_inc [1 + 2 sum_m (-r01 r12)^m cos(2 m delta)], so its Gaussian average
  over delta ~ N(delta_0, s^2) is the series with each term damped by
  e^{-2 m^2 s^2}, s = 2 pi n1 cos(theta_1) sigma / lambda: a closed form.
* An absorbing multilayer: the Gauss-Hermite average against a dense
  trapezoid integral of the coherent R, T over the normal density (an
  independent quadrature of the same expectation).
* sigma = 0 is the coherent stack; energy balance for lossless stacks; the
  series' constant term, the limit of a wide spread, is the incoherent-layer
  result of ``incoherent.py``.
The Gauss-Hermite rule resolves the fringe harmonics only up to a frequency
that grows like sqrt(K): wider spreads need more nodes (measured here: 3 nm
16 nodes, 25 nm 64, 60 nm 256 for errors below 1e-9 on a 2 um film).
"""
import numpy as np
import pytest

import oracle
from oracle import incoherent as inc
from oracle import partial as pc


def film(n0, n1, n2, d, n_lambda):
    n = np.array([[n0, n1, n2]], dtype=np.complex128)
    return np.repeat(n[:, :, None], n_lambda, axis=2), np.array([[d]])


def film_coeffs(pol, n0, n1, n2, theta):
    beta = n0 * np.sin(theta)
    c = [np.sqrt(1 - (beta / n) ** 2) for n in (n0, n1, n2)]
    if pol == "s":
        y = [n * x for n, x in zip((n0, n1, n2), c)]
        r01 = (y[0] - y[1]) / (y[0] + y[1])
        r12 = (y[1] - y[2]) / (y[1] + y[2])
    else:
        r01 = (n1 * c[0] - n0 * c[1]) / (n1 * c[0] + n0 * c[1])
        r12 = (n2 * c[1] - n1 * c[2]) / (n2 * c[1] + n1 * c[2])
    return r01, r12, c


def closed_form_T(pol, n0, n1, n2, d, sigma, theta, lam, terms=60):
    r01, r12, c = film_coeffs(pol, n0, n1, n2, theta)
    rho = r01 * r12
    T_inc = (1 - r01 ** 2) * (1 - r12 ** 2) / (1 - rho ** 2)
    delta0 = 2 * np.pi * n1 * c[1] * d / lam
    s = 2 * np.pi * n1 * c[1] * sigma / lam
    m = np.arange(1, terms + 1)[:, None]
    series = 1 + 2 * np.sum((-rho) ** m * np.cos(2 * m * delta0) * np.exp(-2 * m ** 2 * s ** 2), axis=0)
    return T_inc * series


@pytest.mark.parametrize("pol", ["s", "p"])
@pytest.mark.parametrize("sigma,K,tol", [(3.0, 16, 1e-13), (25.0, 64, 1e-10), (60.0, 256, 1e-9)])
def test_single_film_against_the_closed_form(pol, sigma, K, tol):
    lam = np.linspace(420.0, 780.0, 41)
    th = np.deg2rad([0.0, 35.0])
    n, d = film(1.0, 2.1, 1.52, 2000.0, lam.size)
    R, T = pc.pcoh_tmm(pol, n, d, [1], [sigma], th, lam, n_nodes=K)
    for a, t in enumerate(th):
        ref = closed_form_T(pol, 1.0, 2.1, 1.52, 2000.0, sigma, t, lam)
        assert np.max(np.abs(T[0, a] - ref)) < tol
        assert np.max(np.abs(R[0, a] + T[0, a] - 1.0)) < 1e-13


@pytest.mark.parametrize("pol", ["s", "p"])
def test_absorbing_multilayer_against_a_trapezoid_integral(pol):
    rng = np.random.default_rng(7)
    lam = np.linspace(450.0, 700.0, 9)
    th = np.deg2rad([0.0, 50.0])
    L, j, sigma = 5, 3, 40.0
    n = np.empty((1, L + 2, lam.size), dtype=np.complex128)
    n[:, 0] = 1.0
    n[0, 1:L + 1] = (rng.uniform(1.4, 2.4, L) + 1j * rng.uniform(0.0, 0.08, L))[:, None]
    n[:, L + 1] = 1.52
    d = rng.uniform(50.0, 300.0, (1, L))
    d[0, j - 1] = 900.0
    R, T = pc.pcoh_tmm(pol, n, d, [j], [sigma], th, lam, n_nodes=48)
    # trapezoid over D in [-9 sigma, 9 sigma] against the normal density
    D = np.linspace(-9 * sigma, 9 * sigma, 3601)
    dens = np.exp(-0.5 * (D / sigma) ** 2) / (sigma * np.sqrt(2 * np.pi))
    dd = np.repeat(d, D.size, axis=0)
    dd[:, j - 1] += D
    Rd, Td = oracle.coh_tmm(pol, np.repeat(n, D.size, axis=0), dd, th, lam)
    wt = dens * (D[1] - D[0])
    wt[[0, -1]] *= 0.5
    assert np.max(np.abs(R[0] - np.einsum("kab,k->ab", Rd, wt))) < 1e-10
    assert np.max(np.abs(T[0] - np.einsum("kab,k->ab", Td, wt))) < 1e-10
    assert np.all(R + T < 1.0)


def test_zero_spread_and_no_layer_are_coherent():
    rng = np.random.default_rng(8)
    lam = np.linspace(400.0, 800.0, 7)
    th = np.deg2rad([10.0, 60.0])
    n = np.empty((3, 6, lam.size), dtype=np.complex128)
    n[:, 0] = 1.0
    n[:, 1:5] = (rng.uniform(1.3, 2.5, (3, 4)) + 1j * rng.uniform(0, 0.1, (3, 4)))[:, :, None]
    n[:, 5] = 1.52
    d = rng.uniform(20.0, 400.0, (3, 4))
    for pol in "sp":
        R0, T0 = oracle.coh_tmm(pol, n, d, th, lam)
        R, T = pc.pcoh_tmm(pol, n, d, [2, 0, 4], [0.0, 50.0, 0.0], th, lam, n_nodes=9)
        assert np.max(np.abs(R - R0)) < 1e-14 and np.max(np.abs(T - T0)) < 1e-14


@pytest.mark.parametrize("pol", ["s", "p"])
def test_wide_spread_limit_is_the_incoherent_layer(pol):
    # the series' constant term (1 - r01^2)(1 - r12^2) / (1 - r01^2 r12^2) is
    # the film treated as an incoherent layer by the intensity method
    lam = np.linspace(450.0, 750.0, 7)
    th = np.deg2rad([0.0, 40.0])
    n = np.repeat(np.array([[1.0, 2.1, 1.52]])[:, :, None], lam.size, axis=2).astype(np.complex128)
    _, Ti = inc.inc_tmm(pol, n, np.array([[2000.0]]), np.array([[1]], dtype=bool), th, lam)
    for a, t in enumerate(th):
        r01, r12, _ = film_coeffs(pol, 1.0, 2.1, 1.52, t)
        T_inc = (1 - r01 ** 2) * (1 - r12 ** 2) / (1 - (r01 * r12) ** 2)
        assert np.max(np.abs(Ti[0, a] - T_inc)) < 1e-13


def test_node_count_is_bounded():
    with pytest.raises(ValueError):
        pc.gauss_hermite(257)


def test_ragged_and_invalid_stacks():
    lam = np.array([500.0, 650.0])
    th = np.array([0.3])
    n = np.empty((4, 5, 2), dtype=np.complex128)
    n[:, 0] = 1.0
    n[:, 1:4] = 1.8 + 0.01j
    n[:, 4] = 1.52
    d = np.full((4, 3), 150.0)
    Ls = np.array([3, 1, 2, 3])
    for s in range(4):
        n[s, Ls[s] + 1:] = 1.52
    R, T = pc.pcoh_tmm("s", n, d, [3, 1, 3, 2], [20.0, 20.0, 20.0, -1.0], th, lam, n_nodes=8, L_per_stack=Ls)
    assert np.all(np.isfinite(R[:2])) and np.all(np.isnan(R[2:])) and np.all(np.isnan(T[2:]))
    # a partial layer in the one-layer stack: its own thickness average
    R1, _ = pc.pcoh_tmm("s", n[1:2, :3], d[1:2, :1], [1], [20.0], th, lam, n_nodes=8)
    assert np.max(np.abs(R[1] - R1[0])) < 1e-14
