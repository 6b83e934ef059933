"""Pins for the oracle: closed forms, invariants and an independent formulation.

Each test fixes the oracle against something other than itself: textbook
values (single interface, Brewster, total internal reflection), closed forms
(Airy single layer, quarter-wave stack, half-wave absentee layer), physical
invariants stated in the paper (R + T = 1 without absorption, s = p at normal
incidence; Sec. 2 after Eqs. 1-2) or implied by the method (zero-thickness and
index-matched layers, transmittance reciprocity, independence of the interior
square-root choice), the characteristic-matrix formulation of the same problem,
and central finite differences for the gradient.
"""
import numpy as np
import pytest

import oracle
from oracle.admittance import coh_tmm_admittance
from paper_2111_13667_gb300 import workloads as W
from tests.helpers import oracle_index, oracle_RT, stack


def RT(pol, n_media, d, theta, lam):
    n, dd = stack(n_media, d, n_lambda=np.size(lam))
    R, T = oracle.coh_tmm(pol, n, dd, np.atleast_1d(theta), np.atleast_1d(lam))
    return R[0], T[0]


# ---------------------------------------------------------------- single interface
def test_single_interface_normal_incidence_air_glass():
    # ((1 - 1.5) / (1 + 1.5))^2 = 0.04 exactly; T = 0.96.
    for pol in "sp":
        R, T = RT(pol, [1.0, 1.5], [], 0.0, 500.0)
        assert abs(R[0, 0] - 0.04) < 1e-15
        assert abs(T[0, 0] - 0.96) < 1e-15


def test_single_interface_brewster_and_s_value():
    n1, n2 = 1.0, 1.5
    tb = np.arctan(n2 / n1)
    Rs, _ = RT("s", [n1, n2], [], tb, 600.0)
    Rp, Tp = RT("p", [n1, n2], [], tb, 600.0)
    assert Rp[0, 0] < 1e-28
    assert abs(Tp[0, 0] - 1.0) < 1e-14
    # At Brewster's angle r_s = (n1^2 - n2^2) / (n1^2 + n2^2).
    assert abs(Rs[0, 0] - ((n1**2 - n2**2) / (n1**2 + n2**2)) ** 2) < 1e-14


def test_total_internal_reflection():
    th = np.deg2rad([45.0, 60.0, 89.0])  # critical angle asin(1/1.5) = 41.8 deg
    for pol in "sp":
        R, T = RT(pol, [1.5, 1.0], [], th, 500.0)
        assert np.allclose(R[:, 0], 1.0, atol=1e-14)
        assert np.allclose(T[:, 0], 0.0, atol=1e-14)


def test_grazing_incidence_reading():
    for pol in "sp":
        R, T = RT(pol, [1.0, 1.8, 1.52], [100.0], np.pi / 2, 500.0)
        assert R[0, 0] == 1.0 and T[0, 0] == 0.0


# ---------------------------------------------------------------- closed forms
def _airy(pol, n0, n1, n2, d, theta, lam):
    """Single film by summing the multiple-reflection series (Airy form)."""
    beta = n0 * np.sin(theta)
    c = [np.sqrt(1 - (beta / n) ** 2 + 0j) for n in (n0, n1, n2)]
    c = [(-x if (n * x).imag < 0 else x) for n, x in zip((n0, n1, n2), c)]
    if pol == "s":
        y = [n * x for n, x in zip((n0, n1, n2), c)]
        r01 = (y[0] - y[1]) / (y[0] + y[1])
        r12 = (y[1] - y[2]) / (y[1] + y[2])
    else:
        r01 = (n1 * c[0] - n0 * c[1]) / (n1 * c[0] + n0 * c[1])
        r12 = (n2 * c[1] - n1 * c[2]) / (n2 * c[1] + n1 * c[2])
    ph = np.exp(2j * 2 * np.pi * n1 * d * c[1] / lam)
    r = (r01 + r12 * ph) / (1 + r01 * r12 * ph)
    return abs(r) ** 2


@pytest.mark.parametrize("n1", [1.9, 2.3 + 0.05j, 1.3 + 0.4j])
@pytest.mark.parametrize("pol", ["s", "p"])
def test_airy_single_layer(n1, pol):
    lam = np.linspace(400, 900, 37)
    th = np.deg2rad([0.0, 30.0, 65.0])
    n, d = stack([1.0, n1, 1.52], [137.0], n_lambda=lam.size)
    R, _ = oracle.coh_tmm(pol, n, d, th, lam)
    for a, t in enumerate(th):
        ref = np.array([_airy(pol, 1.0, n1, 1.52, 137.0, t, l) for l in lam])
        assert np.max(np.abs(R[0, a] - ref)) < 1e-13


@pytest.mark.parametrize("N", list(range(1, 11)))
def test_quarter_wave_stack(N):
    # ambient | (H L)^N | substrate at the design wavelength, normal incidence:
    # admittance Y = (nH / nL)^(2N) ns, R = ((n0 - Y) / (n0 + Y))^2.
    n0, nH, nL, ns, lam0 = 1.0, 2.35, 1.46, 1.52, 600.0
    media = [n0] + [nH, nL] * N + [ns]
    d = [lam0 / (4 * nH), lam0 / (4 * nL)] * N
    Y = (nH / nL) ** (2 * N) * ns
    ref = ((n0 - Y) / (n0 + Y)) ** 2
    for pol in "sp":
        R, T = RT(pol, media, d, 0.0, lam0)
        assert abs(R[0, 0] - ref) < 1e-13
        assert abs(R[0, 0] + T[0, 0] - 1.0) < 1e-13


def test_half_wave_absentee_layer():
    n0, nf, ns, lam0 = 1.0, 2.1, 1.52, 550.0
    R, _ = RT("s", [n0, nf, ns], [lam0 / (2 * nf)], 0.0, lam0)
    assert abs(R[0, 0] - ((n0 - ns) / (n0 + ns)) ** 2) < 1e-14


# ---------------------------------------------------------------- invariants
def _random_stack(rng, L, absorbing, S=4):
    n = np.empty((S, L + 2), dtype=np.complex128)
    n[:, 0] = 1.0
    n[:, 1:L + 1] = rng.uniform(1.3, 2.6, (S, L)) + (1j * rng.uniform(0, 0.3, (S, L)) if absorbing else 0)
    n[:, L + 1] = 1.52
    d = rng.uniform(5, 400, (S, L))
    return n, d


LAM = np.linspace(380.0, 1100.0, 41)
THETA = np.deg2rad(np.linspace(0, 85, 9))


def _full(n):
    return np.repeat(n[:, :, None], LAM.size, axis=2)


@pytest.mark.parametrize("pol", ["s", "p"])
def test_lossless_R_plus_T_is_one(pol):
    rng = np.random.default_rng(10)
    n, d = _random_stack(rng, 17, absorbing=False)
    R, T = oracle.coh_tmm(pol, _full(n), d, THETA, LAM)
    assert np.max(np.abs(R + T - 1.0)) < 1e-12


@pytest.mark.parametrize("pol", ["s", "p"])
def test_lossless_with_total_internal_reflection(pol):
    # injection index 2, outcoupling into air: beyond 30 deg T = 0 and R = 1.
    w = W.map_x3()
    R, T = oracle.coh_tmm(pol, oracle_index(w), w.d, w.theta, w.lam)
    assert np.max(np.abs(R + T - 1.0)) < 1e-11
    beyond = np.sin(w.theta) * 2.0 > 1.0 + 1e-9
    assert np.max(np.abs(T[0, beyond])) < 1e-12


@pytest.mark.parametrize("pol", ["s", "p"])
def test_absorbing_R_plus_T_below_one(pol):
    rng = np.random.default_rng(11)
    n, d = _random_stack(rng, 11, absorbing=True)
    R, T = oracle.coh_tmm(pol, _full(n), d, THETA, LAM)
    assert np.all(R >= 0) and np.all(T >= 0)
    assert np.all(R + T < 1.0)


def test_s_equals_p_at_normal_incidence():
    rng = np.random.default_rng(12)
    n, d = _random_stack(rng, 13, absorbing=True)
    Rs, Ts = oracle.coh_tmm("s", _full(n), d, [0.0], LAM)
    Rp, Tp = oracle.coh_tmm("p", _full(n), d, [0.0], LAM)
    assert np.max(np.abs(Rs - Rp)) < 1e-13 and np.max(np.abs(Ts - Tp)) < 1e-13


@pytest.mark.parametrize("pol", ["s", "p"])
def test_zero_thickness_layer_changes_nothing(pol):
    rng = np.random.default_rng(13)
    n, d = _random_stack(rng, 9, absorbing=True)
    R0, T0 = oracle.coh_tmm(pol, _full(n), d, THETA, LAM)
    n2 = np.insert(n, 5, 2.9 + 0.7j, axis=1)
    d2 = np.insert(d, 4, 0.0, axis=1)
    R1, T1 = oracle.coh_tmm(pol, _full(n2), d2, THETA, LAM)
    assert np.max(np.abs(R1 - R0)) < 1e-12 and np.max(np.abs(T1 - T0)) < 1e-12


@pytest.mark.parametrize("pol", ["s", "p"])
def test_split_layer_changes_nothing(pol):
    rng = np.random.default_rng(14)
    n, d = _random_stack(rng, 9, absorbing=True)
    R0, T0 = oracle.coh_tmm(pol, _full(n), d, THETA, LAM)
    j = 3  # finite layer j+1 (column j of d) split into 0.3 / 0.7 of its thickness
    n2 = np.insert(n, j + 1, n[:, j + 1], axis=1)
    d2 = np.insert(d, j, 0.3 * d[:, j], axis=1)
    d2[:, j + 1] = 0.7 * d[:, j]
    R1, T1 = oracle.coh_tmm(pol, _full(n2), d2, THETA, LAM)
    assert np.max(np.abs(R1 - R0)) < 1e-12 and np.max(np.abs(T1 - T0)) < 1e-12


@pytest.mark.parametrize("pol", ["s", "p"])
def test_index_matched_layer_before_substrate(pol):
    # A finite layer of the (lossless) outcoupling medium only moves the
    # reference plane inside that medium: R and T unchanged.
    rng = np.random.default_rng(15)
    n, d = _random_stack(rng, 7, absorbing=True)
    R0, T0 = oracle.coh_tmm(pol, _full(n), d, THETA, LAM)
    n2 = np.insert(n, 8, 1.52, axis=1)
    d2 = np.concatenate([d, np.full((d.shape[0], 1), 333.0)], axis=1)
    R1, T1 = oracle.coh_tmm(pol, _full(n2), d2, THETA, LAM)
    assert np.max(np.abs(R1 - R0)) < 1e-12 and np.max(np.abs(T1 - T0)) < 1e-12


@pytest.mark.parametrize("pol", ["s", "p"])
@pytest.mark.parametrize("absorbing", [False, True])
def test_transmittance_reciprocity(pol, absorbing):
    # Light from the other side, with the angle mapped through Snell's law,
    # sees the same transmittance (reciprocity), for lossless outer media.
    rng = np.random.default_rng(16)
    n, d = _random_stack(rng, 8, absorbing=absorbing)
    th = np.deg2rad(np.linspace(0, 60, 7))
    R0, T0 = oracle.coh_tmm(pol, _full(n), d, th, LAM)
    nr, dr = n[:, ::-1].copy(), d[:, ::-1].copy()
    th_r = np.arcsin(np.sin(th) * 1.0 / 1.52)
    for a in range(th.size):
        _, Tb = oracle.coh_tmm(pol, _full(nr), dr, [th_r[a]], LAM)
        assert np.max(np.abs(Tb[:, 0] - T0[:, a])) < 1e-12


@pytest.mark.parametrize("pol", ["s", "p"])
def test_interior_root_choice_does_not_matter(pol):
    rng = np.random.default_rng(17)
    n, d = _random_stack(rng, 12, absorbing=True)
    R0, T0 = oracle.coh_tmm(pol, _full(n), d, THETA, LAM)
    flips = rng.integers(1, 2**12, size=n.shape[0]).astype(np.uint32)
    R1, T1 = oracle.coh_tmm(pol, _full(n), d, THETA, LAM, flip_mask=flips)
    assert np.max(np.abs(R1 - R0)) < 1e-12 and np.max(np.abs(T1 - T0)) < 1e-12


def test_opaque_layer_clamp():
    # 100 um of an index 2 + 1i absorber right after the ambient: only the
    # front interface is seen; Im(delta) is clamped at 35.
    lam = np.linspace(400, 800, 11)
    for pol in "sp":
        R, T = RT(pol, [1.0, 2.0 + 1.0j, 1.7, 1.52], [1e5, 80.0], np.deg2rad([0, 40]), lam)
        Rb, _ = RT(pol, [1.0, 2.0 + 1.0j], [], np.deg2rad([0, 40]), lam)
        assert np.all(np.isfinite(R)) and np.all(np.isfinite(T))
        assert np.max(np.abs(R - Rb)) < 1e-13
        assert np.max(T) < 1e-25


def test_many_opaque_layers_stay_finite():
    lam = np.linspace(400, 800, 5)
    media = [1.0] + [2.0 + 1.0j, 1.5] * 20 + [1.52]
    d = [1e5, 100.0] * 20
    for pol in "sp":
        R, T = RT(pol, media, d, np.deg2rad([0, 30]), lam)
        assert np.all(np.isfinite(R)) and np.all(np.isfinite(T))


# ---------------------------------------------------------------- second formulation
@pytest.mark.parametrize("pol", ["s", "p"])
@pytest.mark.parametrize("case", ["lossless", "absorbing", "dispersive", "tir", "metal_substrate"])
def test_matches_characteristic_matrix_form(pol, case):
    if case == "dispersive":
        w = W.dispersive(S=6, L=15, n_lambda=33, n_theta=7)
        n, d, th, lam = oracle_index(w), w.d, w.theta, w.lam
    elif case == "tir":
        w = W.map_x3()
        n, d = oracle_index(w), w.d
        th, lam = w.theta[::7], w.lam
    else:
        rng = np.random.default_rng({"lossless": 18, "absorbing": 19, "metal_substrate": 20}[case])
        nn, d = _random_stack(rng, 21, absorbing=(case != "lossless"))
        if case == "metal_substrate":  # absorbing outcoupling medium: T needs the conjugates of Eq. 2's reading
            nn[:, -1] = 0.3 + 2.5j
        n, th, lam = _full(nn), THETA, LAM
    # Under total internal reflection with evanescent interior layers (index
    # up to 4.6 next to 1.2) the two forms round differently near grazing
    # incidence: a few 1e-12, still far below the 1e-10 GPU tolerance.
    tol = 1e-11 if case == "tir" else 1e-12
    R, T = oracle.coh_tmm(pol, n, d, th, lam)
    for s in range(n.shape[0]):
        Ra, Ta = coh_tmm_admittance(pol, n[s], d[s], th, lam)
        assert np.max(np.abs(R[s] - Ra)) < tol
        assert np.max(np.abs(T[s] - Ta)) < tol


# ---------------------------------------------------------------- ragged stacks
def test_ragged_equals_truncated_and_padded():
    w = W.ragged(S=12, L_max=20, n_lambda=17, n_theta=5)
    Rr, Tr = oracle_RT(w)
    n = oracle_index(w)
    # padded: same arrays, every stack run at L_max (zero-thickness outcoupling layers)
    Rp, Tp = oracle.coh_tmm_pols(w.pols, n, w.d, w.theta, w.lam)
    assert np.max(np.abs(Rr - Rp)) < 1e-13 and np.max(np.abs(Tr - Tp)) < 1e-13
    for s in range(w.S):
        L = int(w.L_per_stack[s])
        nt = np.ascontiguousarray(n[s:s + 1, :L + 2])
        Rt, Tt = oracle.coh_tmm_pols(w.pols, nt, w.d[s:s + 1, :L], w.theta, w.lam)
        assert np.max(np.abs(Rt[:, 0] - Rr[:, s])) == 0.0
        assert np.max(np.abs(Tt[:, 0] - Tr[:, s])) == 0.0


# ---------------------------------------------------------------- gradient
def _fd_setup():
    w = W.adjoint(S=3, L=6, n_lambda=9, n_theta=3)
    return w, oracle_index(w)


def test_gradient_merit_matches_plain_forward():
    w, n = _fd_setup()
    m, _, _ = oracle.merit_grad(w.pols, n, w.d, w.theta, w.lam, w.R_target)
    m2 = oracle.merit(w.pols, n, w.d, w.theta, w.lam, w.R_target)
    assert np.max(np.abs(m - m2)) < 1e-15


def test_gradient_matches_central_differences():
    w, n = _fd_setup()
    _, dd, dn = oracle.merit_grad(w.pols, n, w.d, w.theta, w.lam, w.R_target)
    f = lambda nn, d: oracle.merit(w.pols, nn, d, w.theta, w.lam, w.R_target)
    h_d, h_n = 1e-4, 1e-6
    for j in range(w.L_max):
        dp, dm = w.d.copy(), w.d.copy()
        dp[:, j] += h_d
        dm[:, j] -= h_d
        fd = (f(n, dp) - f(n, dm)) / (2 * h_d)
        assert np.allclose(dd[:, j], fd, rtol=1e-6, atol=1e-11)
        np_, nm_ = n.copy(), n.copy()
        np_[:, j + 1, :] += h_n
        nm_[:, j + 1, :] -= h_n
        fd = (f(np_, w.d) - f(nm_, w.d)) / (2 * h_n)
        assert np.allclose(dn[:, j], fd, rtol=1e-6, atol=1e-9)


def test_gradient_ragged_zero_past_layer_count():
    w = W.ragged(S=4, L_max=6, n_lambda=5, n_theta=2)
    w.R_target = W.band_stop_target(w.lam, 2, w.n_theta)
    n = oracle_index(w)
    m, dd, dn = oracle.merit_grad(w.pols, n, w.d, w.theta, w.lam, w.R_target, L_per_stack=w.L_per_stack)
    for s in range(w.S):
        L = int(w.L_per_stack[s])
        assert np.all(dd[s, L:] == 0.0) and np.all(dn[s, L:] == 0.0)
        mt, ddt, dnt = oracle.merit_grad(w.pols, np.ascontiguousarray(n[s:s + 1, :L + 2]),
                                         w.d[s:s + 1, :L], w.theta, w.lam, w.R_target)
        assert abs(mt[0] - m[s]) == 0.0
        assert np.max(np.abs(ddt[0] - dd[s, :L])) == 0.0


def test_rejects_bad_arguments():
    n, d = stack([1.0, 1.5, 1.52], [10.0])
    with pytest.raises(ValueError):
        oracle.coh_tmm("s", n, np.zeros((1, 2)), [0.0], [500.0])
    with pytest.raises(ValueError):
        oracle.coh_tmm("s", n, d, [0.0], [500.0], L_per_stack=np.array([5], dtype=np.int32))


def test_reward_closed_forms():
    # air | glass at normal incidence: R = ((1 - 1.5) / 2.5)^2 = 0.04 at every
    # lambda, so against a zero target the reward is -0.04 per (plane, lambda)
    lam = np.linspace(400.0, 800.0, 7)
    n = np.repeat(np.array([[1.0, 1.5]], dtype=np.complex128)[:, :, None], 7, axis=2)
    th = np.array([0.0])
    r = oracle.reward("sp", n, np.zeros((1, 0)), th, lam, np.zeros((2, 1, 7)))
    assert abs(r[0] + 2 * 7 * 0.04) < 1e-14
    r = oracle.reward("sp", n, np.zeros((1, 0)), th, lam, np.zeros((1, 1, 7)), average=True)
    assert abs(r[0] + 7 * 0.04) < 1e-14
    # a target of 1 (a perfect mirror wanted): -sum (1 - R)
    r = oracle.reward("s", n, np.zeros((1, 0)), th, lam, np.ones((1, 1, 7)))
    assert abs(r[0] + 7 * 0.96) < 1e-13
    # the target equal to the stack's own R gives zero, any other target less
    rng = np.random.default_rng(3)
    nd = np.repeat(np.array([[1.0, 2.1, 1.4, 1.52]], dtype=np.complex128)[:, :, None], 7, axis=2)
    d = np.array([[120.0, 80.0]])
    R, _ = oracle.coh_tmm_pols("sp", nd, d, np.deg2rad([0.0, 40.0]), lam)
    assert abs(oracle.reward("sp", nd, d, np.deg2rad([0.0, 40.0]), lam, R[:, 0])[0]) < 1e-15
    assert oracle.reward("sp", nd, d, np.deg2rad([0.0, 40.0]), lam, rng.uniform(0, 1, R[:, 0].shape))[0] < 0
