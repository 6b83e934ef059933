"""Pins of the CPU thickness optimiser (``oracle/optimize.py``, Adam over d).

Physics pins: a single layer of index sqrt(n_0 n_s) on a substrate n_s has
R = 0 at normal incidence exactly when its optical thickness is an odd number
of quarter waves, d* = (2k + 1) lambda / (4 n); starts on either side of d*
and near 3 d* must reach those minima.  Definition pins: the first Adam step
moves every live coordinate by lr against the sign of its gradient; the box
constraint holds exactly; layers past L_s do not move."""
import numpy as np

import oracle
from oracle import optimize

N_S = 1.52
N_AR = np.sqrt(N_S)
LAM = np.array([550.0])
TH = np.array([0.0])
D_STAR = 550.0 / (4.0 * N_AR)


def ar_index(S):
    return np.tile(np.array([[[1.0], [N_AR], [N_S]]], dtype=np.complex128), (S, 1, 1))


def test_quarter_wave_antireflection_optimum_is_reached_from_several_starts():
    d0 = np.array([[90.0], [130.0], [3 * D_STAR - 25.0]])
    d, merits = optimize.adam("s", ar_index(3), d0, TH, LAM, np.zeros((1, 1, 1)), 300, 2.0,
                              d_min=10.0, d_max=400.0)
    assert abs(d[0, 0] - D_STAR) < 2.0 and abs(d[1, 0] - D_STAR) < 2.0
    assert abs(d[2, 0] - 3 * D_STAR) < 2.0
    assert np.all(merits[-1] < 1e-9)
    assert np.all(merits[-1] < 1e-3 * merits[0])
    # the exact optimum reflects nothing (R = 0 closed form)
    R, _ = oracle.coh_tmm_pols("s", ar_index(1), np.array([[D_STAR]]), TH, LAM)
    assert R[0, 0, 0, 0] < 1e-28


def test_box_constraint_holds_exactly():
    d, _ = optimize.adam("s", ar_index(1), np.array([[90.0]]), TH, LAM, np.zeros((1, 1, 1)), 100, 2.0,
                         d_min=10.0, d_max=100.0)
    assert d[0, 0] == 100.0


def test_first_step_moves_each_live_coordinate_by_lr():
    rng = np.random.default_rng(5)
    S, L = 4, 3
    n = np.empty((S, L + 2, 1), dtype=np.complex128)
    n[:, 0] = 1.0
    n[:, 1:L + 1, 0] = rng.uniform(1.3, 2.4, (S, L))
    n[:, L + 1] = 1.52
    lam = np.linspace(450.0, 650.0, 5)
    th = np.deg2rad([0.0, 30.0])
    n = np.repeat(n, lam.size, axis=2)
    d0 = rng.uniform(50.0, 200.0, (S, L))
    Rt = np.full((2, th.size, lam.size), 0.3)
    _, g, _ = oracle.merit_grad("sp", n, d0, th, lam, Rt)
    lr = 1.5
    d1, merits = optimize.adam("sp", n, d0, th, lam, Rt, 1, lr, d_min=0.0, d_max=1e4)
    move = d1 - d0
    # opposite to the gradient, never longer than lr, and lr itself wherever
    # |g| >> eps (bias-corrected m^ / sqrt(v^) = g / |g| on the first step)
    assert np.all(np.sign(move) == -np.sign(g)) and np.all(np.abs(move) <= lr)
    big = np.abs(g) > 1e-5
    assert big.sum() >= 6
    assert np.allclose(np.abs(move[big]), lr, rtol=1e-3, atol=0)
    assert np.allclose(merits[0], oracle.merit("sp", n, d0, th, lam, Rt), rtol=1e-12)


def test_layers_past_L_s_do_not_move():
    rng = np.random.default_rng(6)
    S, L = 3, 4
    n = np.empty((S, L + 2, 1), dtype=np.complex128)
    n[:, 0] = 1.0
    n[:, 1:L + 1, 0] = rng.uniform(1.3, 2.4, (S, L))
    n[:, L + 1] = 1.52
    Ls = np.array([4, 2, 1], dtype=np.int32)
    for s in range(S):  # the outcoupling medium follows layer L_s
        n[s, Ls[s] + 1:] = 1.52
    d0 = rng.uniform(50.0, 200.0, (S, L))
    d, _ = optimize.adam("s", n, d0, TH, LAM, np.full((1, 1, 1), 0.1), 5, 3.0, L_per_stack=Ls)
    for s in range(S):
        assert np.array_equal(d[s, Ls[s]:], d0[s, Ls[s]:])
        assert np.all(d[s, :Ls[s]] != d0[s, :Ls[s]])
