"""Stacks with one partially coherent layer, on the CPU.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The paper treats
coherent stacks only and gives no model of partial coherence; this is the
reading the library implements:

* one finite layer j of a stack (``layer[s]`` = j, 1-based; 0 = none) has a
  thickness spread by a Gaussian, d_j + D with D ~ N(0, sigma_s^2) (sigma in
  nm), as from a nonuniform thick layer or a finite coherence length;
* the stack's R and T are the expectations of the coherent R and T (Eqs. 1-6)
  over D;
* the expectation is the Gauss-Hermite rule with ``n_nodes`` nodes x_k and
  weights w_k:  E[f(D)] = sum_k (w_k / sqrt(pi)) f(sqrt(2) sigma x_k),
  1 <= n_nodes <= 256; the rule resolves the fringe harmonics up to a
  frequency growing like sqrt(n_nodes), so wide spreads need many nodes (the
  incoherent limit itself is the intensity method's, ``incoherent.py``);
* a node whose thickness d_j + sqrt(2) sigma x_k falls below zero counts as a
  layer of zero thickness.

sigma = 0 gives the coherent stack; for a non-absorbing layer whose phase
spread 2 pi Re(n_j cos theta_j) sigma / lambda is well above 1 the result
tends to that of the same layer treated as incoherent (``incoherent.py``).
Each node's R, T come from ``coh_tmm``; the nodes and weights from numpy's
Gauss-Hermite routine.  A stack whose ``layer`` is outside [0, L_s] or whose
sigma is negative or not finite gets NaN.
"""
from __future__ import annotations

import numpy as np

from . import coh_tmm


MAX_NODES = 256


def gauss_hermite(n_nodes):
    """Nodes x_k and normalised weights w_k / sqrt(pi) (summing to 1),
    1 <= n_nodes <= 256 (numpy's routine overflows further out)."""
    if not 1 <= int(n_nodes) <= MAX_NODES:
        raise ValueError("n_nodes must be in [1, 256]")
    x, w = np.polynomial.hermite.hermgauss(int(n_nodes))
    return x, w / np.sqrt(np.pi)


def pcoh_tmm(pol, n, d, layer, sigma, theta, lam, n_nodes=32, L_per_stack=None):
    """R, T (float64 [S][N_theta][N_lambda]) for one polarisation.

    ``n`` complex [S][L_max+2][N_lambda] (or [S][L_max+2]), ``d`` [S][L_max]
    nm, ``layer`` int [S] (0 = coherent stack), ``sigma`` [S] nm.
    """
    n = np.asarray(n, dtype=np.complex128)
    d = np.asarray(d, dtype=np.float64)
    layer = np.asarray(layer, dtype=np.int64)
    sigma = np.asarray(sigma, dtype=np.float64)
    theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    lam = np.atleast_1d(np.asarray(lam, dtype=np.float64))
    S, L_max = d.shape
    Ls = np.full(S, L_max) if L_per_stack is None else np.asarray(L_per_stack, dtype=np.int64)
    x, w = gauss_hermite(n_nodes)
    K = x.size
    # every stack repeated once per node, the partial layer's thickness moved
    d_big = np.repeat(d, K, axis=0).reshape(S, K, L_max)
    bad = np.zeros(S, dtype=bool)
    for s in range(S):
        j = int(layer[s])
        if j < 0 or j > Ls[s] or not np.isfinite(sigma[s]) or sigma[s] < 0:
            bad[s] = True
            continue
        if j >= 1:
            d_big[s, :, j - 1] = np.maximum(d[s, j - 1] + np.sqrt(2.0) * sigma[s] * x, 0.0)
    n_big = np.repeat(n, K, axis=0)
    Ls_big = None if L_per_stack is None else np.repeat(Ls, K).astype(np.int32)
    R, T = coh_tmm(pol, n_big, d_big.reshape(S * K, L_max), theta, lam, L_per_stack=Ls_big)
    R = np.einsum("skab,k->sab", R.reshape(S, K, theta.size, lam.size), w)
    T = np.einsum("skab,k->sab", T.reshape(S, K, theta.size, lam.size), w)
    R[bad] = np.nan
    T[bad] = np.nan
    return R, T
