"""Stacks with incoherent (thick) layers, on the CPU.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The paper treats
coherent stacks only; thick layers whose interference fringes are washed out
(a substrate under a coating) are handled here in the usual way: the stack is
cut at the incoherent media into coherent blocks, each block is described by
the power coefficients it has for light from its left (R_f, T_f) and from its
right (R_b, T_b), and the blocks are combined through the incoherent layers
by intensities instead of amplitudes.

Readings (the paper gives none):
* media 0 and L_s+1 are incoherent; finite layer j is incoherent where the
  caller flags it.  Incoherent layers must be non-absorbing (real index);
* with forward / backward intensities (I+, I-) on either side of a block
  between incoherent media a and b,
      I-_a = R_f I+_a + T_b I-_b,    I+_b = T_f I+_a + R_b I-_b,
  and an incoherent layer passes intensities unchanged (no absorption); with
  I+ = 1, I- = 0 in the exit medium, R = I-_0 / I+_0 and T = 1 / I+_0;
* an incoherent layer in which the wave is evanescent (n_j <= n_0 sin theta)
  passes no power: R is that of the structure in front of it, with it as the
  exit medium, and T = 0.
Each block's coefficients come from ``oracle.coh_tmm`` run on the block
(incidence from a) and on the reversed block (incidence from b, at the angle
Snell's law gives in medium b); no reciprocity is assumed.
"""
from __future__ import annotations

import numpy as np

from . import coh_tmm


def _block_RT(pol, n_blk, d_blk, theta, lam):
    """R, T [N_theta][N_lambda] of one coherent block (one stack)."""
    R, T = coh_tmm(pol, n_blk[None], d_blk[None], theta, lam)
    return R[0], T[0]


def inc_tmm(pol, n, d, incoherent, theta, lam, L_per_stack=None):
    """R, T (float64 [S][N_theta][N_lambda]) for one polarisation.

    n [S][L_max+2][N_lambda] complex, d [S][L_max], incoherent [S][L_max]
    (nonzero: the finite layer is incoherent), theta [N_theta] in medium 0.
    """
    n = np.asarray(n, dtype=np.complex128)
    d = np.asarray(d, dtype=np.float64)
    inc = np.asarray(incoherent).astype(bool)
    theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    lam = np.atleast_1d(np.asarray(lam, dtype=np.float64))
    S, Lp2, Nl = n.shape
    Nt = theta.size
    R_out = np.empty((S, Nt, Nl))
    T_out = np.empty((S, Nt, Nl))
    for s in range(S):
        L = int(L_per_stack[s]) if L_per_stack is not None else Lp2 - 2
        is_inc = [True] + [bool(inc[s, j - 1]) for j in range(1, L + 1)] + [True]
        if np.any(n[s, 0].imag != 0) or any(np.any(n[s, j].imag != 0) for j in range(1, L + 1) if is_inc[j]):
            R_out[s] = T_out[s] = np.nan
            continue
        n0 = n[s, 0].real  # [N_lambda]
        for it, th in enumerate(theta):
            beta = n0 * np.sin(th)  # [N_lambda]
            for il in range(Nl):
                R_out[s, it, il], T_out[s, it, il] = _one_point(pol, n[s, :, il], d[s], is_inc, L,
                                                               beta[il], lam[il])
    return R_out, T_out


def _one_point(pol, n_s, d_s, is_inc, L, beta, lam):
    lamv = np.array([lam])
    # the first incoherent layer in which the wave is evanescent ends the stack
    exit_ = L + 1
    cut = False
    for j in range(1, L + 1):
        if is_inc[j] and n_s[j].real <= beta:
            exit_, cut = j, True
            break
    inc_media = [j for j in range(exit_ + 1) if j == 0 or j == exit_ or is_inc[j]]
    # blocks between consecutive incoherent media, combined right to left.
    # (P, M) are I+ and I- on the left of the blocks done so far, scaled by the
    # product t of their T_f (so no division by a vanishing T_f):
    #   I+_a = (I+_b - R_b I-_b) / T_f,  I-_a = R_f I+_a + T_b I-_b
    P, M, t = 1.0, 0.0, 1.0
    for a, b in reversed(list(zip(inc_media[:-1], inc_media[1:]))):
        n_blk = n_s[a:b + 1][:, None]
        d_blk = d_s[a:b - 1] if b - 1 > a else np.zeros(0)
        th_a = np.arcsin(beta / n_s[a].real)
        Rf, Tf = _block_RT(pol, n_blk, d_blk, np.array([th_a]), lamv)
        Rf, Tf = float(Rf[0, 0]), float(Tf[0, 0])
        if b == exit_:
            Rb = Tb = 0.0  # nothing returns from the exit medium
        else:
            th_b = np.arcsin(beta / n_s[b].real)
            Rb, Tb = _block_RT(pol, n_blk[::-1].copy(), d_blk[::-1].copy(), np.array([th_b]), lamv)
            Rb, Tb = float(Rb[0, 0]), float(Tb[0, 0])
        P, M, t = P - Rb * M, Rf * (P - Rb * M) + Tf * Tb * M, t * Tf
    return M / P, (0.0 if cut else t / P)
