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
  caller flags it.  Medium 0 must be non-absorbing (else NaN);
* q_j = n_j cos(theta_j) is the root of n_j^2 - beta^2 (beta = n_0 sin theta)
  with Im q_j >= 0 (Re q_j >= 0 if Im q_j is zero to rounding), in every
  medium;
* a block's coefficients follow the coherent method: the Fresnel
  coefficients of Eq. 1 and the layer phases of Eq. 3 with these roots, the
  product of Eq. 4, and R = |r|^2, T = Re(n_b conj-or-not cos theta_b) /
  Re(n_a ... cos theta_a) |t|^2 (the Poynting form of Eq. 2 with complex
  bounding media); each block is evaluated once from each side,
  no reciprocity is assumed;
* an incoherent layer with a complex index attenuates every single pass of
  light by P_j = |exp(i delta_j)|^2 = exp(-4 pi Im(q_j) d_j / lambda);
* with forward / backward intensities (I+, I-) on either side of a block
  between incoherent media a and b,
      I-_a = R_f I+_a + T_b I-_b,    I+_b = T_f I+_a + R_b I-_b,
  across incoherent layer j: I+ at its right boundary = P_j I+ at its left,
  I- at its left = P_j I- at its right; with I+ = 1, I- = 0 in the exit
  medium, R = I-_0 / I+_0 and T = 1 / I+_0;
* an incoherent layer with Re(n_j^2 - beta^2) <= 0 (for a real index
  n_j <= n_0 sin theta: the wave is evanescent) passes no power: R is that of
  the structure in front of it, with it as the exit medium, and T = 0.
"""
from __future__ import annotations

import cmath
import math

import numpy as np

IM_DELTA_MAX = 35.0  # the coherent method's opaque-layer clamp Im(delta) <= 35 (not in the paper)


def forward_root(z):
    """Root of z with Im >= 0; the principal root (Re >= 0) where the imaginary
    part is zero to rounding (|Im| <= 100 eps |q|); the paper leaves the branch open."""
    q = cmath.sqrt(complex(z))  # principal: Re q >= 0
    if q.imag < -100 * 2.220446049250313e-16 * abs(q):
        q = -q
    return q


def block_RT(pol, n_blk, d_blk, beta, lam):
    """(R, T) of one coherent block for light from its first medium, by the
    coherent method written out for one point: media n_blk[0..m] (complex),
    finite thicknesses d_blk[0..m-2] (nm), Snell invariant beta (real),
    vacuum wavelength lam (nm).  Eq. 1 coefficients, Eq. 3 matrices
    multiplied left to right (Eq. 4), Eqs. 5-6, Eq. 2 in its Poynting form."""
    n = [complex(x) for x in n_blk]
    m = len(n) - 1
    q = [forward_root(x * x - beta * beta) for x in n]
    c = [qj / nj for qj, nj in zip(q, n)]  # cos(theta_j)

    def rt(j):  # interface j | j+1
        if pol == "s":
            a, b = n[j] * c[j], n[j + 1] * c[j + 1]
            return (a - b) / (a + b), 2 * a / (a + b)
        a, b = n[j + 1] * c[j], n[j] * c[j + 1]
        return (a - b) / (a + b), 2 * n[j] * c[j] / (a + b)

    r, t = rt(0)
    M = np.array([[1, r], [r, 1]], dtype=np.complex128) / t
    for j in range(1, m):
        delta = 2 * math.pi * q[j] * d_blk[j - 1] / lam
        delta = complex(delta.real, min(delta.imag, IM_DELTA_MAX))
        r, t = rt(j)
        Mj = np.array([[cmath.exp(-1j * delta), 0], [0, cmath.exp(1j * delta)]]) @ np.array([[1, r], [r, 1]]) / t
        M = M @ Mj
    rr, tt = M[1, 0] / M[0, 0], 1 / M[0, 0]
    if pol == "s":
        f = (n[m] * c[m]).real / (n[0] * c[0]).real
    else:
        f = (n[m] * np.conj(c[m])).real / (n[0] * np.conj(c[0])).real
    return float(abs(rr) ** 2), float(f * abs(tt) ** 2)


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
        if np.any(n[s, 0].imag != 0):
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
    # the first incoherent layer in which the wave is evanescent ends the stack
    exit_ = L + 1
    cut = False
    for j in range(1, L + 1):
        if is_inc[j] and (n_s[j] * n_s[j] - beta * beta).real <= 0:
            exit_, cut = j, True
            break
    inc_media = [j for j in range(exit_ + 1) if j == 0 or j == exit_ or is_inc[j]]
    # blocks between consecutive incoherent media, combined right to left.
    # (P, M) are I+ and I- on the left of the blocks done so far, scaled by the
    # product t of their T_f and single-pass factors (no division by a
    # vanishing one):
    #   across layer b:  I+_left = I+_right / P_b,  I-_left = P_b I-_right
    #   across a block:  I+_a = (I+_b - R_b I-_b) / T_f,  I-_a = R_f I+_a + T_b I-_b
    P, M, t = 1.0, 0.0, 1.0
    for a, b in reversed(list(zip(inc_media[:-1], inc_media[1:]))):
        if b != exit_:
            qb = forward_root(complex(n_s[b]) ** 2 - beta * beta)
            Pb = math.exp(-4 * math.pi * qb.imag * d_s[b - 1] / lam)
            M, t = M * Pb * Pb, t * Pb
        n_blk = n_s[a:b + 1]
        d_blk = d_s[a:b - 1] if b - 1 > a else np.zeros(0)
        Rf, Tf = block_RT(pol, n_blk, d_blk, beta, lam)
        if b == exit_:
            Rb = Tb = 0.0  # nothing returns from the exit medium
        else:
            Rb, Tb = block_RT(pol, n_blk[::-1], d_blk[::-1], beta, lam)
        P, M, t = P - Rb * M, Rf * (P - Rb * M) + Tf * Tb * M, t * Tf
    return M / P, (0.0 if cut else t / P)
