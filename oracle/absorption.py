"""Absorbed fraction of the incident power in every layer, on the CPU.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The paper notes that
partial coefficients follow from multiplying Eq. 4 only part of the way; here
the partial products from the right give the field amplitudes at the left
boundary of every layer, and the absorption in layer j is the integral of the
absorption density over its thickness,
    A_j = k0 / P_in * integral_0^d_j Im(n_j^2) |E(z)|^2 dz,   k0 = 2 pi / lambda,
with P_in the incident flux (per unit of the common field constants):
  s: E = E_y = a e^{i kappa z} + b e^{-i kappa z} (kappa = k0 q_j), P_in = q_0 |a_0|^2;
  p: with H_y = a e^{i kappa z} + b e^{-i kappa z}, E_x = (q_j / n_j^2)(a e - b e)
     and E_z = -(beta / n_j^2)(a e + b e), P_in = Re(q_0 / n_0^2) |a_0|^2.
The amplitudes come from the boundary conditions written as 2x2 matrices
(continuity of E_y and q E-difference for s; of H_y and (q / n^2) H-difference
for p), multiplied in full (complex128), the incident amplitude set to 1.
The integral of |a e^{i kappa z} + b e^{-i kappa z}|^2 (and of the difference)
is taken in closed form, the backward term with its amplitude at the layer's
right boundary (no growing exponential).  Layers past L_s give 0; the clamp Im delta <= 35
applies to the propagation matrices as in the other oracles.
"""
from __future__ import annotations

import numpy as np

IM_DELTA_MAX = 35.0


def _root(z):
    """Forward branch of sqrt(z): Im >= 0, the principal root where Im is zero to rounding."""
    q = np.sqrt(z + 0j)
    flip = (q.imag < 0) & (np.abs(q.imag) > 100 * np.finfo(float).eps * np.abs(q))
    q = np.where(flip, -q, q)
    flip2 = (np.abs(q.imag) <= 100 * np.finfo(float).eps * np.abs(q)) & (q.real < 0)
    return np.where(flip2, -q, q)


def _int_exp(c, d):
    """integral_0^d e^{c z} dz for complex c (c -> 0 handled)."""
    c = np.asarray(c, dtype=np.complex128)
    small = np.abs(c * d) < 1e-8
    safe = np.where(small, 1.0, c)
    return np.where(small, d * (1 + c * d / 2), np.expm1(safe * d) / safe)


def _int_mod2(a, b, b_right, kappa, d, sign):
    """integral_0^d |a e^{i kappa z} + sign b e^{-i kappa z}|^2 dz, where the
    backward wave's own term is written with its amplitude at z = d,
    b_right = b e^{-i kappa d}, so that every exponential decays."""
    decay = _int_exp(-2 * kappa.imag, d).real
    return ((np.abs(a) ** 2 + np.abs(b_right) ** 2) * decay
            + 2 * sign * (a * np.conj(b) * _int_exp(2j * kappa.real, d)).real)


def absorption(pol, n, d, theta, lam, L_per_stack=None):
    """A [S][L_max][N_theta][N_lambda] plus R, T [S][N_theta][N_lambda] for one polarisation.

    n [S][L_max+2][N_lambda] complex, d [S][L_max] nm, theta [N_theta] in medium 0.
    """
    n = np.asarray(n, dtype=np.complex128)
    d = np.asarray(d, dtype=np.float64)
    theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    lam = np.atleast_1d(np.asarray(lam, dtype=np.float64))
    S, Lp2, Nl = n.shape
    L_max = Lp2 - 2
    A = np.zeros((S, L_max, theta.size, Nl))
    R = np.empty((S, theta.size, Nl))
    T = np.empty((S, theta.size, Nl))
    for s in range(S):
        L = int(L_per_stack[s]) if L_per_stack is not None else L_max
        med = n[s, :L + 2]  # medium L+1 is the outcoupling medium of a ragged stack
        for it, th in enumerate(theta):
            beta = med[0].real * np.sin(th)                      # [N_lambda]
            q = _root(med ** 2 - beta ** 2)                      # [L+2][N_lambda]
            q[0] = med[0].real * np.cos(th)
            k = q if pol == "s" else q / med ** 2
            # transfer matrices: v_left(j) = P_j F_{j,j+1} v_left(j+1), v_left(0) = F_{0,1} v_left(1)
            def interface(j):
                a, b = k[j], k[j + 1]
                return np.array([[a + b, a - b], [a - b, a + b]]) / (2 * a)
            def phase(j):
                delta = 2 * np.pi * q[j] * d[s, j - 1] / lam
                delta = delta.real + 1j * np.minimum(delta.imag, IM_DELTA_MAX)
                z = np.zeros_like(delta)
                return np.array([[np.exp(-1j * delta), z], [z, np.exp(1j * delta)]])
            # right partial products: Pr[j] maps v_left(L+1) to v_left(j), Pq[j]
            # to the amplitudes at the right boundary of layer j
            eye = np.array([[np.ones(Nl), np.zeros(Nl)], [np.zeros(Nl), np.ones(Nl)]], dtype=np.complex128)
            Pr = [None] * (L + 2)
            Pq = [None] * (L + 2)
            Pr[L + 1] = eye
            for j in range(L, 0, -1):
                Pq[j] = np.einsum("ikl,kjl->ijl", interface(j), Pr[j + 1])
                Pr[j] = np.einsum("ikl,kjl->ijl", phase(j), Pq[j])
            M = np.einsum("ikl,kjl->ijl", interface(0), Pr[1])
            t = 1.0 / M[0, 0]
            r = M[1, 0] * t
            p_in = k[0].real  # |a_0| = 1; k_0 real for s (q_0) and p (q_0 / n_0^2)
            R[s, it] = np.abs(r) ** 2
            T[s, it] = (k[L + 1].real * np.abs(t) ** 2) / p_in
            k0 = 2 * np.pi / lam
            for j in range(1, L + 1):
                v = Pr[j][:, 0] * t   # amplitudes at the left boundary of layer j
                b_right = Pq[j][1, 0] * t
                kappa = k0 * q[j]
                dj = d[s, j - 1]
                im_eps = (med[j] ** 2).imag
                if pol == "s":
                    e2 = _int_mod2(v[0], v[1], b_right, kappa, dj, +1)
                else:
                    n4 = np.abs(med[j]) ** 4
                    e2 = (np.abs(q[j]) ** 2 * _int_mod2(v[0], v[1], b_right, kappa, dj, -1)
                          + beta ** 2 * _int_mod2(v[0], v[1], b_right, kappa, dj, +1)) / n4
                A[s, j - 1, it] = k0 * im_eps * e2 / p_in
    return A, R, T


def field_profile(pol, n, d, theta, lam, n_z, L_per_stack=None):
    """|E(z) / E_inc|^2 at the depths z_k = (k + 1/2) d_j / n_z of every layer:
    [S][L_max][n_z][N_theta][N_lambda] (0 past L_s).  E_inc is the incident
    plane wave's field amplitude: for p, |E|^2 = (|q|^2 |a e - b e|^2 +
    beta^2 |a e + b e|^2) / |n|^4 in units of the incident H amplitude, and
    the incident E = H / n_0 in those units, so the ratio carries n_0^2."""
    n = np.asarray(n, dtype=np.complex128)
    d = np.asarray(d, dtype=np.float64)
    theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    lam = np.atleast_1d(np.asarray(lam, dtype=np.float64))
    S, Lp2, Nl = n.shape
    L_max = Lp2 - 2
    out = np.zeros((S, L_max, n_z, theta.size, Nl))
    for s in range(S):
        L = int(L_per_stack[s]) if L_per_stack is not None else L_max
        med = n[s, :L + 2]
        for it, th in enumerate(theta):
            beta = med[0].real * np.sin(th)
            q = _root(med ** 2 - beta ** 2)
            q[0] = med[0].real * np.cos(th)
            k = q if pol == "s" else q / med ** 2
            def interface(j):
                a, b = k[j], k[j + 1]
                return np.array([[a + b, a - b], [a - b, a + b]]) / (2 * a)
            def phase(j):
                delta = 2 * np.pi * q[j] * d[s, j - 1] / lam
                delta = delta.real + 1j * np.minimum(delta.imag, IM_DELTA_MAX)
                z = np.zeros_like(delta)
                return np.array([[np.exp(-1j * delta), z], [z, np.exp(1j * delta)]])
            eye = np.array([[np.ones(Nl), np.zeros(Nl)], [np.zeros(Nl), np.ones(Nl)]], dtype=np.complex128)
            Pr = [None] * (L + 2)
            Pq = [None] * (L + 2)
            Pr[L + 1] = eye
            for j in range(L, 0, -1):
                Pq[j] = np.einsum("ikl,kjl->ijl", interface(j), Pr[j + 1])
                Pr[j] = np.einsum("ikl,kjl->ijl", phase(j), Pq[j])
            M = np.einsum("ikl,kjl->ijl", interface(0), Pr[1])
            t = 1.0 / M[0, 0]
            k0 = 2 * np.pi / lam
            for j in range(1, L + 1):
                # forward wave from the left boundary, backward wave from the
                # right boundary: both decay away from where they are taken
                a, b_right = Pr[j][0, 0] * t, Pq[j][1, 0] * t
                kappa = k0 * q[j]
                dj = d[s, j - 1]
                for kz in range(n_z):
                    z = (kz + 0.5) * dj / n_z
                    fw, bw = a * np.exp(1j * kappa * z), b_right * np.exp(1j * kappa * (dj - z))
                    if pol == "s":
                        e2 = np.abs(fw + bw) ** 2
                    else:
                        e2 = (np.abs(q[j]) ** 2 * np.abs(fw - bw) ** 2 + beta ** 2 * np.abs(fw + bw) ** 2) \
                            / np.abs(med[j]) ** 4 * med[0].real ** 2
                    out[s, j - 1, kz, it] = e2
    return out
