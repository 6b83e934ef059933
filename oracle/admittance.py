"""Characteristic-matrix (tilted-admittance) formulation of the thin-film problem.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  This is a second,
independent formulation used to pin the paper-following oracle on random
stacks; it follows the textbook derivation, not the paper's Eq. 3.

Derivation (time dependence e^{-i omega t}, forward wave e^{+i k_z z}, the
convention under which the paper's Eq. 3 carries diag(e^{-i delta}, e^{i delta})):
in layer j the tangential fields are E(z) = A e^{i k z} + B e^{-i k z} and
H(z) = eta_j (A e^{i k z} - B e^{-i k z}), with eta_j = n_j cos(theta_j) for s
and n_j / cos(theta_j) for p.  Eliminating A, B between z = 0 and z = d_j gives

    [E(0), H(0)]^T = [[cos delta, -i sin delta / eta], [-i eta sin delta, cos delta]] [E(d), H(d)]^T

with delta = 2 pi n_j d_j cos(theta_j) / lambda.  Chaining every finite layer
and closing with [E, H] = [1, eta_out] in the outcoupling medium gives [B, C];
then the input admittance Y = C / B and

    R = |(eta_in - Y) / (eta_in + Y)|^2,
    T = 4 Re(eta_in) Re(eta_out) / |eta_in B + C|^2.

The root of cos(theta_j) and the Im(delta) <= 35 clamp follow the same
readings as the paper-following oracle.
"""
from __future__ import annotations

import numpy as np

IM_DELTA_MAX = 35.0


def _cos_theta(n, beta):
    c = np.sqrt(1.0 - (beta / n) ** 2 + 0j)
    nc = n * c
    tiny = np.abs(nc.imag) <= 100.0 * np.finfo(float).eps * np.abs(nc)
    flip = np.where(tiny, nc.real < 0.0, nc.imag < 0.0)
    return np.where(flip, -c, c)


def coh_tmm_admittance(pol, n_row, d, theta, lam):
    """R, T [N_theta][N_lambda] for one stack.

    n_row: complex [L+2][N_lambda] (media 0..L+1); d: [L] nm; theta radians; lam nm.
    """
    n_row = np.asarray(n_row, dtype=np.complex128)
    d = np.asarray(d, dtype=np.float64)
    theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    lam = np.atleast_1d(np.asarray(lam, dtype=np.float64))
    L = n_row.shape[0] - 2
    beta = (n_row[0].real[None, :] * np.sin(theta)[:, None])  # [Nt, Nl]
    nj = n_row[:, None, :]  # [L+2, 1, Nl]
    c = _cos_theta(nj, beta[None, :, :])  # [L+2, Nt, Nl]
    eta = nj * c if pol == "s" else nj / c
    B = np.ones(beta.shape, dtype=np.complex128)
    C = eta[L + 1] * B
    for j in range(L, 0, -1):
        delta = 2.0 * np.pi * nj[j] * d[j - 1] * c[j] / lam[None, :]
        delta = np.where(delta.imag > IM_DELTA_MAX, delta.real + 1j * IM_DELTA_MAX, delta)
        cd, sd = np.cos(delta), np.sin(delta)
        B, C = cd * B - 1j * sd / eta[j] * C, -1j * eta[j] * sd * B + cd * C
    with np.errstate(divide="ignore", invalid="ignore"):
        Y = C / B
        r = (eta[0] - Y) / (eta[0] + Y)
        R = np.abs(r) ** 2
        T = 4.0 * eta[0].real * eta[L + 1].real / np.abs(eta[0] * B + C) ** 2
    grazing = c[0] == 0
    R = np.where(grazing, 1.0, R)
    T = np.where(grazing, 0.0, T)
    return R, T
