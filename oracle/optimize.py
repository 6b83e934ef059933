"""Merit-driven thickness optimisation on the CPU: many-start Adam over d.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The paper's optimisation
use case (Fig. 1c: a merit of R over wavelength and angle, minimised over the
layer thicknesses with gradients from the differentiable TMM) does not fix an
optimiser; this follows Adam as Kingma and Ba define it (2015, Algorithm 1),
written out step by step.  Every stack is an independent start; its merit and
gradient come from ``oracle.merit_grad`` (forward-mode dual numbers).

Per step t = 1, 2, ... and every finite layer j < L_s of every stack:
    g   = d merit / d d_j                     (at the current d)
    m   = beta1 m + (1 - beta1) g             first-moment estimate
    v   = beta2 v + (1 - beta2) g^2           second-moment estimate
    m^  = m / (1 - beta1^t),  v^ = v / (1 - beta2^t)      bias correction
    d   = d - lr m^ / (sqrt(v^) + eps), then clipped to [d_min, d_max]
Layers past L_s of a ragged stack are left as they are.
"""
from __future__ import annotations

import numpy as np

from . import merit_grad


def adam(pols, n, d0, theta, lam, R_target, steps, lr, beta1=0.9, beta2=0.999, eps=1e-8,
         d_min=0.0, d_max=np.inf, L_per_stack=None, nthreads=None, lib=None):
    """Run ``steps`` Adam steps from d0 [S][L_max].

    Returns ``(d [S][L_max], merits [steps][S])``; ``merits[k]`` is the merit
    at the thicknesses the k-th step starts from.
    """
    d = np.array(d0, dtype=np.float64, copy=True)
    S, L_max = d.shape
    Ls = np.full(S, L_max) if L_per_stack is None else np.asarray(L_per_stack)
    live = np.arange(L_max)[None, :] < Ls[:, None]
    m = np.zeros_like(d)
    v = np.zeros_like(d)
    merits = np.empty((steps, S))
    for t in range(1, steps + 1):
        merit, g, _ = merit_grad(pols, n, d, theta, lam, R_target, L_per_stack=L_per_stack,
                                 nthreads=nthreads, lib=lib)
        merits[t - 1] = merit
        g = np.where(live, g, 0.0)
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        m_hat = m / (1.0 - beta1 ** t)
        v_hat = v / (1.0 - beta2 ** t)
        step = lr * m_hat / (np.sqrt(v_hat) + eps)
        d = np.where(live, np.clip(d - step, d_min, d_max), d)
    return d, merits
