"""Shared test helpers: feed a seeded workload to the oracle."""
import numpy as np

import oracle


def oracle_index(w):
    """complex [S][L_max+2][N_lambda] index array for the oracle."""
    return oracle.assemble_index(w.n_direct, w.table, w.mat_idx, w.n_lambda)


def oracle_RT(w, pols=None, nthreads=None):
    """Oracle R, T as [P][S][N_theta][N_lambda] for a Workload."""
    return oracle.coh_tmm_pols(pols or w.pols, oracle_index(w), w.d, w.theta, w.lam,
                               L_per_stack=w.L_per_stack, nthreads=nthreads)


def oracle_grad(w, nthreads=None):
    return oracle.merit_grad(w.pols, oracle_index(w), w.d, w.theta, w.lam, w.R_target,
                             L_per_stack=w.L_per_stack, nthreads=nthreads)


def stack(n_media, d, n_lambda=1):
    """One-stack oracle input from a list of media indices and finite thicknesses."""
    n = np.asarray(n_media, dtype=np.complex128)[None, :, None]
    n = np.repeat(n, n_lambda, axis=2)
    return n, np.asarray(d, dtype=np.float64).reshape(1, -1)
