"""The oracle: plain, slow FP64 CPU implementations of TMM-Fast's hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product package never imports it, and this package imports nothing from the
product package.

Two independent formulations live here:

* ``tmm_oracle.c`` (loaded through ctypes) follows the paper's own steps,
  Sec. 2, Eqs. 1-6: Snell's law, Fresnel coefficients, the layer matrices of
  Eq. 3 multiplied left to right as full 2x2 complex matrices (Eq. 4), and the
  extraction of Eqs. 5-6 and Eq. 2.  It also differentiates the per-stack MSE
  merit (Sec. 4, appendix A.3) by forward-mode dual numbers.
* ``admittance.py`` is the textbook characteristic-matrix (tilted admittance)
  form of the same thin-film problem, written independently in numpy; it is
  used only to pin the first formulation on random stacks.

Beside them: ``mlp.py`` (the surrogate network's reference forward/backward),
``optimize.py`` (many-start Adam over the thicknesses on top of
``merit_grad``, the merit-driven optimisation of the paper's Fig. 1c) and
``incoherent.py`` (thick incoherent layers combined by intensities between
coherent blocks evaluated with ``coh_tmm``), ``absorption.py`` (absorbed
fraction per layer from the field amplitudes of right partial products) and
``partial.py`` (one partially coherent layer: the Gauss-Hermite expectation
of ``coh_tmm`` over a Gaussian spread of its thickness).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tmm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_tmm.so")
_lib = None
_lock = threading.Lock()

IM_DELTA_MAX = 35.0  # opaque-layer clamp on Im(delta), a reading (not in the paper)


def build(force: bool = False) -> str:
    """Compile ``tmm_oracle.c`` into ``liboracle_tmm.so`` next to it (gcc)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(path):
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    up = ctypes.POINTER(ctypes.c_uint32)
    i = ctypes.c_int
    lib.oracle_coh_tmm.argtypes = [i, i, i, i, i, dp, dp, ip, dp, dp, up, dp, dp, i]
    lib.oracle_coh_tmm.restype = i
    lib.oracle_merit_grad.argtypes = [i, i, i, i, i, dp, dp, ip, dp, dp, dp, dp, dp, dp, i]
    lib.oracle_merit_grad.restype = i
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB_PATH)
    return _lib


def build_variant(src_text: str, out_path: str):
    """Compile a modified copy of tmm_oracle.c (used by the mutation tests,
    which plant mistakes in the oracle to show that the pins catch them) and
    return its loaded library."""
    src = out_path + ".c"
    with open(src, "w") as fh:
        fh.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", src, "-o",
                    out_path, "-lm"], check=True)
    return _bind(out_path)


def source() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def _prep(n, d, theta, lam, L_per_stack):
    n = np.ascontiguousarray(n, dtype=np.complex128)
    d = np.ascontiguousarray(d, dtype=np.float64)
    theta = np.ascontiguousarray(np.atleast_1d(theta), dtype=np.float64)
    lam = np.ascontiguousarray(np.atleast_1d(lam), dtype=np.float64)
    if n.ndim != 3:
        raise ValueError("n must be complex [S][L_max+2][N_lambda]")
    S, Lp2, Nl = n.shape
    L_max = Lp2 - 2
    if d.shape != (S, L_max):
        raise ValueError(f"d must be [S][L_max] = {(S, L_max)}, got {d.shape}")
    if Nl != lam.shape[0]:
        raise ValueError("n's last axis must match lambda")
    if L_per_stack is not None:
        L_per_stack = np.ascontiguousarray(L_per_stack, dtype=np.int32)
        if L_per_stack.shape != (S,):
            raise ValueError("L_per_stack must be [S]")
    return n, d, theta, lam, L_per_stack, S, L_max, Nl


def coh_tmm(pol, n, d, theta, lam, L_per_stack=None, flip_mask=None, nthreads=None, lib=None):
    """R, T (each float64 [S][N_theta][N_lambda]) for one polarisation.

    ``pol`` is ``'s'`` or ``'p'``; ``n`` is complex [S][L_max+2][N_lambda]
    (media 0..L+1, index 0 the injection medium), ``d`` [S][L_max] in nm,
    ``theta`` radians in medium 0, ``lam`` nm.  Follows Sec. 2, Eqs. 1-6.
    ``lib`` selects another build of the oracle (mutation tests only).
    """
    lib = lib or _load()
    n, d, theta, lam, L_per_stack, S, L_max, Nl = _prep(n, d, theta, lam, L_per_stack)
    Nt = theta.shape[0]
    if flip_mask is not None:
        flip_mask = np.ascontiguousarray(flip_mask, dtype=np.uint32)
    R = np.empty((S, Nt, Nl))
    T = np.empty((S, Nt, Nl))
    rc = lib.oracle_coh_tmm(0 if pol == "s" else 1, S, L_max, Nl, Nt,
                            _ptr(n.view(np.float64), ctypes.c_double), _ptr(d, ctypes.c_double),
                            _ptr(L_per_stack, ctypes.c_int32), _ptr(theta, ctypes.c_double),
                            _ptr(lam, ctypes.c_double), _ptr(flip_mask, ctypes.c_uint32),
                            _ptr(R, ctypes.c_double), _ptr(T, ctypes.c_double),
                            int(nthreads or default_threads()))
    if rc != 0:
        raise ValueError("oracle_coh_tmm rejected its arguments")
    return R, T


def coh_tmm_pols(pols, n, d, theta, lam, L_per_stack=None, nthreads=None, lib=None):
    """R, T stacked as [P][S][N_theta][N_lambda] for the polarisations in ``pols``."""
    Rs, Ts = [], []
    for p in pols:
        R, T = coh_tmm(p, n, d, theta, lam, L_per_stack=L_per_stack, nthreads=nthreads, lib=lib)
        Rs.append(R)
        Ts.append(T)
    return np.stack(Rs), np.stack(Ts)


def merit_grad(pols, n, d, theta, lam, R_target, L_per_stack=None, nthreads=None, lib=None):
    """Per-stack MSE merit and its gradients wrt d_j and a real offset of n_j.

    Returns ``(merit [S], dm_dd [S][L_max], dm_dn [S][L_max])``; ``R_target``
    is [P][N_theta][N_lambda] with P = len(pols), s before p.
    """
    lib = lib or _load()
    n, d, theta, lam, L_per_stack, S, L_max, Nl = _prep(n, d, theta, lam, L_per_stack)
    Nt = theta.shape[0]
    mask = (1 if "s" in pols else 0) | (2 if "p" in pols else 0)
    P = bin(mask).count("1")
    R_target = np.ascontiguousarray(R_target, dtype=np.float64)
    if R_target.shape != (P, Nt, Nl):
        raise ValueError(f"R_target must be [P][N_theta][N_lambda] = {(P, Nt, Nl)}")
    merit = np.empty(S)
    dd = np.empty((S, L_max))
    dn = np.empty((S, L_max))
    rc = lib.oracle_merit_grad(mask, S, L_max, Nl, Nt,
                               _ptr(n.view(np.float64), ctypes.c_double), _ptr(d, ctypes.c_double),
                               _ptr(L_per_stack, ctypes.c_int32), _ptr(theta, ctypes.c_double),
                               _ptr(lam, ctypes.c_double), _ptr(R_target, ctypes.c_double),
                               _ptr(merit, ctypes.c_double), _ptr(dd, ctypes.c_double),
                               _ptr(dn, ctypes.c_double), int(nthreads or default_threads()))
    if rc != 0:
        raise ValueError("oracle_merit_grad rejected its arguments")
    return merit, dd, dn


def merit(pols, n, d, theta, lam, R_target, L_per_stack=None, nthreads=None, lib=None):
    """Per-stack merit from the plain forward: mean of (R - R_target)^2."""
    R, _ = coh_tmm_pols(pols, n, d, theta, lam, L_per_stack=L_per_stack, nthreads=nthreads, lib=lib)
    e = R - np.asarray(R_target)[:, None, :, :]
    return np.mean(e * e, axis=(0, 2, 3))


def reward(pols, n, d, theta, lam, R_target, L_per_stack=None, average=False, nthreads=None, lib=None):
    """Reward of the paper's RL environment (Sec. 5) for every stack:
    -sum over (plane, theta, lambda) of |R_target - R|.  The planes are the
    polarisations in ``pols`` (s before p), or their mean with ``average``;
    ``R_target`` is [planes][N_theta][N_lambda]."""
    R, _ = coh_tmm_pols(pols, n, d, theta, lam, L_per_stack=L_per_stack, nthreads=nthreads, lib=lib)
    if average:
        R = R.mean(axis=0, keepdims=True)
    return -np.sum(np.abs(np.asarray(R_target)[:, None, :, :] - R), axis=(0, 2, 3))


def gather_index(table, mat_idx):
    """Index assembly: n[s, j, lambda] = table[mat_idx[s, j], lambda] (plain indexing)."""
    return np.asarray(table, dtype=np.complex128)[np.asarray(mat_idx)]


def assemble_index(n_direct=None, table=None, mat_idx=None, n_lambda=None):
    """complex [S][L_max+2][N_lambda] from either form of the index input.

    ``n_direct`` [S][L+2] (non-dispersive, repeated along lambda) or
    [S][L+2][N_lambda]; otherwise ``table[mat_idx]``.
    """
    if n_direct is not None:
        n_direct = np.asarray(n_direct, dtype=np.complex128)
        if n_direct.ndim == 2:
            return np.ascontiguousarray(np.repeat(n_direct[:, :, None], int(n_lambda), axis=2))
        return np.ascontiguousarray(n_direct)
    return np.ascontiguousarray(gather_index(table, mat_idx))
