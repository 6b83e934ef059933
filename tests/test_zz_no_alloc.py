"""tmm_coh_batched_noalloc: the persistent launch for callers that cannot
allocate device memory at call time (its scratch is a fixed array inside the
library).  Checked through the C ABI against tmm_coh_batched_ex with a caller
workspace -- the same kernels on the same inputs, so bit for bit -- on two
calls in a row (the second one starts from the first one's leftover scratch
contents), and once against the CPU oracle.  Kept in a file of its own,
collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2111_13667_gb300 import abi
from paper_2111_13667_gb300 import workloads as W
from tests.helpers import oracle_RT

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-4, "f32d": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def _with_workspace(prob, cfg, with_T=True):
    R = prob.empty_out()
    T = prob.empty_out() if with_T else None
    ws = abi.alloc_workspace(abi.tmm_workspace_size(prob, cfg))
    abi.tmm_coh_batched_ex(prob, cfg, ws, R, T)
    return R, T


def _noalloc_status(prob, cfg, R, T):
    s = prob.struct()
    return abi.load().tmm_coh_batched_noalloc(ctypes.byref(s), ctypes.byref(cfg) if cfg is not None else None,
                                              R.data_ptr(), None if T is None else T.data_ptr(),
                                              torch.cuda.current_stream().cuda_stream)


def _noalloc(prob, cfg, with_T=True):
    R = prob.empty_out()
    T = prob.empty_out() if with_T else None
    st = _noalloc_status(prob, cfg, R, T)
    assert st == abi.TMM_OK, abi.status_text(st)
    return R, T


@pytest.mark.parametrize("prec", ["f64", "f32", "f32d"])
def test_noalloc_matches_workspace_launch_twice(prec):
    cfg = abi.launch_cfg(persistent=1)
    for seed, S, L in ((51, 2000, 40), (52, 777, 17)):
        w = W.ragged(seed=seed, S=S, L_max=L, n_lambda=33, n_theta=5)
        prob = abi.to_device(w, prec)
        Rw, Tw = _with_workspace(prob, cfg)
        Rn, Tn = _noalloc(prob, cfg)
        torch.cuda.synchronize()
        assert torch.equal(Rn, Rw) and torch.equal(Tn, Tw)
        assert bool(torch.isfinite(Rn).all())


@pytest.mark.parametrize("prec", ["f64", "f32", "f32d"])
def test_noalloc_against_oracle_and_R_only(prec):
    w = W.ragged(seed=54, S=97, L_max=23, n_lambda=29, n_theta=7)
    prob = abi.to_device(w, prec)
    Ro, To = oracle_RT(w)
    R, T = _noalloc(prob, None)
    torch.cuda.synchronize()
    assert np.max(np.abs(R.double().cpu().numpy() - Ro)) <= TOL[prec]
    assert np.max(np.abs(T.double().cpu().numpy() - To)) <= TOL[prec]
    # T = NULL: R only, a separately compiled kernel instance; bit for bit the
    # R-only workspace launch, and within the tolerance of the oracle
    R1, _ = _noalloc(prob, None, with_T=False)
    Rw, _ = _with_workspace(prob, abi.launch_cfg(persistent=1), with_T=False)
    torch.cuda.synchronize()
    assert torch.equal(R1, Rw)
    assert np.max(np.abs(R1.double().cpu().numpy() - Ro)) <= TOL[prec]


def test_noalloc_rejects_problem_beyond_its_scratch():
    w = W.ragged(seed=53, S=300_000, L_max=4, n_lambda=8, n_theta=1)
    prob = abi.to_device(w, "f32")
    assert _noalloc_status(prob, None, prob.empty_out(), None) == abi.TMM_ERR_NOMEM


def test_noalloc_rejects_double_float():
    w = W.ragged(seed=55, S=10, L_max=4, n_lambda=8, n_theta=2)
    prob = abi.to_device(w, "f64x")
    assert _noalloc_status(prob, None, prob.empty_out(), None) == abi.TMM_ERR_UNSUPPORTED
