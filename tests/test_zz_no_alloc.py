"""tmm_coh_batched_noalloc: the persistent launch for callers that cannot
allocate device memory at call time (its scratch is a fixed array inside the
library).  Checked through the C ABI against tmm_coh_batched_ex with a caller
workspace, on two calls in a row (the second one starts from the first one's
leftover scratch contents).  Kept in a file of its own, collected last."""
import ctypes

import pytest
import torch

from paper_2111_13667_gb300 import abi
from paper_2111_13667_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def _with_workspace(prob, cfg):
    R, T = prob.empty_out(), prob.empty_out()
    ws = abi.alloc_workspace(abi.tmm_workspace_size(prob, cfg))
    abi.tmm_coh_batched_ex(prob, cfg, ws, R, T)
    return R, T


def _noalloc(prob, cfg):
    R, T = prob.empty_out(), prob.empty_out()
    s = prob.struct()
    st = abi.load().tmm_coh_batched_noalloc(ctypes.byref(s), ctypes.byref(cfg), R.data_ptr(), T.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
    assert st == abi.TMM_OK, abi.status_text(st)
    return R, T


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_matches_workspace_launch_twice(prec):
    cfg = abi.launch_cfg(persistent=1)
    for seed, S, L in ((51, 2000, 40), (52, 777, 17)):
        w = W.ragged(seed=seed, S=S, L_max=L, n_lambda=33, n_theta=5)
        prob = abi.to_device(w, prec)
        Rw, Tw = _with_workspace(prob, cfg)
        Rn, Tn = _noalloc(prob, cfg)
        torch.cuda.synchronize()
        assert float((Rn - Rw).abs().max()) <= TOL[prec]
        assert float((Tn - Tw).abs().max()) <= TOL[prec]
        assert bool(torch.isfinite(Rn).all())


def test_noalloc_rejects_problem_beyond_its_scratch():
    w = W.ragged(seed=53, S=300_000, L_max=4, n_lambda=8, n_theta=1)
    prob = abi.to_device(w, "f32")
    R = prob.empty_out()
    s = prob.struct()
    st = abi.load().tmm_coh_batched_noalloc(ctypes.byref(s), None, R.data_ptr(), None,
                                            torch.cuda.current_stream().cuda_stream)
    assert st == abi.TMM_ERR_NOMEM
