"""The stored oracle sample (tests/golden, written by make_golden.py from the
oracle alone): the oracle must keep reproducing it, and the GPU FP64 path must
match it without running the oracle."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2111_13667_gb300 import workloads as W

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden():
    with open(os.path.join(HERE, "oracle_plain_fp64_sample.json")) as fh:
        g = json.load(fh)
    to = lambda a: np.array([[[[float(v) for v in row] for row in plane] for plane in pol] for pol in a])
    return g, to(g["R"]), to(g["T"])


def test_oracle_reproduces_golden():
    g, Rg, Tg = golden()
    w = W.plain_fp64().subset(g["stacks"])
    n = oracle.assemble_index(w.n_direct, None, None, w.n_lambda)
    R, T = oracle.coh_tmm_pols("sp", n, w.d, w.theta, w.lam)
    pick = np.ix_(range(2), range(len(g["stacks"])), g["theta_index"], g["lambda_index"])
    assert np.max(np.abs(R[pick] - Rg)) <= 1e-15 and np.max(np.abs(T[pick] - Tg)) <= 1e-15


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f64x"])
def test_gpu_matches_golden(prec):
    import torch
    from paper_2111_13667_gb300 import abi
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, Rg, Tg = golden()
    w = W.plain_fp64()
    R, T = abi.coh_tmm(abi.to_device(w, prec))
    torch.cuda.synchronize()
    s = torch.as_tensor(g["stacks"], device=R.device)
    R = R[:, s].cpu().numpy()[:, :, g["theta_index"]][:, :, :, g["lambda_index"]]
    T = T[:, s].cpu().numpy()[:, :, g["theta_index"]][:, :, :, g["lambda_index"]]
    assert np.max(np.abs(R - Rg)) <= 1e-10 and np.max(np.abs(T - Tg)) <= 1e-10
