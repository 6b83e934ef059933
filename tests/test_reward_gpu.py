"""The batched environment reward (tmm_coh_reward) against the oracle's
-sum |R_target - R|, for uniform and ragged stacks, both launches, every
plane choice, and with the unpolarised mean.

Tolerances: FP64 within 1e-12 relative; FP32 within 1e-5 per summed term
(the forward's FP32 error on these workloads is a few 1e-6 per R)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_13667_gb300 import abi
from paper_2111_13667_gb300 import workloads as W
from tests.helpers import oracle_index

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def target(w, planes, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, (planes, w.n_theta, w.n_lambda))


def gpu_reward(w, prec, Rt, pols=None, cfg=None):
    prob = abi.to_device(w, prec, pols=pols)
    dt = prob.real_dtype
    out = torch.empty(w.S, dtype=dt, device="cuda")
    abi.tmm_coh_reward(prob, torch.as_tensor(Rt).to(device="cuda", dtype=dt).contiguous(), out, cfg=cfg)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


def check(got, ref, prec, n_terms):
    if prec == "f64":
        assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-12
    else:
        assert np.max(np.abs(got - ref)) <= 1e-5 * n_terms


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("pols", ["s", "p", "sp", "u"])
def test_reward_matches_oracle(prec, pols):
    w = W.dispersive(seed=31, S=13, L=8, n_lambda=45, n_theta=7)
    planes = 2 if pols == "sp" else 1
    Rt = target(w, planes, 1)
    opols = "sp" if pols == "u" else pols
    ref = oracle.reward(opols, oracle_index(w), w.d, w.theta, w.lam, Rt, average=pols == "u")
    got = gpu_reward(w, prec, Rt, pols=pols)
    check(got, ref, prec, planes * w.n_theta * w.n_lambda)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("persistent", [0, 1])
def test_reward_ragged_stacks(prec, persistent):
    w = W.ragged(seed=32, S=57, L_max=30, n_lambda=33, n_theta=5)
    Rt = target(w, 2, 2)
    ref = oracle.reward("sp", oracle_index(w), w.d, w.theta, w.lam, Rt, L_per_stack=w.L_per_stack)
    got = gpu_reward(w, prec, Rt, cfg=abi.launch_cfg(persistent=persistent))
    check(got, ref, prec, 2 * w.n_theta * w.n_lambda)


def test_reward_is_deterministic_and_launch_independent():
    w = W.ragged(seed=33, S=200, L_max=20, n_lambda=64, n_theta=8)
    Rt = target(w, 2, 3)
    a = gpu_reward(w, "f32", Rt, cfg=abi.launch_cfg(persistent=1))
    b = gpu_reward(w, "f32", Rt, cfg=abi.launch_cfg(persistent=1))
    c = gpu_reward(w, "f32", Rt)
    assert np.array_equal(a, b)  # fixed-order sums: bit-reproducible
    # the other launch is compiled separately: equal to FP32 rounding
    assert np.max(np.abs(a - c)) <= 1e-5 * 2 * w.n_theta * w.n_lambda


def test_reward_argument_checks():
    w = W.dispersive(seed=34, S=300, L=2, n_lambda=8, n_theta=2)
    prob = abi.to_device(w, "f32")
    Rt = torch.zeros(2, 2, 8, device="cuda")
    out = torch.empty(300, device="cuda")
    assert abi.tmm_reward_workspace_size(prob) > 256
    with pytest.raises(abi.TmmError) as e:
        abi.tmm_coh_reward(prob, Rt, out, workspace=torch.empty(256, dtype=torch.uint8, device="cuda"))
    assert e.value.status == abi.TMM_ERR_NOMEM
    with pytest.raises(abi.TmmError) as e:
        abi.tmm_coh_reward(prob, Rt, out, cfg=abi.launch_cfg(persistent=1, max_items_per_block=4))
    assert e.value.status == abi.TMM_ERR_INVALID_ARG
    probx = abi.to_device(w, "f64x")
    with pytest.raises(abi.TmmError) as e:
        abi.tmm_coh_reward(probx, Rt.double(), out.double(), workspace=torch.empty(256, dtype=torch.uint8,
                                                                                   device="cuda"))
    assert e.value.status == abi.TMM_ERR_UNSUPPORTED
