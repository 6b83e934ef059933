"""The GPU thickness optimiser (tmm_optimize_adam) against the CPU Adam of
``oracle/optimize.py`` on the same seeded starts, plus the physics optimum,
resumption, ragged stacks and argument checks.

Tolerances: FP64 trajectories within 1e-8 nm and merits within 1e-10 relative
after 8 steps (the gradients agree to ~1e-12 and Adam's normalised step keeps
that scale); FP32 within 2e-2 nm (1e-4 relative gradient error times the step
length lr over the steps) and merits within 1e-3 relative.
"""
import numpy as np
import pytest
import torch

from oracle import optimize
from paper_2111_13667_gb300 import abi
from paper_2111_13667_gb300 import workloads as W
from tests.helpers import oracle_index

pytestmark = pytest.mark.gpu

LR, STEPS = 2.0, 8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def gpu_adam(w, prec, steps, lr, d_min=1.0, d_max=500.0, chunks=None):
    prob = abi.to_device(w, prec)
    dt = prob.real_dtype
    Rt = torch.as_tensor(w.R_target).to(device="cuda", dtype=dt).contiguous()
    hist = torch.empty(steps, w.S, dtype=dt, device="cuda")
    ws, done = None, 0
    for k in (chunks or [steps]):
        cfg = abi.adam_cfg(lr, d_min=d_min, d_max=d_max, step0=done)
        ws = abi.tmm_optimize_adam(prob, Rt, cfg, k, merit_hist=hist[done:done + k], workspace=ws)
        done += k
    torch.cuda.synchronize()
    return prob.d.double().cpu().numpy(), hist.double().cpu().numpy()


def cpu_adam(w, steps, lr, d_min=1.0, d_max=500.0):
    return optimize.adam(w.pols, oracle_index(w), w.d, w.theta, w.lam, w.R_target, steps, lr, d_min=d_min,
                         d_max=d_max, L_per_stack=w.L_per_stack)


def small_adjoint():
    return W.adjoint(seed=21, S=7, L=6, n_lambda=24, n_theta=3)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_adam_trajectory_matches_oracle(prec):
    w = small_adjoint()
    d_ref, m_ref = cpu_adam(w, STEPS, LR)
    d, m = gpu_adam(w, prec, STEPS, LR)
    dtol, mtol = (1e-8, 1e-10) if prec == "f64" else (2e-2, 1e-3)
    assert np.max(np.abs(d - d_ref)) <= dtol, np.max(np.abs(d - d_ref))
    assert np.max(np.abs(m - m_ref) / m_ref) <= mtol
    assert np.all(np.abs(d - w.d) > 0)  # every layer moved
    assert np.all(m_ref[-1] < m_ref[0])


def test_resumed_calls_equal_one_call():
    w = small_adjoint()
    d1, m1 = gpu_adam(w, "f64", STEPS, LR)
    d2, m2 = gpu_adam(w, "f64", STEPS, LR, chunks=[3, 1, 4])
    assert np.array_equal(d1, d2) and np.array_equal(m1, m2)


def test_ragged_stacks_keep_layers_past_L_s():
    w = W.ragged(seed=22, S=9, L_max=7, n_lambda=16, n_theta=2)
    w.R_target = W.band_stop_target(w.lam, 2, w.n_theta)
    d_ref, m_ref = cpu_adam(w, 5, LR)
    d, m = gpu_adam(w, "f64", 5, LR)
    assert np.max(np.abs(d - d_ref)) <= 1e-8 and np.max(np.abs(m - m_ref) / m_ref) <= 1e-10
    for s in range(w.S):
        assert np.array_equal(d[s, w.L_per_stack[s]:], w.d[s, w.L_per_stack[s]:])


def test_quarter_wave_antireflection_optimum_on_the_gpu():
    n_ar = np.sqrt(1.52)
    d_star = 550.0 / (4.0 * n_ar)
    nd = np.tile(np.array([[1.0, n_ar, 1.52]], dtype=np.complex128), (3, 1))
    w = W.Workload("ar", theta=np.array([0.0]), lam=np.array([550.0]),
                   d=np.array([[90.0], [130.0], [3 * d_star - 25.0]]), n_direct=nd, pols="s",
                   R_target=np.zeros((1, 1, 1)))
    d, m = gpu_adam(w, "f64", 300, 2.0, d_min=10.0, d_max=400.0)
    assert abs(d[0, 0] - d_star) < 2.0 and abs(d[1, 0] - d_star) < 2.0 and abs(d[2, 0] - 3 * d_star) < 2.0
    assert np.all(m[-1] < 1e-9)


def test_argument_checks():
    w = small_adjoint()
    prob = abi.to_device(w, "f64")
    Rt = torch.as_tensor(w.R_target, device="cuda")
    with pytest.raises(abi.TmmError) as e:
        abi.tmm_optimize_adam(prob, Rt, abi.adam_cfg(0.0), 1)
    assert e.value.status == abi.TMM_ERR_INVALID_ARG
    with pytest.raises(abi.TmmError) as e:
        abi.tmm_optimize_adam(prob, Rt, abi.adam_cfg(1.0, d_min=5.0, d_max=1.0), 1)
    assert e.value.status == abi.TMM_ERR_INVALID_ARG
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(abi.TmmError) as e:
        abi.tmm_optimize_adam(prob, Rt, abi.adam_cfg(1.0), 1, workspace=small)
    assert e.value.status == abi.TMM_ERR_NOMEM
    probx = abi.to_device(w, "f64x")
    with pytest.raises(abi.TmmError) as e:
        abi.tmm_optimize_adam(probx, Rt, abi.adam_cfg(1.0), 1, workspace=small)
    assert e.value.status == abi.TMM_ERR_UNSUPPORTED
    d0 = prob.d.clone()
    abi.tmm_optimize_adam(prob, Rt, abi.adam_cfg(1.0), 0)  # zero steps: nothing moves
    torch.cuda.synchronize()
    assert torch.equal(prob.d, d0)
