"""GPU parity of the adjoint (tmm_coh_grad) against the oracle's forward-mode
FP64 gradient and central finite differences.

Tolerances: merit within 1e-10 (FP64) / 1e-5 (FP32) absolute; gradients within
1e-9 (FP64) / 1e-4 (FP32) of the largest gradient magnitude of the stack set.
"""
import numpy as np
import pytest
import torch

from paper_2111_13667_gb300 import abi
from paper_2111_13667_gb300 import autograd as ag
from paper_2111_13667_gb300 import workloads as W
from tests.helpers import oracle_grad

pytestmark = pytest.mark.gpu

GTOL = {"f64": 1e-9, "f32": 1e-4}
MTOL = {"f64": 1e-10, "f32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def gpu_grad(w, prec, with_ws=False):
    prob = abi.to_device(w, prec)
    dt = prob.real_dtype
    Rt = torch.as_tensor(w.R_target).to(device="cuda", dtype=dt).contiguous()
    m = torch.empty(w.S, dtype=dt, device="cuda")
    dd = torch.empty(w.S, w.L_max, dtype=dt, device="cuda")
    dn = torch.empty(w.S, w.L_max, dtype=dt, device="cuda")
    ws = ag.grad_workspace(prob) if with_ws else None
    abi.tmm_coh_grad(prob, Rt, m, dd, dn, ws)
    torch.cuda.synchronize()
    return m.double().cpu().numpy(), dd.double().cpu().numpy(), dn.double().cpu().numpy()


def check(got, ref, prec):
    m, dd, dn = got
    mo, ddo, dno = ref
    assert np.all(np.isfinite(dd)) and np.all(np.isfinite(dn))
    assert np.max(np.abs(m - mo)) <= MTOL[prec]
    scale = max(np.max(np.abs(ddo)), 1e-30)
    assert np.max(np.abs(dd - ddo)) <= GTOL[prec] * scale, np.max(np.abs(dd - ddo)) / scale
    scale = max(np.max(np.abs(dno)), 1e-30)
    assert np.max(np.abs(dn - dno)) <= GTOL[prec] * scale, np.max(np.abs(dn - dno)) / scale


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("with_ws", [False, True])
def test_adjoint_small_vs_oracle(prec, with_ws):
    w = W.adjoint(seed=31, S=6, L=9, n_lambda=41, n_theta=5)
    check(gpu_grad(w, prec, with_ws), oracle_grad(w), prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("with_ws", [False, True])
def test_thickness_only_launch(prec, with_ws):
    # dm_dn = NULL takes the instance without the index terms (the optimiser's
    # launch): merit and dm_dd against the oracle, and against the full launch
    w = W.adjoint(seed=33, S=7, L=11, n_lambda=37, n_theta=6)
    prob = abi.to_device(w, prec)
    dt = prob.real_dtype
    Rt = torch.as_tensor(w.R_target).to(device="cuda", dtype=dt).contiguous()
    m = torch.empty(w.S, dtype=dt, device="cuda")
    dd = torch.empty(w.S, w.L_max, dtype=dt, device="cuda")
    abi.tmm_coh_grad(prob, Rt, m, dd, None, ag.grad_workspace(prob) if with_ws else None)
    torch.cuda.synchronize()
    mo, ddo, _ = oracle_grad(w)
    m, dd = m.double().cpu().numpy(), dd.double().cpu().numpy()
    assert np.max(np.abs(m - mo)) <= MTOL[prec]
    scale = np.max(np.abs(ddo))
    assert np.max(np.abs(dd - ddo)) <= GTOL[prec] * scale
    mf, ddf, _ = gpu_grad(w, prec, with_ws)
    assert np.max(np.abs(dd - ddf)) <= (1e-12 if prec == "f64" else 1e-6) * scale
    assert np.max(np.abs(m - mf)) <= (1e-14 if prec == "f64" else 1e-7)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_adjoint_single_pol_and_nondispersive(prec):
    w = W.plain_fp64(seed=32, S=4, L=7)
    w.theta = w.theta[:4]
    w.lam = w.lam[:50]
    for pols in ("s", "p"):
        w.pols = pols
        w.R_target = W.band_stop_target(w.lam, 1, w.n_theta)
        check(gpu_grad(w, prec), oracle_grad(w), prec)


def test_adjoint_with_opaque_layer():
    lam = np.linspace(400, 800, 21)
    th = np.deg2rad([0.0, 25.0, 50.0])
    media = np.array([[1.0, 2.1, 2.0 + 1.0j, 1.7, 1.45, 1.52]], dtype=np.complex128)
    d = np.array([[120.0, 1e5, 80.0, 95.0]])
    w = W.Workload("opaque", theta=th, lam=lam, d=d, n_direct=media,
                   R_target=W.band_stop_target(lam, 2, 3))
    check(gpu_grad(w, "f64"), oracle_grad(w), "f64")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_adjoint_ragged(prec):
    w = W.ragged(seed=33, S=7, L_max=12, n_lambda=19, n_theta=3)
    w.R_target = W.band_stop_target(w.lam, 2, w.n_theta)
    got = gpu_grad(w, prec)
    check(got, oracle_grad(w), prec)
    for s in range(w.S):
        assert np.all(got[1][s, w.L_per_stack[s]:] == 0.0)


def test_adjoint_is_deterministic_and_workspace_agrees():
    w = W.adjoint(seed=34, S=3, L=20, n_lambda=128, n_theta=16)
    a = gpu_grad(w, "f64")
    b = gpu_grad(w, "f64")
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    c = gpu_grad(w, "f64", with_ws=True)
    for x, y in zip(a, c):
        assert np.max(np.abs(x - y)) <= 1e-12 * max(1.0, np.max(np.abs(x)))


def test_adjoint_full_size_sampled_and_fd():
    """The 4096 x 40 x 512 x 16 problem in FP64: two sampled stacks against the
    oracle's forward-mode gradient, and 64 sampled stacks against central
    differences (step 1e-4 nm) of the GPU merit."""
    w = W.adjoint()
    m, dd, dn = gpu_grad(w, "f64", with_ws=True)
    idx = np.array([0, 2917])
    ref = oracle_grad(w.subset(idx))
    check((m[idx], dd[idx], dn[idx]), ref, "f64")

    rng = np.random.default_rng(2)
    sel = np.sort(rng.choice(w.S, size=64, replace=False))
    sub = w.subset(sel)
    h = 1e-4
    L = w.L_max
    # one batch: for each sampled stack and layer, d_j + h and d_j - h
    rep = np.repeat(np.arange(64), 2 * L)
    big = sub.subset(rep)
    big.d = big.d.copy()
    k = np.arange(64 * 2 * L)
    layer = (k // 2) % L
    sign = np.where(k % 2 == 0, 1.0, -1.0)
    big.d[k, layer] += sign * h
    mb, _, _ = gpu_grad(big, "f64", with_ws=True)
    fd = ((mb[0::2] - mb[1::2]) / (2 * h)).reshape(64, L)
    adj = dd[sel]
    assert np.max(np.abs(adj - fd)) <= 1e-6 * np.max(np.abs(adj)) + 1e-12


def test_adjoint_fp32_full_size_against_fp64():
    w = W.adjoint()
    _, dd64, dn64 = gpu_grad(w, "f64", with_ws=True)
    _, dd32, dn32 = gpu_grad(w, "f32", with_ws=True)
    assert np.max(np.abs(dd32 - dd64)) <= GTOL["f32"] * np.max(np.abs(dd64))
    assert np.max(np.abs(dn32 - dn64)) <= GTOL["f32"] * np.max(np.abs(dn64))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_autograd_function(prec):
    w = W.plain_fp64(seed=35, S=3, L=6)
    w.lam = w.lam[::4]
    w.R_target = W.band_stop_target(w.lam, 2, w.n_theta)
    prob = abi.to_device(w, prec)
    dt = prob.real_dtype
    Rt = torch.as_tensor(w.R_target).to(device="cuda", dtype=dt)
    d = prob.d.clone().requires_grad_(True)
    nl = torch.as_tensor(w.n_direct[:, 1:-1].real).to(device="cuda", dtype=dt).requires_grad_(True)
    m = ag.merit(prob, Rt, d=d, n_layers=nl)
    wts = torch.arange(1, w.S + 1, dtype=dt, device="cuda")
    (m * wts).sum().backward()
    mo, ddo, dno = oracle_grad(w)
    wn = np.arange(1, w.S + 1)[:, None]
    tol = GTOL[prec]
    assert np.max(np.abs(d.grad.double().cpu().numpy() - wn * ddo)) <= tol * np.max(np.abs(wn * ddo))
    assert np.max(np.abs(nl.grad.double().cpu().numpy() - wn * dno)) <= tol * np.max(np.abs(wn * dno))
    assert np.max(np.abs(m.detach().double().cpu().numpy() - mo)) <= MTOL[prec]


def test_grad_rejects_too_many_layers():
    w = W.adjoint(seed=36, S=2, L=130, n_lambda=8, n_theta=2)
    with pytest.raises(abi.TmmError) as e:
        gpu_grad(w, "f32")
    assert e.value.status == abi.TMM_ERR_UNSUPPORTED
