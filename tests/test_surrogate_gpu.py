"""The learned surrogate on the GPU: exact training spectra, gradients of the
tcgen05 training step against a CPU reference, training progress, the exact
judge with per-row fallback, and checkpoint / resume."""

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
from paper_2111_13667_gb300 import abi
from paper_2111_13667_gb300 import workloads as W
from paper_2111_13667_gb300.surrogate import Surrogate, make_dataset, random_thicknesses, train

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def small(hidden=128, depth=2, seed=3, n_lambda=64, n_theta=4):
    w = W.surrogate(B=1)
    lam = np.linspace(400.0, 900.0, n_lambda)
    th = np.deg2rad(np.linspace(0, 70, n_theta))
    return Surrogate(hidden=hidden, depth=depth, seed=seed, lam=lam, theta=th)


def test_generate_matches_oracle():
    sur = Surrogate(hidden=64, depth=1)
    d = random_thicknesses(9, seed=61)
    R = sur.generate(d).double().cpu().numpy()
    w = W.surrogate(B=9)
    w.d = d.double().cpu().numpy()
    n = oracle.assemble_index(w.n_direct, None, None, w.n_lambda)
    Ro, _ = oracle.coh_tmm_pols("sp", n, w.d, w.theta, w.lam)
    Ro = np.transpose(Ro, (1, 0, 2, 3)).reshape(9, -1)
    assert np.max(np.abs(R - Ro)) <= 1e-4


def test_training_step_gradients_match_cpu_reference():
    sur = small()
    B = 256
    d = random_thicknesses(B, seed=62)
    T = sur.generate(d)
    layers = [sur.layer_tensors(i)[:2] for i in range(sur.depth + 1)]
    sur.train_step(d, T, lr=1e-6)
    torch.cuda.synchronize()
    assert sur.status() == abi.TMM_OK
    loss, grads, _ = mlp.forward_backward([(W_.cpu(), b.cpu()) for W_, b in layers], d.cpu(), T.cpu(),
                                          *sur.d_range)
    for i in range(sur.depth + 1):
        _, _, dW, db = [t.cpu().double() for t in sur.layer_tensors(i)]
        gW, gb = grads[i]
        rel_w = float((dW - gW).norm() / gW.norm())
        rel_b = float((db - gb).norm() / gb.norm())
        assert rel_w < 2e-2 and rel_b < 2e-2, (i, rel_w, rel_b)


def test_training_reduces_loss_and_judge_guarantees_tolerance(tmp_path):
    sur = Surrogate(hidden=256, depth=3, seed=5)
    d, R = make_dataset(sur, 16384, seed=63)
    rep = train(sur, d, R, steps=200, batch=1024, lr_max=2e-3, warmup=20)
    assert sur.status() == abi.TMM_OK
    assert rep.loss_last < 0.5 * rep.loss_first
    dt = random_thicknesses(3000, seed=64)
    exact = sur.generate(dt)
    stats = torch.zeros(2, dtype=torch.int32, device="cuda")
    out = sur.infer(dt, judge_fraction=1.0, tol=1e-3, stats=stats)
    torch.cuda.synchronize()
    err = (out - exact).abs().amax(dim=1)
    assert float(err.max()) <= 1e-3 + 1e-7  # every row judged: fallback rows are exact
    raw = sur.infer(dt, judge_fraction=0.0)
    raw_err = (raw - exact).abs().amax(dim=1)
    n_fb = int(stats[0].item())
    assert n_fb == int((raw_err > 1e-3).sum().item())
    max_bits = int(stats[1].item())
    assert abs(np.array([max_bits], dtype=np.int32).view(np.float32)[0] - float(raw_err.max())) < 1e-6
    # judging every 4th row only touches those rows
    part = sur.infer(dt, judge_fraction=0.25, tol=1e-3)
    rows = torch.arange(0, 3000, 4, device="cuda")
    assert float((part[rows] - out[rows]).abs().max()) == 0.0
    other = torch.ones(3000, dtype=torch.bool, device="cuda")
    other[rows] = False
    assert float((part[other] - raw[other]).abs().max()) == 0.0


def test_checkpoint_resume_is_exact(tmp_path):
    sur = small(seed=7)
    d, R = make_dataset(sur, 4096, seed=65)
    train(sur, d, R, steps=5, batch=1024, warmup=1)
    path = str(tmp_path / "sur.bin")
    sur.save(path)
    other = small(seed=99)
    other.load(path)
    x = random_thicknesses(500, seed=66)
    assert torch.equal(sur.infer(x), other.infer(x))
    for s in (sur, other):
        s.train_step(d[:1024], R[:1024], 1e-3)
    torch.cuda.synchronize()
    for i in range(sur.depth + 1):
        assert torch.equal(sur.layer_tensors(i)[0], other.layer_tensors(i)[0])


def test_mlp_inference_outruns_exact_kernel():
    """The gain the network buys: spectra per second of the network alone vs
    the exact kernel on the same 65536 stacks (full-size network)."""
    sur = Surrogate()
    d = random_thicknesses(65536, seed=67)
    for _ in range(2):
        sur.infer(d)
        sur.generate(d)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    sur.infer(d)
    ev[1].record()
    ev[2].record()
    sur.generate(d)
    ev[3].record()
    torch.cuda.synchronize()
    t_mlp, t_exact = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    print(f"network {65536 / t_mlp * 1e3:.3e} spectra/s, exact {65536 / t_exact * 1e3:.3e} spectra/s")
    assert t_mlp < t_exact
