"""Pins of the surrogate-network oracle (``oracle/mlp.py``) on the CPU.

The network is a design of this project (the paper defines none), so its pins
are mathematical: its GELU against scipy's normal CDF (z Phi(z), a different
routine from torch's erf), the odd-part identity, a brute-force forward pass
of a tiny network with the input map (d - d_min)/(d_max - d_min), and finite
differences of the loss for every bias and for weights at bf16-exact values."""
import math

import numpy as np
import pytest
import torch
from scipy.special import ndtr

from oracle import mlp


def test_gelu_is_z_times_normal_cdf():
    z = torch.linspace(-8.0, 8.0, 16001, dtype=torch.float64)
    exact = z * torch.as_tensor(ndtr(z.numpy()))
    # torch's erf is accurate to a few ulp; its vectorised and scalar paths
    # (chosen by how a tensor is split over threads) differ by up to ~16 ulp
    # of GELU values near 8
    assert float(((mlp.gelu(z) - exact) / z.abs().clamp(min=1.0)).abs().max()) < 1e-14


def test_gelu_odd_part_is_half_identity():
    # z Phi(z) - (-z) Phi(-z) = z (Phi(z) + Phi(-z)) = z
    z = torch.linspace(-6.0, 6.0, 1201, dtype=torch.float64)
    assert float((mlp.gelu(z) - mlp.gelu(-z) - z).abs().max()) < 1e-14
    assert float(mlp.gelu(torch.tensor(0.0, dtype=torch.float64))) == 0.0


def _net(sizes, seed, kin=64):
    g = torch.Generator().manual_seed(seed)
    layers = []
    k = kin
    for n in sizes:
        W = (torch.randn(n, k, generator=g) / k ** 0.5).to(torch.bfloat16).float()
        b = torch.randn(n, generator=g) * 0.3
        layers.append((W, b))
        k = n
    return layers


def test_forward_matches_brute_force_loops():
    layers = _net([5, 4, 3], seed=1)
    d = torch.tensor([[30.0, 100.0, 240.0], [25.0, 60.0, 200.0]])
    t = torch.zeros(2, 3)
    _, _, y = mlp.forward_backward(layers, d, t, 20.0, 250.0)
    for b in range(2):
        h = [0.0] * 64
        for i in range(3):
            x = (float(d[b, i]) - 20.0) / 230.0
            h[i] = float(torch.tensor(x).to(torch.bfloat16))
        for li, (W, bias) in enumerate(layers):
            out = []
            for n in range(W.shape[0]):
                s = float(bias[n]) + sum(float(W[n, k]) * h[k] for k in range(len(h)))
                if li < len(layers) - 1:
                    s = 0.5 * s * (1.0 + math.erf(s / math.sqrt(2.0)))
                out.append(s)
            h = out
        assert np.allclose(h, y[b].numpy(), rtol=1e-12, atol=1e-12)


def _loss(layers, d, t):
    return mlp.forward_backward(layers, d, t, 20.0, 250.0)[0]


@pytest.fixture(scope="module")
def problem():
    layers = _net([6, 6, 4], seed=2)
    g = torch.Generator().manual_seed(3)
    d = 20.0 + 230.0 * torch.rand(7, 5, generator=g)
    t = torch.rand(7, 4, generator=g)
    return layers, d, t


def test_bias_gradients_match_finite_differences(problem):
    layers, d, t = problem
    _, grads, _ = mlp.forward_backward(layers, d, t, 20.0, 250.0)
    h = 1e-5
    for li, (W, b) in enumerate(layers):
        for n in range(b.shape[0]):
            plus = [(W_, b_.double().clone()) for W_, b_ in layers]
            minus = [(W_, b_.double().clone()) for W_, b_ in layers]
            plus[li][1][n] += h
            minus[li][1][n] -= h
            fd = (_loss(plus, d, t) - _loss(minus, d, t)) / (2 * h)
            assert abs(fd - float(grads[li][1][n])) <= 1e-7 + 1e-6 * abs(fd), (li, n)


def test_weight_gradients_match_finite_differences(problem):
    # weights pass through bf16 rounding, so the step is one bf16 spacing at a
    # bf16-exact value (0.5: spacing 2^-8); central differences stay smooth
    layers, d, t = problem
    for li, (n, k) in enumerate([(1, 2), (3, 0), (2, 5)]):
        base = [(W.clone(), b) for W, b in layers]
        base[li][0][n, k] = 0.5
        _, grads, _ = mlp.forward_backward(base, d, t, 20.0, 250.0)
        h = 2.0 ** -8
        plus = [(W.clone(), b) for W, b in base]
        minus = [(W.clone(), b) for W, b in base]
        plus[li][0][n, k] = 0.5 + h
        minus[li][0][n, k] = 0.5 - h
        fd = (_loss(plus, d, t) - _loss(minus, d, t)) / (2 * h)
        g = float(grads[li][0][n, k])
        assert abs(fd - g) <= 1e-6 + 1e-3 * abs(g), (li, fd, g)
        assert abs(g) > 1e-6


def test_written_out_backward_equals_autograd():
    # the layer-by-layer backward of forward_backward_stored, rounding off, is
    # the autograd gradient of the same loss (a transposed operand, a missing
    # GELU' factor or a wrong loss scale would fail here)
    layers = _net([16, 12, 9], seed=5)
    g = torch.Generator().manual_seed(6)
    d = 20.0 + 230.0 * torch.rand(7, 5, generator=g)
    t = torch.rand(7, 9, generator=g)
    loss_a, grads_a, y_a = mlp.forward_backward(layers, d, t, 20.0, 250.0)
    Wr = [(W.to(torch.bfloat16).double(), b) for W, b in layers]  # the rounding forward_backward applies
    x = torch.zeros(7, 64, dtype=torch.float64)
    x[:, :5] = (d.double() - 20.0) / 230.0
    # forward_backward rounds its input to bf16; feed the same input here
    d_r = (x[:, :5].to(torch.bfloat16).double() * 230.0 + 20.0)
    loss_b, grads_b, y_b = mlp.forward_backward_stored(Wr, d_r, t, 20.0, 250.0, bf16=False)
    assert abs(loss_a - loss_b) < 1e-12
    assert float((y_a - y_b).abs().max()) < 1e-12
    for (gw, gb), (hw, hb) in zip(grads_a, grads_b):
        assert float((gw - hw).abs().max()) < 1e-12 and float((gb - hb).abs().max()) < 1e-12


def test_gelu_grad_is_the_derivative():
    z = torch.linspace(-6.0, 6.0, 601, dtype=torch.float64)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert float((mlp.gelu_grad(z) - fd).abs().max()) < 1e-9
