"""Reference forward/backward of the surrogate MLP (plain torch on the CPU, fp64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The network is not in
the paper; this restates its definition -- x = (d - d_min)/(d_max - d_min) in
[0, 1], zero-padded to 64 inputs, hidden layers z = W h + b, h' = GELU(z) in
its erf form z Phi(z) = 0.5 z (1 + erf(z / sqrt 2)),
linear head y = W h + b, loss = mean (y - t)^2 -- and differentiates it with
autograd.  The GPU kernels store GEMM operands and activations in bf16; the
reference rounds the network input and the weights the same way and keeps
activations in fp64, so the two differ by the bf16 rounding of stored
activations and by accumulation order.
"""
from __future__ import annotations

import torch


def bf(t):
    return t.to(torch.bfloat16).to(torch.float64)


def gelu(z):
    return 0.5 * z * (1.0 + torch.erf(z / 2.0 ** 0.5))


def forward_backward(layers, d, target, d_min, d_max, kin=64):
    """layers: list of (W [N][K] fp32, b [N] fp32) tensors (CPU).  Returns
    (loss, [(dW, db)], y) in fp64, with the input and the weights rounded to
    bf16 like the kernels' operands."""
    B, L = d.shape
    x = torch.zeros(B, kin, dtype=torch.float64)
    x[:, :L] = (d.double() - d_min) / (d_max - d_min)
    h = bf(x)
    Ws = [bf(W.double()).requires_grad_(True) for W, _ in layers]
    bs = [b.double().requires_grad_(True) for _, b in layers]
    for i in range(len(layers) - 1):
        z = h @ Ws[i].T + bs[i]
        h = gelu(z)
    y = h @ Ws[-1].T + bs[-1]
    loss = ((y - target.double()) ** 2).mean()
    loss.backward()
    return float(loss.detach()), [(W.grad, b.grad) for W, b in zip(Ws, bs)], y.detach()
