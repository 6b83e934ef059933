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

``forward_backward_stored`` is the same network and loss with the backward
pass written out layer by layer (no autograd) and, with ``bf16=True``, every
tensor the training step stores rounded to bf16 where the kernels round it:
the input, the weights, each pre-activation z, each activation GELU(z) (of
the rounded z), the loss gradient 2 (y - t) / (B O) and each back-propagated
dZ = (dH) GELU'(z).  Products and sums stay exact (fp64), so it differs from
the GPU only by fp32 accumulation order.  With ``bf16=False`` it must equal
the autograd gradient of ``forward_backward`` (its pin).
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


def gelu_grad(z):
    """d/dz z Phi(z) = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + torch.erf(z / 2.0 ** 0.5)) + z * torch.exp(-0.5 * z * z) / (2.0 * torch.pi) ** 0.5


def forward_backward_stored(layers, d, target, d_min, d_max, kin=64, bf16=True):
    """(loss, [(dW, db)], y) in fp64 with the training step's stored tensors
    rounded to bf16 where the kernels round them (see the module docstring)."""
    r = bf if bf16 else (lambda t: t)
    B, L = d.shape
    x = torch.zeros(B, kin, dtype=torch.float64)
    x[:, :L] = (d.double() - d_min) / (d_max - d_min)
    hs = [r(x)]
    zs = []
    Ws = [r(W.double()) for W, _ in layers]
    bs = [b.double() for _, b in layers]
    for i in range(len(layers) - 1):
        z = r(hs[-1] @ Ws[i].T + bs[i])
        zs.append(z)
        hs.append(r(gelu(z)))
    y = hs[-1] @ Ws[-1].T + bs[-1]
    t = target.double()
    O = y.shape[1]
    loss = float(((y - t) ** 2).mean())
    g = r(2.0 * (y - t) / (B * O))  # d loss / d y
    grads = [None] * len(layers)
    for i in range(len(layers) - 1, -1, -1):
        grads[i] = (g.T @ hs[i], g.sum(dim=0))
        if i > 0:
            g = r((g @ Ws[i]) * gelu_grad(zs[i - 1]))
    return loss, grads, y
