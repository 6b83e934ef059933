"""torch.autograd bridge to the adjoint kernel (``tmm_coh_grad``).

``merit(...)`` returns the per-stack merit m_s = mean over (pol, theta,
lambda) of (R - R_target)^2 as a differentiable tensor: its backward hands
autograd the gradients the adjoint kernel computed in the same launch as the
merit, wrt the thicknesses and, for a non-dispersive real index given per
layer, wrt the layer indices.  This is the role TMM-Torch plays in the paper
(Sec. 4, appendix A.3), without taping any per-layer intermediate.
"""
from __future__ import annotations

from dataclasses import replace
from typing import Optional

import torch

from . import abi


def _index_from_layers(prob: abi.DeviceProblem, n_layers: torch.Tensor) -> torch.Tensor:
    """complex [S][L+2] index rows: the template's outer media around n_layers."""
    base = prob.n_direct
    cd = torch.complex128 if prob.prec == abi.TMM_F64 else torch.complex64
    if base is None or base.dim() != 2:
        raise ValueError("index gradients need a non-dispersive direct index (n_direct [S][L+2])")
    mid = n_layers.to(cd)
    return torch.cat([base[:, :1], mid, base[:, -1:]], dim=1).contiguous()


class TmmMerit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, d, n_layers, prob, R_target, workspace):
        p = replace(prob, d=d.detach().contiguous())
        if n_layers is not None:
            p = replace(p, n_direct=_index_from_layers(prob, n_layers.detach()))
        S, L = p.S, p.L_max
        dt = p.real_dtype
        m = torch.empty(S, dtype=dt, device=d.device)
        dd = torch.empty(S, L, dtype=dt, device=d.device)
        dn = torch.empty(S, L, dtype=dt, device=d.device) if n_layers is not None else None
        abi.tmm_coh_grad(p, R_target, m, dd, dn, workspace)
        ctx.has_n = n_layers is not None
        ctx.save_for_backward(dd, dn if dn is not None else dd)
        return m

    @staticmethod
    def backward(ctx, gm):
        dd, dn = ctx.saved_tensors
        g = gm[:, None]
        return g * dd, (g * dn if ctx.has_n else None), None, None, None


def grad_workspace(prob: abi.DeviceProblem) -> Optional[torch.Tensor]:
    return abi.alloc_workspace(abi.tmm_workspace_size(prob), prob.d.device)


def merit(prob: abi.DeviceProblem, R_target: torch.Tensor, d: Optional[torch.Tensor] = None,
          n_layers: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Differentiable per-stack merit [S].

    ``d`` [S][L] (defaults to the problem's thicknesses) and, for a
    non-dispersive direct index, ``n_layers`` [S][L] (real indices of the
    finite layers) may require grad.
    """
    d = prob.d if d is None else d
    return TmmMerit.apply(d, n_layers, prob, R_target, workspace)
