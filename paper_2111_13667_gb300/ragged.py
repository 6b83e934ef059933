"""Ragged batches: stacks with uneven layer counts in one persistent launch,
captured in a CUDA graph.

The launch sequence of ``tmm_coh_batched_ex`` with ``persistent = 1`` (zero the
work counter, counting-sort the stacks longest first, one persistent grid that
pulls (stack, tile) items) is fixed for a given problem, so it is recorded
once in a CUDA graph and replayed; the launch shape comes from the autotuner.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import abi, autotune


class RaggedRunner:
    def __init__(self, prob: abi.DeviceProblem, cfg: Optional[abi.TmmLaunchCfg] = None, with_T: bool = True,
                 tune: bool = True):
        self.prob = prob
        if cfg is None:
            cfg = autotune.tune(prob, with_T=with_T) if tune else abi.launch_cfg(persistent=1)
        self.cfg = cfg
        self.R = prob.empty_out()
        self.T = prob.empty_out() if with_T else None
        need = abi.tmm_workspace_size(prob, cfg) if cfg.persistent else 0
        self.ws = abi.alloc_workspace(need, prob.d.device)
        self.graph = None

    def launch(self):
        """One eager launch on the current stream."""
        abi.tmm_coh_batched_ex(self.prob, self.cfg, self.ws, self.R, self.T)

    def capture(self):
        side = torch.cuda.Stream(device=self.R.device)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.launch()  # warm-up: kernel attributes are set outside the capture
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.launch()
        self.graph = g
        return self

    def __call__(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()
        return self.R, self.T

    def status(self) -> int:
        """TMM_OK or TMM_ERR_TIMEOUT recorded by the last persistent launch."""
        if self.ws is None:
            return abi.TMM_OK
        return abi.tmm_workspace_status(self.ws)
