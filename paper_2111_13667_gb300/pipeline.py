"""R, T for problems whose inputs and outputs live in host memory.

``HostPipeline`` copies the (small) inputs to the device, then evaluates the
stacks in chunks with ``tmm_coh_batched`` on a compute stream while a copy
stream brings each finished chunk's R, T back into the caller's pinned host
arrays; chunk k's copies overlap the kernels of the chunks after it.  Chunks
are small (32 by default) and three ring slots let the kernels run two chunks
ahead of the copies, so only the last chunk's copy is exposed.  The copies
can be spread over more streams (``N_COPY_STREAMS``): on GB300 two streams
measured the same as one in quiet conditions and about three times slower in
some full benchmark runs, so one is the default.  Only argument marshalling
and copies happen here; every evaluation is the library kernel.
"""
from __future__ import annotations

from dataclasses import replace
from typing import Dict, Optional

import torch

from . import abi

_INPUTS = ("theta", "lam", "d", "n_direct", "table", "mat_idx", "L_per_stack")


class HostPipeline:
    N_SLOTS = 3
    N_COPY_STREAMS = 1

    def __init__(self, prob: abi.DeviceProblem, n_chunks: int = 32, with_T: bool = True):
        """``prob`` holds device buffers sized for the whole problem (they
        receive the host inputs on every run)."""
        self.prob = prob
        self.with_T = with_T
        S = prob.S
        self.n_chunks = max(1, min(n_chunks, S))
        self.bounds = [(S * c) // self.n_chunks for c in range(self.n_chunks + 1)]
        cmax = max(b - a for a, b in zip(self.bounds[:-1], self.bounds[1:]))
        self.plane = int(prob.theta.shape[0]) * int(prob.lam.shape[0])
        n = prob.n_pol * cmax * self.plane
        dev = prob.d.device
        # ring slots of flat storage, each viewed as a contiguous [P][chunk][theta][lambda]
        ns = self.N_SLOTS
        self.Rbuf = [torch.empty(n, dtype=prob.real_dtype, device=dev) for _ in range(ns)]
        self.Tbuf = [torch.empty(n, dtype=prob.real_dtype, device=dev) for _ in range(ns)] if with_T else None
        self.copy_streams = [torch.cuda.Stream(device=dev) for _ in range(self.N_COPY_STREAMS)]
        self.done = [torch.cuda.Event() for _ in range(ns)]
        # free[slot][i]: copy stream i has finished reading the slot
        self.free = [[torch.cuda.Event() for _ in self.copy_streams] for _ in range(ns)]
        self.used = [False] * ns

    def _sub(self, s0: int, s1: int) -> abi.DeviceProblem:
        p = self.prob
        cut = lambda t: None if t is None else t[s0:s1]
        return replace(p, d=p.d[s0:s1], n_direct=cut(p.n_direct) if p.n_direct is not None else None,
                       mat_idx=cut(p.mat_idx), L_per_stack=cut(p.L_per_stack))

    def run(self, host_inputs: Dict[str, torch.Tensor], R_host: torch.Tensor, T_host: Optional[torch.Tensor] = None):
        """``host_inputs`` maps DeviceProblem field names to (pinned) host
        tensors to upload; R_host, T_host: pinned [P][S][N_theta][N_lambda]."""
        compute = torch.cuda.current_stream()
        for k, v in host_inputs.items():
            if k not in _INPUTS:
                raise KeyError(k)
            getattr(self.prob, k).copy_(v, non_blocking=True)
        ns = self.N_SLOTS
        for c in range(self.n_chunks):
            s0, s1 = self.bounds[c], self.bounds[c + 1]
            slot = c % ns
            if self.used[slot]:
                for ev in self.free[slot]:
                    compute.wait_event(ev)
            n = s1 - s0
            shape = (self.prob.n_pol, n, int(self.prob.theta.shape[0]), int(self.prob.lam.shape[0]))
            size = self.prob.n_pol * n * self.plane
            Rv = self.Rbuf[slot][:size].view(shape)
            Tv = self.Tbuf[slot][:size].view(shape) if self.with_T else None
            abi.tmm_coh_batched(self._sub(s0, s1), Rv, Tv, stream=compute)
            self.done[slot].record(compute)
            copies = []
            for p in range(Rv.shape[0]):
                copies.append((R_host[p, s0:s1], Rv[p]))
                if T_host is not None and Tv is not None:
                    copies.append((T_host[p, s0:s1], Tv[p]))
            for i, cs in enumerate(self.copy_streams):
                with torch.cuda.stream(cs):
                    cs.wait_event(self.done[slot])
                    for dst, src in copies[i::len(self.copy_streams)]:
                        dst.copy_(src, non_blocking=True)
                    self.free[slot][i].record(cs)
            self.used[slot] = True
        for cs in self.copy_streams:
            compute.wait_stream(cs)
        return R_host, T_host
