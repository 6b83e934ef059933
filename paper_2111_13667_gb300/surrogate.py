"""Learned surrogate of the batched transfer-matrix method (binding + driver).

The C ABI (``tmm_surrogate_*``) owns the network and runs every step on the
GPU: exact spectra for the training set come from the library's transfer-matrix
kernel, training steps and inference run on the tcgen05 bf16 GEMM, and
inference outputs are judged by the exact kernel with a per-row fallback.
This module only marshals arguments and walks contiguous slices of a dataset
that lives in HBM (its thicknesses are i.i.d., so consecutive rows form random
batches and no shuffling is needed).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import abi
from . import workloads as W


class Surrogate:
    def __init__(self, hidden: int = 1024, depth: int = 6, seed: int = 4, n_media=None, lam=None, theta=None,
                 d_range=W.SURROGATE_D_RANGE):
        w = W.surrogate(B=1)
        n_media = np.asarray(w.n_direct[0] if n_media is None else n_media, dtype=np.complex128)
        self.lam = np.ascontiguousarray(w.lam if lam is None else lam, dtype=np.float64)
        self.theta = np.ascontiguousarray(w.theta if theta is None else theta, dtype=np.float64)
        self._media = np.ascontiguousarray(n_media.view(np.float64))
        self.L = n_media.shape[0] - 2
        self.d_range = d_range
        dp = ctypes.POINTER(ctypes.c_double)
        desc = abi.TmmSurrogateDesc(self.L, self._media.ctypes.data_as(dp), self.lam.shape[0],
                                    self.lam.ctypes.data_as(dp), self.theta.shape[0], self.theta.ctypes.data_as(dp),
                                    float(d_range[0]), float(d_range[1]), hidden, depth, seed)
        h = ctypes.c_void_p()
        abi._check("tmm_surrogate_create", abi.load().tmm_surrogate_create(ctypes.byref(desc), ctypes.byref(h)))
        self.handle = h
        self.outputs = int(abi.load().tmm_surrogate_outputs(h))
        self.parameters = int(abi.load().tmm_surrogate_parameters(h))
        self.hidden, self.depth = hidden, depth

    def close(self):
        if getattr(self, "handle", None):
            abi.load().tmm_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls
    def generate(self, d: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        B = int(d.shape[0])
        out = torch.empty(B, self.outputs, device=d.device) if out is None else out
        abi._check("tmm_surrogate_generate", abi.load().tmm_surrogate_generate(
            self.handle, abi._ptr(d), B, abi._ptr(out), abi._stream(stream)))
        return out

    def train_step(self, d: torch.Tensor, R: torch.Tensor, lr: float, loss: Optional[torch.Tensor] = None,
                   stream=None):
        abi._check("tmm_surrogate_train_step", abi.load().tmm_surrogate_train_step(
            self.handle, abi._ptr(d), abi._ptr(R), int(d.shape[0]), float(lr), abi._ptr(loss), abi._stream(stream)))

    def infer(self, d: torch.Tensor, judge_fraction: float = 0.0, tol: float = 1e-3,
              out: Optional[torch.Tensor] = None, stats: Optional[torch.Tensor] = None, stream=None):
        """R [B][outputs]; ``stats`` (device int32 [2]) receives (fallback rows, max judged error bits)."""
        B = int(d.shape[0])
        out = torch.empty(B, self.outputs, device=d.device) if out is None else out
        nf = me = None
        if stats is not None:
            nf = stats.data_ptr()
            me = stats.data_ptr() + 4
        abi._check("tmm_surrogate_infer", abi.load().tmm_surrogate_infer(
            self.handle, abi._ptr(d), B, abi._ptr(out), float(judge_fraction), float(tol), nf, me,
            abi._stream(stream)))
        return out

    def status(self) -> int:
        return int(abi.load().tmm_surrogate_status(self.handle, abi._stream(None)))

    def layer(self, i: int):
        v = abi.TmmSurrogateLayerView()
        abi._check("tmm_surrogate_layer", abi.load().tmm_surrogate_layer(self.handle, i, ctypes.byref(v)))
        return v

    def layer_tensors(self, i: int):
        """Copies of (W [N][K], b [N], dW [N][K], db [N]) of layer i, on the device."""
        v = self.layer(i)
        torch.cuda.synchronize()
        return [torch.as_tensor(_DeviceArray(ptr, shape), device="cuda").clone()
                for ptr, shape in ((v.W, (v.N, v.K)), (v.b, (v.N,)), (v.dW, (v.N, v.K)), (v.db, (v.N,)))]

    def save(self, path: str):
        abi._check("tmm_surrogate_save", abi.load().tmm_surrogate_save(self.handle, path.encode()))

    def load(self, path: str):
        abi._check("tmm_surrogate_load", abi.load().tmm_surrogate_load(self.handle, path.encode()))


class _DeviceArray:
    """A float32 device buffer owned by the library, exposed for a copy."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def random_thicknesses(n: int, seed: int, L: int = W.SURROGATE_L, d_range=W.SURROGATE_D_RANGE,
                       device="cuda") -> torch.Tensor:
    rng = np.random.default_rng(seed)
    d = rng.uniform(d_range[0], d_range[1], (n, L)).astype(np.float32)
    return torch.as_tensor(d).to(device)


def make_dataset(sur: Surrogate, n: int, seed: int, chunk: int = 65536):
    """(d [n][L], R [n][outputs]) with R from the exact transfer-matrix kernel."""
    d = random_thicknesses(n, seed, sur.L, sur.d_range)
    R = torch.empty(n, sur.outputs, device="cuda")
    for i in range(0, n, chunk):
        sur.generate(d[i:i + chunk], R[i:i + chunk])
    return d, R


@dataclass
class TrainReport:
    steps: int
    batch: int
    seconds: float
    loss_first: float
    loss_last: float


def train(sur: Surrogate, d: torch.Tensor, R: torch.Tensor, steps: int, batch: int = 8192, lr_max: float = 1e-3,
          lr_min: float = 1e-5, warmup: int = 100, log_every: int = 0, on_eval=None, eval_every: int = 0) -> TrainReport:
    """Adam with linear warm-up and cosine decay over contiguous dataset slices.
    ``on_eval(step, loss)`` is called every ``eval_every`` steps and after the
    last (for a learning curve)."""
    import time
    n = (int(d.shape[0]) // batch) * batch
    loss = torch.zeros(1, device=d.device)
    first = None
    t0 = time.perf_counter()
    for k in range(steps):
        lr = lr_max * min(1.0, (k + 1) / max(1, warmup))
        if k >= warmup:
            frac = (k - warmup) / max(1, steps - warmup)
            lr = lr_min + 0.5 * (lr_max - lr_min) * (1 + math.cos(math.pi * frac))
        o = (k * batch) % n
        sur.train_step(d[o:o + batch], R[o:o + batch], lr, loss)
        if k == 0:
            first = float(loss.item())
        if log_every and k % log_every == 0:
            print(f"step {k} lr {lr:.2e} loss {float(loss.item()):.3e}", flush=True)
        if on_eval is not None and ((eval_every and (k + 1) % eval_every == 0) or k + 1 == steps):
            on_eval(k + 1, float(loss.item()))
    torch.cuda.synchronize()
    return TrainReport(steps, batch, time.perf_counter() - t0, first or float("nan"), float(loss.item()))


def _gemm_shape(M, N, K, epilogue, repeat, seed=2):
    """`repeat` launches of one tcgen05 GEMM on random bf16 operands (profiling
    helper; the kernel form follows the library's choice unless TMM_GEMM_FORM is set)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = (torch.randn(M, K, generator=g) / K ** 0.5).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    bias = torch.randn(N, generator=g).cuda()
    f32 = epilogue in (0, 3)
    out = torch.empty(M, N, device="cuda", dtype=torch.float32 if f32 else torch.bfloat16)
    aux = None if epilogue == 1 else (torch.randn(M, N, generator=g).to(torch.bfloat16).cuda() if epilogue == 2 else None)
    for _ in range(repeat):
        abi.tmm_gemm_bf16(A, B, None if epilogue == 2 else bias, epilogue, out, aux)
    torch.cuda.synchronize()


def _main():
    import argparse
    ap = argparse.ArgumentParser(description="run surrogate inference, or one GEMM shape (profiling helper)")
    ap.add_argument("--infer-batch", type=int, default=65536)
    ap.add_argument("--repeat", type=int, default=4)
    ap.add_argument("--gemm", type=int, nargs=3, metavar=("M", "N", "K"), default=None,
                    help="time one GEMM shape instead of the inference")
    ap.add_argument("--epilogue", type=int, default=1, help="0 fp32, 1 GELU, 2 GELU', 3 clamp (with --gemm)")
    a = ap.parse_args()
    abi.load()
    if a.gemm:
        _gemm_shape(*a.gemm, a.epilogue, a.repeat)
        print("gemm", a.gemm, "epilogue", a.epilogue, "status ok")
        return
    sur = Surrogate()
    d = random_thicknesses(a.infer_batch, seed=44)
    out = torch.empty(a.infer_batch, sur.outputs, device="cuda")
    for _ in range(a.repeat):
        sur.infer(d, out=out)
    torch.cuda.synchronize()
    print("status", sur.status())


if __name__ == "__main__":
    _main()
