"""Thin ctypes binding of libtmm's C ABI (``include/tmm.h``).

Functions carry the C names and only marshal arguments: torch tensors become
device pointers, the current torch stream becomes the ``cudaStream_t``.  Every
step of the computation runs in libtmm's CUDA kernels; there is no CPU path.
If libtmm.so is missing (not built) every call raises instead of computing.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtmm.so")

TMM_OK = 0
TMM_ERR_INVALID_ARG = -1
TMM_ERR_UNSUPPORTED = -2
TMM_ERR_CUDA = -3
TMM_ERR_TIMEOUT = -4
TMM_ERR_NOMEM = -5
TMM_F64 = 0
TMM_F32 = 1
TMM_F64X = 2
TMM_F32D = 3
TMM_POL_S = 1
TMM_POL_P = 2
TMM_POL_AVG = 4

EXPORTED = ("tmm_coh_batched", "tmm_coh_batched_ex", "tmm_workspace_size", "tmm_workspace_status",
            "tmm_coh_grad", "tmm_status_string", "tmm_last_cuda_error", "tmm_version",
            "tmm_probe_fma_rate", "tmm_gemm_bf16", "tmm_gemm_bf16_t", "tmm_coh_batched_noalloc",
            "tmm_optimize_workspace_size", "tmm_optimize_adam", "tmm_reward_workspace_size", "tmm_coh_reward",
            "tmm_host_workspace_size", "tmm_coh_batched_host",
            "tmm_inc_batched", "tmm_absorption_batched", "tmm_field_profile", "tmm_pcoh_batched", "tmm_surrogate_create", "tmm_surrogate_destroy", "tmm_surrogate_outputs", "tmm_surrogate_parameters",
            "tmm_surrogate_generate", "tmm_surrogate_train_step", "tmm_surrogate_infer", "tmm_surrogate_layer",
            "tmm_surrogate_status", "tmm_surrogate_save", "tmm_surrogate_load")


class TmmProblem(ctypes.Structure):
    """Mirror of ``tmm_problem``."""
    _fields_ = [
        ("S", ctypes.c_int32), ("L_max", ctypes.c_int32), ("n_lambda", ctypes.c_int32),
        ("n_theta", ctypes.c_int32), ("pol_mask", ctypes.c_uint32), ("prec", ctypes.c_int32),
        ("n_direct", ctypes.c_void_p), ("n_direct_per_lambda", ctypes.c_int32),
        ("mat_table", ctypes.c_void_p), ("mat_idx", ctypes.c_void_p), ("n_materials", ctypes.c_int32),
        ("d", ctypes.c_void_p), ("L_per_stack", ctypes.c_void_p), ("theta", ctypes.c_void_p),
        ("lambda_", ctypes.c_void_p),
    ]


class TmmLaunchCfg(ctypes.Structure):
    """Mirror of ``tmm_launch_cfg``."""
    _fields_ = [("tile_lambda", ctypes.c_int32), ("tile_theta", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("max_items_per_block", ctypes.c_int32)]


class TmmAdamCfg(ctypes.Structure):
    """Mirror of ``tmm_adam_cfg``."""
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("d_min", ctypes.c_double), ("d_max", ctypes.c_double),
                ("step0", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class TmmSurrogateDesc(ctypes.Structure):
    """Mirror of ``tmm_surrogate_desc``."""
    _fields_ = [("n_layers", ctypes.c_int32), ("n_media", ctypes.POINTER(ctypes.c_double)),
                ("n_lambda", ctypes.c_int32), ("lambda_", ctypes.POINTER(ctypes.c_double)),
                ("n_theta", ctypes.c_int32), ("theta", ctypes.POINTER(ctypes.c_double)),
                ("d_min", ctypes.c_double), ("d_max", ctypes.c_double), ("hidden", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class TmmSurrogateLayerView(ctypes.Structure):
    """Mirror of ``tmm_surrogate_layer_view``."""
    _fields_ = [("N", ctypes.c_int32), ("K", ctypes.c_int32), ("Kvalid", ctypes.c_int32),
                ("W", ctypes.c_void_p), ("b", ctypes.c_void_p), ("dW", ctypes.c_void_p), ("db", ctypes.c_void_p)]


class TmmError(RuntimeError):
    def __init__(self, fn, status, detail=""):
        self.status = status
        msg = f"{fn} failed: {status} ({status_text(status)})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


_lib = None
_lock = threading.Lock()


def load(path: Optional[str] = None):
    """Load libtmm.so (no device work).  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libtmm.so is not built ({p}); run __graft_entry__.build() first")
        lib = ctypes.CDLL(p)
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        P = ctypes.POINTER(TmmProblem)
        C = ctypes.POINTER(TmmLaunchCfg)
        lib.tmm_coh_batched.argtypes = [P, vp, vp, vp]
        lib.tmm_coh_batched_ex.argtypes = [P, C, vp, sz, vp, vp, vp]
        lib.tmm_workspace_size.argtypes = [P, C, ctypes.POINTER(sz)]
        lib.tmm_workspace_status.argtypes = [vp, vp]
        lib.tmm_host_workspace_size.argtypes = [P, ctypes.c_int32, ctypes.POINTER(sz)]
        lib.tmm_coh_batched_host.argtypes = [P, ctypes.c_int32, vp, sz, vp, vp, vp]
        lib.tmm_coh_grad.argtypes = [P, vp, vp, vp, vp, vp, sz, vp]
        lib.tmm_status_string.argtypes = [ctypes.c_int]
        lib.tmm_status_string.restype = ctypes.c_char_p
        lib.tmm_last_cuda_error.argtypes = []
        lib.tmm_last_cuda_error.restype = ctypes.c_char_p
        lib.tmm_version.restype = ctypes.c_int32
        lib.tmm_probe_fma_rate.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_float), vp]
        lib.tmm_gemm_bf16.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      vp, vp, vp]
        lib.tmm_gemm_bf16_t.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        vp, vp, vp, ctypes.c_int32, vp]
        lib.tmm_coh_batched_noalloc.argtypes = [P, C, vp, vp, vp]
        lib.tmm_optimize_workspace_size.argtypes = [P, ctypes.POINTER(sz)]
        lib.tmm_reward_workspace_size.argtypes = [P, C, ctypes.POINTER(sz)]
        lib.tmm_coh_reward.argtypes = [P, C, vp, vp, vp, sz, vp]
        lib.tmm_inc_batched.argtypes = [P, vp, vp, vp, vp]
        lib.tmm_absorption_batched.argtypes = [P, vp, vp, vp, vp]
        lib.tmm_field_profile.argtypes = [P, ctypes.c_int32, vp, vp]
        lib.tmm_pcoh_batched.argtypes = [P, vp, vp, ctypes.c_int32, vp, vp, vp]
        lib.tmm_optimize_adam.argtypes = [P, vp, ctypes.POINTER(TmmAdamCfg), ctypes.c_int32, vp, vp, sz, vp]
        i32, f32 = ctypes.c_int32, ctypes.c_float
        lib.tmm_surrogate_create.argtypes = [ctypes.POINTER(TmmSurrogateDesc), ctypes.POINTER(vp)]
        lib.tmm_surrogate_destroy.argtypes = [vp]
        lib.tmm_surrogate_destroy.restype = None
        lib.tmm_surrogate_outputs.argtypes = [vp]
        lib.tmm_surrogate_outputs.restype = i32
        lib.tmm_surrogate_parameters.argtypes = [vp]
        lib.tmm_surrogate_parameters.restype = ctypes.c_int64
        lib.tmm_surrogate_generate.argtypes = [vp, vp, i32, vp, vp]
        lib.tmm_surrogate_train_step.argtypes = [vp, vp, vp, i32, f32, vp, vp]
        lib.tmm_surrogate_infer.argtypes = [vp, vp, i32, vp, f32, f32, vp, vp, vp]
        lib.tmm_surrogate_layer.argtypes = [vp, i32, ctypes.POINTER(TmmSurrogateLayerView)]
        lib.tmm_surrogate_status.argtypes = [vp, vp]
        lib.tmm_surrogate_save.argtypes = [vp, ctypes.c_char_p]
        lib.tmm_surrogate_load.argtypes = [vp, ctypes.c_char_p]
        for name in ("tmm_surrogate_create", "tmm_surrogate_generate", "tmm_surrogate_train_step",
                     "tmm_surrogate_infer", "tmm_surrogate_layer", "tmm_surrogate_status", "tmm_surrogate_save",
                     "tmm_surrogate_load"):
            getattr(lib, name).restype = ctypes.c_int
        for name in ("tmm_coh_batched", "tmm_coh_batched_ex", "tmm_workspace_size",
                     "tmm_workspace_status", "tmm_coh_grad", "tmm_probe_fma_rate", "tmm_gemm_bf16",
                     "tmm_gemm_bf16_t", "tmm_coh_batched_noalloc", "tmm_optimize_workspace_size",
                     "tmm_optimize_adam", "tmm_reward_workspace_size", "tmm_coh_reward", "tmm_inc_batched",
                     "tmm_absorption_batched", "tmm_field_profile", "tmm_pcoh_batched"):
            getattr(lib, name).restype = ctypes.c_int
        if path is None:
            _lib = lib
        return lib


def status_text(status: int) -> str:
    try:
        return load().tmm_status_string(int(status)).decode()
    except Exception:  # library missing: plain text
        return str(status)


def _check(fn, status):
    if status != TMM_OK:
        detail = load().tmm_last_cuda_error().decode() if status == TMM_ERR_CUDA else ""
        raise TmmError(fn, status, detail)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libtmm takes device tensors only")
    if not t.is_contiguous():
        raise ValueError("libtmm takes contiguous tensors only")
    return t.data_ptr()


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


# ---------------------------------------------------------------- problems on the device
@dataclass
class DeviceProblem:
    """A ``tmm_problem`` whose arrays are torch tensors on one CUDA device."""

    prec: int
    pol_mask: int
    theta: torch.Tensor
    lam: torch.Tensor
    d: torch.Tensor
    n_direct: Optional[torch.Tensor] = None      # complex, [S][L+2] or [S][L+2][N_lambda]
    table: Optional[torch.Tensor] = None         # complex [M][N_lambda]
    mat_idx: Optional[torch.Tensor] = None       # int32 [S][L+2]
    L_per_stack: Optional[torch.Tensor] = None   # int32 [S]

    @property
    def real_dtype(self):
        """dtype of the outputs (float for TMM_F32 and TMM_F32D)."""
        return torch.float32 if self.prec in (TMM_F32, TMM_F32D) else torch.float64

    @property
    def S(self):
        return int(self.d.shape[0])

    @property
    def L_max(self):
        return int(self.d.shape[1])

    @property
    def n_pol(self):
        """Output planes: one per polarisation, or one for the s/p average."""
        return 1 if self.pol_mask & TMM_POL_AVG else bin(self.pol_mask & 3).count("1")

    def struct(self) -> TmmProblem:
        p = TmmProblem()
        p.S, p.L_max = self.S, self.L_max
        p.n_lambda, p.n_theta = int(self.lam.shape[0]), int(self.theta.shape[0])
        p.pol_mask, p.prec = self.pol_mask, self.prec
        if self.n_direct is not None:
            p.n_direct = _ptr(self.n_direct)
            p.n_direct_per_lambda = 1 if self.n_direct.dim() == 3 else 0
        else:
            p.mat_table, p.mat_idx = _ptr(self.table), _ptr(self.mat_idx)
            p.n_materials = int(self.table.shape[0])
        p.d, p.theta, p.lambda_ = _ptr(self.d), _ptr(self.theta), _ptr(self.lam)
        p.L_per_stack = _ptr(self.L_per_stack)
        return p

    def out_shape(self):
        return (self.n_pol, self.S, int(self.theta.shape[0]), int(self.lam.shape[0]))

    def empty_out(self):
        return torch.empty(self.out_shape(), dtype=self.real_dtype, device=self.d.device)


def pol_mask_of(pols: str) -> int:
    """"s", "p", "sp", or "u" (unpolarised: the mean of s and p, one plane)."""
    if pols == "u":
        return TMM_POL_S | TMM_POL_P | TMM_POL_AVG
    return (TMM_POL_S if "s" in pols else 0) | (TMM_POL_P if "p" in pols else 0)


def to_device(w, prec="f64", device="cuda", pols=None) -> DeviceProblem:
    """Upload a ``workloads.Workload`` (numpy arrays) as a DeviceProblem.
    prec: "f64", "f32", "f64x" or "f32d" (FP32 arithmetic on double inputs)."""
    pr = {"f64": TMM_F64, "f32": TMM_F32, "f64x": TMM_F64X, "f32d": TMM_F32D}.get(prec, prec)
    rd = torch.float32 if pr == TMM_F32 else torch.float64
    cd = torch.complex64 if pr == TMM_F32 else torch.complex128
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=dt).contiguous()
    return DeviceProblem(
        prec=pr, pol_mask=pol_mask_of(pols or w.pols), theta=t(w.theta, rd), lam=t(w.lam, rd), d=t(w.d, rd),
        n_direct=None if w.n_direct is None else t(w.n_direct, cd),
        table=None if w.table is None else t(w.table, cd),
        mat_idx=None if w.mat_idx is None else t(w.mat_idx, torch.int32),
        L_per_stack=None if w.L_per_stack is None else t(w.L_per_stack, torch.int32))


def launch_cfg(tile_lambda=0, tile_theta=0, persistent=0, blocks_per_sm=0, max_items_per_block=0):
    return TmmLaunchCfg(tile_lambda, tile_theta, persistent, blocks_per_sm, max_items_per_block)


# ---------------------------------------------------------------- the C entry points
def tmm_coh_batched(prob: DeviceProblem, R: torch.Tensor, T: Optional[torch.Tensor] = None, stream=None):
    s = prob.struct()
    _check("tmm_coh_batched", load().tmm_coh_batched(ctypes.byref(s), _ptr(R), _ptr(T), _stream(stream)))


def tmm_workspace_size(prob: DeviceProblem, cfg: Optional[TmmLaunchCfg] = None) -> int:
    s = prob.struct()
    n = ctypes.c_size_t(0)
    _check("tmm_workspace_size", load().tmm_workspace_size(ctypes.byref(s), ctypes.byref(cfg) if cfg else None,
                                                           ctypes.byref(n)))
    return int(n.value)


def tmm_coh_batched_ex(prob: DeviceProblem, cfg: Optional[TmmLaunchCfg], workspace: Optional[torch.Tensor],
                       R: torch.Tensor, T: Optional[torch.Tensor] = None, stream=None):
    s = prob.struct()
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check("tmm_coh_batched_ex", load().tmm_coh_batched_ex(ctypes.byref(s), ctypes.byref(cfg) if cfg else None,
                                                           _ptr(workspace), ws_bytes, _ptr(R), _ptr(T),
                                                           _stream(stream)))


def tmm_coh_batched_noalloc(prob: DeviceProblem, cfg: Optional[TmmLaunchCfg], R: torch.Tensor,
                            T: Optional[torch.Tensor] = None, stream=None):
    """Persistent launch whose scratch is the library's own static device array
    (no allocation; calls that overlap on the GPU race)."""
    s = prob.struct()
    _check("tmm_coh_batched_noalloc", load().tmm_coh_batched_noalloc(
        ctypes.byref(s), ctypes.byref(cfg) if cfg else None, _ptr(R), _ptr(T), _stream(stream)))


def tmm_host_workspace_size(prob_struct: TmmProblem, n_chunks: int) -> int:
    n = ctypes.c_size_t(0)
    _check("tmm_host_workspace_size", load().tmm_host_workspace_size(ctypes.byref(prob_struct), int(n_chunks),
                                                                     ctypes.byref(n)))
    return int(n.value)


def host_problem(prob: "DeviceProblem", host: dict) -> TmmProblem:
    """The tmm_problem of ``prob`` with its arrays replaced by the (pinned) host
    tensors in ``host`` (keys: the DeviceProblem field names)."""
    p = prob.struct()
    hp = lambda t: None if t is None else t.data_ptr()
    if prob.n_direct is not None:
        p.n_direct = hp(host["n_direct"])
    else:
        p.mat_table, p.mat_idx = hp(host["table"]), hp(host["mat_idx"])
    p.d, p.theta, p.lambda_ = hp(host["d"]), hp(host["theta"]), hp(host["lam"])
    p.L_per_stack = hp(host.get("L_per_stack"))
    return p


def tmm_coh_batched_host(prob_struct: TmmProblem, n_chunks: int, workspace: torch.Tensor, R: torch.Tensor,
                         T: Optional[torch.Tensor] = None, stream=None):
    """Host-memory problem and outputs (``prob_struct`` from ``host_problem``);
    ``R``, ``T`` host tensors, ``workspace`` a device tensor."""
    for t in (R, T):
        if t is not None and (t.is_cuda or not t.is_contiguous()):
            raise ValueError("R, T must be contiguous host tensors")
    _check("tmm_coh_batched_host", load().tmm_coh_batched_host(
        ctypes.byref(prob_struct), int(n_chunks), _ptr(workspace), workspace.numel() * workspace.element_size(),
        R.data_ptr(), None if T is None else T.data_ptr(), _stream(stream)))


def tmm_workspace_status(workspace: torch.Tensor, stream=None) -> int:
    """TMM_OK or TMM_ERR_TIMEOUT recorded by a persistent launch (synchronises)."""
    st = load().tmm_workspace_status(_ptr(workspace), _stream(stream))
    if st not in (TMM_OK, TMM_ERR_TIMEOUT):
        _check("tmm_workspace_status", st)
    return st


def tmm_coh_grad(prob: DeviceProblem, R_target: torch.Tensor, merit: torch.Tensor, dm_dd: torch.Tensor,
                 dm_dn: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None, stream=None):
    s = prob.struct()
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check("tmm_coh_grad", load().tmm_coh_grad(ctypes.byref(s), _ptr(R_target), _ptr(merit), _ptr(dm_dd),
                                               _ptr(dm_dn), _ptr(workspace), ws_bytes, _stream(stream)))


def tmm_probe_fma_rate(prec: int, stream=None):
    """(flops per second, kernel ms) of the FMA issue-rate probe."""
    f = ctypes.c_double(0)
    ms = ctypes.c_float(0)
    _check("tmm_probe_fma_rate", load().tmm_probe_fma_rate(int(prec), ctypes.byref(f), ctypes.byref(ms),
                                                           _stream(stream)))
    return f.value, ms.value


def tmm_gemm_bf16(A: torch.Tensor, B: torch.Tensor, bias: Optional[torch.Tensor], epilogue: int,
                  out: torch.Tensor, aux: Optional[torch.Tensor] = None, stream=None):
    """out = epilogue(A @ B^T) on the tcgen05 GEMM (A [M][K], B [N][K] bf16)."""
    M, K = A.shape
    N = B.shape[0]
    _check("tmm_gemm_bf16", load().tmm_gemm_bf16(_ptr(A), _ptr(B), _ptr(bias), M, N, K, epilogue, _ptr(out),
                                                 _ptr(aux), _stream(stream)))


def tmm_gemm_bf16_t(A: torch.Tensor, B: torch.Tensor, bias: Optional[torch.Tensor], epilogue: int,
                    out: torch.Tensor, aux: Optional[torch.Tensor], outT: torch.Tensor, stream=None):
    """tmm_gemm_bf16 (GELU or GELU' epilogue) plus the transposed copy outT [N][ldoT]."""
    M, K = A.shape
    N = B.shape[0]
    _check("tmm_gemm_bf16_t", load().tmm_gemm_bf16_t(_ptr(A), _ptr(B), _ptr(bias), M, N, K, epilogue, _ptr(out),
                                                     _ptr(aux), _ptr(outT), int(outT.stride(0)), _stream(stream)))


def tmm_reward_workspace_size(prob: DeviceProblem, cfg: Optional[TmmLaunchCfg] = None) -> int:
    s = prob.struct()
    n = ctypes.c_size_t(0)
    _check("tmm_reward_workspace_size", load().tmm_reward_workspace_size(ctypes.byref(s),
                                                                         ctypes.byref(cfg) if cfg else None,
                                                                         ctypes.byref(n)))
    return n.value


def tmm_coh_reward(prob: DeviceProblem, R_target: torch.Tensor, reward: torch.Tensor,
                   cfg: Optional[TmmLaunchCfg] = None, workspace: Optional[torch.Tensor] = None, stream=None):
    """reward[s] = -sum |R_target - R| over the output planes, theta, lambda."""
    if workspace is None:
        workspace = alloc_workspace(tmm_reward_workspace_size(prob, cfg), device=prob.d.device)
    nbytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    s = prob.struct()
    _check("tmm_coh_reward", load().tmm_coh_reward(ctypes.byref(s), ctypes.byref(cfg) if cfg else None,
                                                   _ptr(R_target), _ptr(reward), _ptr(workspace), nbytes,
                                                   _stream(stream)))
    return workspace


def tmm_inc_batched(prob: DeviceProblem, incoherent: Optional[torch.Tensor], R: torch.Tensor,
                    T: Optional[torch.Tensor] = None, stream=None):
    """R, T with incoherent layers; ``incoherent`` uint8 [S][L_max] on the device or None."""
    _check("tmm_inc_batched", load().tmm_inc_batched(ctypes.byref(prob.struct()), _ptr(incoherent), _ptr(R),
                                                     _ptr(T), _stream(stream)))


def tmm_absorption_batched(prob: DeviceProblem, A: torch.Tensor, R: Optional[torch.Tensor] = None,
                           T: Optional[torch.Tensor] = None, stream=None):
    """A [P][S][L_max][N_theta][N_lambda] (and R, T) from the partial products."""
    _check("tmm_absorption_batched", load().tmm_absorption_batched(ctypes.byref(prob.struct()), _ptr(A), _ptr(R),
                                                                   _ptr(T), _stream(stream)))


def tmm_field_profile(prob: DeviceProblem, n_z: int, E: torch.Tensor, stream=None):
    """|E(z) / E_inc|^2 into E [P][S][L_max][n_z][N_theta][N_lambda]."""
    _check("tmm_field_profile", load().tmm_field_profile(ctypes.byref(prob.struct()), int(n_z), _ptr(E),
                                                         _stream(stream)))


def tmm_pcoh_batched(prob: DeviceProblem, layer: torch.Tensor, sigma: torch.Tensor, n_nodes: int, R: torch.Tensor,
                     T: Optional[torch.Tensor] = None, stream=None):
    """R, T with one partially coherent layer per stack: layer int32 [S]
    (1-based, 0 = none), sigma [S] nm in the problem's real type."""
    _check("tmm_pcoh_batched", load().tmm_pcoh_batched(ctypes.byref(prob.struct()), _ptr(layer), _ptr(sigma),
                                                       int(n_nodes), _ptr(R), _ptr(T), _stream(stream)))


def adam_cfg(lr, beta1=0.9, beta2=0.999, eps=1e-8, d_min=0.0, d_max=1e30, step0=0) -> TmmAdamCfg:
    return TmmAdamCfg(float(lr), float(beta1), float(beta2), float(eps), float(d_min), float(d_max), int(step0), 0)


def tmm_optimize_workspace_size(prob: DeviceProblem) -> int:
    s = prob.struct()
    n = ctypes.c_size_t(0)
    _check("tmm_optimize_workspace_size", load().tmm_optimize_workspace_size(ctypes.byref(s), ctypes.byref(n)))
    return n.value


def tmm_optimize_adam(prob: DeviceProblem, R_target: torch.Tensor, cfg: TmmAdamCfg, steps: int,
                      merit_hist: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                      stream=None) -> Optional[torch.Tensor]:
    """``steps`` Adam steps on prob.d (updated in place).  Returns the
    workspace (holding the moment estimates) for a later call with
    cfg.step0 = steps taken so far."""
    if workspace is None:
        workspace = alloc_workspace(tmm_optimize_workspace_size(prob), device=prob.d.device)
    nbytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    s = prob.struct()
    _check("tmm_optimize_adam", load().tmm_optimize_adam(ctypes.byref(s), _ptr(R_target), ctypes.byref(cfg),
                                                         int(steps), _ptr(merit_hist), _ptr(workspace), nbytes,
                                                         _stream(stream)))
    return workspace


def tmm_version() -> int:
    return int(load().tmm_version())


def alloc_workspace(nbytes: int, device="cuda") -> Optional[torch.Tensor]:
    """A 256-byte aligned device buffer of at least nbytes (None for 0)."""
    if nbytes <= 0:
        return None
    return torch.empty((nbytes + 255) // 256 * 256, dtype=torch.uint8, device=device)


# ---------------------------------------------------------------- convenience
def coh_tmm(prob: DeviceProblem, with_T=True, cfg: Optional[TmmLaunchCfg] = None, stream=None):
    """R (and T) as [P][S][N_theta][N_lambda] device tensors for a DeviceProblem."""
    R = prob.empty_out()
    T = prob.empty_out() if with_T else None
    if cfg is not None and cfg.persistent:
        ws = alloc_workspace(tmm_workspace_size(prob, cfg), R.device)
        tmm_coh_batched_ex(prob, cfg, ws, R, T, stream)
    elif cfg is not None:
        tmm_coh_batched_ex(prob, cfg, None, R, T, stream)
    else:
        tmm_coh_batched(prob, R, T, stream)
    return R, T
