"""Launch-shape autotuner for the forward kernels.

Candidates (tile of wavelengths x angles per block, one-block-per-item or
persistent longest-first scheduling) are timed with CUDA events on the real
problem; the fastest is cached in a JSON file keyed by GPU name and a shape
class of the problem (precision, polarisations, ragged or not, stack-count
bucket, L_max, grid sizes).
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, List, Optional

import torch

from . import abi

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CACHE_PATH = os.environ.get("TMM_AUTOTUNE_CACHE", os.path.join(_ROOT, "_build", "autotune_cache.json"))
_lock = threading.Lock()


def shape_key(prob: abi.DeviceProblem, with_T: bool) -> str:
    dev = prob.d.device
    name = torch.cuda.get_device_name(dev).replace(" ", "_")
    S = prob.S
    bucket = 1 << max(0, (S - 1).bit_length())
    return (f"{name}|prec{prob.prec}|pol{prob.pol_mask}|T{int(with_T)}|ragged{int(prob.L_per_stack is not None)}"
            f"|S{bucket}|L{prob.L_max}|nl{prob.lam.shape[0]}|nt{prob.theta.shape[0]}")


def candidates(prob: abi.DeviceProblem, persistent_options=(0, 1)) -> List[abi.TmmLaunchCfg]:
    """Launch shapes to time.  The library's own shape for the problem (tile
    fields 0) comes first, so the tuned choice is never slower than the default
    beyond timing noise, and a problem too small for every listed tile still
    has a candidate; then tiles of 128, 256 or 512 (lambda, theta) points."""
    nt = int(prob.theta.shape[0])
    nl = int(prob.lam.shape[0])
    tts = sorted({t for t in (nt, (nt + 1) // 2, (nt + 3) // 4, 32, 16, 8) if 1 <= t <= min(nt, 32)})
    out = [abi.launch_cfg(persistent=pers) for pers in persistent_options]
    for tt in tts:
        for threads in (128, 256, 512):
            tl = threads // tt
            if tl < 4 or tl * tt < 64 or tl > 2 * max(nl, 1):
                continue
            for pers in persistent_options:
                out.append(abi.launch_cfg(tile_lambda=tl, tile_theta=tt, persistent=pers))
    return out


def _time(prob, cfg, R, T, ws, reps):
    stream = torch.cuda.current_stream()
    launch = (lambda: abi.tmm_coh_batched_ex(prob, cfg, ws, R, T))
    launch()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        launch()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _load_cache() -> Dict[str, dict]:
    try:
        with open(CACHE_PATH) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(key, entry):
    with _lock:
        data = _load_cache()
        data[key] = entry
        os.makedirs(os.path.dirname(CACHE_PATH), exist_ok=True)
        tmp = CACHE_PATH + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, CACHE_PATH)


def tune(prob: abi.DeviceProblem, with_T: bool = True, reps: int = 3, use_cache: bool = True,
         persistent_options=(0, 1), report: Optional[list] = None) -> abi.TmmLaunchCfg:
    """Fastest launch shape for this problem (cached per GPU and shape class);
    tile fields 0 in the result mean the library's default shape."""
    key = shape_key(prob, with_T)
    if use_cache:
        ent = _load_cache().get(key)
        if ent:
            return abi.launch_cfg(**ent["cfg"])
    R = prob.empty_out()
    T = prob.empty_out() if with_T else None
    best, best_ms = None, float("inf")
    for cfg in candidates(prob, persistent_options):
        ws = abi.alloc_workspace(abi.tmm_workspace_size(prob, cfg), prob.d.device) if cfg.persistent else None
        try:
            ms = _time(prob, cfg, R, T, ws, reps)
        except abi.TmmError:
            continue
        if report is not None:
            report.append({"tile_lambda": cfg.tile_lambda, "tile_theta": cfg.tile_theta,
                           "persistent": cfg.persistent, "ms": ms})
        if ms < best_ms:
            best, best_ms = cfg, ms
    if best is None:
        raise RuntimeError("no launch shape could be timed")
    entry = {"cfg": {"tile_lambda": best.tile_lambda, "tile_theta": best.tile_theta,
                     "persistent": best.persistent, "blocks_per_sm": best.blocks_per_sm,
                     "max_items_per_block": 0}, "ms": best_ms}
    if use_cache:
        _store(key, entry)
    return best
