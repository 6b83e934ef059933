"""Ragged batches on the GPU: persistent longest-first launch recorded in a
CUDA graph, autotuned launch shapes, against the FP64 oracle and the padded
launch (zero-thickness outcoupling layers up to L_max, exact by invariance)."""
import numpy as np
import pytest
import torch

from paper_2111_13667_gb300 import abi, autotune
from paper_2111_13667_gb300 import workloads as W
from paper_2111_13667_gb300.ragged import RaggedRunner
from tests.helpers import oracle_RT

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()
    autotune.CACHE_PATH = str(tmp_path_factory.mktemp("tune") / "cache.json")


def np_(t):
    return t.double().cpu().numpy()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_graph_replay_matches_oracle(prec):
    w = W.ragged(seed=41, S=157, L_max=40, n_lambda=37, n_theta=6)
    prob = abi.to_device(w, prec)
    run = RaggedRunner(prob, cfg=abi.launch_cfg(persistent=1)).capture()
    R1, T1 = [np_(x) for x in run()]
    run.R.zero_()
    R2, T2 = [np_(x) for x in run()]
    torch.cuda.synchronize()
    assert run.status() == abi.TMM_OK
    assert np.array_equal(R1, R2) and np.array_equal(T1, T2)
    Ro, To = oracle_RT(w)
    assert np.max(np.abs(R1 - Ro)) <= TOL[prec]
    assert np.max(np.abs(T1 - To)) <= TOL[prec]


def test_autotuned_shape_is_correct_and_cached():
    w = W.ragged(seed=42, S=300, L_max=30, n_lambda=64, n_theta=8)
    prob = abi.to_device(w, "f32")
    report = []
    cfg = autotune.tune(prob, report=report)
    assert len(report) >= 4 and all(r["ms"] > 0 for r in report)
    assert cfg.tile_lambda * cfg.tile_theta <= 512
    again = autotune.tune(prob)  # from the cache
    assert (again.tile_lambda, again.tile_theta, again.persistent) == (cfg.tile_lambda, cfg.tile_theta,
                                                                       cfg.persistent)
    run = RaggedRunner(prob, cfg=cfg).capture()
    R, T = [np_(x) for x in run()]
    Ro, To = oracle_RT(w)
    assert np.max(np.abs(R - Ro)) <= TOL["f32"] and np.max(np.abs(T - To)) <= TOL["f32"]


def test_full_size_ragged_sampled():
    """131072 stacks, L_s ~ U{1..120}, 256 lambda x 16 theta, FP32, in the
    graph-captured persistent launch the benchmark times."""
    w = W.ragged()
    prob = abi.to_device(w, "f32")
    run = RaggedRunner(prob, cfg=abi.launch_cfg(persistent=1)).capture()
    R, T = run()
    torch.cuda.synchronize()
    assert run.status() == abi.TMM_OK
    Ls = w.L_per_stack
    idx = np.unique(np.concatenate([[0, w.S - 1], [int(np.argmax(Ls)), int(np.argmin(Ls))],
                                    np.random.default_rng(3).choice(w.S, 6, replace=False)]))
    Ro, To = oracle_RT(w.subset(idx))
    it = torch.as_tensor(idx, device=R.device)
    assert np.max(np.abs(np_(R[:, it]) - Ro)) <= TOL["f32"]
    assert np.max(np.abs(np_(T[:, it]) - To)) <= TOL["f32"]
    assert bool(torch.isfinite(R).all()) and bool(torch.isfinite(T).all())
    # every element against the double-float launch of the same ragged problem
    # (held to 1e-10 on its own oracle samples), then the padded FP32 launch
    R64, T64 = abi.coh_tmm(abi.to_device(w, "f64x"))
    assert float((R.double() - R64).abs().max()) <= TOL["f32"]
    assert float((T.double() - T64).abs().max()) <= TOL["f32"]
    R64s, T64s = R64[:, it].cpu().numpy(), T64[:, it].cpu().numpy()
    assert np.max(np.abs(R64s - Ro)) <= 1e-10 and np.max(np.abs(T64s - To)) <= 1e-10
    del R64, T64
    padded = abi.DeviceProblem(prob.prec, prob.pol_mask, prob.theta, prob.lam, prob.d, table=prob.table,
                               mat_idx=prob.mat_idx)
    Rp, Tp = abi.coh_tmm(padded)
    assert float((Rp - R).abs().max()) <= 2 * TOL["f32"]
    assert float((Tp - T).abs().max()) <= 2 * TOL["f32"]
