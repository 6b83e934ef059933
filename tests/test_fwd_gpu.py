"""GPU parity of the forward path (tmm_coh_batched) against the FP64 oracle.

Tolerances: FP64 paths (f64, f64x) within 1e-10 absolute in R and T, FP32
paths within 1e-4 absolute, element by element on the same seeded inputs.
"f32" takes its inputs as float (rounded from the seeded doubles), "f32d" as
double; both compute in FP32 and are held to 1e-4 against the oracle on the
double inputs.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

from paper_2111_13667_gb300 import abi
from paper_2111_13667_gb300 import workloads as W
from tests.helpers import oracle_index, oracle_RT

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-4, "f64x": 1e-10, "f32d": 1e-4}
ALL = ["f64", "f32", "f64x", "f32d"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def gpu_RT(w, prec, cfg=None, with_T=True, pols=None):
    prob = abi.to_device(w, prec, pols=pols)
    R, T = abi.coh_tmm(prob, with_T=with_T, cfg=cfg)
    torch.cuda.synchronize()
    return R.double().cpu().numpy(), (T.double().cpu().numpy() if with_T else None)


def assert_close(got, ref, tol, what=""):
    assert got.shape == ref.shape, (got.shape, ref.shape)
    assert np.all(np.isfinite(got)), f"non-finite {what}"
    err = np.max(np.abs(got - ref)) if got.size else 0.0
    assert err <= tol, f"{what}: max |err| = {err:.3e} > {tol:.0e}"


@pytest.mark.parametrize("prec", ALL)
def test_plain_fp64_workload_full(prec):
    w = W.plain_fp64()
    Ro, To = oracle_RT(w)
    R, T = gpu_RT(w, prec)
    assert_close(R, Ro, TOL[prec], "R")
    assert_close(T, To, TOL[prec], "T")


@pytest.mark.parametrize("prec", ALL)
def test_dispersive_small_ragged_tail(prec):
    # several lambda / theta tiles with a partial last tile, gathered index
    w = W.dispersive(seed=11, S=37, L=24, n_lambda=203, n_theta=13)
    Ro, To = oracle_RT(w)
    R, T = gpu_RT(w, prec)
    assert_close(R, Ro, TOL[prec], "R")
    assert_close(T, To, TOL[prec], "T")


@pytest.mark.parametrize("prec", ALL)
def test_direct_per_lambda_index(prec):
    w = W.dispersive(seed=12, S=9, L=10, n_lambda=40, n_theta=5)
    w.n_direct = oracle_index(w)  # same indices given directly, [S][L+2][N_lambda]
    w.table = w.mat_idx = None
    Ro, To = oracle_RT(w)
    R, T = gpu_RT(w, prec)
    assert_close(R, Ro, TOL[prec], "R")
    assert_close(T, To, TOL[prec], "T")


@pytest.mark.parametrize("prec", ALL)
@pytest.mark.parametrize("pols", ["s", "p"])
def test_single_polarisation_and_R_only(prec, pols):
    w = W.plain_fp64(seed=13, S=5, L=7)
    Ro, _ = oracle_RT(w, pols=pols)
    R, _ = gpu_RT(w, prec, with_T=False, pols=pols)
    assert_close(R, Ro, TOL[prec], "R")


@pytest.mark.parametrize("prec", ALL)
def test_unpolarised_average_mode(prec):
    # pol_mask 7: one plane of (R_s + R_p) / 2 and (T_s + T_p) / 2, as the paper
    # averages s and p for unpolarised light
    w = W.dispersive(seed=15, S=11, L=9, n_lambda=70, n_theta=9)
    Ro, To = oracle_RT(w)
    R, T = gpu_RT(w, prec, pols="u")
    assert R.shape == (1,) + Ro.shape[1:]
    assert_close(R[0], 0.5 * (Ro[0] + Ro[1]), TOL[prec], "R unpolarised")
    assert_close(T[0], 0.5 * (To[0] + To[1]), TOL[prec], "T unpolarised")
    # the same as averaging the two planes of the s+p launch, to rounding of a
    # separately compiled kernel
    Rsp, Tsp = gpu_RT(w, prec)
    same = 1e-12 if prec in ("f64", "f64x") else 2e-6
    assert_close(R[0], 0.5 * (Rsp[0] + Rsp[1]), same, "R vs s+p launch")
    assert_close(T[0], 0.5 * (Tsp[0] + Tsp[1]), same, "T vs s+p launch")


@pytest.mark.parametrize("prec", ALL)
def test_total_internal_reflection_and_grazing(prec):
    # injection index 2 into air, interior indices up to 4.6, theta up to
    # exactly 90 deg (the paper's reflectivity-map shape)
    w = W.map_x3()
    Ro, To = oracle_RT(w)
    R, T = gpu_RT(w, prec)
    if prec == "f64x":  # cos(theta) of the rounded pi/2 is 6e-17: R, T within rounding of 1, 0
        assert np.max(np.abs(R[:, 0, -1, :] - 1.0)) <= 1e-12 and np.max(np.abs(T[:, 0, -1, :])) <= 1e-12
    else:
        assert np.all(R[:, 0, -1, :] == 1.0) and np.all(T[:, 0, -1, :] == 0.0)  # grazing reading
    # every precision meets its standard tolerance on the whole map, total
    # internal reflection with its high-Q guided modes included
    assert_close(R, Ro, TOL[prec], "R")
    assert_close(T, To, TOL[prec], "T")
    below = np.sin(w.theta) * 2.0 < 1.0
    assert (~below).sum() > 100  # the map reaches far into total internal reflection


@pytest.mark.parametrize("prec", ALL)
def test_timing_shape_to_grazing(prec):
    # Sec. 4 timing run: 19 layers of real index 1.2-5 between air, theta
    # 0-90 deg.  Near grazing incidence (85.3 deg) this resonant stack turns a
    # phase error of 1e-6 rad per layer into 1e-4 in R: the FP32 kernels hold
    # the plain tolerance because the large, angle-independent part of every
    # layer phase is staged in double-float arithmetic.
    w = W.speedup_x1()
    Ro, To = oracle_RT(w)
    R, T = gpu_RT(w, prec)
    assert_close(R, Ro, TOL[prec], "R")
    assert_close(T, To, TOL[prec], "T")


@pytest.mark.parametrize("prec", ALL)
def test_alternating_shared_memory_sizes(prec):
    # One kernel launched for a deeper, a shallower and again the deeper stack;
    # all three stage more than the 48 KiB default of shared memory, so the
    # limit granted for the first launch must still hold for the third.  These
    # stacks (71 and 97 layers of index 1.3-2.5) reflect up to 0.9996.
    for L in (97, 71, 97):
        w = W.plain_fp64(seed=40 + L, S=3, L=L)
        Ro, To = oracle_RT(w)
        R, T = gpu_RT(w, prec)
        assert_close(R, Ro, TOL[prec], f"R L={L}")
        assert_close(T, To, TOL[prec], f"T L={L}")


@pytest.mark.parametrize("prec", ALL)
def test_single_interface_and_opaque_layers(prec):
    lam = np.linspace(400, 800, 33)
    th = np.deg2rad(np.linspace(0, 70, 6))
    cases = [
        ([1.0, 1.5], []),                                    # L = 0
        ([1.0, 2.0 + 1.0j, 1.7, 1.52], [1e5, 80.0]),         # clamp: thick absorber
        ([1.0] + [2.0 + 1.0j, 1.5] * 12 + [1.52], [1e5, 100.0] * 12),  # many opaque layers
    ]
    for media, d in cases:
        L = len(d)
        nd = np.asarray(media, dtype=np.complex128)[None, :]
        w = W.Workload("case", theta=th, lam=lam, d=np.asarray(d, dtype=np.float64).reshape(1, L), n_direct=nd)
        Ro, To = oracle_RT(w)
        R, T = gpu_RT(w, prec)
        assert_close(R, Ro, TOL[prec], f"R {media[:3]}")
        assert_close(T, To, TOL[prec], f"T {media[:3]}")


@pytest.mark.parametrize("prec", ALL)
def test_interior_gain_and_evanescent_layers(prec):
    # interior roots on both sides of the branch rule: a gain layer (Im n < 0,
    # so Im(n^2 - beta^2) < 0), absorbing layers, and lossless layers that turn
    # evanescent (Re(n^2 - beta^2) < 0) past their critical angle for light
    # injected from index 1.8.  R and T do not depend on which root an interior
    # layer takes (the sign flips cancel), so every path matches the oracle at its tolerance.
    lam = np.linspace(400, 800, 41)
    th = np.deg2rad(np.linspace(0, 80, 10))
    for media, d in (([1.8, 1.35, 2.1 - 0.02j, 1.45, 1.9 + 0.01j, 1.3, 1.9], [120.0, 80.0, 60.0, 150.0, 40.0]),
                     ([1.8, 1.6 - 0.005j, 1.2, 2.4 + 0.1j, 1.2, 1.52 + 0.001j], [200.0, 30.0, 90.0, 25.0])):
        L = len(d)
        nd = np.asarray(media, dtype=np.complex128)[None, :]
        w = W.Workload("case", theta=th, lam=lam, d=np.asarray(d, dtype=np.float64).reshape(1, L), n_direct=nd)
        Ro, To = oracle_RT(w)
        R, T = gpu_RT(w, prec)
        assert_close(R, Ro, TOL[prec], f"R {media}")
        assert_close(T, To, TOL[prec], f"T {media}")


@pytest.mark.parametrize("prec,persistent", [("f64", 0), ("f64", 1), ("f32", 0), ("f32", 1), ("f64x", 0),
                                             ("f32d", 0), ("f32d", 1)])
def test_ragged_layer_counts(prec, persistent):
    w = W.ragged(seed=14, S=301, L_max=60, n_lambda=45, n_theta=7)
    Ro, To = oracle_RT(w)
    cfg = abi.launch_cfg(persistent=persistent)
    R, T = gpu_RT(w, prec, cfg=cfg)
    assert_close(R, Ro, TOL[prec], "R")
    assert_close(T, To, TOL[prec], "T")
    # padded problem (zero-thickness outcoupling layers up to L_max) gives the same
    wp = W.Workload(w.name, theta=w.theta, lam=w.lam, d=w.d, table=w.table, mat_idx=w.mat_idx)
    Rp, Tp = gpu_RT(wp, prec)
    assert_close(Rp, Ro, TOL[prec], "R padded")


def test_bad_material_index_poisons_only_its_stack():
    w = W.dispersive(seed=15, S=6, L=5, n_lambda=16, n_theta=3)
    w.mat_idx = w.mat_idx.copy()
    w.mat_idx[2, 3] = 99
    R, T = gpu_RT(w, "f64")
    assert np.all(np.isnan(R[:, 2])) and np.all(np.isnan(T[:, 2]))
    ok = [0, 1, 3, 4, 5]
    Ro, To = oracle_RT(w.subset(ok))
    assert_close(R[:, ok], Ro, TOL["f64"], "R")


def test_bad_layer_count_poisons_only_its_stack():
    w = W.ragged(seed=16, S=5, L_max=8, n_lambda=16, n_theta=3)
    w.L_per_stack = w.L_per_stack.copy()
    w.L_per_stack[1] = 9
    w.L_per_stack[3] = -1
    for persistent in (0, 1):
        R, _ = gpu_RT(w, "f32", cfg=abi.launch_cfg(persistent=persistent))
        assert np.all(np.isnan(R[:, 1])) and np.all(np.isnan(R[:, 3]))
        assert np.all(np.isfinite(R[:, [0, 2, 4]]))


def test_persistent_iteration_limit_reports_timeout():
    # a deliberately small per-block item budget: blocks stop early and the
    # workspace records TMM_ERR_TIMEOUT (no fault, no hang)
    w = W.ragged(seed=17, S=2000, L_max=10, n_lambda=64, n_theta=4)
    prob = abi.to_device(w, "f32")
    cfg = abi.launch_cfg(persistent=1, blocks_per_sm=1, max_items_per_block=1)
    ws = abi.alloc_workspace(abi.tmm_workspace_size(prob, cfg))
    R = prob.empty_out()
    abi.tmm_coh_batched_ex(prob, cfg, ws, R, None)
    assert abi.tmm_workspace_status(ws) == abi.TMM_ERR_TIMEOUT
    cfg = abi.launch_cfg(persistent=1)
    abi.tmm_coh_batched_ex(prob, cfg, ws, R, None)
    assert abi.tmm_workspace_status(ws) == abi.TMM_OK


def test_workspace_checks():
    w = W.ragged(seed=18, S=10, L_max=10, n_lambda=8, n_theta=2)
    prob = abi.to_device(w, "f32")
    cfg = abi.launch_cfg(persistent=1)
    R = prob.empty_out()
    with pytest.raises(abi.TmmError) as e:
        abi.tmm_coh_batched_ex(prob, cfg, None, R, None)
    assert e.value.status == abi.TMM_ERR_INVALID_ARG
    small = abi.alloc_workspace(256)
    with pytest.raises(abi.TmmError) as e:
        abi.tmm_coh_batched_ex(prob, cfg, small, R, None)
    assert e.value.status == abi.TMM_ERR_NOMEM


def max_abs_diff(a, b, chunk=1 << 26):
    """max |a - b| over two equally shaped device tensors, in FP64, chunk by chunk."""
    a, b = a.reshape(-1), b.reshape(-1)
    m = 0.0
    for i in range(0, a.numel(), chunk):
        m = max(m, float((a[i:i + chunk].double() - b[i:i + chunk].double()).abs().max()))
    return m


_full_f64x = {}


def full_dispersive_f64x():
    """The full dispersive workload in double-float (held to 1e-10 on its
    oracle samples), the reference for whole-tensor checks of the FP32 paths."""
    if not _full_f64x:
        R, T = abi.coh_tmm(abi.to_device(W.dispersive(), "f64x"))
        _full_f64x["RT"] = (R, T)
    return _full_f64x["RT"]


@pytest.mark.parametrize("prec", ALL)
def test_dispersive_full_size_sampled(prec):
    """The full 16384 x 24 x 512 x 32 problem in the launch the benchmark
    times.  A seeded sample of stacks is checked against the oracle; the FP32
    paths are also checked element by element on the whole output against
    the double-float launch, which meets 1e-10 on its own oracle sample."""
    w = W.dispersive()
    prob = abi.to_device(w, prec)
    R, T = abi.coh_tmm(prob)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(99).choice(w.S, size=6, replace=False))
    idx = np.concatenate([[0], idx, [w.S - 1]])
    Ro, To = oracle_RT(w.subset(idx))
    it = torch.as_tensor(idx, device=R.device)
    Rg = R[:, it].double().cpu().numpy()
    Tg = T[:, it].double().cpu().numpy()
    assert_close(Rg, Ro, TOL[prec], "R")
    assert_close(Tg, To, TOL[prec], "T")
    assert bool(torch.isfinite(R).all()) and bool(torch.isfinite(T).all())
    if prec in ("f32", "f32d"):
        Rx, Tx = full_dispersive_f64x()
        eR, eT = max_abs_diff(R, Rx), max_abs_diff(T, Tx)
        assert eR <= TOL[prec] and eT <= TOL[prec], (eR, eT)
    else:
        # properties that hold everywhere: 0 <= R, T and R + T <= 1
        assert float(R.min()) >= -TOL[prec] and float(T.min()) >= -TOL[prec]
        assert float((R + T).max()) <= 1 + TOL[prec]
    del R, T
    if prec == "f32d":
        _full_f64x.clear()
        torch.cuda.empty_cache()


def test_empty_batch():
    w = W.plain_fp64(S=3, L=2)
    prob = abi.to_device(w, "f64")
    prob.d = prob.d[:0]
    prob.n_direct = prob.n_direct[:0]
    R = prob.empty_out()
    abi.tmm_coh_batched(prob, R, None)
    assert R.numel() == 0


def test_f64x_rejects_persistent_and_grad():
    w = W.ragged(seed=19, S=4, L_max=5, n_lambda=8, n_theta=2)
    prob = abi.to_device(w, "f64x")
    R = prob.empty_out()
    cfg = abi.launch_cfg(persistent=1)
    ws = abi.alloc_workspace(abi.tmm_workspace_size(prob, cfg))
    with pytest.raises(abi.TmmError) as e:
        abi.tmm_coh_batched_ex(prob, cfg, ws, R, None)
    assert e.value.status == abi.TMM_ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", ["f32", "f64x", "f32d"])
@pytest.mark.parametrize("n_chunks", [1, 3, 8])
def test_host_entry_matches_device_launch(prec, n_chunks):
    # tmm_coh_batched_host: host inputs and outputs, chunked, copies behind the
    # kernels -- the same kernels on the same values, so bit for bit the device
    # launch; twice in a row on one workspace, pinned and pageable host memory
    w = W.dispersive(seed=20, S=53, L=9, n_lambda=37, n_theta=6)
    prob = abi.to_device(w, prec)
    Rd, Td = abi.coh_tmm(prob)
    for pinned in (True, False):
        pin = (lambda t: t.pin_memory()) if pinned else (lambda t: t)
        h_in = {k: pin(getattr(prob, k).cpu()) for k in ("theta", "lam", "d", "table", "mat_idx")}
        hR = pin(torch.zeros(Rd.shape, dtype=Rd.dtype))
        hT = pin(torch.zeros(Td.shape, dtype=Td.dtype))
        hp = abi.host_problem(prob, h_in)
        ws = torch.empty(abi.tmm_host_workspace_size(hp, n_chunks), dtype=torch.uint8, device="cuda")
        for _ in range(2):
            abi.tmm_coh_batched_host(hp, n_chunks, ws, hR, hT)
            torch.cuda.synchronize()
            assert torch.equal(hR, Rd.cpu()) and torch.equal(hT, Td.cpu())


def test_host_entry_ragged_direct_index_and_checks():
    w = W.ragged(seed=21, S=40, L_max=12, n_lambda=19, n_theta=5)
    w2 = W.plain_fp64(seed=22, S=17, L=6)
    for ww in (w, w2):
        prob = abi.to_device(ww, "f64")
        Rd, _ = abi.coh_tmm(prob, with_T=False)
        keys = [k for k in ("theta", "lam", "d", "table", "mat_idx", "n_direct", "L_per_stack")
                if getattr(prob, k) is not None]
        h_in = {k: getattr(prob, k).cpu() for k in keys}
        hp = abi.host_problem(prob, h_in)
        ws = torch.empty(abi.tmm_host_workspace_size(hp, 4), dtype=torch.uint8, device="cuda")
        hR = torch.zeros(Rd.shape, dtype=Rd.dtype)
        abi.tmm_coh_batched_host(hp, 4, ws, hR, None)
        torch.cuda.synchronize()
        assert torch.equal(hR, Rd.cpu())
        with pytest.raises(abi.TmmError) as e:  # workspace too small
            abi.tmm_coh_batched_host(hp, 4, ws[:256], hR, None)
        assert e.value.status == abi.TMM_ERR_NOMEM
        with pytest.raises(abi.TmmError) as e:  # more chunks than stacks
            abi.tmm_coh_batched_host(hp, ww.S + 1, ws, hR, None)
        assert e.value.status == abi.TMM_ERR_INVALID_ARG
