"""GPU parity of the partially coherent layer (tmm_pcoh_batched) against the
oracle (``oracle/partial.py``: the Gauss-Hermite expectation of the
coherent oracle over the layer's thickness spread).

Tolerances: FP64 1e-10 absolute, FP32 1e-4, element by element in R and T.
The kernel computes its own Gauss-Hermite rule (Sturm bisection); the
oracle takes numpy's.
"""
import numpy as np
import pytest
import torch

from oracle import partial as pc
from paper_2111_13667_gb300 import abi
from paper_2111_13667_gb300 import workloads as W
from tests.helpers import oracle_index

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def gpu_pcoh(w, prec, layer, sigma, K, pols=None):
    prob = abi.to_device(w, prec, pols=pols)
    lay = torch.as_tensor(np.asarray(layer, dtype=np.int32), device="cuda")
    sig = torch.as_tensor(np.asarray(sigma, dtype=np.float64), device="cuda").to(prob.real_dtype)
    R, T = prob.empty_out(), prob.empty_out()
    abi.tmm_pcoh_batched(prob, lay, sig, K, R, T)
    torch.cuda.synchronize()
    return R.double().cpu().numpy(), T.double().cpu().numpy()


def oracle_pcoh(w, layer, sigma, K, pols="sp"):
    n = oracle_index(w)
    out = [pc.pcoh_tmm(pol, n, w.d, layer, sigma, w.theta, w.lam, n_nodes=K, L_per_stack=w.L_per_stack)
           for pol in pols]
    return np.stack([o[0] for o in out]), np.stack([o[1] for o in out])


def lossy_workload(seed, S=8, L=7, n_lambda=23, n_theta=5):
    rng = np.random.default_rng(seed)
    lam = np.linspace(420.0, 780.0, n_lambda)
    n = np.empty((S, L + 2, n_lambda), dtype=np.complex128)
    n[:, 0] = 1.0
    n[:, 1:L + 1] = (rng.uniform(1.3, 2.6, (S, L)) + 1j * rng.uniform(0.0, 0.05, (S, L)))[:, :, None] \
        * (1.0 + 0.03 * (lam - 600.0) / 180.0)
    n[:, L + 1] = 1.52
    d = rng.uniform(15.0, 300.0, (S, L))
    return W.Workload("lossy", theta=np.deg2rad(np.linspace(0, 80, n_theta)), lam=lam, d=d, n_direct=n)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_matches_oracle(prec):
    w = lossy_workload(61)
    rng = np.random.default_rng(62)
    layer = np.array([0, 1, 7, 3, 4, 2, 5, 6])
    sigma = np.array([10.0, 0.0, 12.0, 25.0, 4.0, 30.0, 18.0, 8.0])
    w.d[np.arange(8), np.maximum(layer, 1) - 1] = rng.uniform(600.0, 2000.0, 8)
    Ro, To = oracle_pcoh(w, layer, sigma, 24)
    R, T = gpu_pcoh(w, prec, layer, sigma, 24)
    assert np.max(np.abs(R - Ro)) <= TOL[prec], np.max(np.abs(R - Ro))
    assert np.max(np.abs(T - To)) <= TOL[prec], np.max(np.abs(T - To))


@pytest.mark.parametrize("K", [1, 2, 7, 64, 256])
def test_node_counts(K):
    # every rule size, odd and even, the largest one included
    w = lossy_workload(63, S=3, L=4, n_lambda=9, n_theta=3)
    layer, sigma = [2, 3, 1], [20.0, 5.0, 40.0]
    w.d[:, :] = np.maximum(w.d, 200.0)
    Ro, To = oracle_pcoh(w, layer, sigma, K)
    R, T = gpu_pcoh(w, "f64", layer, sigma, K)
    assert np.max(np.abs(R - Ro)) <= 1e-10 and np.max(np.abs(T - To)) <= 1e-10


def test_zero_spread_is_the_coherent_kernel():
    w = lossy_workload(64, S=5)
    prob = abi.to_device(w, "f64")
    R0, T0 = prob.empty_out(), prob.empty_out()
    abi.tmm_coh_batched(prob, R0, T0)
    R, T = gpu_pcoh(w, "f64", [3, 0, 1, 7, 5], [0.0] * 5, 9)
    assert np.max(np.abs(R - R0.cpu().numpy())) < 1e-12 and np.max(np.abs(T - T0.cpu().numpy())) < 1e-12


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ragged_unpolarised_and_invalid(prec):
    w = W.ragged(seed=65, S=12, L_max=10, n_lambda=11, n_theta=4)
    Ls = w.L_per_stack
    layer = np.minimum(np.arange(12) % 4, Ls)
    layer[10] = Ls[10] + 1      # beyond the stack: NaN
    sigma = np.full(12, 15.0)
    sigma[11] = -1.0            # negative spread: NaN
    Ro, To = oracle_pcoh(w, layer, sigma, 16)
    R, T = gpu_pcoh(w, prec, layer, sigma, 16)
    good = np.ones(12, dtype=bool)
    good[[10, 11]] = False
    assert np.max(np.abs(R[:, good] - Ro[:, good])) <= TOL[prec]
    assert np.max(np.abs(T[:, good] - To[:, good])) <= TOL[prec]
    assert np.all(np.isnan(R[:, ~good])) and np.all(np.isnan(T[:, ~good]))
    Ru, Tu = gpu_pcoh(w, prec, layer, sigma, 16, pols="u")
    assert np.max(np.abs(Ru[0, good] - 0.5 * (Ro[0, good] + Ro[1, good]))) <= TOL[prec]
    assert np.max(np.abs(Tu[0, good] - 0.5 * (To[0, good] + To[1, good]))) <= TOL[prec]


def test_thick_plate_under_coatings_sampled():
    # the coated-substrate workload with its 1 mm plate partially coherent
    # (sigma 30 nm), checked on sampled stacks at full size
    w = W.coated_substrate(S=512, n_lambda=64, n_theta=8)
    layer = np.full(w.S, w.L_max)
    sigma = np.full(w.S, 30.0)
    R, T = gpu_pcoh(w, "f64", layer, sigma, 32)
    idx = np.array([0, 77, 311, 511])
    ws = W.Workload("sample", theta=w.theta, lam=w.lam, d=w.d[idx], table=w.table, mat_idx=w.mat_idx[idx])
    Ro, To = oracle_pcoh(ws, layer[idx], sigma[idx], 32)
    assert np.max(np.abs(R[:, idx] - Ro)) <= 1e-10 and np.max(np.abs(T[:, idx] - To)) <= 1e-10
    assert np.all(R + T <= 1.0 + 1e-12)
