"""GPU parity of stacks with incoherent layers (tmm_inc_batched) against the
oracle's intensity combination of coherent blocks (``oracle/incoherent.py``).

Tolerances as for the coherent path: FP64 within 1e-10, FP32 within 1e-4
absolute in R and T."""
import numpy as np
import pytest
import torch

from oracle import incoherent as inc
from paper_2111_13667_gb300 import abi
from paper_2111_13667_gb300 import workloads as W
from tests.helpers import oracle_RT, oracle_index

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def random_inc_workload(seed, S=5, L=6, n_lambda=17, n_theta=5, L_per_stack=None, inc_k=0.0):
    """Coherent layers may absorb; flagged (incoherent) layers are thick, with
    extinction coefficients up to inc_k."""
    rng = np.random.default_rng(seed)
    lam = np.linspace(450.0, 750.0, n_lambda)
    flags = (rng.uniform(size=(S, L)) < 0.35).astype(np.uint8)
    n = np.empty((S, L + 2, n_lambda), dtype=np.complex128)
    n[:, 0] = 1.0
    re = rng.uniform(1.3, 2.4, (S, L))
    im = np.where(flags == 0, rng.uniform(0.0, 0.08, (S, L)), rng.uniform(0.0, inc_k, (S, L)))
    n[:, 1:L + 1] = (re + 1j * im)[:, :, None] * (1.0 + 0.02 * (lam[None, None, :] - 600.0) / 300.0)
    n[:, L + 1] = 1.52
    d = np.where(flags == 1, rng.uniform(2e4, 5e5, (S, L)), rng.uniform(20.0, 250.0, (S, L)))
    if L_per_stack is not None:
        for s in range(S):
            n[s, L_per_stack[s] + 1:] = 1.52
            d[s, L_per_stack[s]:] = 0.0
            flags[s, L_per_stack[s]:] = 0
    w = W.Workload("inc", theta=np.deg2rad(np.linspace(0, 80, n_theta)), lam=lam, d=d, n_direct=n,
                   L_per_stack=L_per_stack)
    return w, flags


def gpu_inc(w, flags, prec, pols=None):
    prob = abi.to_device(w, prec, pols=pols)
    R, T = prob.empty_out(), prob.empty_out()
    fl = None if flags is None else torch.as_tensor(flags, dtype=torch.uint8, device="cuda").contiguous()
    abi.tmm_inc_batched(prob, fl, R, T)
    torch.cuda.synchronize()
    return R.double().cpu().numpy(), T.double().cpu().numpy()


def oracle_inc(w, flags):
    out = [inc.inc_tmm(pol, w.n_direct, w.d, flags, w.theta, w.lam, L_per_stack=w.L_per_stack) for pol in "sp"]
    return np.stack([o[0] for o in out]), np.stack([o[1] for o in out])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_incoherent_layers_match_oracle(prec):
    w, flags = random_inc_workload(41)
    assert flags.sum() >= 4
    Ro, To = oracle_inc(w, flags)
    R, T = gpu_inc(w, flags, prec)
    assert np.max(np.abs(R - Ro)) <= TOL[prec] and np.max(np.abs(T - To)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ragged_stacks_and_unpolarised_mode(prec):
    Ls = np.array([6, 3, 1, 5, 4], dtype=np.int32)
    w, flags = random_inc_workload(42, L_per_stack=Ls)
    Ro, To = oracle_inc(w, flags)
    R, T = gpu_inc(w, flags, prec)
    assert np.max(np.abs(R - Ro)) <= TOL[prec] and np.max(np.abs(T - To)) <= TOL[prec]
    Ru, Tu = gpu_inc(w, flags, prec, pols="u")
    assert np.max(np.abs(Ru[0] - 0.5 * (Ro[0] + Ro[1]))) <= TOL[prec]
    assert np.max(np.abs(Tu[0] - 0.5 * (To[0] + To[1]))) <= TOL[prec]


def test_no_flags_is_the_coherent_result():
    w, _ = random_inc_workload(43)
    Ro, To = oracle_RT(w)
    R, T = gpu_inc(w, None, "f64")
    assert np.max(np.abs(R - Ro)) <= 1e-10 and np.max(np.abs(T - To)) <= 1e-10


def test_evanescent_cut_and_absorbing_incoherent_layer():
    lam = np.array([600.0, 650.0])
    th = np.deg2rad([0.0, 70.0])
    nd = np.array([[1.8, 2.2, 1.5, 2.0, 1.0],        # at 70 deg the 1.5 slab is evanescent
                   [1.0, 2.0, 1.5 + 0.01j, 1.7, 1.0]], dtype=np.complex128)  # absorbing incoherent
    d = np.array([[110.0, 1e6, 90.0], [100.0, 1e3, 80.0]])
    flags = np.array([[0, 1, 0], [0, 1, 0]], dtype=np.uint8)
    w = W.Workload("cut", theta=th, lam=lam, d=d, n_direct=nd)
    Ro, To = oracle_inc(W.Workload("cut", theta=th, lam=lam, d=d, n_direct=np.repeat(nd[:, :, None], 2, 2)), flags)
    R, T = gpu_inc(w, flags, "f64")
    assert np.max(np.abs(R - Ro)) <= 1e-10 and np.max(np.abs(T - To)) <= 1e-10
    assert np.all(T[:, 0, 1, :] == 0.0)
    assert np.all(T[:, 1] > 0.0) and np.all(R[:, 1] + T[:, 1] < 1.0)  # the absorber transmits part


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_absorbing_incoherent_layers_match_oracle(prec):
    # flagged layers with extinction coefficients up to 1e-4 (0.2 - 500 um
    # thick: single-pass factors down to ~0.3), next to absorbing coherent ones
    w, flags = random_inc_workload(44, S=6, inc_k=1e-4)
    assert flags.sum() >= 4
    Ro, To = oracle_inc(w, flags)
    R, T = gpu_inc(w, flags, prec)
    assert np.max(np.abs(R - Ro)) <= TOL[prec] and np.max(np.abs(T - To)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("plate_k", [1e-6, 2e-5])
def test_coated_absorbing_plate(prec, plate_k):
    # coatings on a 1 mm plate of weakly absorbing glass (1.52 + i plate_k)
    w = W.coated_substrate(S=4, n_lambda=23, n_theta=6, plate_k=plate_k)
    flags = w.meta["incoherent"]
    n = oracle_index(w)
    Ro = np.stack([inc.inc_tmm(pol, n, w.d, flags, w.theta, w.lam)[0] for pol in "sp"])
    To = np.stack([inc.inc_tmm(pol, n, w.d, flags, w.theta, w.lam)[1] for pol in "sp"])
    R, T = gpu_inc(w, flags, prec)
    assert np.max(np.abs(R - Ro)) <= TOL[prec] and np.max(np.abs(T - To)) <= TOL[prec]
    # the plate absorbs: less transmitted than the lossless plate
    w0 = W.coated_substrate(S=4, n_lambda=23, n_theta=6)
    R0, T0 = gpu_inc(w0, flags, prec)
    assert np.all(T <= T0 + TOL[prec])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_evanescent_cut_at_some_angles(prec):
    # FP32 runs two angles per thread: the pairs (0, 70 deg) end at different
    # layers (one-angle fallback), (72, 75 deg) both at the evanescent slab,
    # and the odd fifth angle rides alone
    lam = np.array([600.0, 650.0, 700.0])
    th = np.deg2rad([0.0, 70.0, 72.0, 75.0, 30.0])
    nd = np.array([[1.8, 2.2, 1.5, 2.0, 1.0], [1.8, 1.6, 1.5, 2.3, 1.2]], dtype=np.complex128)
    d = np.array([[110.0, 1e6, 90.0], [140.0, 1e5, 60.0]])
    flags = np.array([[0, 1, 0], [0, 1, 0]], dtype=np.uint8)
    w = W.Workload("cut", theta=th, lam=lam, d=d, n_direct=np.repeat(nd[:, :, None], 3, 2))
    Ro, To = oracle_inc(w, flags)
    R, T = gpu_inc(w, flags, prec)
    assert np.max(np.abs(R - Ro)) <= TOL[prec] and np.max(np.abs(T - To)) <= TOL[prec]
    assert np.all(T[:, :, 1:4, :] == 0.0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_coated_substrate_workload_sample(prec):
    # the benchmark's workload (gathered material table, 1 mm incoherent plate)
    w = W.coated_substrate(S=4, n_lambda=23, n_theta=6)
    flags = w.meta["incoherent"]
    n = oracle_index(w)
    Ro = np.stack([inc.inc_tmm(pol, n, w.d, flags, w.theta, w.lam)[0] for pol in "sp"])
    To = np.stack([inc.inc_tmm(pol, n, w.d, flags, w.theta, w.lam)[1] for pol in "sp"])
    R, T = gpu_inc(w, flags, prec)
    assert np.max(np.abs(R - Ro)) <= TOL[prec] and np.max(np.abs(T - To)) <= TOL[prec]
