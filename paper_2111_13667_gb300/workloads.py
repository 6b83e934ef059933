"""Seeded synthetic inputs for the batched transfer-matrix workloads.

This module only draws inputs: layer thicknesses, refractive indices (given
directly or as a per-material dispersion table plus per-layer material
indices), angle and wavelength grids, ragged layer counts and merit targets.
It contains none of the transfer-matrix arithmetic, so both the CUDA path and
the CPU oracle can be fed from it.

Units: thickness and wavelength in nm, angles in radians (in the injection
medium), complex indices n + i k with k >= 0.  Medium 0 is the injection
medium, medium L+1 the outcoupling medium; ``d`` holds the L finite layers.

Workloads (all seeded with ``numpy.random.default_rng(seed)``):

* ``plain_fp64``  -- 64 stacks x 12 layers, real n ~ U[1.3, 2.5],
  d ~ U[10, 300] nm, ambient 1.0, substrate 1.52, 200 lambda in 400-800 nm,
  10 theta in 0-80 deg, s and p.
* ``dispersive``  -- 16384 stacks x 24 layers, 8 Cauchy materials
  n = A + B / lambda_um^2 (A ~ U[1.3, 2.4], B ~ U[0, 0.02] um^2) with
  k = k0 exp(-lambda_um / 0.3) (k0 ~ U[0, 0.05]); d ~ U[5, 400] nm;
  512 lambda in 300-1200 nm, 32 theta in 0-85 deg.
* ``adjoint``     -- 4096 stacks x 40 layers of the same material model,
  512 lambda in 400-800 nm, 16 theta in 0-60 deg, with a smooth band-stop
  target R_t = 0.02 + 0.93 sig((lambda-550)/5) sig((650-lambda)/5).
* ``ragged``      -- 131072 stacks with L_s ~ U{1..120}, d ~ U[5, 500] nm,
  the same material model, 256 lambda in 350-1000 nm, 16 theta in 0-75 deg.
* ``surrogate``   -- 20 layers alternating 1.46 / 2.35 (layer 1 = 1.46),
  ambient 1.0, substrate 1.52, d ~ U[20, 250] nm, 256 lambda in 400-900 nm,
  8 theta in 0-70 deg.
* ``speedup_x1``, ``dataset_x2``, ``map_x3`` -- the shapes of the paper's own
  timing run (Sec. "Core functionality speedup"), its dataset example
  (appendix A.2) and its reflectivity map (appendix A.1, Fig. 2).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

AMBIENT_N = 1.0
SUBSTRATE_N = 1.52
N_MATERIALS = 8


@dataclass
class Workload:
    """One batched problem.  Exactly one of ``n_direct`` / (``table``, ``mat_idx``) is set.

    n_direct : complex [S][L_max+2] (non-dispersive) or [S][L_max+2][N_lambda]
    table    : complex [M][N_lambda] dispersion table
    mat_idx  : int32 [S][L_max+2] material of every medium (0 and L_s+1 included)
    d        : float64 [S][L_max] thicknesses, nm (entries past L_s are 0)
    L_per_stack : int32 [S] or None (uniform L_max)
    R_target : float64 [P][N_theta][N_lambda] or None
    """

    name: str
    theta: np.ndarray
    lam: np.ndarray
    d: np.ndarray
    pols: str = "sp"
    n_direct: Optional[np.ndarray] = None
    table: Optional[np.ndarray] = None
    mat_idx: Optional[np.ndarray] = None
    L_per_stack: Optional[np.ndarray] = None
    R_target: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def S(self) -> int:
        return int(self.d.shape[0])

    @property
    def L_max(self) -> int:
        return int(self.d.shape[1])

    @property
    def n_lambda(self) -> int:
        return int(self.lam.shape[0])

    @property
    def n_theta(self) -> int:
        return int(self.theta.shape[0])

    @property
    def n_pol(self) -> int:
        return len(self.pols)

    @property
    def evals(self) -> int:
        """Number of (stack, lambda, theta, pol) evaluations."""
        return self.S * self.n_lambda * self.n_theta * self.n_pol

    def layer_steps(self) -> int:
        """Sum over evaluations of (finite layers + 1) interfaces."""
        Ls = self.L_per_stack if self.L_per_stack is not None else np.full(self.S, self.L_max)
        return int(np.sum(Ls.astype(np.int64) + 1)) * self.n_lambda * self.n_theta * self.n_pol

    def subset(self, idx) -> "Workload":
        """The same problem restricted to the stacks ``idx``."""
        idx = np.asarray(idx)
        return replace(
            self,
            d=np.ascontiguousarray(self.d[idx]),
            n_direct=None if self.n_direct is None else np.ascontiguousarray(self.n_direct[idx]),
            mat_idx=None if self.mat_idx is None else np.ascontiguousarray(self.mat_idx[idx]),
            L_per_stack=None if self.L_per_stack is None else np.ascontiguousarray(self.L_per_stack[idx]),
        )


def deg(a):
    return np.deg2rad(np.asarray(a, dtype=np.float64))


def cauchy_table(rng, lam_nm, n_materials=N_MATERIALS, extra=(AMBIENT_N, SUBSTRATE_N)):
    """Material table [n_materials + len(extra)][N_lambda] of complex indices.

    Rows 0..n_materials-1: Cauchy n = A + B / lambda_um^2 with A ~ U[1.3, 2.4],
    B ~ U[0, 0.02] um^2, and k = k0 exp(-lambda_um / 0.3), k0 ~ U[0, 0.05].
    The remaining rows are the constant real indices in ``extra``
    (ambient, substrate).
    """
    A = rng.uniform(1.3, 2.4, n_materials)
    B = rng.uniform(0.0, 0.02, n_materials)
    k0 = rng.uniform(0.0, 0.05, n_materials)
    lu = np.asarray(lam_nm, dtype=np.float64) / 1000.0
    rows = [A[m] + B[m] / lu ** 2 + 1j * k0[m] * np.exp(-lu / 0.3) for m in range(n_materials)]
    rows += [np.full(lu.shape, complex(v)) for v in extra]
    return np.ascontiguousarray(np.array(rows, dtype=np.complex128))


def band_stop_target(lam_nm, n_pol, n_theta):
    """Smooth band-stop target: ~0.95 in 550-650 nm, 0.02 elsewhere, any angle and pol."""
    lam = np.asarray(lam_nm, dtype=np.float64)
    sig = lambda x: 1.0 / (1.0 + np.exp(-x))
    prof = 0.02 + 0.93 * sig((lam - 550.0) / 5.0) * sig((650.0 - lam) / 5.0)
    return np.ascontiguousarray(np.broadcast_to(prof, (n_pol, n_theta, lam.shape[0])).copy())


def _mat_rows(rng, S, L, n_materials=N_MATERIALS):
    """[S][L+2] material indices: ambient row index, L random materials, substrate."""
    amb, sub = n_materials, n_materials + 1
    m = np.empty((S, L + 2), dtype=np.int32)
    m[:, 0] = amb
    m[:, 1:L + 1] = rng.integers(0, n_materials, size=(S, L), dtype=np.int32)
    m[:, L + 1] = sub
    return m


def plain_fp64(seed=0, S=64, L=12):
    rng = np.random.default_rng(seed)
    n = rng.uniform(1.3, 2.5, (S, L))
    d = rng.uniform(10.0, 300.0, (S, L))
    nd = np.empty((S, L + 2), dtype=np.complex128)
    nd[:, 0] = AMBIENT_N
    nd[:, 1:L + 1] = n
    nd[:, L + 1] = SUBSTRATE_N
    return Workload("plain_fp64 (64 stacks x 12 layers, 200 lambda x 10 theta)",
                    theta=deg(np.linspace(0, 80, 10)), lam=np.linspace(400.0, 800.0, 200),
                    d=d, n_direct=nd)


def dispersive(seed=1, S=16384, L=24, n_lambda=512, n_theta=32, shard=0):
    """``shard`` r > 0 draws its own stacks (materials, thicknesses) from a
    stream of its own, with the same material table: the r-th GPU's share of a
    larger batch of independent stacks.  Shard 0 is the single-GPU workload."""
    rng = np.random.default_rng(seed)
    lam = np.linspace(300.0, 1200.0, n_lambda)
    table = cauchy_table(rng, lam)
    if shard:
        rng = np.random.default_rng([seed, shard])
    mat = _mat_rows(rng, S, L)
    d = rng.uniform(5.0, 400.0, (S, L))
    return Workload(f"dispersive ({S} stacks x {L} layers, {n_lambda} lambda x {n_theta} theta, 8 materials)",
                    theta=deg(np.linspace(0, 85, n_theta)), lam=lam, d=d, table=table, mat_idx=mat)


def adjoint(seed=2, S=4096, L=40, n_lambda=512, n_theta=16):
    rng = np.random.default_rng(seed)
    lam = np.linspace(400.0, 800.0, n_lambda)
    table = cauchy_table(rng, lam)
    mat = _mat_rows(rng, S, L)
    d = rng.uniform(5.0, 400.0, (S, L))
    th = deg(np.linspace(0, 60, n_theta))
    return Workload(f"adjoint ({S} stacks x {L} layers, {n_lambda} lambda x {n_theta} theta, MSE merit)",
                    theta=th, lam=lam, d=d, table=table, mat_idx=mat,
                    R_target=band_stop_target(lam, 2, n_theta))


def ragged(seed=3, S=131072, L_max=120, n_lambda=256, n_theta=16):
    """Layer counts L_s ~ U{1..L_max}.  Past L_s the stack is padded with
    zero-thickness layers of the outcoupling medium, so the same arrays also
    describe the padded problem (``L_per_stack`` dropped)."""
    rng = np.random.default_rng(seed)
    lam = np.linspace(350.0, 1000.0, n_lambda)
    table = cauchy_table(rng, lam)
    Ls = rng.integers(1, L_max + 1, size=S, dtype=np.int32)
    mat = _mat_rows(rng, S, L_max)
    d = rng.uniform(5.0, 500.0, (S, L_max))
    j = np.arange(L_max)[None, :]
    d[j >= Ls[:, None]] = 0.0
    jm = np.arange(L_max + 2)[None, :]
    mat[jm >= (Ls[:, None] + 1)] = N_MATERIALS + 1
    return Workload(f"ragged ({S} stacks, L_s~U{{1..{L_max}}}, {n_lambda} lambda x {n_theta} theta)",
                    theta=deg(np.linspace(0, 75, n_theta)), lam=lam, d=d, table=table, mat_idx=mat,
                    L_per_stack=Ls)


def coated_substrate(seed=5, S=16384, L=24, n_lambda=512, n_theta=32, plate_k=0.0):
    """Coatings on a thick glass plate in air: layers 1..L-1 as the dispersive
    workload (8 Cauchy materials, d ~ U[5, 400] nm), layer L a 1 mm plate of
    the substrate index 1.52 (plus i plate_k, a weakly absorbing glass, when
    plate_k > 0) flagged incoherent, air behind it.  Returns the workload with
    ``meta["incoherent"]`` = uint8 [S][L] flags."""
    rng = np.random.default_rng(seed)
    lam = np.linspace(300.0, 1200.0, n_lambda)
    table = cauchy_table(rng, lam)
    if plate_k > 0.0:
        table = np.ascontiguousarray(np.concatenate([table, table[N_MATERIALS + 1:N_MATERIALS + 2] + 1j * plate_k]))
    mat = _mat_rows(rng, S, L)
    mat[:, L] = N_MATERIALS + 1 if plate_k <= 0.0 else N_MATERIALS + 2  # the plate
    mat[:, L + 1] = N_MATERIALS       # air behind it (the ambient row)
    d = rng.uniform(5.0, 400.0, (S, L))
    d[:, L - 1] = 1.0e6
    flags = np.zeros((S, L), dtype=np.uint8)
    flags[:, L - 1] = 1
    return Workload(f"coated substrate ({S} stacks x {L - 1} coherent layers on a 1 mm incoherent plate, "
                    f"{n_lambda} lambda x {n_theta} theta)",
                    theta=deg(np.linspace(0, 85, n_theta)), lam=lam, d=d, table=table, mat_idx=mat,
                    meta={"incoherent": flags})


SURROGATE_L = 20
SURROGATE_D_RANGE = (20.0, 250.0)


def surrogate_stack_index(L=SURROGATE_L):
    """Index row [L+2] of the fixed alternating stack: 1.0 | 1.46 2.35 ... | 1.52."""
    row = np.empty(L + 2, dtype=np.complex128)
    row[0] = AMBIENT_N
    row[1:L + 1] = [1.46 if (j % 2 == 0) else 2.35 for j in range(L)]
    row[L + 1] = SUBSTRATE_N
    return row


def surrogate(seed=4, B=65536):
    rng = np.random.default_rng(seed)
    d = rng.uniform(SURROGATE_D_RANGE[0], SURROGATE_D_RANGE[1], (B, SURROGATE_L))
    nd = np.ascontiguousarray(np.broadcast_to(surrogate_stack_index(), (B, SURROGATE_L + 2)).copy())
    return Workload(f"surrogate ({B} stacks x 20 layers, 256 lambda x 8 theta)",
                    theta=deg(np.linspace(0, 70, 8)), lam=np.linspace(400.0, 900.0, 256),
                    d=d, n_direct=nd)


def speedup_x1(seed=5, S=10):
    """Shape of the paper's timing run: 10 stacks, 21 media (19 finite layers),
    100 lambda in 400-700 nm, 20 theta in 0-90 deg, s only."""
    rng = np.random.default_rng(seed)
    L = 19
    nd = np.empty((S, L + 2), dtype=np.complex128)
    nd[:, 0] = AMBIENT_N
    nd[:, 1:L + 1] = rng.uniform(1.2, 5.0, (S, L))
    nd[:, L + 1] = AMBIENT_N
    d = rng.uniform(20.0, 150.0, (S, L))
    return Workload("speedup_x1 (10 stacks x 19 layers, 100 lambda x 20 theta, s)",
                    theta=deg(np.linspace(0, 90, 20)), lam=np.linspace(400.0, 700.0, 100),
                    d=d, n_direct=nd, pols="s")


def dataset_x2(seed=6, S=1_000_000):
    """Shape of the paper's dataset example: 10 finite layers
    [2.5 | 2.0, 1.4 x5 | 1.0], d ~ U[5, 180] nm, 100 lambda in 1000-1700 nm,
    normal incidence, s only."""
    rng = np.random.default_rng(seed)
    row = np.array([2.5] + [2.0, 1.4] * 5 + [1.0], dtype=np.complex128)
    L = row.shape[0] - 2
    nd = np.ascontiguousarray(np.broadcast_to(row, (S, L + 2)).copy())
    d = rng.uniform(5.0, 180.0, (S, L))
    return Workload(f"dataset_x2 ({S} stacks x {L} layers, 100 lambda, normal incidence, s)",
                    theta=np.zeros(1), lam=np.linspace(1000.0, 1700.0, 100), d=d, n_direct=nd, pols="s")


def map_x3(seed=7, L=10):
    """Shape of the paper's reflectivity map: one stack, 300 lambda in 500-900 nm
    x 300 theta in 0-90 deg; injection index 2, outcoupling into air."""
    rng = np.random.default_rng(seed)
    nd = np.empty((1, L + 2), dtype=np.complex128)
    nd[0, 0] = 2.0
    nd[0, 1:L + 1] = rng.uniform(1.2, 5.0, L)
    nd[0, L + 1] = 1.0
    d = rng.uniform(20.0, 150.0, (1, L))
    return Workload("map_x3 (1 stack, 300 lambda x 300 theta)",
                    theta=deg(np.linspace(0, 90, 300)), lam=np.linspace(500.0, 900.0, 300),
                    d=d, n_direct=nd)


WORKLOADS = {
    "plain_fp64": plain_fp64,
    "dispersive": dispersive,
    "adjoint": adjoint,
    "ragged": ragged,
    "surrogate": surrogate,
    "speedup_x1": speedup_x1,
    "dataset_x2": dataset_x2,
    "map_x3": map_x3,
    "coated_substrate": coated_substrate,
}
