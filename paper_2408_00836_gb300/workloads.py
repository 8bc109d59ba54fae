"""Seeded synthetic inputs for the five Hubbard workloads (shared by the CUDA
path's tests and benchmark and by the oracle-side tests).

This module only draws random numbers and assembles coefficient arrays from
a bond list the caller supplies; it holds none of the method's arithmetic and
imports nothing from the library or the oracle.  Every draw uses numpy's
PCG64 generator seeded with 1000 + workload number, in the order listed for
each workload.

Workloads (the paper's lattices and couplings, Sec. 3: open 1D/2D lattices,
U/t in {2, 8}, hopping/on-site disorder and NN V of Eqs. 15, 16):

1. chain1x4   1x4 chain, 8 qubits, N = 2+2, t = 1, U = 4; layers of
              (odd, even, U) hops/on-site in application order, 2 layers;
              draws: theta ~ U(-pi, pi) [6].
2. grid2x4    2x4 snake-ordered grid, 16 qubits, N = 4+4, t = 1,
              U in {1, 2, 4, 8}; 4 layers of (U, h1, v1, h2, v2); draws:
              Z ~ N(0,1) [8,8] (orbital perturbation 1e-3 (Z + Z^T)/2),
              theta sets ~ U(-pi, pi) [1024, 20]; batch element b uses theta
              set b // 4 and U value b % 4.
3. grid3x4    3x4 grid, 24 qubits, N = 6+6; t_ij = 1 + 0.1 z_ij on bonds,
              U_i = 4 (1 + 0.1 w_i), V = 0.5 on bonds; 6 layers of
              (U, V, h1, v1, h2, v2); draws: z ~ N(0,1) [12,12] (entry
              [min(i,j), max(i,j)] is used), w ~ N(0,1) [12],
              theta ~ U(-pi, pi) [36].
4. grid2x7    2x7 grid, 28 qubits, N = 7+7, t = 1, U = 8; 8 layers of
              (U, h1, v1, h2, v2); draws: theta_0 ~ N(0, 1e-5) [40]
              (variance 1e-5, the paper's initialisation, Sec. 2.1).
5. grid4x4    4x4 grid, 32 qubits, N = 8+8; t_ij = 1 + z_ij,
              U_i = 8 (1 + w_i) with z, w ~ U(-0.1, 0.1); 4 layers of
              (U, h1, v1, h2, v2); draws: z [16,16], w [16],
              theta ~ U(-pi, pi) [20].
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    number: int
    nx: int
    ny: int
    order: str                 # 'rowmajor' | 'snake'
    n_up: int
    n_dn: int
    layers: int
    classes: list              # one layer, application order
    t: float
    U: list                    # one value per instance
    V: float
    batch: int
    draws: dict = field(default_factory=dict)
    t_noise: str = "none"      # 'none' | 'gauss0.1' | 'uniform'
    U_noise: str = "none"

    @property
    def n_sites(self) -> int:
        return self.nx * self.ny

    @property
    def n_qubits(self) -> int:
        return 2 * self.n_sites

    @property
    def n_params(self) -> int:
        return self.layers * len(self.classes)

    @property
    def n_instances(self) -> int:
        return len(self.U)

    def coefficients(self, bonds, instance: int = 0):
        """(t [L,L], U [L], V [L,L]) for one instance, given the bond list."""
        L = self.n_sites
        t = np.zeros((L, L))
        V = np.zeros((L, L))
        z = self.draws.get("t_noise")
        for (i, j) in bonds:
            a, b = min(i, j), max(i, j)
            if self.t_noise == "gauss0.1":
                v = self.t * (1.0 + 0.1 * z[a, b])
            elif self.t_noise == "uniform":
                v = self.t * (1.0 + z[a, b])
            else:
                v = self.t
            t[a, b] = t[b, a] = v
            if self.V:
                V[a, b] = V[b, a] = self.V
        w = self.draws.get("U_noise")
        U0 = self.U[instance]
        if self.U_noise == "gauss0.1":
            U = U0 * (1.0 + 0.1 * w)
        elif self.U_noise == "uniform":
            U = U0 * (1.0 + w)
        else:
            U = np.full(L, float(U0))
        return t, np.asarray(U, dtype=np.float64), V

    def theta(self) -> np.ndarray:
        """Parameters [batch, P]."""
        th = self.draws["theta"]
        if th.ndim == 1:
            return th[None, :].copy()
        return np.repeat(th, self.n_instances, axis=0)

    def orbital_perturbation(self):
        Z = self.draws.get("perturb_Z")
        if Z is None:
            return None
        return 1e-3 * (Z + Z.T) / 2.0


def workload(number: int, batch_sets: int | None = None) -> Workload:
    """The seeded inputs of workload ``number`` (1..5)."""
    rng = np.random.default_rng(1000 + number)
    H = ["U", "h1", "v1", "h2", "v2"]
    if number == 1:
        w = Workload("chain1x4", 1, 1, 4, "rowmajor", 2, 2, 2, ["odd", "even", "U"], 1.0, [4.0], 0.0, 1)
        w.draws["theta"] = rng.uniform(-math.pi, math.pi, 6)
    elif number == 2:
        w = Workload("grid2x4", 2, 2, 4, "snake", 4, 4, 4, list(H), 1.0, [1.0, 2.0, 4.0, 8.0], 0.0, 4096)
        w.draws["perturb_Z"] = rng.standard_normal((8, 8))
        sets = rng.uniform(-math.pi, math.pi, (1024, 20))
        if batch_sets is not None:
            sets = sets[:batch_sets]
        w.draws["theta"] = sets
        w.batch = sets.shape[0] * 4
    elif number == 3:
        w = Workload("grid3x4", 3, 3, 4, "rowmajor", 6, 6, 6, ["U", "V", "h1", "v1", "h2", "v2"],
                     1.0, [4.0], 0.5, 1, t_noise="gauss0.1", U_noise="gauss0.1")
        w.draws["t_noise"] = rng.standard_normal((12, 12))
        w.draws["U_noise"] = rng.standard_normal(12)
        w.draws["theta"] = rng.uniform(-math.pi, math.pi, 36)
    elif number == 4:
        w = Workload("grid2x7", 4, 2, 7, "rowmajor", 7, 7, 8, list(H), 1.0, [8.0], 0.0, 1)
        w.draws["theta"] = rng.normal(0.0, math.sqrt(1e-5), 40)
    elif number == 5:
        w = Workload("grid4x4", 5, 4, 4, "rowmajor", 8, 8, 4, list(H), 1.0, [8.0], 0.0, 1,
                     t_noise="uniform", U_noise="uniform")
        w.draws["t_noise"] = rng.uniform(-0.1, 0.1, (16, 16))
        w.draws["U_noise"] = rng.uniform(-0.1, 0.1, 16)
        w.draws["theta"] = rng.uniform(-math.pi, math.pi, 20)
    elif number == 6:
        # profiling proxy of workload 5 at 24 qubits: 3x4 grid, N = 6+6,
        # t = 1, U = 8, 4 layers of (U, h1, v1, h2, v2); theta ~ U(-pi, pi)
        w = Workload("grid3x4u", 6, 3, 4, "rowmajor", 6, 6, 4, list(H), 1.0, [8.0], 0.0, 1)
        w.draws["theta"] = rng.uniform(-math.pi, math.pi, 20)
    else:
        raise ValueError(number)
    return w


def random_theta(seed: int, batch: int, P: int, scale: float = math.pi) -> np.ndarray:
    """Extra seeded parameter sets for tests: U(-scale, scale) [batch, P]."""
    return np.random.default_rng(seed).uniform(-scale, scale, (batch, P))


def disordered_grid(nx: int, ny: int, seed: int):
    """Seeded couplings of an nx x ny grid for the NP-ansatz tests: t_ij =
    1 + 0.1 N(0, 1) on every site pair (callers keep the bonds' entries),
    U_i = 4 (1 + 0.1 N(0, 1)), and a diagonal orbital perturbation of
    1e-3 x site index that splits degenerate levels of the Slater start.
    Drawn for all pairs in index order, so the values do not depend on the
    order in which a lattice lists its bonds."""
    L = nx * ny
    rng = np.random.default_rng(seed)
    tt = 1.0 + 0.1 * rng.standard_normal((L, L))
    U = 4.0 * (1.0 + 0.1 * rng.standard_normal(L))
    return tt, U, np.diag(1e-3 * np.arange(L))


def bond_matrix(tt: np.ndarray, bonds) -> np.ndarray:
    """t_ij = tt[min(i,j), max(i,j)] on the listed bonds, 0 elsewhere."""
    t = np.zeros_like(tt)
    for (i, j) in bonds:
        a, b = min(i, j), max(i, j)
        t[i, j] = t[j, i] = tt[a, b]
    return t
