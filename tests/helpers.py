"""Shared test helpers: build the same problem on the CUDA path and in the
oracle from the same seeded inputs, and compare results.

Tolerances (relative to the scale of the quantity):
  energies     c128 1e-10, c64 1e-6   (the stated parity targets)
  gradients    c128 1e-10, c64 1e-6   (relative to max(1, |grad|_inf))
  state        c128 1e-10, c64 1e-6   (relative L2 error of the vector)
"""

import json
import os

import numpy as np

import oracle as O
import paper_2408_00836_gb300 as H

TOL = {H.C128: 1e-10, H.C64: 1e-6}


class Problem:
    def __init__(self, nx, ny, order="rowmajor", modes="blocked", t=None, U=None, V=None,
                 n_up=None, n_dn=None, layers=2, classes=("U", "h1", "v1", "h2", "v2"),
                 perturb=None, instances=None):
        import torch  # noqa: F401  (CUDA side only)
        self.nx, self.ny, self.L = nx, ny, nx * ny
        self.bonds, self.cls = H.square_lattice(nx, ny, order)
        self.lat = O.square_lattice(nx, ny, order)
        L = self.L
        self.n_up = L // 2 if n_up is None else n_up
        self.n_dn = L // 2 if n_dn is None else n_dn
        # instances: list of (t, U, V)
        if instances is None:
            instances = [(t, U, V)]
        self.instances = instances
        self.models = [H.Model(L, self.bonds, ti, Ui, Vi, self.n_up, self.n_dn, modes=modes)
                       for (ti, Ui, Vi) in instances]
        self.groups = H.hva_groups(self.bonds, self.cls, L, layers, list(classes))
        self.ans = H.Ansatz(self.models, self.groups, layers)
        self.P = self.ans.P
        self.n = 2 * L
        self.omodels = [O.make_model(self.lat, ti, Ui, Vi, self.n_up, self.n_dn, modes=modes)
                        for (ti, Ui, Vi) in instances]
        # the oracle names the on-site potential group 'eps'
        self.ogroups = O.hva_groups(self.lat, layers, ["eps" if c == "pot" else c for c in classes])
        self.basis = O.sector_basis(self.omodels[0])
        self.perturb = perturb
        self._psi0 = {}
        self._H = {}

    def psi0(self, r=0):
        if r not in self._psi0:
            pu, pd, _ = O.orbitals(self.omodels[r], self.perturb)
            self._psi0[r] = O.slater_state(self.omodels[r], pu, pd)
        return self._psi0[r]

    def Hmat(self, r=0):
        if r not in self._H:
            self._H[r] = O.hamiltonian(self.omodels[r], self.basis)
        return self._H[r]

    def full(self, vec):
        out = np.zeros(1 << self.n, dtype=np.complex128)
        out[self.basis.astype(np.int64)] = vec
        return out

    def oracle_energy_grad(self, theta, r=0):
        return O.energy_and_gradient(self.omodels[r], self.basis, self.ogroups, theta, self.psi0(r),
                                     self.Hmat(r))

    def oracle_state(self, theta, r=0):
        return O.ansatz_state(self.omodels[r], self.basis, self.ogroups, theta, self.psi0(r))


def grad_scale(prob, theta, r=0):
    """Per-parameter scale of a gradient comparison: max(1, S_p) with S_p =
    sum over the groups of parameter p of 2 ||lam_k|| ||G_k psi_k||, the
    Cauchy-Schwarz bound of the terms 2 Im<lam_k|G_k|psi_k> that make up g_p
    (Sec. 2.1).  Rounding in a given precision is relative to the size of
    these terms, not to |g_p|, which cancellation can make small (on a single
    basis state g = 0 exactly while each term is of size ||H psi|| ||G psi||)."""
    om, basis, groups = prob.omodels[r], prob.basis, prob.ogroups
    psi = prob.oracle_state(theta, r)
    lam = prob.Hmat(r) @ psi
    S = np.zeros(len(theta))
    cache = {}
    for g in reversed(groups):
        Gpsi = O.apply_generator(om, basis, g, psi, cache)
        S[g.param] += 2.0 * float(np.linalg.norm(lam) * np.linalg.norm(Gpsi))
        th = float(theta[g.param])
        psi = O.apply_group(om, basis, g, th, psi, cache, inverse=True)
        lam = O.apply_group(om, basis, g, th, lam, cache, inverse=True)
    return np.maximum(1.0, S)


def rel_err(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def grad_err(g, go):
    """c64/c128 gradient error in units of the stated target: max_p |g_p -
    g_ref,p| / max(1, |g_ref|_inf)."""
    return float(np.max(np.abs(np.asarray(g) - np.asarray(go))) / max(1.0, float(np.max(np.abs(go)))))


def energy_err(E, Eo):
    return float(abs(E - Eo) / max(1.0, abs(Eo)))


def log_errors(test: str, dtype: int, engine: str, **errs):
    """Appends the measured errors of one result (relative, see grad_err /
    energy_err) to the JSON-lines file named by HUBSV_ERR_LOG, if set, so
    that a GPU run states the error of each result against the oracle."""
    path = os.environ.get("HUBSV_ERR_LOG")
    if not path:
        return
    rec = {"test": test, "dtype": "c64" if dtype == H.C64 else "c128", "engine": engine,
           "tol": TOL[dtype]}
    rec.update({k: float(v) for k, v in errs.items()})
    with open(path, "a") as f:
        f.write(json.dumps(rec) + "\n")
