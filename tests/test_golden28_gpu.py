"""28-qubit parity against stored oracle values.

tests/golden/grid2x7_28q.txt holds the oracle's energy and adjoint gradient
of the 28-qubit workload (2x7 grid, U = 8, 8 HVA layers, Slater start) at the
workload's seeded theta_0 ~ N(0, 1e-5) and at a seeded theta ~ U(-1, 1),
written by tests/golden/make_grid2x7_golden.py, which calls only the oracle
(its 11.8 M sector amplitudes fit the CPU).  The row engine (the library's
choice at this size) and the dense 2^28 sweeps are compared with them at the
stated bounds, in complex64 and complex128."""

import os

import numpy as np
import pytest

import oracle as O
import paper_2408_00836_gb300 as H
from paper_2408_00836_gb300 import workloads as W

from helpers import TOL, energy_err, grad_err, log_errors

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "grid2x7_28q.txt")


def _golden():
    rows = {}
    with open(GOLD) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows[parts[0]] = (float(parts[1]), np.array([float(x) for x in parts[2:]]))
    return rows


def test_golden_file_is_consistent():
    """CPU: the stored Hartree-Fock row equals the oracle's closed form, and
    each stored gradient has one entry per parameter."""
    w = W.workload(4)
    lat = O.square_lattice(w.nx, w.ny, w.order)
    t, U, _ = w.coefficients(lat.bonds)
    m = O.make_model(lat, t, U, None, w.n_up, w.n_dn)
    pu, pd, _ = O.orbitals(m, None)
    rows = _golden()
    assert abs(rows["hartree_fock"][0] - O.hartree_fock_energy(m, pu, pd)) < 1e-12
    for name in ("theta0", "seed44"):
        assert len(rows[name][1]) == w.n_params


@pytest.mark.gpu
@pytest.mark.parametrize("engine", ["auto", "sweeps"])
@pytest.mark.parametrize("dtype", [H.C64, H.C128])
def test_28q_energy_gradient_against_golden(dtype, engine):
    torch = pytest.importorskip("torch")
    w = W.workload(4)
    bonds, cls = H.square_lattice(w.nx, w.ny, w.order)
    t, U, _ = w.coefficients(bonds)
    a = H.Ansatz(H.Model(w.n_sites, bonds, t, U, None, w.n_up, w.n_dn),
                 H.hva_groups(bonds, cls, w.n_sites, w.layers, w.classes), w.layers)
    rows = _golden()
    thetas = {"theta0": w.theta()[0], "seed44": W.random_theta(44, 1, w.n_params, 1.0)[0]}
    td = torch.complex64 if dtype == H.C64 else torch.complex128
    psi = torch.empty((1, 1 << w.n_qubits), dtype=td, device="cuda")
    lam = torch.empty_like(psi)
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty((1, a.P), dtype=torch.float64, device="cuda")
    for name, theta in thetas.items():
        Eo, go = rows[name]
        a.state_prepare(H.PREP_SLATER, None, None, None, dtype, 1)
        th = torch.tensor(theta[None, :], device="cuda")
        a.energy_grad(th, psi, lam, E, g, dtype=dtype, sweeps=engine == "sweeps")
        H.sync()
        e, gg = float(E[0]), g.cpu().numpy()[0]
        log_errors(f"workload4_28q[{name}]", dtype, engine, energy=energy_err(e, Eo), grad=grad_err(gg, go))
        assert abs(e - Eo) < TOL[dtype] * max(1.0, abs(Eo)), (name, e, Eo)
        assert grad_err(gg, go) < TOL[dtype], (name, grad_err(gg, go))


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [H.C64, H.C128])
def test_28q_batch_of_three_on_rows(dtype):
    """Three parameter sets in one row-engine call (the multi-start shape):
    the first two against the golden values, the third against its own
    single-state call; then the overlap loss of the same batch against one
    shared reference, element by element against single-state calls."""
    torch = pytest.importorskip("torch")
    w = W.workload(4)
    bonds, cls = H.square_lattice(w.nx, w.ny, w.order)
    t, U, _ = w.coefficients(bonds)
    a = H.Ansatz(H.Model(w.n_sites, bonds, t, U, None, w.n_up, w.n_dn),
                 H.hva_groups(bonds, cls, w.n_sites, w.layers, w.classes), w.layers)
    rows = _golden()
    th3 = np.stack([w.theta()[0], W.random_theta(44, 1, w.n_params, 1.0)[0],
                    W.random_theta(45, 1, w.n_params, 1.0)[0]])
    assert a.workspace(1, dtype, 3)[1] == 1                  # the row engine
    td = torch.complex64 if dtype == H.C64 else torch.complex128
    n = w.n_qubits

    def run(th):
        b = th.shape[0]
        a.state_prepare(H.PREP_SLATER, None, None, None, dtype, b)
        psi = torch.empty((b, 1 << n), dtype=td, device="cuda")
        lam = torch.empty_like(psi)
        E = torch.empty(b, dtype=torch.float64, device="cuda")
        g = torch.empty((b, a.P), dtype=torch.float64, device="cuda")
        a.energy_grad(torch.tensor(th, device="cuda"), psi, lam, E, g, dtype=dtype, batch=b)
        H.sync()
        return E.cpu().numpy(), g.cpu().numpy()

    E3, g3 = run(th3)
    for b, name in enumerate(("theta0", "seed44")):
        Eo, go = rows[name]
        assert abs(E3[b] - Eo) < TOL[dtype] * max(1.0, abs(Eo)), (b, E3[b], Eo)
        assert grad_err(g3[b], go) < TOL[dtype], (b, grad_err(g3[b], go))
    E1, g1 = run(th3[2:])
    assert abs(E3[2] - E1[0]) < TOL[dtype] * max(1.0, abs(E1[0]))
    assert grad_err(g3[2], g1[0]) < TOL[dtype]
    # the overlap loss, batch of three against the state at theta0
    a.state_prepare(H.PREP_SLATER, None, None, None, dtype, 1)
    ref = torch.empty((1, 1 << n), dtype=td, device="cuda")
    Er = torch.empty(1, dtype=torch.float64, device="cuda")
    a.energy(torch.tensor(th3[:1], device="cuda"), ref, Er, dtype=dtype, keep_state=True)

    def ovl(th):
        b = th.shape[0]
        a.state_prepare(H.PREP_SLATER, None, None, None, dtype, b)
        psi = torch.empty((b, 1 << n), dtype=td, device="cuda")
        lam = torch.empty_like(psi)
        F = torch.empty(b, dtype=torch.float64, device="cuda")
        f = torch.empty_like(F)
        g = torch.empty((b, a.P), dtype=torch.float64, device="cuda")
        a.overlap_grad(torch.tensor(th, device="cuda"), ref, psi, lam, F, f, g, dtype=dtype, batch=b)
        H.sync()
        return F.cpu().numpy(), g.cpu().numpy()

    F3, gf3 = ovl(th3)
    assert abs(F3[0] - 1.0) < 10 * TOL[dtype]                 # the reference itself
    for b in (1, 2):
        F1, gf1 = ovl(th3[b:b + 1])
        assert abs(F3[b] - F1[0]) < TOL[dtype]
        assert grad_err(gf3[b], gf1[0]) < TOL[dtype]
