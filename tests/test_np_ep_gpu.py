"""The NP ansatz (Sec. 2.2.1: per-term Givens and controlled-phase factors
of Eq. 8, on-site spin mixing, R_z pre-layer) and the EP ansatz (Sec. 2.2.2:
Eq. 10 on neighbouring qubits, R_z before and after) through the C ABI
against the oracle.

Both mix the two spin species (the on-site NP gate moves an electron from
an up to a down mode; EP gates join qubits of either spin), so only the
total electron number is conserved: the oracle works in the total-N basis
and the library runs dense sweeps over every tile.  Energies and gradients
are compared at the stated bounds, the final state amplitude by amplitude
(including the weight that leaves the (N_up, N_dn) sector), in both JW
orders, complex64 and complex128."""

import numpy as np
import pytest

import oracle as O
import paper_2408_00836_gb300 as H

from helpers import TOL, energy_err, grad_err, log_errors, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {H.C64: torch.complex64, H.C128: torch.complex128}
_CACHE = {}


def _case(kind, nx, ny, layers, modes):
    key = (kind, nx, ny, layers, modes)
    if key in _CACHE:
        return _CACHE[key]
    rng = np.random.default_rng(70 + nx * ny + layers)
    bonds, cls = H.square_lattice(nx, ny)
    L = nx * ny
    t = np.zeros((L, L))
    for (i, j) in bonds:
        t[i, j] = t[j, i] = 1.0 + 0.1 * rng.standard_normal()
    U = 4.0 * (1 + 0.1 * rng.standard_normal(L))
    n_up, n_dn = L // 2, L - L // 2
    model = H.Model(L, bonds, t, U, None, n_up, n_dn, modes=modes)
    if kind == "np":
        groups = H.np_groups(bonds, cls, L, layers, modes=modes)
    else:
        groups = H.ep_groups(2 * L, layers)
    ans = H.Ansatz(model, groups, 1)
    lat = O.square_lattice(nx, ny)
    om = O.make_model(lat, t, U, None, n_up, n_dn, modes=modes)
    og = O.np_groups(lat, om, layers) if kind == "np" else O.ep_groups(2 * L, layers)
    assert ans.P == max(g.param for g in og) + 1
    basis = O.number_basis(om, n_up + n_dn)
    perturb = np.diag(1e-3 * np.arange(L))          # splits degenerate levels
    pu, pd, _ = O.orbitals(om, perturb)
    sec = O.sector_basis(om)
    psi0 = np.zeros(len(basis), dtype=complex)
    psi0[np.searchsorted(basis, sec)] = O.slater_state(om, pu, pd)
    Hm = O.hamiltonian(om, basis)
    theta = rng.uniform(-1.0, 1.0, ans.P)
    Eo, go = O.energy_and_gradient(om, basis, og, theta, psi0, Hm)
    st = O.ansatz_state(om, basis, og, theta, psi0)
    full = np.zeros(1 << (2 * L), dtype=complex)
    full[basis.astype(np.int64)] = st
    outside = float(np.sum(np.abs(st[~np.isin(basis, sec)]) ** 2))
    _CACHE[key] = (ans, perturb, theta, Eo, go, full, outside)
    return _CACHE[key]


CASES = [("np", 2, 2, 2, "interleaved"), ("np", 2, 2, 2, "blocked"), ("np", 2, 4, 2, "blocked"),
         ("np", 2, 3, 3, "interleaved"), ("ep", 2, 3, 2, "interleaved"), ("ep", 2, 2, 3, "blocked")]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(map(str, c)))
@pytest.mark.parametrize("dtype", [H.C64, H.C128])
def test_np_ep_energy_gradient_and_state(dtype, case):
    ans, perturb, theta, Eo, go, full, outside = _case(*case)
    assert outside > 1e-4            # the circuit leaves the (N_up, N_dn) sector
    n = ans.n
    ans.state_prepare(H.PREP_SLATER, perturb, None, None, dtype, 1)
    th = torch.tensor(theta[None, :], device="cuda")
    psi = torch.empty((1, 1 << n), dtype=DT[dtype], device="cuda")
    lam = torch.empty_like(psi)
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty((1, ans.P), dtype=torch.float64, device="cuda")
    ans.energy_grad(th, psi, lam, E, g, dtype=dtype)
    H.sync()
    e, gg = float(E[0]), g.cpu().numpy()[0]
    log_errors("-".join(map(str, case)), dtype, "sweeps", energy=energy_err(e, Eo), grad=grad_err(gg, go))
    assert abs(e - Eo) < TOL[dtype] * max(1.0, abs(Eo))
    assert grad_err(gg, go) < TOL[dtype], grad_err(gg, go)
    ans.energy(th, psi, E, dtype=dtype, keep_state=True)
    H.sync()
    got = psi.cpu().numpy()[0]
    assert rel_err(got, full) < TOL[dtype]
    assert abs(float(E[0]) - Eo) < TOL[dtype] * max(1.0, abs(Eo))


def _golden_np3x4():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "np3x4_24q.txt")
    with open(path) as f:
        row = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")][0]
    return float(row[1]), np.array([float(x) for x in row[2:]])


@pytest.mark.parametrize("dtype", [H.C64, H.C128])
def test_np3x4_24_qubits_against_golden(dtype):
    """The NP ansatz at 24 qubits (3x4, one layer, 116 parameters, spin
    mixing: dense sweeps over all 4096 tiles) against the oracle's energy
    and gradient stored by tests/golden/make_np3x4_golden.py from the same
    seeded inputs."""
    from paper_2408_00836_gb300 import workloads as W
    Eo, go = _golden_np3x4()
    tt, U, perturb = W.disordered_grid(3, 4, 71)
    bonds, cls = H.square_lattice(3, 4)
    model = H.Model(12, bonds, W.bond_matrix(tt, bonds), U, None, 6, 6)
    ans = H.Ansatz(model, H.np_groups(bonds, cls, 12, 1), 1)
    assert ans.P == len(go) == 116
    theta = W.random_theta(72, 1, ans.P, 1.0)
    ans.state_prepare(H.PREP_SLATER, perturb, None, None, dtype, 1)
    th = torch.tensor(theta, device="cuda")
    psi = torch.empty((1, 1 << 24), dtype=DT[dtype], device="cuda")
    lam = torch.empty_like(psi)
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty((1, ans.P), dtype=torch.float64, device="cuda")
    ans.energy_grad(th, psi, lam, E, g, dtype=dtype)
    H.sync()
    e, gg = float(E[0]), g.cpu().numpy()[0]
    log_errors("np3x4_24q_golden", dtype, "sweeps", energy=energy_err(e, Eo), grad=grad_err(gg, go))
    assert abs(e - Eo) < TOL[dtype] * max(1.0, abs(Eo))
    assert grad_err(gg, go) < TOL[dtype], grad_err(gg, go)
