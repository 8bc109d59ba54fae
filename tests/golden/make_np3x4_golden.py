"""Writes np3x4_24q.txt: the oracle's energy and adjoint gradient of the NP
ansatz (Sec. 2.2.1, Eq. 8: per-term Givens and controlled-phase factors,
on-site spin mixing, R_z pre-layer; one layer, 116 parameters) on a 3x4
grid (24 qubits, N = 6 + 6, spin-blocked order) with seeded disordered
couplings (workloads.disordered_grid, seed 71), from the Slater start, at
theta ~ U(-1, 1) (workloads.random_theta, seed 72).  The NP gates conserve
only the total electron number, so the oracle works in the total-N basis
(2 704 156 states).  Also checks the oracle gradient against a central
difference along one seeded direction.

Calls only the oracle (and the seeded input draws); run from the repository
root:  python tests/golden/make_np3x4_golden.py   (a few minutes)."""

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2408_00836_gb300 import workloads as W  # noqa: E402

NX, NY, LAYERS, N_UP, N_DN = 3, 4, 1, 6, 6


def main():
    L = NX * NY
    lat = O.square_lattice(NX, NY)
    tt, U, perturb = W.disordered_grid(NX, NY, 71)
    t = W.bond_matrix(tt, lat.bonds)
    m = O.make_model(lat, t, U, None, N_UP, N_DN)
    groups = O.np_groups(lat, m, LAYERS)
    P = max(g.param for g in groups) + 1
    assert P == O.np_param_count(NX, NY, LAYERS)
    theta = W.random_theta(72, 1, P, 1.0)[0]
    t0 = time.time()
    basis = O.number_basis(m, N_UP + N_DN)
    sec = O.sector_basis(m)
    pu, pd, _ = O.orbitals(m, perturb)
    psi0 = np.zeros(len(basis), dtype=complex)
    psi0[np.searchsorted(basis, sec)] = O.slater_state(m, pu, pd)
    H = O.hamiltonian(m, basis)
    cache = {}
    E, g = O.energy_and_gradient(m, basis, groups, theta, psi0, H, cache)
    print("E", E, time.time() - t0, flush=True)
    d = np.random.default_rng(9).standard_normal(P)
    d /= np.linalg.norm(d)
    h = 1e-4
    ep = O.energy(m, basis, groups, theta + h * d, psi0, H, cache)
    em = O.energy(m, basis, groups, theta - h * d, psi0, H, cache)
    fd = (ep - em) / (2 * h)
    ad = float(np.dot(g, d))
    assert abs(fd - ad) < 1e-6 * max(1.0, abs(ad)), (fd, ad)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "np3x4_24q.txt")
    with open(out, "w") as f:
        f.write("# NP ansatz, 3x4 grid (24 qubits, N = 6+6, spin-blocked), 1 layer, 116 parameters,\n")
        f.write("# disordered couplings (workloads.disordered_grid seed 71), theta seed 72, Slater start:\n")
        f.write("# oracle energy E and adjoint gradient (Sec. 2.1), complex128, total-N basis, written by\n")
        f.write("# tests/golden/make_np3x4_golden.py (oracle only).  Columns: name E g_0 .. g_115\n")
        f.write(f"# directional FD check along the seed-9 direction: fd={fd!r} adjoint={ad!r}\n")
        f.write("theta72 " + repr(float(E)) + " " + " ".join(repr(float(x)) for x in g) + "\n")
    print("wrote", out, time.time() - t0)


if __name__ == "__main__":
    main()
