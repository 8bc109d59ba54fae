"""Writes grid2x7_28q.txt: the oracle's energy and adjoint gradient of the
28-qubit workload (2x7 grid, t = 1, U = 8, N = 7 + 7, 8 layers of (U, h1, v1,
h2, v2), Slater-determinant start) at two seeded parameter vectors: the
workload's own theta_0 ~ N(0, 1e-5) (the paper's initialisation, Sec. 2.1)
and a theta ~ U(-1, 1) drawn with seed 44.  Also records the Hartree-Fock
closed form of the start and checks the oracle gradient against central
differences along one seeded direction.

Calls only the oracle (and the seeded input draws); run from the repository
root:  python tests/golden/make_grid2x7_golden.py   (about ten minutes)."""

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2408_00836_gb300 import workloads as W  # noqa: E402


def main():
    w = W.workload(4)
    lat = O.square_lattice(w.nx, w.ny, w.order)
    t, U, V = w.coefficients(lat.bonds)
    m = O.make_model(lat, t, U, None, w.n_up, w.n_dn)
    t0 = time.time()
    basis = O.sector_basis(m)
    H = O.hamiltonian(m, basis)
    pu, pd, _ = O.orbitals(m, w.orbital_perturbation())
    psi0 = O.slater_state(m, pu, pd)
    groups = O.hva_groups(lat, w.layers, w.classes)
    e_hf = O.hartree_fock_energy(m, pu, pd)
    rows = [("hartree_fock", e_hf, [])]
    cache = {}
    thetas = {"theta0": w.theta()[0], "seed44": W.random_theta(44, 1, w.n_params, 1.0)[0]}
    for name, th in thetas.items():
        E, g = O.energy_and_gradient(m, basis, groups, th, psi0, H, cache)
        rows.append((name, E, list(g)))
        print(name, E, time.time() - t0, flush=True)
    # the oracle's own consistency at this size: the adjoint gradient of the
    # second point against a central difference along a seeded direction
    th = thetas["seed44"]
    d = np.random.default_rng(9).standard_normal(len(th))
    d /= np.linalg.norm(d)
    h = 1e-4
    ep = O.energy(m, basis, groups, th + h * d, psi0, H, cache)
    em = O.energy(m, basis, groups, th - h * d, psi0, H, cache)
    fd = (ep - em) / (2 * h)
    ad = float(np.dot(rows[-1][2], d))
    assert abs(fd - ad) < 1e-6 * max(1.0, abs(ad)), (fd, ad)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "grid2x7_28q.txt")
    with open(out, "w") as f:
        f.write("# 28-qubit workload (2x7 grid, U = 8, N = 7+7, 8 HVA layers, Slater start):\n")
        f.write("# oracle energy E and adjoint gradient (Sec. 2.1), complex128, written by\n")
        f.write("# tests/golden/make_grid2x7_golden.py (oracle only).  Columns: name E g_0 .. g_39\n")
        f.write(f"# directional FD check of seed44 along seed-9 direction: fd={fd!r} adjoint={ad!r}\n")
        for name, E, g in rows:
            f.write(" ".join([name, repr(float(E))] + [repr(float(x)) for x in g]) + "\n")
    print("wrote", out, time.time() - t0)


if __name__ == "__main__":
    main()
