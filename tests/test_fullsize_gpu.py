"""Parity at the full benchmark sizes (28 and 32 qubits), in the launch
configuration bench.py times.  The oracle cannot evolve 2^32 amplitudes, so
these tests use what it computes exactly at any size -- the Hartree-Fock
closed form of the Slater start, H applied to sampled basis states one by
one from its Jordan-Wigner operators, exact periodicities of the ansatz --
and properties that hold at any size (complex64 against complex128, the
adjoint gradient against a finite difference)."""

import math

import numpy as np
import pytest

import oracle as O
import paper_2408_00836_gb300 as H
from paper_2408_00836_gb300 import workloads as W

from helpers import TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {H.C64: torch.complex64, H.C128: torch.complex128}


def _setup(number):
    w = W.workload(number)
    bonds, cls = H.square_lattice(w.nx, w.ny, w.order)
    t, U, V = w.coefficients(bonds)
    m = H.Model(w.n_sites, bonds, t, U, V if w.V else None, w.n_up, w.n_dn)
    a = H.Ansatz(m, H.hva_groups(bonds, cls, w.n_sites, w.layers, w.classes), w.layers)
    lat = O.square_lattice(w.nx, w.ny, w.order)
    om = O.make_model(lat, t, U, V if w.V else None, w.n_up, w.n_dn)
    return w, a, om


def _energy(a, w, theta, dtype, psi=None, keep=False):
    if psi is None:
        psi = torch.empty((1, 1 << w.n_qubits), dtype=DT[dtype], device="cuda")
    a.state_prepare(H.PREP_SLATER, w.orbital_perturbation(), None, None, dtype, 1)
    th = torch.tensor(np.asarray(theta, dtype=np.float64).reshape(1, -1), device="cuda")
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    a.energy(th, psi, E, dtype=dtype, batch=1, keep_state=keep)
    H.sync()
    return float(E[0])


@pytest.mark.parametrize("number", [4, 5])
def test_slater_start_energy_is_hartree_fock(number):
    """theta = 0: the ansatz is the identity and E is the HF closed form."""
    w, a, om = _setup(number)
    pu, pd, _ = O.orbitals(om, w.orbital_perturbation())
    e_hf = O.hartree_fock_energy(om, pu, pd)
    for dtype in (H.C64, H.C128):
        e = _energy(a, w, np.zeros(a.P), dtype)
        assert abs(e - e_hf) < TOL[dtype] * max(1.0, abs(e_hf)), (dtype, e, e_hf)
        torch.cuda.empty_cache()


def test_32q_apply_h_on_sampled_states():
    """lam = H psi at 32 qubits, checked element by element on 1500 sampled
    sector states against the oracle's operators applied one state at a
    time (psi read back from the GPU at the partners)."""
    w, a, om = _setup(5)
    n = w.n_qubits
    psi = torch.empty((1, 1 << n), dtype=torch.complex64, device="cuda")
    a.state_prepare(H.PREP_SLATER, None, None, psi, H.C64, 1)
    lam = torch.empty_like(psi)
    a.apply_h(psi, lam, H.C64)
    H.sync()
    rng = np.random.default_rng(3)
    L = w.n_sites
    ups = np.array([sum(1 << int(s) for s in rng.choice(L, 8, replace=False)) for _ in range(1500)], dtype=np.uint64)
    dns = np.array([sum(1 << (L + int(s)) for s in rng.choice(L, 8, replace=False)) for _ in range(1500)], dtype=np.uint64)
    xs = ups | dns
    # oracle: off-diagonal partners y of each x with the matrix element, from a+ a
    rows, partners, coefs = [], [], []
    for (i, j) in om.bonds:
        for m in (om.up, om.dn):
            for (p, q) in ((int(m[i]), int(m[j])), (int(m[j]), int(m[i]))):
                v1, s1, y = O.annihilate(xs, q)
                v2, s2, z = O.create(y, p)
                ok = v1 & v2
                rows.append(np.flatnonzero(ok))
                partners.append(z[ok])
                coefs.append(-om.t[i, j] * (s1 * s2)[ok])
    d = O.hubbard.diagonal_energy(om, xs)
    allidx = np.concatenate([xs] + partners).astype(np.int64)
    uniq, inv = np.unique(allidx, return_inverse=True)
    vals = psi[0, torch.tensor(uniq, device="cuda")].cpu().numpy().astype(np.complex128)
    lam_got = lam[0, torch.tensor(xs.astype(np.int64), device="cuda")].cpu().numpy()
    psi_x = vals[inv[:len(xs)]]
    ref = d * psi_x
    off = len(xs)
    for r, z, c in zip(rows, partners, coefs):
        ref[r] += c * vals[inv[off:off + len(z)]]
        off += len(z)
    scale = np.max(np.abs(ref))
    assert scale > 0
    assert np.max(np.abs(lam_got - ref)) < 5e-6 * scale


def test_28q_periodicity_and_precisions():
    """Uniform t = 1 and U = 8: exp(-i 2 pi G_hop) = exp(-i (2 pi / 8) G_U) = 1,
    so shifting a hop parameter by 2 pi or an on-site one by 2 pi / 8 leaves E
    unchanged; complex64 agrees with complex128."""
    w, a, om = _setup(4)
    theta = W.random_theta(44, 1, a.P, 1.0)[0]
    e128 = _energy(a, w, theta, H.C128)
    e64 = _energy(a, w, theta, H.C64)
    assert abs(e64 - e128) < TOL[H.C64] * max(1.0, abs(e128))
    t2 = theta.copy()
    t2[1] += 2 * math.pi      # h1 of layer 0
    t2[5] += 2 * math.pi / 8  # U of layer 1
    t2[13] += 2 * math.pi     # h2 of layer 2
    assert abs(_energy(a, w, t2, H.C128) - e128) < TOL[H.C128] * max(1.0, abs(e128))
    t3 = theta.copy()
    t3[5] += math.pi / 8      # half a period moves it
    assert abs(_energy(a, w, t3, H.C128) - e128) > 1e-6


def test_32q_c64_energy_gradient_against_c128_and_fd():
    """Workload 5 at full size: c64 energy + adjoint gradient (the benchmarked
    call, row engine) against c128 energies: the energy within the c64
    tolerance and the gradient's directional derivative against a central
    difference; the dense sweeps with the layer checkpoint give the same."""
    w, a, om = _setup(5)
    theta = w.theta()[0]
    n = w.n_qubits
    psi = torch.empty((1, 1 << n), dtype=torch.complex64, device="cuda")
    lam = torch.empty_like(psi)
    a.state_prepare(H.PREP_SLATER, w.orbital_perturbation(), None, None, H.C64, 1)
    th = torch.tensor(theta[None, :], device="cuda")
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty((1, a.P), dtype=torch.float64, device="cuda")
    a.energy_grad(th, psi, lam, E, g, dtype=H.C64, batch=1)
    H.sync()
    e64 = float(E[0])
    g64 = g.cpu().numpy()[0]
    # the dense 2^32 sweeps with a checkpoint of psi at the middle layer
    # (three 2^32 vectors resident, 103 GB): the same energy and gradient
    ck = torch.empty_like(psi)
    a.energy_grad(th, psi, lam, E, g, ckpt=ck, dtype=H.C64, batch=1, sweeps=True)
    H.sync()
    g64c = g.cpu().numpy()[0]
    assert abs(float(E[0]) - e64) < TOL[H.C64] * max(1.0, abs(e64))
    assert np.max(np.abs(g64c - g64)) < 2 * TOL[H.C64] * max(1.0, np.max(np.abs(g64)))
    del psi, lam, ck
    torch.cuda.empty_cache()
    psi = torch.empty((1, 1 << n), dtype=torch.complex128, device="cuda")
    e128 = _energy(a, w, theta, H.C128, psi)
    assert abs(e64 - e128) < TOL[H.C64] * max(1.0, abs(e128))
    d = np.random.default_rng(8).standard_normal(a.P)
    d /= np.linalg.norm(d)
    h = 1e-4
    ep = _energy(a, w, theta + h * d, H.C128, psi)
    em = _energy(a, w, theta - h * d, H.C128, psi)
    fd = (ep - em) / (2 * h)
    # central difference error ~ h^2 |E'''| / 6 plus c128 rounding / h; c64 gradient relative 1e-6
    assert abs(float(g64 @ d) - fd) < 1e-5 * max(1.0, np.linalg.norm(g64))
    assert abs(float(g64c @ d) - fd) < 1e-5 * max(1.0, np.linalg.norm(g64c))


def test_32q_c128_gradient_on_row_clusters_against_dense_sweeps():
    """Workload 5 in complex128: the row engine stages each psi row and its
    lam row (2 x 206 KB) on a two-CTA cluster; its energy and gradient agree
    with the dense 2^32 sweeps' at the complex128 bound."""
    w, a, om = _setup(5)
    theta = w.theta()[0]
    assert a.workspace(1, H.C128, 1)[1] == 1          # the row engine takes the call
    a.state_prepare(H.PREP_SLATER, w.orbital_perturbation(), None, None, H.C128, 1)
    th = torch.tensor(theta[None, :], device="cuda")
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty((1, a.P), dtype=torch.float64, device="cuda")
    psi = H.workspace_tensor(a, 1, H.C128, 1)
    lam = H.workspace_tensor(a, 1, H.C128, 1)
    a.energy_grad(th, psi, lam, E, g, dtype=H.C128, batch=1)
    H.sync()
    e_rows, g_rows = float(E[0]), g.cpu().numpy()[0]
    del psi, lam
    torch.cuda.empty_cache()
    psi = torch.empty((1, 1 << w.n_qubits), dtype=torch.complex128, device="cuda")
    lam = torch.empty_like(psi)
    a.energy_grad(th, psi, lam, E, g, dtype=H.C128, batch=1, sweeps=True)
    H.sync()
    e_sw, g_sw = float(E[0]), g.cpu().numpy()[0]
    del psi, lam
    torch.cuda.empty_cache()
    assert abs(e_rows - e_sw) < TOL[H.C128] * max(1.0, abs(e_sw))
    assert np.max(np.abs(g_rows - g_sw)) < TOL[H.C128] * max(1.0, np.max(np.abs(g_sw)))
