"""The overlap loss of Eq. 5, the fidelity and the spin correlation C_ij
(Sec. 3) through the C ABI against the oracle.

The reference state stands in for the paper's DMRG wavefunction: the
oracle's Lanczos ground state at 12 qubits, and an oracle ansatz state at
other parameters at 24 qubits (a Lanczos vector there costs minutes on the
CPU).  F, f and df/dtheta are compared at the stated bounds (f and its
gradient relative to max(1, |.|)); C_ij element by element, on the ansatz
state the library leaves in psi and on the reference itself."""

import math

import numpy as np
import pytest

import oracle as O
import paper_2408_00836_gb300 as H
from paper_2408_00836_gb300 import workloads as W

from helpers import TOL, Problem, grad_err, log_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {H.C64: torch.complex64, H.C128: torch.complex128}
_CACHE = {}


def _case(name):
    if name in _CACHE:
        return _CACHE[name]
    if name in ("2x3", "2x2"):
        ny = 3 if name == "2x3" else 2
        rng = np.random.default_rng(61 if ny == 3 else 64)
        bonds, _ = H.square_lattice(2, ny)
        t = np.zeros((2 * ny, 2 * ny))
        for (i, j) in bonds:
            t[i, j] = t[j, i] = 1.0 + 0.1 * rng.standard_normal()
        prob = Problem(2, ny, t=t, U=np.full(2 * ny, 8.0), V=None, layers=3, classes=("U", "h1", "v1", "h2", "v2"))
        _, ref = O.lanczos_ground(prob.Hmat())
        thetas = rng.uniform(-1, 1, (2, prob.P))
    else:
        w = W.workload(6)
        bonds, _ = H.square_lattice(3, 4)
        t, U, _ = w.coefficients(bonds)
        prob = Problem(3, 4, t=t, U=U, V=None, layers=w.layers, classes=w.classes)
        ref = O.ansatz_state(prob.omodels[0], prob.basis, prob.ogroups, W.random_theta(62, 1, prob.P, 0.5)[0],
                             prob.psi0())
        thetas = W.random_theta(63, 2, prob.P, 0.5)
    refs = [ref, O.ansatz_state(prob.omodels[0], prob.basis, prob.ogroups, thetas[1] * 0.9, prob.psi0())]
    oracle = [[O.overlap_loss_and_gradient(prob.omodels[0], prob.basis, prob.ogroups, thetas[b], prob.psi0(), r)
               for b in range(2)] for r in refs]
    _CACHE[name] = (prob, thetas, refs, oracle)
    return _CACHE[name]


@pytest.mark.parametrize("fused,engine", [(True, "rows"), (True, "sweeps"), (False, "sweeps")])
@pytest.mark.parametrize("case", ["2x3", "3x4"])
@pytest.mark.parametrize("dtype", [H.C64, H.C128])
def test_overlap_loss_and_gradient_against_oracle(dtype, case, fused, engine):
    """F, f and df/dtheta against the oracle, on the row engine (a prepared
    state: the overlap and lam_K formed on the sector amplitudes) and on the
    dense sweeps (also from a caller-given state)."""
    prob, thetas, refs, oracle = _case(case)
    sweeps = engine == "sweeps"
    a = prob.ans
    batch = 2
    n = prob.n
    psi = torch.empty((batch, 1 << n), dtype=DT[dtype], device="cuda")
    lam = torch.empty_like(psi)
    th = torch.tensor(thetas, device="cuda")
    # one reference for both elements, then one per element
    for mode in ("shared", "per_element"):
        if mode == "shared":
            ref = torch.tensor(prob.full(refs[0])[None, :], dtype=DT[dtype], device="cuda")
            exp = [oracle[0][0], oracle[0][1]]
        else:
            ref = torch.tensor(np.stack([prob.full(refs[0]), prob.full(refs[1])]), dtype=DT[dtype], device="cuda")
            exp = [oracle[0][0], oracle[1][1]]
        if fused:
            a.state_prepare(H.PREP_SLATER, None, None, None, dtype, batch)
        else:
            a.state_prepare(H.PREP_SLATER, None, None, psi, dtype, batch)
        F = torch.empty(batch, dtype=torch.float64, device="cuda")
        f = torch.empty_like(F)
        g = torch.empty((batch, a.P), dtype=torch.float64, device="cuda")
        a.overlap_grad(th, ref, psi, lam, F, f, g, dtype=dtype, batch=batch, fused=fused, sweeps=sweeps)
        H.sync()
        Fv, fv, gv = F.cpu().numpy(), f.cpu().numpy(), g.cpu().numpy()
        for b in range(batch):
            Fo, fo, go = exp[b]
            log_errors(f"overlap_{case}_{mode}", dtype, engine, F=abs(Fv[b] - Fo), f=abs(fv[b] - fo) / max(1, abs(fo)),
                       grad=grad_err(gv[b], go))
            assert abs(Fv[b] - Fo) < TOL[dtype], (b, Fv[b], Fo)
            assert abs(fv[b] - fo) < TOL[dtype] * max(1.0, abs(fo))
            assert grad_err(gv[b], go) < TOL[dtype], (b, grad_err(gv[b], go))
        # fidelity only (no gradient, no lam)
        if fused:
            a.state_prepare(H.PREP_SLATER, None, None, None, dtype, batch)
        else:
            a.state_prepare(H.PREP_SLATER, None, None, psi, dtype, batch)
        F2 = torch.empty(batch, dtype=torch.float64, device="cuda")
        a.overlap_grad(th, ref, psi, None, F2, None, None, dtype=dtype, batch=batch, fused=fused, sweeps=sweeps)
        H.sync()
        assert np.max(np.abs(F2.cpu().numpy() - Fv)) < TOL[dtype]


@pytest.mark.parametrize("case", ["2x2", "2x3", "3x4"])
@pytest.mark.parametrize("dtype", [H.C64, H.C128])
def test_spin_correlation_against_oracle(dtype, case):
    """C_ij against the oracle: 8 qubits (runs of 2^8 amplitudes per
    thread), 12 and 24 qubits (runs of 2^10 per warp)."""
    prob, thetas, refs, _ = _case(case)
    a = prob.ans
    L, n = prob.L, prob.n
    om = prob.omodels[0]
    # the ansatz state left in psi by energy(..., keep_state)
    a.state_prepare(H.PREP_SLATER, None, None, None, dtype, 1)
    psi = torch.empty((1, 1 << n), dtype=DT[dtype], device="cuda")
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    a.energy(torch.tensor(thetas[:1], device="cuda"), psi, E, dtype=dtype, keep_state=True)
    C = torch.empty((1, L, L), dtype=torch.float64, device="cuda")
    a.spin_correlation(psi, C, dtype=dtype)
    H.sync()
    got = C.cpu().numpy()[0]
    ref = O.spin_correlation(om, prob.basis, O.ansatz_state(om, prob.basis, prob.ogroups, thetas[0], prob.psi0()))
    log_errors(f"spin_corr_{case}", dtype, "sweeps", C=float(np.max(np.abs(got - ref))))
    assert np.max(np.abs(got - ref)) < TOL[dtype]
    assert np.max(np.abs(got.sum(axis=1))) < 10 * TOL[dtype]      # S^z_total is fixed in the sector
    # the reference state itself, two batch elements
    st = torch.tensor(np.stack([prob.full(refs[0]), prob.full(refs[1])]), dtype=DT[dtype], device="cuda")
    C2 = torch.empty((2, L, L), dtype=torch.float64, device="cuda")
    a.spin_correlation(st, C2, dtype=dtype, batch=2)
    H.sync()
    for b in range(2):
        exp = O.spin_correlation(om, prob.basis, refs[b])
        assert np.max(np.abs(C2.cpu().numpy()[b] - exp)) < TOL[dtype]
