"""The checkpointed adjoint pass on the dense sweeps (Sec. 2.1's backward
recursion with psi reloaded at the middle layer boundary instead of
un-computed through the second half of the circuit).

energy_grad with a checkpoint buffer runs this plan on the dense-sweep
engine (HUB_FLAG_SWEEPS; the sector engines keep no checkpoint).  Checked
against the oracle: the energy and gradient at the stated bounds, and the
buffer's contents after the call -- psi after the first half of the layers,
amplitude by amplitude -- which shows that the checkpoint was written and is
the state the backward pass reloaded.  Both a generated (sector) start and
a caller-given state (all tiles, no clearing of the buffer) are covered, at
16 and 24 qubits, in complex64 and complex128."""

import numpy as np
import pytest

import oracle as O
import paper_2408_00836_gb300 as H
from paper_2408_00836_gb300 import workloads as W

from helpers import TOL, Problem, energy_err, grad_err, log_errors, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {H.C64: torch.complex64, H.C128: torch.complex128}
_CACHE = {}


def _problem(number):
    if number not in _CACHE:
        w = W.workload(number, batch_sets=1)
        bonds, _ = H.square_lattice(w.nx, w.ny, w.order)
        t, U, V = w.coefficients(bonds, 0)
        prob = Problem(w.nx, w.ny, order=w.order, t=t, U=U, V=V if w.V else None, layers=w.layers,
                       classes=w.classes, perturb=w.orbital_perturbation())
        theta = w.theta()[0]
        half = (w.layers // 2) * len(w.classes)
        mid = O.ansatz_state(prob.omodels[0], prob.basis, prob.ogroups[:half], theta, prob.psi0())
        _CACHE[number] = (prob, theta, prob.oracle_energy_grad(theta), prob.full(mid))
    return _CACHE[number]


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("number", [2, 6])
@pytest.mark.parametrize("dtype", [H.C64, H.C128])
def test_checkpointed_sweeps_gradient_and_buffer(dtype, number, fused):
    prob, theta, (Eo, go), mid = _problem(number)
    a = prob.ans
    n = prob.n
    psi = torch.empty((1, 1 << n), dtype=DT[dtype], device="cuda")
    a.state_prepare(H.PREP_SLATER, prob.perturb, None, None if fused else psi, dtype, 1)
    lam = torch.empty_like(psi)
    nan = complex(float("nan"), float("nan"))
    ck = torch.full_like(psi, nan)
    th = torch.tensor(theta[None, :], device="cuda")
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty((1, a.P), dtype=torch.float64, device="cuda")
    a.energy_grad(th, psi, lam, E, g, ckpt=ck, dtype=dtype, fused=fused, sweeps=True)
    H.sync()
    e, gg = float(E[0]), g.cpu().numpy()[0]
    tag = f"checkpoint_w{number}_{'fused' if fused else 'given'}"
    log_errors(tag, dtype, "sweeps+ckpt", energy=energy_err(e, Eo), grad=grad_err(gg, go))
    assert abs(e - Eo) < TOL[dtype] * max(1.0, abs(Eo))
    assert grad_err(gg, go) < TOL[dtype], grad_err(gg, go)
    st = ck.cpu().numpy()[0]
    assert np.all(np.isfinite(st))          # every amplitude written (or cleared)
    assert rel_err(st, mid) < TOL[dtype]
    # without a checkpoint: the same plan minus the reload agrees as well
    if not fused:
        a.state_prepare(H.PREP_SLATER, prob.perturb, None, psi, dtype, 1)
    a.energy_grad(th, psi, lam, E, g, dtype=dtype, fused=fused, sweeps=True)
    H.sync()
    assert grad_err(g.cpu().numpy()[0], go) < TOL[dtype]
