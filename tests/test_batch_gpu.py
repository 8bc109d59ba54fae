"""The batched workload at its full size, and the autograd face.

* The 16-qubit workload of 1024 seeded parameter sets x 4 U values (4096
  states in one launch): far more states than the on-chip engine's grid
  (a few CTAs per SM), so each CTA's loop over states runs many times and
  must restart its accumulators and coefficients for every new state.  A
  seeded sample of the states is checked against the oracle, state by
  state, on the on-chip and the row engine.
* energy_fn: the torch.autograd.Function whose backward is the adjoint
  gradient of Sec. 2.1; torch.autograd.grad of a scalar loss of the
  energies against the oracle's gradient by the chain rule."""

import math

import numpy as np
import pytest

import paper_2408_00836_gb300 as H
from paper_2408_00836_gb300 import workloads as W

from helpers import TOL, Problem, energy_err, grad_err, log_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {H.C64: torch.complex64, H.C128: torch.complex128}
_W2 = {}


def _workload2():
    if not _W2:
        w = W.workload(2)
        bonds, _ = H.square_lattice(2, 4, "snake")
        inst = [(t, U, None) for (t, U, V) in (w.coefficients(bonds, r) for r in range(4))]
        prob = Problem(2, 4, order="snake", layers=4, classes=w.classes, perturb=w.orbital_perturbation(),
                       instances=inst)
        _W2["v"] = (w, prob)
    return _W2["v"]


@pytest.mark.parametrize("engine", ["auto", "rows"])
@pytest.mark.parametrize("dtype", [H.C64, H.C128])
def test_full_4096_state_batch_sampled_against_oracle(dtype, engine):
    w, prob = _workload2()
    a = prob.ans
    batch = w.batch
    assert batch == 4096
    a.state_prepare(H.PREP_SLATER, prob.perturb, None, None, dtype, batch)
    theta = w.theta()
    th = torch.tensor(theta, device="cuda")
    psi = torch.empty((batch, 1 << prob.n), dtype=DT[dtype], device="cuda")
    lam = torch.empty_like(psi)
    E = torch.full((batch,), float("nan"), dtype=torch.float64, device="cuda")
    g = torch.full((batch, a.P), float("nan"), dtype=torch.float64, device="cuda")
    a.energy_grad(th, psi, lam, E, g, dtype=dtype, batch=batch, rows=engine == "rows")
    H.sync()
    E = E.cpu().numpy()
    g = g.cpu().numpy()
    assert np.all(np.isfinite(E)) and np.all(np.isfinite(g))
    # the first and last states, and a seeded sample across the batch
    sample = sorted({0, 1, batch - 1} | set(np.random.default_rng(17).choice(batch, 32, replace=False).tolist()))
    for b in sample:
        Eo, go = prob.oracle_energy_grad(theta[b], r=b % 4)
        log_errors(f"grid2x4_4096[{b}]", dtype, engine, energy=energy_err(E[b], Eo), grad=grad_err(g[b], go))
        assert abs(E[b] - Eo) < TOL[dtype] * max(1.0, abs(Eo)), b
        assert grad_err(g[b], go) < TOL[dtype], (b, grad_err(g[b], go))
    # the energy-only call over the same batch
    E2 = torch.empty(batch, dtype=torch.float64, device="cuda")
    a.energy(th, psi, E2, dtype=dtype, batch=batch, rows=engine == "rows")
    H.sync()
    assert np.max(np.abs(E2.cpu().numpy() - E)) < TOL[dtype] * max(1.0, np.max(np.abs(E)))


@pytest.mark.parametrize("dtype", [H.C64, H.C128])
def test_energy_fn_autograd_matches_oracle_gradient(dtype):
    rng = np.random.default_rng(41)
    bonds, _ = H.square_lattice(2, 3)
    t = np.zeros((6, 6))
    for (i, j) in bonds:
        t[i, j] = t[j, i] = 1.0 + 0.1 * rng.standard_normal()
    prob = Problem(2, 3, t=t, U=np.full(6, 4.0), V=None, layers=2, classes=("U", "h1", "v1", "h2"))
    a = prob.ans
    batch = 3
    a.state_prepare(H.PREP_SLATER, None, None, None, dtype, batch)
    theta = rng.uniform(-math.pi, math.pi, (batch, prob.P))
    th = torch.tensor(theta, device="cuda", requires_grad=True)
    psi = torch.empty((batch, 1 << prob.n), dtype=DT[dtype], device="cuda")
    lam = torch.empty_like(psi)
    E = H.energy_fn(a, th, psi, lam, dtype=dtype, batch=batch)
    w = torch.tensor([0.5, -1.0, 2.0], dtype=torch.float64, device="cuda")
    loss = (w * E).sum() + (E ** 2).sum()
    (gt,) = torch.autograd.grad(loss, th)
    gt = gt.cpu().numpy()
    Ev = E.detach().cpu().numpy()
    for b in range(batch):
        Eo, go = prob.oracle_energy_grad(theta[b])
        assert abs(Ev[b] - Eo) < TOL[dtype] * max(1.0, abs(Eo))
        ref = (float(w[b]) + 2.0 * Eo) * go          # dL/dtheta_b = (w_b + 2 E_b) dE_b/dtheta_b
        scale = abs(float(w[b]) + 2.0 * Eo)
        assert np.max(np.abs(gt[b] - ref)) < TOL[dtype] * scale * max(1.0, np.max(np.abs(go))), b


def test_engine_autotuner_and_graph_captured_batch():
    """The engine autotuner on the 4096-state batch times the library's
    choice, the on-chip and row engines at each CTA size and the dense
    sweeps, and leaves a valid choice;
    the whole batched evaluation captured in a CUDA graph and replayed
    gives the direct call's results."""
    from paper_2408_00836_gb300.autotune import autotune_engine
    from paper_2408_00836_gb300.vqe import EnergyGradGraph
    w, prob = _workload2()
    a = prob.ans
    batch = w.batch
    a.state_prepare(H.PREP_SLATER, prob.perturb, None, None, H.C64, batch)
    best, times = autotune_engine(a, H.C64, batch=batch, which=1, theta=w.theta(), tiles=(12,), reps=1,
                                  warmup=1)
    assert {"auto", "onchip_t256", "onchip_t512", "rows_t256", "rows_t512", "sweeps_tile12"} <= set(times)
    assert best["name"] == min(times, key=times.get)
    assert best["engine"] in ("on-chip", "rows", "sweeps")
    a.set_tile(H.C64, 0)
    a.set_threads(H.C64, H.ENGINE_ONCHIP, 0)
    a.set_threads(H.C64, H.ENGINE_ROWS, 0)
    fn = EnergyGradGraph(a, dtype=H.C64, batch=batch, use_graph=True, sweeps=best["sweeps"], rows=best["rows"])
    direct = EnergyGradGraph(a, dtype=H.C64, batch=batch, use_graph=False, sweeps=best["sweeps"],
                             rows=best["rows"])
    theta = w.theta()
    E, g = fn(theta)
    Ed, gd = direct(theta)
    assert np.max(np.abs(E - Ed)) < 1e-12 * max(1.0, np.max(np.abs(Ed)))
    assert np.max(np.abs(g - gd)) < 1e-12 * max(1.0, np.max(np.abs(gd)))
    for b in (0, 2047, 4095):
        Eo, go = prob.oracle_energy_grad(theta[b], r=b % 4)
        assert abs(E[b] - Eo) < TOL[H.C64] * max(1.0, abs(Eo))
        assert grad_err(g[b], go) < TOL[H.C64]
