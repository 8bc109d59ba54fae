"""Sector tiles against the oracle and the dense path.

Every operation conserves the numbers of up and down electrons, so when the
initial state is generated by the library (fused preparation) the sweeps
visit only the tiles that meet the (N_up, N_dn) sector and the workspaces
are cleared first.  Checked here: workspaces filled with NaN before the call
do not reach the results; the dense path (a caller's own psi) is exact for a
state spread over all sectors; the plan's moved bytes shrink accordingly."""

import math

import numpy as np
import pytest

import oracle as O
import paper_2408_00836_gb300 as H
from paper_2408_00836_gb300 import workloads as W

from helpers import TOL, Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {H.C64: torch.complex64, H.C128: torch.complex128}


def _grid2x4():
    w = W.workload(2, batch_sets=1)
    bonds, _ = H.square_lattice(2, 4, "snake")
    t, U, _ = w.coefficients(bonds, 0)
    prob = Problem(2, 4, order="snake", t=t, U=U, V=None, layers=4, classes=w.classes,
                   perturb=w.orbital_perturbation())
    return prob, w.theta()[0]


@pytest.mark.parametrize("tile", [0, 8])
@pytest.mark.parametrize("dtype", [H.C128, H.C64])
def test_sector_tiles_ignore_nan_workspaces(dtype, tile):
    prob, theta = _grid2x4()
    a = prob.ans
    a.set_tile(dtype, tile)
    fused_bytes = a.plan_stats(1, dtype, fused=True)[1]
    dense_bytes = a.plan_stats(1, dtype, fused=False)[1]
    assert fused_bytes < dense_bytes
    a.state_prepare(H.PREP_SLATER, prob.perturb, None, None, dtype, 1)
    th = torch.tensor(theta[None, :], device="cuda")
    nan = complex(float("nan"), float("nan"))
    psi = torch.full((1, 1 << prob.n), nan, dtype=DT[dtype], device="cuda")
    lam = torch.full_like(psi, nan)
    ckpt = torch.full_like(psi, nan)
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty((1, a.P), dtype=torch.float64, device="cuda")
    Eo, go = prob.oracle_energy_grad(theta)
    # the checkpoint is kept by the dense sweeps only: force them for it
    for ck in (None, ckpt):
        a.energy_grad(th, psi, lam, E, g, ckpt=ck, dtype=dtype, sweeps=ck is not None)
        H.sync()
        assert abs(E.item() - Eo) < TOL[dtype] * max(1.0, abs(Eo))
        assert np.max(np.abs(g.cpu().numpy()[0] - go)) < TOL[dtype] * max(1.0, np.max(np.abs(go)))
        psi.fill_(nan)
        lam.fill_(nan)
    a.energy(th, psi, E, dtype=dtype, keep_state=True)
    H.sync()
    assert abs(E.item() - Eo) < TOL[dtype] * max(1.0, abs(Eo))
    st = psi.cpu().numpy()[0]
    ref = prob.full(prob.oracle_state(theta))
    assert np.all(st[ref == 0] == 0)        # outside the sector: cleared, not NaN
    a.set_tile(dtype, 0)


@pytest.mark.parametrize("dtype", [H.C128, H.C64])
def test_dense_path_state_over_all_sectors(dtype):
    rng = np.random.default_rng(31)
    bonds, _ = H.square_lattice(2, 3)
    t = np.zeros((6, 6))
    for (i, j) in bonds:
        t[i, j] = t[j, i] = 1.0 + 0.3 * rng.standard_normal()
    U = 3.0 * (1 + 0.2 * rng.standard_normal(6))
    prob = Problem(2, 3, t=t, U=U, V=None, layers=2, classes=("U", "h1", "v1", "h2", "v2"))
    a = prob.ans
    a.set_tile(dtype, 8)                     # 16 tiles
    om = prob.omodels[0]
    fb = O.full_basis(om)
    Hf = O.hamiltonian(om, fb)
    v = rng.standard_normal(len(fb)) + 1j * rng.standard_normal(len(fb))
    v /= np.linalg.norm(v)
    theta = rng.uniform(-math.pi, math.pi, prob.P)
    Eo, go = O.energy_and_gradient(om, fb, prob.ogroups, theta, v, Hf)
    th = torch.tensor(theta[None, :], device="cuda")
    psi = torch.tensor(v[None, :], dtype=DT[dtype], device="cuda")
    lam = torch.empty_like(psi)
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty((1, a.P), dtype=torch.float64, device="cuda")
    a.energy_grad(th, psi, lam, E, g, dtype=dtype, fused=False)
    H.sync()
    assert abs(E.item() - Eo) < TOL[dtype] * max(1.0, abs(Eo))
    assert np.max(np.abs(g.cpu().numpy()[0] - go)) < TOL[dtype] * max(1.0, np.max(np.abs(go)))
    psi = torch.tensor(v[None, :], dtype=DT[dtype], device="cuda")
    a.energy(th, psi, E, dtype=dtype, fused=False)
    H.sync()
    assert abs(E.item() - Eo) < TOL[dtype] * max(1.0, abs(Eo))
    a.set_tile(dtype, 0)


@pytest.mark.parametrize("dtype", [H.C64, H.C128])
def test_sector_sized_workspaces(dtype):
    """ans_workspace_bytes: the row engine needs only the sector matrix and
    its transpose (24 qubits: 2 x 853 776 amplitudes instead of 2^24), the
    on-chip engine none; calls on buffers of exactly that size give the
    oracle's energy and gradient."""
    w = W.workload(6)
    bonds, _ = H.square_lattice(3, 4)
    t, U, _ = w.coefficients(bonds)
    prob = Problem(3, 4, t=t, U=U, V=None, layers=w.layers, classes=w.classes)
    a = prob.ans
    nb, eng = a.workspace(1, dtype, 1)
    amp = 8 if dtype == H.C64 else 16
    assert eng == 1 and nb == 2 * 924 * 924 * amp
    assert a.workspace(1, dtype, 1, sweeps=True) == ((1 << 24) * amp, 2)
    theta = w.theta()[0]
    a.state_prepare(H.PREP_SLATER, None, None, None, dtype, 1)
    psi = H.workspace_tensor(a, 1, dtype, 1)
    lam = H.workspace_tensor(a, 1, dtype, 1)
    assert psi.numel() * psi.element_size() == nb
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty((1, a.P), dtype=torch.float64, device="cuda")
    a.energy_grad(torch.tensor(theta[None, :], device="cuda"), psi, lam, E, g, dtype=dtype)
    H.sync()
    Eo, go = prob.oracle_energy_grad(theta)
    assert abs(E.item() - Eo) < TOL[dtype] * max(1.0, abs(Eo))
    assert np.max(np.abs(g.cpu().numpy()[0] - go)) < TOL[dtype] * max(1.0, np.max(np.abs(go)))
    # on chip: no workspace at all (a one-element buffer is passed)
    p2, _ = _grid2x4()
    assert p2.ans.workspace(1, dtype, 4)[1] == 0 and p2.ans.workspace(1, dtype, 4)[0] == 0
