"""energy_noalloc: the energy call for callers that cannot allocate device
memory (their framework's allocator owns the free memory, or the call sits
on a path where an allocation would synchronise or cannot be recorded).  It
keeps every table and its scratch in a fixed static device array instead of
allocating.  This file is collected last on purpose.

The test calls it through the C ABI twice in a row (the second call reuses
the array the first one filled) and checks both results against energy(),
within the parity tolerances of the other GPU tests, and checks that a
problem too large for the array is refused before anything runs."""

import ctypes

import numpy as np
import pytest

import paper_2408_00836_gb300 as H
from paper_2408_00836_gb300 import _lib
from paper_2408_00836_gb300 import workloads as W

from helpers import TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ansatz(batch_sets):
    w = W.workload(2, batch_sets=batch_sets)
    bonds, cls = H.square_lattice(2, 4, "snake")
    models = [H.Model(8, bonds, *w.coefficients(bonds, r)[:2], None, 4, 4) for r in range(4)]
    a = H.Ansatz(models, H.hva_groups(bonds, cls, 8, w.layers, w.classes), w.layers)
    return w, a


def _call_noalloc(a, theta, psi, E, dtype, batch):
    s = torch.cuda.current_stream().cuda_stream
    return _lib.lib().energy_noalloc(a.handle, ctypes.c_void_p(theta.data_ptr()),
                                     ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(E.data_ptr()),
                                     dtype, batch, H.FLAG_PREP_FUSED, ctypes.c_void_p(s))


@pytest.mark.parametrize("dtype", [H.C64, H.C128])
def test_energy_noalloc_matches_energy_twice(dtype):
    w, a = _ansatz(2)
    batch = w.batch
    a.state_prepare(H.PREP_SLATER, w.orbital_perturbation(), None, None, dtype, batch)
    td = torch.complex64 if dtype == H.C64 else torch.complex128
    theta = torch.tensor(w.theta(), device="cuda")
    psi = torch.empty((batch, 1 << 16), dtype=td, device="cuda")
    E_ref = torch.empty(batch, dtype=torch.float64, device="cuda")
    a.energy(theta, psi, E_ref, dtype=dtype, batch=batch)
    H.sync()
    ref = E_ref.cpu().numpy()
    for _ in range(2):
        E = torch.full((batch,), float("nan"), dtype=torch.float64, device="cuda")
        _lib.check(_call_noalloc(a, theta, psi, E, dtype, batch))
        H.sync()
        got = E.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) < TOL[dtype] * max(1.0, np.max(np.abs(ref)))


def test_energy_noalloc_refuses_problems_beyond_the_array():
    w, a = _ansatz(1024)          # 4096 states: tables far beyond the array
    batch = w.batch
    a.state_prepare(H.PREP_SLATER, w.orbital_perturbation(), None, None, H.C64, 4)
    theta = torch.zeros((batch, a.P), dtype=torch.float64, device="cuda")
    psi = torch.empty((1, 2), dtype=torch.complex64, device="cuda")   # never touched
    E = torch.empty(batch, dtype=torch.float64, device="cuda")
    st = _call_noalloc(a, theta, psi, E, H.C64, batch)
    assert st == _lib.HUB_EINVAL
    assert "bytes of scratch" in _lib.lib().hub_last_error().decode()
