"""energy_noalloc: the energy call for callers that cannot allocate device
memory (their framework's allocator owns the free memory, or the call sits
on a path where an allocation would synchronise the device).  It
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


def _call_noalloc(a, theta, psi, E, dtype, batch, flags=H.FLAG_PREP_FUSED):
    s = torch.cuda.current_stream().cuda_stream
    return _lib.lib().energy_noalloc(a.handle, ctypes.c_void_p(theta.data_ptr()),
                                     ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(E.data_ptr()),
                                     dtype, batch, flags, ctypes.c_void_p(s))


# flags: the library prepares the state (sector sweeps); the caller gives
# psi from state_prepare (dense sweeps over all tiles); and the final state
# kept in psi (compared amplitude by amplitude as well)
FLAG_CASES = {"fused": H.FLAG_PREP_FUSED, "given_psi": 0,
              "fused_keep": H.FLAG_PREP_FUSED | H.FLAG_KEEP_STATE}


@pytest.mark.parametrize("case", list(FLAG_CASES))
@pytest.mark.parametrize("dtype", [H.C64, H.C128])
def test_energy_noalloc_matches_energy_twice(dtype, case):
    flags = FLAG_CASES[case]
    w, a = _ansatz(2)
    batch = w.batch
    td = torch.complex64 if dtype == H.C64 else torch.complex128
    theta = torch.tensor(w.theta(), device="cuda")
    psi = torch.empty((batch, 1 << 16), dtype=td, device="cuda")

    def fresh_psi():
        # psi is clobbered by every call: the caller-given state is rewritten
        a.state_prepare(H.PREP_SLATER, w.orbital_perturbation(), None,
                        None if flags & H.FLAG_PREP_FUSED else psi, dtype, batch)

    fresh_psi()
    E_ref = torch.empty(batch, dtype=torch.float64, device="cuda")
    a.energy(theta, psi, E_ref, dtype=dtype, batch=batch, fused=bool(flags & H.FLAG_PREP_FUSED),
             keep_state=bool(flags & H.FLAG_KEEP_STATE))
    H.sync()
    ref = E_ref.cpu().numpy()
    ref_psi = psi.cpu().numpy() if flags & H.FLAG_KEEP_STATE else None
    for _ in range(2):
        fresh_psi()
        if flags & H.FLAG_KEEP_STATE:
            psi.fill_(float("nan"))
        E = torch.full((batch,), float("nan"), dtype=torch.float64, device="cuda")
        _lib.check(_call_noalloc(a, theta, psi, E, dtype, batch, flags))
        H.sync()
        got = E.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) < TOL[dtype] * max(1.0, np.max(np.abs(ref)))
        if ref_psi is not None:
            st = psi.cpu().numpy()
            for b in range(batch):
                err = np.linalg.norm(st[b] - ref_psi[b]) / np.linalg.norm(ref_psi[b])
                assert err < TOL[dtype], (b, err)


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
