"""Host-side checks of the C ABI that need no GPU: the library loads and
exports every declared entry point, the lattice helper agrees with the
oracle's geometry, argument validation, and the planner's schedules are
valid reorderings of the operation sequence."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2408_00836_gb300 as H
from paper_2408_00836_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    with open(os.path.join(ROOT, "include", "hubsv.h")) as f:
        hdr = f.read()
    declared = set(re.findall(r"^HUB_API\s+[\w\s\*]+?\b(\w+)\s*\(", hdr, flags=re.M))
    assert len(declared) >= 17
    L = _lib.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert declared == set(_lib.EXPORTS)


@pytest.mark.parametrize("nx,ny,order", [(1, 4, "rowmajor"), (2, 4, "snake"), (3, 4, "rowmajor"),
                                         (2, 7, "rowmajor"), (4, 4, "rowmajor"), (4, 4, "snake")])
def test_lattice_matches_oracle(nx, ny, order):
    bonds, cls = H.square_lattice(nx, ny, order)
    lat = O.square_lattice(nx, ny, order)
    assert bonds == lat.bonds
    assert cls == lat.bond_class


def _model(nx=2, ny=3, **kw):
    bonds, cls = H.square_lattice(nx, ny)
    L = nx * ny
    t = np.zeros((L, L))
    for (i, j) in bonds:
        t[i, j] = t[j, i] = 1.0
    return bonds, cls, t


def test_model_validation():
    bonds, cls, t = _model()
    H.Model(6, bonds, t, np.full(6, 4.0), None, 3, 3)
    bad = t.copy()
    bad[0, 1] = 2.0  # not symmetric
    with pytest.raises(H.HubError) as e:
        H.Model(6, bonds, bad, None, None, 3, 3)
    assert e.value.status == _lib.HUB_EINVAL
    bad = t.copy()
    bad[0, 5] = bad[5, 0] = 1.0  # hop off the bond list
    with pytest.raises(H.HubError):
        H.Model(6, bonds, bad, None, None, 3, 3)
    with pytest.raises(H.HubError):
        H.Model(6, bonds + [(0, 1)], t, None, None, 3, 3)  # repeated bond
    with pytest.raises(H.HubError):
        H.Model(6, bonds, t, None, None, 7, 3)  # too many particles
    with pytest.raises(H.HubError) as e:
        H.Model(6, bonds, t, None, None, 3, 3, modes=(np.arange(6), np.arange(6) + 5))
    assert e.value.status == _lib.HUB_EINVAL
    with pytest.raises(H.HubError) as e:  # a valid but unsupported permutation
        H.Model(6, bonds, t, None, None, 3, 3, modes=(np.arange(6)[::-1].copy(), np.arange(6) + 6))
    assert e.value.status == _lib.HUB_EUNSUPPORTED


def test_ansatz_validation():
    bonds, cls, t = _model()
    m = H.Model(6, bonds, t, np.full(6, 4.0), None, 3, 3)
    with pytest.raises(H.HubError):   # two bonds sharing a site in one hop group
        H.Ansatz(m, [(H.HOP, [0, 1], 0)])
    with pytest.raises(H.HubError):
        H.Ansatz(m, [(H.HOP, [99], 0)])
    with pytest.raises(H.HubError):
        H.Ansatz(m, [(H.ONSITE, [0], -1)])
    a = H.Ansatz(m, [(H.HOP, [0], 0), (H.ONSITE, list(range(6)), 3)])
    assert a.P == 4 and a.n == 12


# ---------------------------------------------------------------------------
# schedule validity
# ---------------------------------------------------------------------------

def _sequence(a_groups, bonds, L, which):
    """The operation sequence the planner receives (see ans_plan_describe):
    entries (kind, modes, diagonal, cls) with blocked modes."""
    up = lambda i: i
    dn = lambda i: L + i
    seq = []
    for (kind, terms, p) in a_groups:
        if kind == H.HOP:
            for b in terms:
                i, j = bonds[b]
                for m in (up, dn):
                    seq.append(("giv", {m(i), m(j)}, False, 0))
        else:
            if kind == H.ONSITE:
                sup = {up(i) for i in terms} | {dn(i) for i in terms}
            elif kind == H.NN_V:
                sup = set()
                for b in terms:
                    for s in bonds[b]:
                        sup |= {up(s), dn(s)}
            else:
                sup = set(range(2 * L))
            seq.append(("diag", sup, True, 0))
    fwd = list(seq)
    cls = 1 if which == 0 else 2
    for (i, j) in bonds:
        for m in (up, dn):
            seq.append(("h", {m(i), m(j)}, False, cls))
    seq.append(("hdiag", None, True, cls))   # support: every mode with a coefficient
    if which == 1:
        for op in reversed(fwd):
            seq.append(("grad",) + op[1:3] + (3,))
            seq.append(("inv",) + op[1:3] + (3,))
    return seq


def _check_schedule(plan, seq, n, k, c, all_modes):
    seen = []
    for tile, flags, ids in plan:
        assert bin(tile).count("1") == k
        assert tile & ((1 << c) - 1) == (1 << c) - 1, "coalescing bits missing"
        for i in ids:
            op = seq[i]
            if not op[2]:
                for m in op[1]:
                    assert tile >> m & 1, "operation outside its tile"
        seen.extend(ids)
    assert sorted(seen) == list(range(len(seq))), "every operation exactly once"
    pos = {idx: r for r, idx in enumerate(seen)}
    sup = [all_modes if op[1] is None else op[1] for op in seq]
    for a in range(len(seq)):
        for b in range(a + 1, len(seq)):
            commute = (seq[a][2] and seq[b][2]) or not (sup[a] & sup[b])
            if not commute:
                assert pos[a] < pos[b], f"order of non-commuting ops {a} {b} broken"
    # lam-building steps never precede a forward factor
    last_fwd = max((pos[i] for i, op in enumerate(seq) if op[3] == 0), default=-1)
    for i, op in enumerate(seq):
        if op[3] == 2:
            assert pos[i] > last_fwd


@pytest.mark.parametrize("number", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("which", [0, 1])
def test_schedules_are_valid(number, which):
    w = H.workloads.workload(number, batch_sets=1)
    bonds, cls = H.square_lattice(w.nx, w.ny, w.order)
    t, U, V = w.coefficients(bonds)
    m = H.Model(w.n_sites, bonds, t, U, V if w.V else None, w.n_up, w.n_dn)
    groups = H.hva_groups(bonds, cls, w.n_sites, w.layers, w.classes)
    a = H.Ansatz(m, groups, w.layers)
    seq = _sequence(groups, bonds, w.n_sites, which)
    # default tiles and runs: c64 2^12 amplitudes (2^13 from 28 qubits),
    # runs of 8 (c = 3); c128 2^10 amplitudes, runs of 2 (c = 1)
    for dtype, k, c in [(H.C64, 13 if w.n_qubits >= 28 else 12, 3), (H.C128, 10, 1)]:
        k = min(k, w.n_qubits)
        plan = a.plan_describe(which, dtype)
        _check_schedule(plan, seq, w.n_qubits, k, min(c, k), set(range(w.n_qubits)))
    for kk in (10, 14):
        a.set_tile(H.C64, kk)
        plan = a.plan_describe(which, H.C64)
        # the planner caps c64 tiles at 13 bits (512 threads x 16 amplitudes)
        k_eff = min(kk, 13, w.n_qubits)
        _check_schedule(plan, seq, w.n_qubits, k_eff, min(3, k_eff), set(range(w.n_qubits)))
    a.set_tile(H.C64, 0)
    for runs in (2, 3, 5):
        a.set_runs(H.C64, runs)
        plan = a.plan_describe(which, H.C64)
        k_eff = min(13 if w.n_qubits >= 28 else 12, w.n_qubits)
        _check_schedule(plan, seq, w.n_qubits, k_eff, min(runs, k_eff), set(range(w.n_qubits)))


@pytest.mark.parametrize("number", [2, 4, 5])
def test_sector_plan_bytes(number):
    """With a generated initial state the sweeps visit only tiles whose
    non-tile bits can still hold N_up up and N_dn down electrons; the plan's
    byte count is the count of such tiles times the tile bytes, per sweep."""
    from math import comb
    w = H.workloads.workload(number, batch_sets=1)
    bonds, cls = H.square_lattice(w.nx, w.ny, w.order)
    t, U, V = w.coefficients(bonds)
    m = H.Model(w.n_sites, bonds, t, U, V if w.V else None, w.n_up, w.n_dn)
    a = H.Ansatz(m, H.hva_groups(bonds, cls, w.n_sites, w.layers, w.classes), w.layers)
    L, n = w.n_sites, w.n_qubits
    upm, dnm = (1 << L) - 1, ((1 << L) - 1) << L

    def live(tile, N, mask):
        in_tile = bin(tile & mask).count("1")
        free = L - in_tile
        return sum(comb(free, e) for e in range(max(0, N - in_tile), min(N, free) + 1))

    for dtype, amp in ((H.C64, 8), (H.C128, 16)):
        plan = a.plan_describe(1, dtype)
        k = bin(plan[0][0]).count("1")
        expect = 0
        for tile, flags, _ in plan:
            f = flags & 0xFFFF
            nvec = sum(1 for bit in (2, 4, 16, 32, 64) if f & bit)
            expect += nvec * live(tile, w.n_up, upm) * live(tile, w.n_dn, dnm) * (1 << k) * amp
        assert a.plan_stats(1, dtype, fused=True)[1] == expect
        dense = a.plan_stats(1, dtype, fused=False)[1]
        assert dense == sum(sum(1 for bit in (2, 4, 16, 32, 64) if (fl & 0xFFFF) & bit)
                            for _, fl, _ in a.plan_describe(1, dtype, flags=0)) * (1 << n) * amp


def test_plan_queries_ignore_the_engine_flag():
    """HUB_FLAG_SWEEPS picks the engine; the dense-sweep plan that energy and
    energy_grad run (without a checkpoint) is the same with or without it,
    and plan_stats / plan_describe report that plan."""
    w = H.workloads.workload(4, batch_sets=1)
    bonds, cls = H.square_lattice(w.nx, w.ny, w.order)
    t, U, V = w.coefficients(bonds)
    m = H.Model(w.n_sites, bonds, t, U, None, w.n_up, w.n_dn)
    a = H.Ansatz(m, H.hva_groups(bonds, cls, w.n_sites, w.layers, w.classes), w.layers)
    for which in (0, 1):
        for dtype in (H.C64, H.C128):
            base = a.plan_describe(which, dtype, flags=H.FLAG_PREP_FUSED)
            assert a.plan_describe(which, dtype, flags=H.FLAG_PREP_FUSED | H.FLAG_SWEEPS) == base
            ns = ctypes.c_int32(0)
            by = ctypes.c_double(0.0)
            H.check(H.lib().ans_plan_stats(a.handle, which, dtype, H.FLAG_PREP_FUSED | H.FLAG_SWEEPS,
                                           ctypes.byref(ns), ctypes.byref(by)))
            assert (ns.value, by.value) == a.plan_stats(which, dtype, fused=True)
            assert ns.value == len(base)


@pytest.mark.parametrize("number", [2, 4, 5])
def test_row_plan_bytes(number):
    """The row engine moves whole sector matrices: its bytes per state are a
    whole number of C(L, N_up) C(L, N_dn) amplitude matrices (row sweeps and
    transposes), far fewer than the dense sweeps move."""
    from math import comb
    w = H.workloads.workload(number, batch_sets=1)
    bonds, cls = H.square_lattice(w.nx, w.ny, w.order)
    t, U, V = w.coefficients(bonds)
    m = H.Model(w.n_sites, bonds, t, U, V if w.V else None, w.n_up, w.n_dn)
    a = H.Ansatz(m, H.hva_groups(bonds, cls, w.n_sites, w.layers, w.classes), w.layers)
    C = comb(w.n_sites, w.n_up) * comb(w.n_sites, w.n_dn)
    for which in (0, 1):
        for dtype, amp in ((H.C64, 8), (H.C128, 16)):
            launches, by = a.plan_stats(which, dtype, rows=True)
            units = by / (C * amp)
            assert launches >= 1 and abs(units - round(units)) < 1e-9 and round(units) >= 1
            if w.n_qubits >= 28:
                assert by < a.plan_stats(which, dtype)[1] / 10


@pytest.mark.parametrize("number", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("which", [0, 1])
def test_row_schedules_are_valid(number, which):
    """The row engine's regrouped sequence: every operation once, hops inside
    the spin of their segment, and no two non-commuting operations swapped."""
    w = H.workloads.workload(number, batch_sets=1)
    bonds, cls = H.square_lattice(w.nx, w.ny, w.order)
    t, U, V = w.coefficients(bonds)
    m = H.Model(w.n_sites, bonds, t, U, V if w.V else None, w.n_up, w.n_dn)
    groups = H.hva_groups(bonds, cls, w.n_sites, w.layers, w.classes)
    a = H.Ansatz(m, groups, w.layers)
    seq = _sequence(groups, bonds, w.n_sites, which)
    plan = a.plan_describe(which, H.C64, flags=H.FLAG_PREP_FUSED | H.FLAG_ROWS)
    L = w.n_sites
    for tile, orient, ids in plan:
        assert tile == (((1 << L) - 1) << (L if orient else 0))
    _check_schedule(plan, seq, w.n_qubits, L, 0, set(range(w.n_qubits)))
    # consecutive segments alternate spins (a repeat would be one segment)
    for (_, o1, _), (_, o2, _) in zip(plan, plan[1:]):
        assert o1 != o2


def test_np_ansatz_4x4_12_layers_builds_and_plans():
    """The paper's 4x4 NP ansatz with 12 layers: 1,568 parameters (Sec. 3),
    spin mixing routes it to the dense sweeps, and the sweep planner gives
    every sweep its own small set of accumulator slots."""
    import time
    bonds, cls = H.square_lattice(4, 4)
    t = np.zeros((16, 16))
    for (i, j) in bonds:
        t[i, j] = t[j, i] = 1.0
    m = H.Model(16, bonds, t, np.full(16, 2.0), None, 8, 8, modes="interleaved")
    a = H.Ansatz(m, H.np_groups(bonds, cls, 16, 12, modes="interleaved"), 1)
    assert a.P == 1568
    t0 = time.time()
    ns, by = a.plan_stats(1, H.C64, fused=True)
    assert ns > 0 and by > 0
    assert time.time() - t0 < 60
    # EP: 4 Nx Ny + 2 (2 Nx Ny - 1) l
    e = H.Ansatz(m, H.ep_groups(32, 3), 1)
    assert e.P == 4 * 16 + 2 * 31 * 3


def test_cta_size_override_arguments():
    """ans_set_threads accepts 0 (automatic) and the instantiated CTA sizes
    of each sector engine, and refuses anything else (no GPU needed)."""
    bonds, cls, t = _model()
    m = H.Model(6, bonds, t, np.full(6, 4.0), None, 3, 3)
    a = H.Ansatz([m], H.hva_groups(bonds, cls, 6, 1, ["U", "h1"]), 1)
    for dtype in (H.C64, H.C128):
        for th in (0, 256, 512):
            a.set_threads(dtype, H.ENGINE_ONCHIP, th)
        for th in (0, 256, 512, 1024):
            a.set_threads(dtype, H.ENGINE_ROWS, th)
    for engine, th in [(H.ENGINE_ONCHIP, 1024), (H.ENGINE_ONCHIP, 128), (H.ENGINE_ROWS, 300), (H.ENGINE_ROWS, -1),
                       (2, 256)]:
        with pytest.raises(H.HubError) as e:
            a.set_threads(H.C64, engine, th)
        assert e.value.status == _lib.HUB_EINVAL
    with pytest.raises(H.HubError) as e:
        a.set_threads(7, H.ENGINE_ROWS, 256)
    assert e.value.status == _lib.HUB_EINVAL


def test_misaligned_amplitude_buffers_are_refused():
    """Every call that takes amplitude buffers refuses one that is not
    aligned to its element size (8 bytes for complex64, 16 for complex128)
    with HUB_EINVAL, before it launches or dereferences anything (the
    pointers below are never read; no GPU needed)."""
    bonds, cls, t = _model()
    m = H.Model(6, bonds, t, np.full(6, 4.0), None, 3, 3)
    a = H.Ansatz([m], H.hva_groups(bonds, cls, 6, 1, ["U", "h1"]), 1)
    L = _lib.lib()
    ok = ctypes.c_void_p(1 << 20)   # stands in for the other (valid) buffers
    for dtype, off in ((H.C64, 4), (H.C128, 8)):
        bad = ctypes.c_void_p((1 << 20) + off)
        calls = {
            "state_prepare": lambda: L.state_prepare(a._h, 0, None, None, bad, dtype, 1, None),
            "energy": lambda: L.energy(a._h, ok, bad, ok, dtype, 1, 0, None),
            "energy_noalloc": lambda: L.energy_noalloc(a._h, ok, bad, ok, dtype, 1, 0, None),
            "energy_grad psi": lambda: L.energy_grad(a._h, ok, bad, ok, None, ok, ok, dtype, 1, 0, None),
            "energy_grad lam": lambda: L.energy_grad(a._h, ok, ok, bad, None, ok, ok, dtype, 1, 0, None),
            "energy_grad ckpt": lambda: L.energy_grad(a._h, ok, ok, ok, bad, ok, ok, dtype, 1, 0, None),
            "hub_apply_h": lambda: L.hub_apply_h(a._h, ok, bad, dtype, 1, None),
            "overlap_grad ref": lambda: L.overlap_grad(a._h, ok, bad, 1, ok, None, ok, ok, None, dtype, 1, 0, None),
            "overlap_grad psi": lambda: L.overlap_grad(a._h, ok, ok, 1, bad, None, ok, ok, None, dtype, 1, 0, None),
            "spin_correlation": lambda: L.spin_correlation(a._h, bad, ok, dtype, 1, None),
        }
        for name, call in calls.items():
            assert call() == _lib.HUB_EINVAL, name
            assert b"aligned" in L.hub_last_error(), name
