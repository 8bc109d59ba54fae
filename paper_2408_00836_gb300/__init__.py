"""GB300 statevector engine for Hubbard-model VQE (arxiv 2408.00836).

Python face of libhubsv.so: the C ABI of include/hubsv.h with the same names,
PyTorch used only for device memory and streams.  Every amplitude operation
runs in the sm_103a kernels; there is no CPU or PyTorch fallback.

Main entry points (all take and return torch CUDA tensors):

* ``square_lattice(nx, ny, order)`` -- open grid bonds and HVA bond classes.
* ``Model`` -- the Hamiltonian of Eqs. 1, 2, 15, 16 (``hub_create``).
* ``Ansatz`` -- the layered HVA of Eq. 7 (``ans_create``) with
  ``state_prepare``, ``energy``, ``energy_grad`` and ``apply_h``.
* ``energy_fn`` -- ``torch.autograd`` function whose backward is the adjoint
  gradient of Sec. 2.1.
"""

from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np

from ._lib import HubError, HubGroup, HubLattice, check, lib  # noqa: F401
from . import workloads  # noqa: F401

C64, C128 = 0, 1
HOP, ONSITE, NN_V, POT, RZ, GIVENS, CPHASE = 0, 1, 2, 3, 4, 5, 6
PAIR_KINDS = (GIVENS, CPHASE)   # their terms are mode pairs, flattened
PREP_SLATER, PREP_NEEL = 0, 1
FLAG_PREP_FUSED = 1
FLAG_KEEP_STATE = 2
FLAG_SWEEPS = 4
FLAG_ROWS = 8
FLAG_ROW_CLUSTER = 16
ENGINE_ONCHIP, ENGINE_ROWS = 0, 1
CLASS_IDS = {"h1": 0, "h2": 1, "v1": 2, "v2": 3, "even": 0, "odd": 1}


def _i32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def square_lattice(nx: int, ny: int, order: str = "rowmajor"):
    """Open nx x ny grid: (bonds [(i, j)], classes ['h1'|'h2'|'v1'|'v2'])."""
    o = {"rowmajor": 0, "snake": 1}[order]
    nb = ctypes.c_int32(0)
    check(lib().hub_square_lattice(nx, ny, o, None, None, ctypes.byref(nb)))
    b = np.zeros(2 * nb.value, dtype=np.int32)
    c = np.zeros(nb.value, dtype=np.int32)
    check(lib().hub_square_lattice(nx, ny, o, b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(nb)))
    names = ["h1", "h2", "v1", "v2"]
    return [(int(b[2 * i]), int(b[2 * i + 1])) for i in range(nb.value)], [names[k] for k in c]


class Model:
    """Hubbard Hamiltonian handle (``hub_create``)."""

    def __init__(self, n_sites: int, bonds, t, U=None, V=None, n_up=None, n_dn=None,
                 modes="blocked"):
        L = n_sites
        self.n_sites = L
        self.bonds = [tuple(b) for b in bonds]
        bnd, bp = _i32(np.array(self.bonds, dtype=np.int32).reshape(-1))
        keep = [bnd]
        if isinstance(modes, str):
            if modes == "blocked":
                up = dn = None
            elif modes == "interleaved":
                up, dn = np.arange(L) * 2, np.arange(L) * 2 + 1
            else:
                raise ValueError(modes)
        else:
            up, dn = modes
        lat = HubLattice(L, len(self.bonds), bp, None, None)
        if up is not None:
            ua, upp = _i32(up)
            da, dpp = _i32(dn)
            keep += [ua, da]
            lat.mode_up, lat.mode_dn = upp, dpp
        ta, tp = _f64(np.asarray(t, dtype=np.float64).reshape(L, L))
        Ua, Up = _f64(U) if U is not None else (None, None)
        Va, Vp = _f64(np.asarray(V).reshape(L, L)) if V is not None else (None, None)
        self.n_up = L // 2 if n_up is None else n_up
        self.n_dn = L // 2 if n_dn is None else n_dn
        h = ctypes.c_void_p()
        check(lib().hub_create(ctypes.byref(lat), tp, Up, Vp, self.n_up, self.n_dn, ctypes.byref(h)))
        self._h = h
        del keep, ta, Ua, Va

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and h.value and _lib_loaded():
            lib().hub_destroy(h)
            self._h = None


def _lib_loaded():
    try:
        from . import _lib as m
        return m._lib is not None
    except Exception:  # interpreter shutdown
        return False


def hva_groups(bonds, classes, n_sites: int, n_layers: int, layer: Sequence[str]):
    """Groups of a layered HVA in application order (Eq. 7): one parameter per
    entry of ``layer`` ('U', 'V', 'pot' or a bond class), index l*len + g."""
    out = []
    G = len(layer)
    for l in range(n_layers):
        for g, name in enumerate(layer):
            p = l * G + g
            if name == "U":
                out.append((ONSITE, list(range(n_sites)), p))
            elif name == "V":
                out.append((NN_V, list(range(len(bonds))), p))
            elif name == "pot":
                out.append((POT, list(range(n_sites)), p))
            else:
                cid = CLASS_IDS[name]
                terms = [i for i, c in enumerate(classes) if CLASS_IDS[c] == cid]
                out.append((HOP, terms, p))
    return out


def site_modes(n_sites: int, modes="blocked"):
    """(up, dn) mode of every site for a mode layout ('blocked', the
    default: up i -> i, dn i -> L + i; 'interleaved', the paper's order:
    up i -> 2i, dn i -> 2i + 1; or explicit (up, dn) arrays)."""
    L = n_sites
    if isinstance(modes, str):
        if modes == "blocked":
            return list(range(L)), [L + i for i in range(L)]
        if modes == "interleaved":
            return [2 * i for i in range(L)], [2 * i + 1 for i in range(L)]
        raise ValueError(modes)
    return [int(x) for x in modes[0]], [int(x) for x in modes[1]]


def np_groups(bonds, classes, n_sites: int, n_layers: int, modes="blocked", rz: bool = True):
    """Groups of the number-preserving ansatz of Sec. 2.2.1 in application
    order: an R_z pre-layer (one parameter per qubit), then per layer every
    term of Eq. 7 in its order -- the on-site terms, then the h1, v1, h2,
    v2 hopping classes, each bond for both spins -- replaced by its own NP
    gate of Eq. 8: a GIVENS factor (theta) and a CPHASE factor (phi) on the
    term's two modes.  (10 Nx Ny - 4 Nx - 4 Ny) parameters a layer plus
    2 Nx Ny for R_z."""
    up, dn = site_modes(n_sites, modes)
    out, p = [], 0
    if rz:
        for k in range(2 * n_sites):
            out.append((RZ, [k], p))
            p += 1
    for _ in range(n_layers):
        pairs = [(up[i], dn[i]) for i in range(n_sites)]
        for cc in ("h1", "v1", "h2", "v2"):
            for (i, j), c in zip(bonds, classes):
                if c == cc:
                    pairs += [(up[i], up[j]), (dn[i], dn[j])]
        for (a, b) in pairs:
            a, b = min(a, b), max(a, b)
            out.append((GIVENS, [a, b], p))
            out.append((CPHASE, [a, b], p + 1))
            p += 2
    return out


def ep_groups(n_modes: int, n_layers: int):
    """Groups of the excitation-preserving ansatz of Sec. 2.2.2: R_z on
    every qubit, per layer Eq. 10's gate on each pair of neighbouring qubits
    (k, k+1) as a GIVENS and a CPHASE factor, then R_z on every qubit again
    (4 Nx Ny + 2 (2 Nx Ny - 1) l parameters).  Eq. 10's U_EP(theta, phi) is
    GIVENS(-theta / 2) CPHASE(-phi): the parameters here are -theta / 2 and
    -phi.  Qubit k is mode k (the paper's order is the interleaved one)."""
    out, p = [], 0
    for k in range(n_modes):
        out.append((RZ, [k], p))
        p += 1
    for _ in range(n_layers):
        for k in range(n_modes - 1):
            out.append((GIVENS, [k, k + 1], p))
            out.append((CPHASE, [k, k + 1], p + 1))
            p += 2
    for k in range(n_modes):
        out.append((RZ, [k], p))
        p += 1
    return out


def _ptr(t, nbytes: int, what: str):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.numel() * t.element_size() < nbytes:
        raise ValueError(f"{what} holds {t.numel() * t.element_size()} bytes, needs {nbytes}")
    return ctypes.c_void_p(t.data_ptr())


class Ansatz:
    """Layered HVA handle (``ans_create`` / ``ans_create_multi``)."""

    def __init__(self, models, groups, n_layers: int = 1):
        if isinstance(models, Model):
            models = [models]
        self.models = list(models)
        self.groups = list(groups)
        arrs = []
        garr = (HubGroup * max(1, len(self.groups)))()
        for i, (kind, terms, param) in enumerate(self.groups):
            a, p = _i32(terms if len(terms) else [0])
            arrs.append(a)
            n_terms = len(terms) // 2 if kind in PAIR_KINDS else len(terms)
            garr[i] = HubGroup(kind, n_terms, p, param)
        G = len(self.groups)
        if G % n_layers:
            raise ValueError("number of groups must be a multiple of n_layers")
        h = ctypes.c_void_p()
        hs = (ctypes.c_void_p * len(self.models))(*[m.handle.value for m in self.models])
        check(lib().ans_create_multi(hs, len(self.models), n_layers, G // n_layers, garr, ctypes.byref(h)))
        self._h = h
        del arrs
        self.P = lib().ans_num_params(h)
        self.n = lib().ans_num_qubits(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and h.value and _lib_loaded():
            lib().ans_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def amp_bytes(self, dtype: int) -> int:
        return (8 if dtype == C64 else 16) << self.n

    def state_prepare(self, kind=PREP_SLATER, orb_perturb=None, neel_up=None, psi=None,
                      dtype=C64, batch: int = 1, stream=None):
        pa, pp = _f64(orb_perturb) if orb_perturb is not None else (None, None)
        na, npp = _i32(neel_up) if neel_up is not None else (None, None)
        ptr = _ptr(psi, batch * self.amp_bytes(dtype), "psi")
        check(lib().state_prepare(self._h, kind, pp, npp, ptr, dtype, batch, _stream(stream)))
        del pa, na

    @staticmethod
    def _flags(fused=True, keep_state=False, sweeps=False, rows=False):
        return ((FLAG_PREP_FUSED if fused else 0) | (FLAG_KEEP_STATE if keep_state else 0)
                | (FLAG_SWEEPS if sweeps else 0) | (FLAG_ROWS if rows else 0))

    def workspace(self, which: int, dtype=C64, batch: int = 1, fused: bool = True, keep_state: bool = False,
                  sweeps: bool = False, rows: bool = False):
        """(bytes psi and lam must each hold, engine) of a call (which: 0
        energy, 1 energy_grad); engine 0 on chip, 1 rows, 2 dense sweeps."""
        by = ctypes.c_uint64(0)
        eng = ctypes.c_int32(0)
        check(lib().ans_workspace_bytes(self._h, which, dtype, self._flags(fused, keep_state, sweeps, rows),
                                        batch, ctypes.byref(by), ctypes.byref(eng)))
        return by.value, eng.value

    def energy(self, theta, psi, E, dtype=C64, batch: int = 1, fused: bool = True,
               keep_state: bool = False, sweeps: bool = False, rows: bool = False, stream=None):
        flags = self._flags(fused, keep_state, sweeps, rows)
        nb = self.workspace(0, dtype, batch, fused, keep_state, sweeps, rows)[0]
        check(lib().energy(self._h, _ptr(theta, 8 * batch * self.P, "theta"),
                           _ptr(psi, max(nb, 1), "psi"), _ptr(E, 8 * batch, "E"),
                           dtype, batch, flags, _stream(stream)))
        return E

    def energy_grad(self, theta, psi, lam, E, grad, ckpt=None, dtype=C64, batch: int = 1,
                    fused: bool = True, sweeps: bool = False, rows: bool = False, row_cluster: bool = False,
                    stream=None):
        """row_cluster: HUB_FLAG_ROW_CLUSTER (rows of psi and lam on two-CTA
        clusters wherever the row engine runs them)."""
        nb = self.workspace(1, dtype, batch, fused, False, sweeps, rows)[0]
        dense = batch * self.amp_bytes(dtype)
        flags = self._flags(fused, False, sweeps, rows) | (FLAG_ROW_CLUSTER if row_cluster else 0)
        check(lib().energy_grad(self._h, _ptr(theta, 8 * batch * self.P, "theta"), _ptr(psi, max(nb, 1), "psi"),
                                _ptr(lam, max(nb, 1), "lam"), _ptr(ckpt, dense, "ckpt"), _ptr(E, 8 * batch, "E"),
                                _ptr(grad, 8 * batch * self.P, "grad"), dtype, batch, flags, _stream(stream)))
        return E, grad

    def apply_h(self, psi, lam, dtype=C64, batch: int = 1, stream=None):
        nb = batch * self.amp_bytes(dtype)
        check(lib().hub_apply_h(self._h, _ptr(psi, nb, "psi"), _ptr(lam, nb, "lam"), dtype, batch,
                                _stream(stream)))
        return lam

    def overlap_grad(self, theta, psi_ref, psi, lam=None, F=None, f=None, grad=None, dtype=C64,
                     batch: int = 1, fused: bool = True, sweeps: bool = False, stream=None):
        """Fidelity F = |<psi_ref|psi(theta)>|^2, the overlap loss of Eq. 5
        f = log10(1 - F) and (grad given) df/dtheta; psi_ref holds one
        reference or one per batch element.  sweeps: the dense sweeps even
        where the row engine applies."""
        nb = batch * self.amp_bytes(dtype)
        ref_batch = psi_ref.numel() * psi_ref.element_size() // self.amp_bytes(dtype)
        if ref_batch not in (1, batch):
            raise ValueError("psi_ref must hold 1 or batch states")
        check(lib().overlap_grad(self._h, _ptr(theta, 8 * batch * self.P, "theta"),
                                 _ptr(psi_ref, ref_batch * self.amp_bytes(dtype), "psi_ref"), ref_batch,
                                 _ptr(psi, nb, "psi"), _ptr(lam, nb, "lam"), _ptr(F, 8 * batch, "F"),
                                 _ptr(f, 8 * batch, "f"), _ptr(grad, 8 * batch * self.P, "grad"), dtype, batch,
                                 (FLAG_PREP_FUSED if fused else 0) | (FLAG_SWEEPS if sweeps else 0),
                                 _stream(stream)))
        return F, f, grad

    def spin_correlation(self, psi, C, dtype=C64, batch: int = 1, stream=None):
        """C[b][i][j] = <S^z_i S^z_j> - <S^z_i><S^z_j> of the state psi (Sec. 3)."""
        L = self.n // 2
        check(lib().spin_correlation(self._h, _ptr(psi, batch * self.amp_bytes(dtype), "psi"),
                                     _ptr(C, 8 * batch * L * L, "C"), dtype, batch, _stream(stream)))
        return C

    def plan_stats(self, which: int, dtype=C64, fused: bool = True, rows: bool = False):
        """(sweeps, HBM bytes per state) of the dense sweep plan, or with
        rows=True (launches, HBM bytes per state) of the row engine."""
        ns = ctypes.c_int32(0)
        by = ctypes.c_double(0.0)
        flags = (FLAG_PREP_FUSED if fused else 0) | (FLAG_ROWS if rows else 0)
        check(lib().ans_plan_stats(self._h, which, dtype, flags, ctypes.byref(ns), ctypes.byref(by)))
        return ns.value, by.value

    def plan_describe(self, which: int, dtype=C64, flags: int = FLAG_PREP_FUSED):
        """[(tile_mask, sweep_flags, [sequence indices])] of a call kind (with
        FLAG_ROWS in flags: the row engine's segments, (spin mode mask,
        orientation, [sequence indices]))."""
        n = ctypes.c_int32(0)
        check(lib().ans_plan_describe(self._h, which, dtype, flags, None, 0, ctypes.byref(n)))
        buf = (ctypes.c_int64 * n.value)()
        check(lib().ans_plan_describe(self._h, which, dtype, flags, buf, n.value, ctypes.byref(n)))
        v = list(buf)
        out, i = [], 1
        for _ in range(v[0]):
            tile, fl, cnt = v[i], v[i + 1], v[i + 2]
            out.append((tile, fl, v[i + 3:i + 3 + cnt]))
            i += 3 + cnt
        return out

    def set_tile(self, dtype: int, log2_tile: int):
        check(lib().ans_set_tile(self._h, dtype, log2_tile))

    def set_runs(self, dtype: int, log2_run: int):
        """log2 of the contiguous amplitudes per HBM run (0 = automatic)."""
        check(lib().ans_set_runs(self._h, dtype, log2_run))

    def set_threads(self, dtype: int, engine: int, threads: int):
        """Threads per CTA of a sector engine (ENGINE_ONCHIP: 256 or 512;
        ENGINE_ROWS: 256, 512 or 1024; 0 = automatic)."""
        check(lib().ans_set_threads(self._h, dtype, engine, threads))


def sync(stream=None):
    check(lib().hub_sync(_stream(stream)))


def workspace_tensor(ans: "Ansatz", which: int, dtype=C64, batch: int = 1, device="cuda", **flags):
    """A psi / lam buffer of exactly the size the call needs (ans.workspace)."""
    import torch
    nb, _ = ans.workspace(which, dtype, batch, **flags)
    td = torch.complex64 if dtype == C64 else torch.complex128
    return torch.empty(max(1, nb // (8 if dtype == C64 else 16)), dtype=td, device=device)


def empty_state(n_qubits: int, dtype=C64, batch: int = 1, device="cuda"):
    import torch
    td = torch.complex64 if dtype == C64 else torch.complex128
    return torch.empty((batch, 1 << n_qubits), dtype=td, device=device)


class _EnergyFn:
    """Builds the torch.autograd.Function lazily (torch imported on use)."""
    fn = None


def energy_fn(ans: Ansatz, theta, psi, lam, dtype=C64, batch: int = 1, ckpt=None):
    """E(theta) with autograd: forward runs energy_grad (the adjoint pass of
    Sec. 2.1) and keeps the gradient; backward scales it by dL/dE."""
    import torch
    if _EnergyFn.fn is None:
        class EnergyFunction(torch.autograd.Function):
            @staticmethod
            def forward(ctx, th, a, ps, lm, dt, bt, ck):
                E = torch.empty(bt, dtype=torch.float64, device=th.device)
                g = torch.empty(bt, a.P, dtype=torch.float64, device=th.device)
                a.energy_grad(th.detach().contiguous(), ps, lm, E, g, ckpt=ck, dtype=dt, batch=bt)
                ctx.save_for_backward(g)
                return E

            @staticmethod
            def backward(ctx, gE):
                (g,) = ctx.saved_tensors
                return gE[:, None] * g, None, None, None, None, None, None
        _EnergyFn.fn = EnergyFunction
    return _EnergyFn.fn.apply(theta, ans, psi, lam, dtype, batch, ckpt)


def profile(ans: Ansatz, enable: bool = True):
    """Enable (or disable) per-launch CUDA-event timing of the sweeps."""
    check(lib().ans_profile(ans.handle, 1 if enable else 0))


def profile_read(ans: Ansatz):
    """[(vectors, dtype, bytes, ms)] of the sweep launches since enabling."""
    n = ctypes.c_int32(0)
    check(lib().ans_profile_read(ans.handle, None, 0, ctypes.byref(n)))
    buf = (ctypes.c_double * max(1, 4 * n.value))()
    check(lib().ans_profile_read(ans.handle, buf, 4 * n.value, ctypes.byref(n)))
    return [(int(buf[4 * i]), int(buf[4 * i + 1]), buf[4 * i + 2], buf[4 * i + 3]) for i in range(n.value)]
