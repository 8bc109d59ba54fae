"""Plain CPU complex128 oracle: Jordan-Wigner Hubbard model, HVA ansatz,
energy, adjoint gradient, Lanczos.  TEST INFRASTRUCTURE ONLY (see the
package docstring); shares no code with the CUDA library.

Conventions (each one follows the paper, or is the reading the paper needs):

* Lattice (Sec. 3, open boundary conditions): an ``nx x ny`` grid, rows
  ``x = 0..nx-1``, columns ``y = 0..ny-1``.  Site numbering is row-major,
  ``s = x*ny + y`` (Sec. 2.2.1, 0-based), or "snake" (odd rows reversed).
* Bond classes (Eq. 7): horizontal bonds ``(x,y)-(x,y+1)`` are ``h1`` for even
  ``y`` and ``h2`` for odd ``y``; vertical bonds ``(x,y)-(x+1,y)`` are ``v1``
  for even ``x`` and ``v2`` for odd ``x``.  Each class is a set of mutually
  commuting hops, as Eq. 7 requires; the paper does not fix the partition.
* Jordan-Wigner (Sec. 2.2.1): one qubit per spin-orbital; mode ``k`` is bit
  ``k`` of the basis index ``x``.  ``a_k|x> = (-1)^{popcount(x & (2^k-1))}
  |x ^ 2^k>`` when bit k is set, and ``|x> = a+_{k1} a+_{k2} ... |vac>`` with
  ``k1 < k2 < ...``.  The site -> mode map is "blocked" (up spins on modes
  0..L-1, down spins on L..2L-1), "interleaved" (the paper's order,
  ``up = 2s``, ``dn = 2s+1``), or any explicit map.
* Hamiltonian (Eqs. 1, 2, 15, 16): ``H = -sum_sigma sum_{i != j} t_ij a+_i a_j
  - sum_{i,sigma} t_ii n_{i sigma} + sum_i U_i n_iu n_id
  + sum_{<ij>} V_ij n_i n_j``.  The hopping sum runs over both orders of each
  pair (Hermitian reading of Eq. 2); the diagonal of ``t`` is the on-site
  potential of Eq. 15; each V bond is counted once (Eq. 2's one-half over
  ordered pairs).
* Ansatz (Eqs. 3 and 7): ``|psi> = U_K ... U_1 |psi_0>``, each group factor
  ``U_g = exp(-i theta_p G_g)``.  The sign of the exponent is read as ``-i``
  throughout (Eq. 7 writes ``+i``; the landscape is mirrored in theta, its
  minima unchanged).  ``G_g`` is the group's Hamiltonian terms with their
  coefficients and signs: hop ``-sum t_ij (a+_i a_j + h.c.)``, on-site
  ``sum U_i n_iu n_id``, NN ``sum V_ij n_i n_j``, potential
  ``-sum t_ii (n_iu + n_id)``, and ``rz``: ``sum_k (1/2 - n_k)`` = ``Z_k/2``.
* Gradient (Sec. 2.1): ``dE/dtheta_k = 2 Im <lambda_k|G_k|psi_k>`` with
  ``psi_k = U_k...U_1 psi_0`` and ``lambda_k = U_{k+1}^+...U_K^+ H psi_K``;
  the printed bra/ket placement is garbled, this is the standard form.
"""

from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Lattice", "square_lattice", "mode_map", "Model", "make_model",
    "Group", "hva_groups", "sector_basis", "full_basis", "popcount",
    "annihilate", "create", "hop_matrix", "number_diag", "hamiltonian",
    "group_terms", "apply_group", "apply_generator", "ansatz_state",
    "energy", "energy_and_gradient", "fd_gradient", "lanczos_ground",
    "orbitals", "slater_state", "neel_state", "hartree_fock_energy",
    "neel_energy", "u0_ground_energy", "fidelity", "overlap_loss_and_gradient",
    "overlap_fd_gradient", "spin_correlation", "number_basis", "np_groups", "ep_groups",
    "np_param_count", "ep_param_count",
]

# ---------------------------------------------------------------------------
# bit helpers
# ---------------------------------------------------------------------------

_POP8 = np.array([bin(i).count("1") for i in range(256)], dtype=np.int64)


def popcount(x) -> np.ndarray:
    """Number of set bits of each entry of a uint64 array (byte-table sum)."""
    x = np.asarray(x, dtype=np.uint64)
    out = np.zeros(x.shape, dtype=np.int64)
    for k in range(8):
        out += _POP8[((x >> np.uint64(8 * k)) & np.uint64(255)).astype(np.intp)]
    return out


def _bit(x: np.ndarray, k: int) -> np.ndarray:
    return ((x >> np.uint64(k)) & np.uint64(1)).astype(np.int64)


# ---------------------------------------------------------------------------
# lattice and modes (Sec. 2.2.1, Sec. 3: open boundary conditions)
# ---------------------------------------------------------------------------

@dataclass
class Lattice:
    nx: int
    ny: int
    order: str
    n_sites: int
    coords: list            # site -> (x, y)
    bonds: list             # [(i, j)] site pairs, i < j
    bond_class: list        # 'h1' | 'h2' | 'v1' | 'v2' per bond


def square_lattice(nx: int, ny: int, order: str = "rowmajor") -> Lattice:
    """Open ``nx x ny`` grid with nearest-neighbour bonds (Eq. 2's <RR'>)."""
    def site(x, y):
        if order == "rowmajor":
            return x * ny + y
        if order == "snake":
            return x * ny + (y if x % 2 == 0 else ny - 1 - y)
        raise ValueError(order)

    coords = [None] * (nx * ny)
    for x in range(nx):
        for y in range(ny):
            coords[site(x, y)] = (x, y)
    bonds, cls = [], []
    for x in range(nx):
        for y in range(ny - 1):
            i, j = site(x, y), site(x, y + 1)
            bonds.append((min(i, j), max(i, j)))
            cls.append("h1" if y % 2 == 0 else "h2")
    for x in range(nx - 1):
        for y in range(ny):
            i, j = site(x, y), site(x + 1, y)
            bonds.append((min(i, j), max(i, j)))
            cls.append("v1" if x % 2 == 0 else "v2")
    return Lattice(nx, ny, order, nx * ny, coords, bonds, cls)


def mode_map(n_sites: int, scheme: str = "blocked"):
    """Site -> qubit maps (up, dn).  'interleaved' is the paper's order."""
    s = np.arange(n_sites)
    if scheme == "blocked":
        return s.copy(), s + n_sites
    if scheme == "interleaved":
        return 2 * s, 2 * s + 1
    raise ValueError(scheme)


# ---------------------------------------------------------------------------
# model
# ---------------------------------------------------------------------------

@dataclass
class Model:
    n_sites: int
    up: np.ndarray          # site -> mode of the up spin-orbital
    dn: np.ndarray          # site -> mode of the down spin-orbital
    t: np.ndarray           # L x L symmetric; diagonal = on-site potential
    U: np.ndarray           # L
    V: np.ndarray           # L x L symmetric, zero diagonal
    n_up: int
    n_dn: int
    bonds: list = field(default_factory=list)   # NN pairs, for V groups

    @property
    def n_modes(self) -> int:
        return 2 * self.n_sites


def make_model(lat: Lattice, t, U, V=None, n_up=None, n_dn=None,
               modes="blocked") -> Model:
    L = lat.n_sites
    t = np.array(t, dtype=np.float64)
    if t.ndim == 0:
        tt = np.zeros((L, L))
        for (i, j) in lat.bonds:
            tt[i, j] = tt[j, i] = float(t)
        t = tt
    U = np.array(U, dtype=np.float64)
    if U.ndim == 0:
        U = np.full(L, float(U))
    if V is None:
        V = np.zeros((L, L))
    else:
        V = np.array(V, dtype=np.float64)
        if V.ndim == 0:
            vv = np.zeros((L, L))
            for (i, j) in lat.bonds:
                vv[i, j] = vv[j, i] = float(V)
            V = vv
    if isinstance(modes, str):
        up, dn = mode_map(L, modes)
    else:
        up, dn = (np.asarray(m, dtype=np.int64) for m in modes)
    n_up = L // 2 if n_up is None else n_up
    n_dn = L // 2 if n_dn is None else n_dn
    return Model(L, np.asarray(up), np.asarray(dn), t, U, V, n_up, n_dn,
                 list(lat.bonds))


# ---------------------------------------------------------------------------
# basis states
# ---------------------------------------------------------------------------

def _configs(modes: Sequence[int], k: int) -> np.ndarray:
    out = [sum(1 << int(m) for m in c) for c in itertools.combinations(modes, k)]
    return np.array(out, dtype=np.uint64)


def sector_basis(model: Model, n_up: int | None = None,
                 n_dn: int | None = None) -> np.ndarray:
    """Sorted basis states with exactly n_up up and n_dn down electrons."""
    n_up = model.n_up if n_up is None else n_up
    n_dn = model.n_dn if n_dn is None else n_dn
    a = _configs(model.up, n_up)
    b = _configs(model.dn, n_dn)
    return np.sort((a[:, None] | b[None, :]).ravel())


def number_basis(model: Model, n_total: int) -> np.ndarray:
    """Sorted basis states with n_total electrons in all (both spins): the
    sector that spin-mixing ansatz factors (the on-site NP gate, the EP
    gates) keep."""
    return np.sort(_configs(list(model.up) + list(model.dn), n_total))


def full_basis(model: Model) -> np.ndarray:
    """All 2^n basis states (small n only)."""
    return np.arange(1 << model.n_modes, dtype=np.uint64)


# ---------------------------------------------------------------------------
# Jordan-Wigner operators from the definition
# ---------------------------------------------------------------------------

def _jw_sign(x: np.ndarray, k: int) -> np.ndarray:
    below = np.uint64((1 << k) - 1)
    return 1 - 2 * (popcount(x & below) & 1)


def annihilate(x: np.ndarray, k: int):
    """a_k on basis states x: (valid, sign, new state)."""
    valid = _bit(x, k) == 1
    return valid, _jw_sign(x, k), x ^ np.uint64(1 << k)


def create(x: np.ndarray, k: int):
    """a+_k on basis states x: (valid, sign, new state)."""
    valid = _bit(x, k) == 0
    return valid, _jw_sign(x, k), x | np.uint64(1 << k)


def _lookup(basis: np.ndarray, states: np.ndarray) -> np.ndarray:
    idx = np.searchsorted(basis, states)
    idx = np.minimum(idx, len(basis) - 1)
    if not np.all(basis[idx] == states):
        raise ValueError("operator leaves the basis")
    return idx


def _cdag_c(basis: np.ndarray, p: int, q: int):
    """Matrix entries of a+_p a_q (p != q) in the basis: rows, cols, values."""
    cols = np.arange(len(basis))
    v1, s1, y = annihilate(basis, q)
    v2, s2, z = create(y, p)
    ok = v1 & v2
    rows = _lookup(basis, z[ok])
    return rows, cols[ok], (s1 * s2)[ok].astype(np.float64)


def hop_matrix(basis: np.ndarray, p: int, q: int) -> sp.csr_matrix:
    """a+_p a_q + a+_q a_p as a sparse matrix on the given basis."""
    r1, c1, v1 = _cdag_c(basis, p, q)
    r2, c2, v2 = _cdag_c(basis, q, p)
    n = len(basis)
    m = sp.coo_matrix((np.concatenate([v1, v2]),
                       (np.concatenate([r1, r2]), np.concatenate([c1, c2]))),
                      shape=(n, n))
    return m.tocsr()


def number_diag(basis: np.ndarray, k: int) -> np.ndarray:
    """Diagonal of n_k = a+_k a_k."""
    return _bit(basis, k).astype(np.float64)


# ---------------------------------------------------------------------------
# Hamiltonian (Eqs. 1, 2, 15, 16)
# ---------------------------------------------------------------------------

def _site_occ(model: Model, basis: np.ndarray):
    nu = np.stack([number_diag(basis, int(model.up[i])) for i in range(model.n_sites)])
    nd = np.stack([number_diag(basis, int(model.dn[i])) for i in range(model.n_sites)])
    return nu, nd


def diagonal_energy(model: Model, basis: np.ndarray) -> np.ndarray:
    """Diagonal part of H: potential, on-site U and NN V terms."""
    nu, nd = _site_occ(model, basis)
    L = model.n_sites
    d = np.zeros(len(basis))
    for i in range(L):
        d += -model.t[i, i] * (nu[i] + nd[i]) + model.U[i] * nu[i] * nd[i]
    for i in range(L):
        for j in range(i + 1, L):
            if model.V[i, j] != 0.0:
                d += model.V[i, j] * (nu[i] + nd[i]) * (nu[j] + nd[j])
    return d


def hamiltonian(model: Model, basis: np.ndarray) -> sp.csr_matrix:
    n = len(basis)
    H = sp.diags(diagonal_energy(model, basis)).tocsr()
    L = model.n_sites
    for i in range(L):
        for j in range(i + 1, L):
            if model.t[i, j] != 0.0:
                for m in (model.up, model.dn):
                    H = H - model.t[i, j] * hop_matrix(basis, int(m[i]), int(m[j]))
    return sp.csr_matrix(H, shape=(n, n))


# ---------------------------------------------------------------------------
# ansatz (Eqs. 3, 7)
# ---------------------------------------------------------------------------

@dataclass
class Group:
    kind: str               # 'hop' | 'onsite_u' | 'nn_v' | 'eps' | 'rz' | 'givens' | 'cphase'
    terms: tuple            # hop/nn_v: site pairs; onsite_u/eps: sites; rz: modes;
                            # givens/cphase: mode pairs
    param: int


def hva_groups(lat: Lattice, n_layers: int, classes: Sequence[str],
               with_v: bool = False) -> list:
    """Groups of a layered HVA, in application order, one parameter each.

    ``classes`` lists the entries of one layer in application order; each is
    'U', 'V', 'eps' or a bond class ('h1', 'h2', 'v1', 'v2', or 'even'/'odd'
    for the h1/h2 classes of a chain).  Parameter index = layer * len + slot.
    """
    alias = {"even": "h1", "odd": "h2"}
    out = []
    G = len(classes)
    for l in range(n_layers):
        for g, c in enumerate(classes):
            p = l * G + g
            if c == "U":
                out.append(Group("onsite_u", tuple(range(lat.n_sites)), p))
            elif c == "V":
                out.append(Group("nn_v", tuple(lat.bonds), p))
            elif c == "eps":
                out.append(Group("eps", tuple(range(lat.n_sites)), p))
            else:
                cc = alias.get(c, c)
                terms = tuple(b for b, k in zip(lat.bonds, lat.bond_class) if k == cc)
                out.append(Group("hop", terms, p))
    return out


def np_groups(lat: Lattice, model: Model, n_layers: int, rz: bool = True) -> list:
    """The number-preserving (NP) ansatz of Sec. 2.2.1, in application order.

    An optional R_z pre-layer (one parameter per qubit, the 'rz' generator
    Z/2), then per layer the terms of Eq. 7 in its order -- on-site terms,
    then the h1, v1, h2, v2 hopping classes -- each replaced by its own NP
    gate U_NP(theta, phi) of Eq. 8 = exp(-i theta G_givens) exp(-i phi
    G_cphase) on the term's two modes: the on-site term on (up(i), dn(i)),
    a hopping term on (sigma(i), sigma(j)) for each spin.  Each factor has its
    own parameter (theta, then phi)."""
    out = []
    p = 0
    if rz:
        for k in range(model.n_modes):
            out.append(Group("rz", (k,), p))
            p += 1
    for _ in range(n_layers):
        pairs = [(int(model.up[i]), int(model.dn[i])) for i in range(lat.n_sites)]
        for cc in ("h1", "v1", "h2", "v2"):
            for (i, j), k in zip(lat.bonds, lat.bond_class):
                if k == cc:
                    for m in (model.up, model.dn):
                        pairs.append((int(m[i]), int(m[j])))
        for (a, b) in pairs:
            a, b = min(a, b), max(a, b)
            out.append(Group("givens", ((a, b),), p))
            out.append(Group("cphase", ((a, b),), p + 1))
            p += 2
    return out


def np_param_count(nx: int, ny: int, n_layers: int, rz: bool = True) -> int:
    """Parameters of the NP ansatz as the paper counts them (Sec. 2.2.1):
    (10 Nx Ny - 4 Nx - 4 Ny) per layer plus 2 Nx Ny for the R_z layer."""
    return (10 * nx * ny - 4 * nx - 4 * ny) * n_layers + (2 * nx * ny if rz else 0)


def ep_groups(n_modes: int, n_layers: int) -> list:
    """The excitation-preserving (EP) ansatz of Sec. 2.2.2, in application
    order: R_z on every qubit, then per layer the two-qubit gate of Eq. 10
    on each pair of neighbouring qubits (k, k+1), k = 0 .. n-2, then R_z on
    every qubit again.  Qubit k is mode k (the paper's interleaved order
    puts site s on qubits 2s, 2s+1).  Eq. 10's gate U_EP(theta, phi) equals
    exp(-i theta' G_givens) exp(-i phi' G_cphase) with theta' = -theta / 2
    and phi' = -phi; the groups here carry theta' and phi' as their
    parameters (a fixed linear change of variables)."""
    out = []
    p = 0
    for k in range(n_modes):
        out.append(Group("rz", (k,), p))
        p += 1
    for _ in range(n_layers):
        for k in range(n_modes - 1):
            out.append(Group("givens", ((k, k + 1),), p))
            out.append(Group("cphase", ((k, k + 1),), p + 1))
            p += 2
    for k in range(n_modes):
        out.append(Group("rz", (k,), p))
        p += 1
    return out


def ep_param_count(nx: int, ny: int, n_layers: int) -> int:
    """4 Nx Ny + 2 (2 Nx Ny - 1) l (Sec. 2.2.2)."""
    return 4 * nx * ny + 2 * (2 * nx * ny - 1) * n_layers


def group_terms(model: Model, basis: np.ndarray, group: Group, cache=None):
    """The group's generator as a list of commuting pieces.

    Returns a list of ('hop', coef, T) with T = a+_p a_q + h.c. (sparse) and
    generator piece ``coef * T``, and at most one ('diag', d) with the
    diagonal generator d(x).
    """
    key = (group.kind, group.terms)
    if cache is not None and key in cache:
        return cache[key]
    pieces = []
    if group.kind == "hop":
        for (i, j) in group.terms:
            for m in (model.up, model.dn):
                T = hop_matrix(basis, int(m[i]), int(m[j]))
                pieces.append(("hop", -model.t[i, j], T))
    elif group.kind == "givens":
        # the theta part of the NP gate (Eq. 8): generator -(a+_p a_q + h.c.),
        # unit coefficient, any two modes (same or opposite spin)
        for (p, q) in group.terms:
            pieces.append(("hop", -1.0, hop_matrix(basis, int(p), int(q))))
    else:
        d = np.zeros(len(basis))
        if group.kind == "onsite_u":
            for i in group.terms:
                d += model.U[i] * number_diag(basis, int(model.up[i])) * number_diag(basis, int(model.dn[i]))
        elif group.kind == "nn_v":
            for (i, j) in group.terms:
                ni = number_diag(basis, int(model.up[i])) + number_diag(basis, int(model.dn[i]))
                nj = number_diag(basis, int(model.up[j])) + number_diag(basis, int(model.dn[j]))
                d += model.V[i, j] * ni * nj
        elif group.kind == "eps":
            for i in group.terms:
                d += -model.t[i, i] * (number_diag(basis, int(model.up[i])) + number_diag(basis, int(model.dn[i])))
        elif group.kind == "rz":
            for k in group.terms:
                d += 0.5 - number_diag(basis, int(k))
        elif group.kind == "cphase":
            # the phi part of the NP gate (Eq. 8): generator -n_p n_q, so that
            # exp(-i phi G) puts exp(+i phi) on |11>
            for (p, q) in group.terms:
                d -= number_diag(basis, int(p)) * number_diag(basis, int(q))
        else:
            raise ValueError(group.kind)
        pieces.append(("diag", d))
    if cache is not None:
        cache[key] = pieces
    return pieces


def _exp_piece(piece, theta: float, psi: np.ndarray, sign: float = -1.0):
    """exp(sign * i * theta * piece) psi, exactly.

    For a hop piece c*T: T has eigenvalues -1, 0, 1 (T^3 = T), so
    exp(i a T) = I + i sin(a) T + (cos(a) - 1) T^2 with a = sign * theta * c.
    """
    if piece[0] == "hop":
        _, c, T = piece
        a = sign * theta * c
        Tpsi = T @ psi
        return psi + 1j * math.sin(a) * Tpsi + (math.cos(a) - 1.0) * (T @ Tpsi)
    _, d = piece
    return np.exp(1j * sign * theta * d) * psi


def apply_group(model, basis, group, theta, psi, cache=None, inverse=False):
    """U_g psi (or U_g^+ psi), one commuting piece at a time."""
    sign = 1.0 if inverse else -1.0
    for piece in group_terms(model, basis, group, cache):
        psi = _exp_piece(piece, theta, psi, sign)
    return psi


def apply_generator(model, basis, group, psi, cache=None):
    """G_g psi."""
    out = np.zeros_like(psi)
    for piece in group_terms(model, basis, group, cache):
        if piece[0] == "hop":
            out += piece[1] * (piece[2] @ psi)
        else:
            out += piece[1] * psi
    return out


def ansatz_state(model, basis, groups, theta, psi0, cache=None):
    psi = np.array(psi0, dtype=np.complex128)
    for g in groups:
        psi = apply_group(model, basis, g, float(theta[g.param]), psi, cache)
    return psi


def energy(model, basis, groups, theta, psi0, H=None, cache=None) -> float:
    """E(theta) = <psi|H|psi> (Eq. 4) with an explicit H|psi>."""
    H = hamiltonian(model, basis) if H is None else H
    psi = ansatz_state(model, basis, groups, theta, psi0, cache)
    return float(np.real(np.vdot(psi, H @ psi)))


def energy_and_gradient(model, basis, groups, theta, psi0, H=None, cache=None):
    """Energy and its adjoint gradient (Sec. 2.1)."""
    H = hamiltonian(model, basis) if H is None else H
    cache = {} if cache is None else cache
    psi = ansatz_state(model, basis, groups, theta, psi0, cache)
    lam = H @ psi
    E = float(np.real(np.vdot(psi, lam)))
    n_par = max(g.param for g in groups) + 1 if groups else 0
    grad = np.zeros(max(n_par, len(theta)))
    for g in reversed(groups):
        Gpsi = apply_generator(model, basis, g, psi, cache)
        grad[g.param] += 2.0 * float(np.imag(np.vdot(lam, Gpsi)))
        th = float(theta[g.param])
        psi = apply_group(model, basis, g, th, psi, cache, inverse=True)
        lam = apply_group(model, basis, g, th, lam, cache, inverse=True)
    return E, grad[:len(theta)]


def fd_gradient(model, basis, groups, theta, psi0, h=1e-4, H=None, cache=None):
    """Central finite differences of E(theta), step h."""
    H = hamiltonian(model, basis) if H is None else H
    cache = {} if cache is None else cache
    theta = np.asarray(theta, dtype=np.float64)
    g = np.zeros(len(theta))
    for k in range(len(theta)):
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        g[k] = (energy(model, basis, groups, tp, psi0, H, cache)
                - energy(model, basis, groups, tm, psi0, H, cache)) / (2 * h)
    return g


# ---------------------------------------------------------------------------
# overlap loss (Eq. 5), fidelity and spin correlations (Sec. 3)
# ---------------------------------------------------------------------------

def fidelity(psi, psi_ref) -> float:
    """F = |<psi_ref|psi>|^2 of two normalised states."""
    return float(abs(np.vdot(psi_ref, psi)) ** 2)


def overlap_loss_and_gradient(model, basis, groups, theta, psi0, psi_ref, cache=None):
    """The overlap loss of Eq. 5, f = log10(1 - F) with F = |<psi(theta)|
    psi_ref>|^2, and its gradient by the adjoint recursion of Sec. 2.1.

    The recursion is the energy's with the projector P = |psi_ref><psi_ref|
    in place of H: F = <psi_K|P|psi_K>, and with lambda_K = P psi_K =
    psi_ref <psi_ref|psi_K> carried back through the inverse factors,
    dF/dtheta_k = 2 Im <lambda_k|G_k|psi_k> (the derivative of the overlap
    a = <psi_ref|psi_K> is -i <chi_k|G_k|psi_k> with chi_k the reference
    carried back, and dF = 2 Re(conj(a) da)).  Then df/dtheta =
    -dF/dtheta / ((1 - F) ln 10).  Returns (F, f, df/dtheta)."""
    cache = {} if cache is None else cache
    psi = ansatz_state(model, basis, groups, theta, psi0, cache)
    a = np.vdot(psi_ref, psi)
    F = float(abs(a) ** 2)
    lam = psi_ref * a
    n_par = max(g.param for g in groups) + 1 if groups else 0
    dF = np.zeros(max(n_par, len(theta)))
    for g in reversed(groups):
        Gpsi = apply_generator(model, basis, g, psi, cache)
        dF[g.param] += 2.0 * float(np.imag(np.vdot(lam, Gpsi)))
        th = float(theta[g.param])
        psi = apply_group(model, basis, g, th, psi, cache, inverse=True)
        lam = apply_group(model, basis, g, th, lam, cache, inverse=True)
    f = math.log10(1.0 - F)
    return F, f, (-dF / ((1.0 - F) * math.log(10.0)))[:len(theta)]


def overlap_fd_gradient(model, basis, groups, theta, psi0, psi_ref, h=1e-5, cache=None):
    """Central finite differences of f(theta) = log10(1 - F(theta))."""
    cache = {} if cache is None else cache
    theta = np.asarray(theta, dtype=np.float64)
    g = np.zeros(len(theta))

    def f_of(th):
        return math.log10(1.0 - fidelity(ansatz_state(model, basis, groups, th, psi0, cache), psi_ref))

    for k in range(len(theta)):
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        g[k] = (f_of(tp) - f_of(tm)) / (2 * h)
    return g


def spin_correlation(model: Model, basis: np.ndarray, psi) -> np.ndarray:
    """C_ij = <S^z_i S^z_j> - <S^z_i><S^z_j> (Sec. 3) for all site pairs,
    S^z_i = (n_{i up} - n_{i dn}) / 2, expectation values in psi."""
    p = np.abs(np.asarray(psi)) ** 2
    nu, nd = _site_occ(model, basis)
    sz = 0.5 * (nu - nd)                      # [L][basis]
    m1 = sz @ p                               # <S^z_i>
    m2 = (sz * p[None, :]) @ sz.T             # <S^z_i S^z_j>
    return m2 - np.outer(m1, m1)


# ---------------------------------------------------------------------------
# Lanczos (stands in for the paper's DMRG reference)
# ---------------------------------------------------------------------------

def lanczos_ground(H, v0=None, m: int = 300, tol: float = 1e-13, seed: int = 7):
    """Lowest eigenvalue of a Hermitian operator by Lanczos with full
    re-orthogonalisation; returns (E0, ground vector)."""
    n = H.shape[0]
    if n <= 2:
        w, v = np.linalg.eigh(H.toarray() if sp.issparse(H) else H)
        return float(w[0]), v[:, 0]
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(n) if v0 is None else np.array(v0, dtype=np.complex128)
    q = q.astype(np.complex128)
    q /= np.linalg.norm(q)
    Q = [q]
    alpha, beta = [], []
    e_old = None
    m = min(m, n)
    for it in range(m):
        w = H @ Q[-1]
        a = float(np.real(np.vdot(Q[-1], w)))
        alpha.append(a)
        w = w - a * Q[-1] - (beta[-1] * Q[-2] if beta else 0.0)
        for qq in Q:                       # full re-orthogonalisation
            w = w - np.vdot(qq, w) * qq
        b = float(np.linalg.norm(w))
        T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
        ev, evec = np.linalg.eigh(T)
        if e_old is not None and abs(ev[0] - e_old) < tol * max(1.0, abs(ev[0])) and it > 5:
            break
        e_old = ev[0]
        if b < 1e-12:
            break
        beta.append(b)
        Q.append(w / b)
    T = np.diag(alpha) + np.diag(beta[:len(alpha) - 1], 1) + np.diag(beta[:len(alpha) - 1], -1)
    ev, evec = np.linalg.eigh(T)
    vec = sum(evec[i, 0] * Q[i] for i in range(len(alpha)))
    return float(ev[0]), vec / np.linalg.norm(vec)


# ---------------------------------------------------------------------------
# initial states
# ---------------------------------------------------------------------------

def orbitals(model: Model, perturb=None):
    """Occupied orbitals of the one-body matrix h = -t (diagonal -t_ii),
    plus an optional symmetric perturbation; returns (Phi_up, Phi_dn, eps).

    Gauge: each eigenvector's entry of largest magnitude (lowest index on a
    tie within 1e-12) is made positive.
    """
    h = -np.array(model.t, dtype=np.float64)
    if perturb is not None:
        h = h + np.asarray(perturb, dtype=np.float64)
    w, v = np.linalg.eigh(h)
    for k in range(v.shape[1]):
        col = v[:, k]
        mags = np.abs(col)
        i = int(np.flatnonzero(mags >= mags.max() - 1e-12)[0])
        if col[i] < 0:
            v[:, k] = -col
    return v[:, :model.n_up].copy(), v[:, :model.n_dn].copy(), w


def _apply_orbital_creation(model, coeffs, spin_modes, vec, basis_from, basis_to):
    out = np.zeros(len(basis_to), dtype=np.complex128)
    for i, c in enumerate(coeffs):
        if c == 0.0:
            continue
        valid, sign, z = create(basis_from, int(spin_modes[i]))
        rows = _lookup(basis_to, z[valid])
        np.add.at(out, rows, c * sign[valid] * vec[valid])
    return out


def slater_state(model: Model, Phi_up, Phi_dn) -> np.ndarray:
    """prod_m b+_{m,up} prod_m b+_{m,dn} |vac> on the sector basis, built by
    applying orbital creation operators b+ = sum_i Phi_im a+_{mode(i)} to the
    vacuum, rightmost first."""
    vec = np.array([1.0 + 0j])
    basis = np.array([0], dtype=np.uint64)
    nu, nd = Phi_up.shape[1], Phi_dn.shape[1]
    for m in reversed(range(nd)):
        nb = sector_basis(model, 0, nd - m)
        vec = _apply_orbital_creation(model, Phi_dn[:, m], model.dn, vec, basis, nb)
        basis = nb
    for m in reversed(range(nu)):
        nb = sector_basis(model, nu - m, nd)
        vec = _apply_orbital_creation(model, Phi_up[:, m], model.up, vec, basis, nb)
        basis = nb
    return vec


def neel_state(model: Model, lat: Lattice, basis: np.ndarray) -> np.ndarray:
    """Checkerboard product state (Sec. 2.1): up on sites with x+y even."""
    x0 = 0
    for s, (x, y) in enumerate(lat.coords):
        x0 |= 1 << int(model.up[s] if (x + y) % 2 == 0 else model.dn[s])
    psi = np.zeros(len(basis), dtype=np.complex128)
    psi[_lookup(basis, np.array([x0], dtype=np.uint64))[0]] = 1.0
    return psi


# ---------------------------------------------------------------------------
# closed forms used as pins
# ---------------------------------------------------------------------------

def hartree_fock_energy(model: Model, Phi_up, Phi_dn) -> float:
    """<SD|H|SD> by Wick's theorem for real orbitals."""
    ru = Phi_up @ Phi_up.T
    rd = Phi_dn @ Phi_dn.T
    h = -model.t
    e = float(np.sum(h * ru) + np.sum(h * rd))
    e += float(np.sum(model.U * np.diag(ru) * np.diag(rd)))
    L = model.n_sites
    for i in range(L):
        for j in range(i + 1, L):
            if model.V[i, j] != 0.0:
                e += model.V[i, j] * ((ru[i, i] + rd[i, i]) * (ru[j, j] + rd[j, j])
                                      - ru[i, j] ** 2 - rd[i, j] ** 2)
    return e


def neel_energy(model: Model) -> float:
    """<Neel|H|Neel>: each site singly occupied, no hopping expectation."""
    L = model.n_sites
    e = -float(np.trace(model.t))
    for i in range(L):
        for j in range(i + 1, L):
            e += model.V[i, j]
    return e


def u0_ground_energy(model: Model) -> float:
    """U = V = 0 ground energy: sum of the lowest one-body levels per spin."""
    w = np.linalg.eigvalsh(-model.t)
    return float(np.sum(w[:model.n_up]) + np.sum(w[:model.n_dn]))
