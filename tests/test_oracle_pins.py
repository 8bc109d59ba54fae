"""Pins of the CPU oracle against facts fixed outside it: closed forms,
the paper's printed gate matrices, invariants, brute force and library
routines.  CPU only; each test names the passage or the mathematics it uses.
"""

import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse.linalg

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _closed_forms():
    rows = []
    with open(os.path.join(GOLD, "closed_forms.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------------------
# Kronecker-product Jordan-Wigner (independent construction of a_k)
# ---------------------------------------------------------------------------

def _kron_annihilator(n, k):
    """a_k = Z x ... x Z (qubits below k) x sigma^- (qubit k) x I (above),
    with qubit j = bit j of the basis index."""
    Z = np.diag([1.0, -1.0])
    I = np.eye(2)
    sm = np.array([[0.0, 1.0], [0.0, 0.0]])   # |0><1|
    M = np.ones((1, 1))
    for j in range(n - 1, -1, -1):
        M = np.kron(M, I if j > k else (sm if j == k else Z))
    return M


def test_jw_operators_match_kronecker_construction_and_car():
    n = 5
    lat = O.square_lattice(1, 3)  # unused geometry; n modes from a map below
    basis = np.arange(1 << n, dtype=np.uint64)
    A = [_kron_annihilator(n, k) for k in range(n)]
    # CAR: {a_i, a_j^+} = delta_ij, {a_i, a_j} = 0
    for i in range(n):
        for j in range(n):
            ac = A[i] @ A[j].T + A[j].T @ A[i]
            assert np.allclose(ac, np.eye(1 << n) * (i == j))
            assert np.allclose(A[i] @ A[j] + A[j] @ A[i], 0)
    # the oracle's hop matrices equal a+_p a_q + a+_q a_p from the Kronecker form
    for p in range(n):
        for q in range(p + 1, n):
            ref = A[p].T @ A[q] + A[q].T @ A[p]
            got = O.hop_matrix(basis, p, q).toarray()
            assert np.array_equal(got, ref)
    for k in range(n):
        assert np.array_equal(np.diag(O.number_diag(basis, k)), A[k].T @ A[k])
    del lat


# ---------------------------------------------------------------------------
# Hamiltonian closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("row", [r for r in _closed_forms() if r[0] == "two_site"])
def test_two_site_ground_energy(row):
    U, t, E0 = float(row[1]), float(row[2]), float(row[3])
    assert abs(E0 - (U - math.sqrt(U * U + 16 * t * t)) / 2) < 1e-11
    lat = O.square_lattice(1, 2)
    m = O.make_model(lat, t, U, n_up=1, n_dn=1)
    b = O.sector_basis(m)
    H = O.hamiltonian(m, b)
    w = np.linalg.eigvalsh(H.toarray())
    assert abs(w[0] - E0) < 1e-11
    e_l, _ = O.lanczos_ground(H)
    assert abs(e_l - E0) < 1e-11


@pytest.mark.parametrize("row", [r for r in _closed_forms() if r[0] == "u0_open_grid"])
def test_u0_energy_equals_sum_of_levels(row):
    A, B, nu, nd, t, E0 = int(row[1]), int(row[2]), int(row[3]), int(row[4]), float(row[5]), float(row[6])
    levels = sorted(-2 * t * math.cos(k * math.pi / (A + 1)) - 2 * t * math.cos(m * math.pi / (B + 1))
                    for k in range(1, A + 1) for m in range(1, B + 1))
    assert abs(sum(levels[:nu]) + sum(levels[:nd]) - E0) < 1e-11
    lat = O.square_lattice(A, B)
    m = O.make_model(lat, t, 0.0, n_up=nu, n_dn=nd)
    assert abs(O.u0_ground_energy(m) - E0) < 1e-10
    b = O.sector_basis(m)
    H = O.hamiltonian(m, b)
    e_l, _ = O.lanczos_ground(H)
    assert abs(e_l - E0) < 1e-9 * abs(E0)


def test_hamiltonian_hermitian_and_sector_dimension():
    lat = O.square_lattice(2, 3)
    rng = np.random.default_rng(0)
    t = np.zeros((6, 6))
    for (i, j) in lat.bonds:
        t[i, j] = t[j, i] = 1 + 0.1 * rng.standard_normal()
    np.fill_diagonal(t, 0.2 * rng.standard_normal(6))
    m = O.make_model(lat, t, 4 * (1 + 0.1 * rng.standard_normal(6)), V=0.5, n_up=3, n_dn=2)
    b = O.sector_basis(m)
    assert len(b) == math.comb(6, 3) * math.comb(6, 2)
    H = O.hamiltonian(m, b)
    assert abs(H - H.getH()).max() == 0.0


def test_dense_full_space_diagonalisation_matches_sector_lanczos():
    """Brute force at 12 qubits: the full-space ground state of the (3,3)
    sector, from a dense eigh of H over all 4096 states, equals Lanczos."""
    lat = O.square_lattice(1, 6)
    m = O.make_model(lat, 1.0, 2.0, n_up=3, n_dn=3)
    full = O.full_basis(m)
    Hf = O.hamiltonian(m, full).toarray()
    n_u = O.popcount(full & np.uint64((1 << 6) - 1))
    n_d = O.popcount(full >> np.uint64(6))
    # H commutes with N_up and N_dn: no matrix element between sectors
    diff = (n_u[:, None] != n_u[None, :]) | (n_d[:, None] != n_d[None, :])
    assert np.all(Hf[diff] == 0)
    sel = (n_u == 3) & (n_d == 3)
    w = np.linalg.eigvalsh(Hf[np.ix_(sel, sel)])
    b = O.sector_basis(m)
    e_l, _ = O.lanczos_ground(O.hamiltonian(m, b))
    assert abs(e_l - w[0]) < 1e-10
    e_a = scipy.sparse.linalg.eigsh(O.hamiltonian(m, b), k=1, which="SA")[0][0]
    assert abs(e_a - w[0]) < 1e-10


# ---------------------------------------------------------------------------
# gates (Eqs. 8, 9) and the FSWAP network (Sec. 2.2.1, Fig. 2)
# ---------------------------------------------------------------------------

def _paper_gates(theta, phi):
    mats, cur = {}, None
    env = {"cos": math.cos, "sin": math.sin, "exp": np.exp, "theta": theta, "phi": phi}
    with open(os.path.join(GOLD, "paper_gates.txt")) as f:
        for line in f:
            s = line.strip()
            if not s or s.startswith("#"):
                continue
            if s in ("NP", "FSWAP", "EP"):
                cur = s
                mats[cur] = []
            else:
                mats[cur].append([complex(eval(tok, {}, env)) for tok in s.split()])
    return {k: np.array(v) for k, v in mats.items()}


def _two_qubit(n, j, G4):
    """Embed a 4x4 gate on qubits (j, j+1); index within = 2*b_{j+1} + b_j."""
    return np.kron(np.kron(np.eye(1 << (n - j - 2)), G4), np.eye(1 << j))


def _fermion_np(n, p, q, theta, phi):
    """exp(-i theta G_hop) exp(+i phi n_p n_q) on the full space, G_hop =
    -(a+_p a_q + h.c.) (t = 1), from the oracle's operators."""
    basis = np.arange(1 << n, dtype=np.uint64)
    T = O.hop_matrix(basis, p, q).toarray()
    npq = O.number_diag(basis, p) * O.number_diag(basis, q)
    return scipy.linalg.expm(1j * theta * T) @ np.diag(np.exp(1j * phi * npq))


def test_np_gate_is_givens_times_cphase_on_adjacent_modes():
    th, ph = 0.37, -1.21
    G = _paper_gates(th, ph)
    got = _fermion_np(2, 0, 1, th, ph)
    assert np.allclose(got, G["NP"], atol=1e-14)
    # the oracle's single hop term exponential (t = 1) is the NP gate at phi = 0
    lat = O.square_lattice(1, 2)
    m = O.make_model(lat, 1.0, 0.0, modes=(np.array([0, 1]), np.array([2, 3])))
    basis = np.arange(4, dtype=np.uint64)
    grp = O.Group("hop", ((0, 1),), 0)
    cols = []
    for k in range(4):
        e = np.zeros(4, dtype=complex)
        e[k] = 1
        cols.append(O.apply_group(m, basis, grp, th, e))
    assert np.allclose(np.array(cols).T, _paper_gates(th, 0.0)["NP"], atol=1e-14)


def test_fswap_network_equals_parity_signed_givens():
    """NP between modes 0 and 3 through FSWAPs (qubit gates on neighbours)
    equals the fermionic exponential with the Jordan-Wigner string."""
    n, th, ph = 4, 0.61, 0.29
    G = _paper_gates(th, ph)
    F = G["FSWAP"]
    fsw = lambda j: _two_qubit(n, j, F)
    net = fsw(2) @ fsw(1) @ _two_qubit(n, 0, G["NP"]) @ fsw(1) @ fsw(2)
    ref = _fermion_np(n, 0, 3, th, ph)
    assert np.allclose(net, ref, atol=1e-13)
    # the same network with plain (bosonic) SWAPs drops the string sign and
    # gives a different operator: the sign is not optional
    S = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex)
    sw = lambda j: _two_qubit(n, j, S)
    naive = sw(2) @ sw(1) @ _two_qubit(n, 0, G["NP"]) @ sw(1) @ sw(2)
    assert not np.allclose(naive, ref, atol=1e-3)


# ---------------------------------------------------------------------------
# ansatz: term products vs matrix exponentials, invariants
# ---------------------------------------------------------------------------

def _model_2x3(V=0.5, modes="blocked", order="rowmajor"):
    lat = O.square_lattice(2, 3, order)
    rng = np.random.default_rng(11)
    t = np.zeros((6, 6))
    for (i, j) in lat.bonds:
        t[i, j] = t[j, i] = 1 + 0.1 * rng.standard_normal()
    np.fill_diagonal(t, 0.3 * rng.standard_normal(6))
    U = 4 * (1 + 0.1 * rng.standard_normal(6))
    return lat, O.make_model(lat, t, U, V=V, n_up=3, n_dn=3, modes=modes)


def test_group_product_equals_expm_of_generator():
    lat, m = _model_2x3()
    b = O.sector_basis(m)
    rng = np.random.default_rng(3)
    psi = rng.standard_normal(len(b)) + 1j * rng.standard_normal(len(b))
    psi /= np.linalg.norm(psi)
    groups = O.hva_groups(lat, 1, ["U", "V", "eps", "h1", "v1", "h2"])
    for g in groups:
        th = rng.uniform(-np.pi, np.pi)
        Gmat = np.zeros((len(b), len(b)), dtype=complex)
        for k in range(len(b)):
            e = np.zeros(len(b), dtype=complex)
            e[k] = 1
            Gmat[:, k] = O.apply_generator(m, b, g, e)
        ref = scipy.linalg.expm(-1j * th * Gmat) @ psi
        got = O.apply_group(m, b, g, th, psi)
        assert np.allclose(got, ref, atol=1e-12), g.kind
        back = O.apply_group(m, b, g, th, got, inverse=True)
        assert np.allclose(back, psi, atol=1e-12)


def test_norm_and_particle_numbers_conserved_in_full_space():
    lat = O.square_lattice(2, 2)
    m = O.make_model(lat, 1.0, 3.0, V=0.4, n_up=2, n_dn=1)
    full = O.full_basis(m)
    sec = O.sector_basis(m)
    pu, pd, _ = O.orbitals(m)
    psi_s = O.slater_state(m, pu, pd)
    psi = np.zeros(len(full), dtype=complex)
    psi[sec.astype(np.int64)] = psi_s
    groups = O.hva_groups(lat, 3, ["U", "V", "h1", "v1"])
    theta = np.random.default_rng(5).uniform(-np.pi, np.pi, 12)
    out = O.ansatz_state(m, full, groups, theta, psi)
    mask = np.ones(len(full), bool)
    mask[sec.astype(np.int64)] = False
    assert np.all(out[mask] == 0)          # exactly: no amplitude leaves
    assert abs(np.linalg.norm(out) - 1) < 1e-13


def test_adjoint_gradient_matches_central_differences():
    lat, m = _model_2x3()
    b = O.sector_basis(m)
    pu, pd, _ = O.orbitals(m)
    psi0 = O.slater_state(m, pu, pd)
    H = O.hamiltonian(m, b)
    groups = O.hva_groups(lat, 2, ["U", "V", "h1", "v1", "h2", "v2"])
    theta = np.random.default_rng(2).uniform(-np.pi, np.pi, 12)
    E, g = O.energy_and_gradient(m, b, groups, theta, psi0, H)
    gf = O.fd_gradient(m, b, groups, theta, psi0, h=1e-4, H=H)
    assert np.max(np.abs(g - gf)) < 1e-7 * max(1.0, np.max(np.abs(g)))
    assert g[5] == 0.0 and g[11] == 0.0    # v2 is empty on a 2-row lattice
    assert abs(E - O.energy(m, b, groups, theta, psi0, H)) < 1e-12


def test_variational_bound_and_lanczos():
    lat, m = _model_2x3()
    b = O.sector_basis(m)
    H = O.hamiltonian(m, b)
    e0, v0 = O.lanczos_ground(H)
    w = np.linalg.eigvalsh(H.toarray())
    assert abs(e0 - w[0]) < 1e-10
    assert np.linalg.norm(H @ v0 - e0 * v0) < 1e-6
    pu, pd, _ = O.orbitals(m)
    psi0 = O.slater_state(m, pu, pd)
    groups = O.hva_groups(lat, 2, ["U", "V", "h1", "v1", "h2"])
    rng = np.random.default_rng(9)
    for _ in range(5):
        th = rng.uniform(-np.pi, np.pi, 10)
        assert O.energy(m, b, groups, th, psi0, H) >= e0 - 1e-12


def test_periodicity_for_integer_generators():
    """Uniform t = 1 gives hop generators with integer spectra (period 2 pi);
    uniform integer U gives period 2 pi / U for the on-site parameter."""
    lat = O.square_lattice(2, 3)
    m = O.make_model(lat, 1.0, 4.0, n_up=3, n_dn=3)
    b = O.sector_basis(m)
    pu, pd, _ = O.orbitals(m, perturb=np.diag(1e-3 * np.arange(6)))
    psi0 = O.slater_state(m, pu, pd)
    H = O.hamiltonian(m, b)
    groups = O.hva_groups(lat, 2, ["U", "h1", "v1", "h2"])
    th = np.random.default_rng(4).uniform(-np.pi, np.pi, 8)
    e = O.energy(m, b, groups, th, psi0, H)
    for k, period in [(0, 2 * np.pi / 4.0), (1, 2 * np.pi), (2, 2 * np.pi), (7, 2 * np.pi)]:
        t2 = th.copy()
        t2[k] += period
        assert abs(O.energy(m, b, groups, t2, psi0, H) - e) < 1e-11
    t2 = th.copy()
    t2[0] += np.pi / 4.0        # half a period moves the energy
    assert abs(O.energy(m, b, groups, t2, psi0, H) - e) > 1e-6


def _generator_sum_residual(m, b, groups, vec, terms_fn=None):
    """|| sum_g G_g vec - H vec || / || H vec || over one layer of groups.

    Under the reading that each generator is its class's Hamiltonian terms
    with their coefficients and signs (Sec. 2.2.1: the HVA layer of Eq. 7
    exponentiates the terms of the Hamiltonian), the generators of one layer
    that covers every term class (on-site U, NN V, potential, and every
    hopping class) add up to H exactly.  H itself is pinned by the closed
    forms above (two-site dimer, U = 0 levels, Neel and Hartree-Fock
    energies) and by the Kronecker-product Jordan-Wigner construction."""
    cache = {}
    if terms_fn is None:
        acc = sum(O.apply_generator(m, b, g, vec, cache) for g in groups)
    else:
        acc = np.zeros_like(vec)
        for g in groups:
            for piece in terms_fn(m, b, g):
                acc = acc + (piece[1] * (piece[2] @ vec) if piece[0] == "hop" else piece[1] * vec)
    ref = O.hamiltonian(m, b) @ vec
    return float(np.linalg.norm(acc - ref) / np.linalg.norm(ref))


def test_layer_generators_sum_to_hamiltonian():
    """Every group kind's generator carries exactly its Hamiltonian terms:
    one layer over all term classes sums to H (disordered t, on-site
    potential, site-dependent U and bond-dependent V, both JW orders)."""
    for modes in ("blocked", "interleaved"):
        lat, m = _model_2x3(modes=modes)
        rng = np.random.default_rng(21)
        Vm = np.zeros((6, 6))
        for (i, j) in lat.bonds:
            Vm[i, j] = Vm[j, i] = 0.5 + 0.3 * rng.standard_normal()
        m = O.make_model(lat, m.t, m.U, V=Vm, n_up=3, n_dn=2, modes=modes)
        b = O.sector_basis(m)
        vec = rng.standard_normal(len(b)) + 1j * rng.standard_normal(len(b))
        groups = O.hva_groups(lat, 1, ["U", "V", "eps", "h1", "v1", "h2", "v2"])
        assert _generator_sum_residual(m, b, groups, vec) < 1e-13


def test_energy_period_in_theta_V_is_two_pi_over_V():
    """Uniform integer V: G_V = V sum n_i n_j has eigenvalues V x (integer),
    so E is 2 pi / V-periodic in theta_V, and (generically) not pi /
    V-periodic -- which a doubled V coefficient would make it."""
    lat = O.square_lattice(2, 3)
    m = O.make_model(lat, 1.0, 4.0, V=2.0, n_up=3, n_dn=3)
    b = O.sector_basis(m)
    pu, pd, _ = O.orbitals(m, perturb=np.diag(1e-3 * np.arange(6)))
    psi0 = O.slater_state(m, pu, pd)
    H = O.hamiltonian(m, b)
    groups = O.hva_groups(lat, 2, ["U", "V", "h1", "v1", "h2"])
    th = np.random.default_rng(8).uniform(-np.pi, np.pi, 10)
    e = O.energy(m, b, groups, th, psi0, H)
    for k in (1, 6):                       # the V parameter of each layer
        t2 = th.copy()
        t2[k] += 2 * np.pi / 2.0
        assert abs(O.energy(m, b, groups, t2, psi0, H) - e) < 1e-11
        t2 = th.copy()
        t2[k] += np.pi / 2.0
        assert abs(O.energy(m, b, groups, t2, psi0, H) - e) > 1e-6


def _kron_rz_product(n, theta):
    """prod_k exp(-i theta Z_k / 2) in the full 2^n space, qubit k = bit k,
    Z = diag(1, -1) on (|0>, |1>): the textbook single-qubit R_z(theta)."""
    rz = np.diag([np.exp(-0.5j * theta), np.exp(0.5j * theta)])
    M = np.ones((1, 1), dtype=complex)
    for _ in range(n):
        M = np.kron(M, rz)
    return M


def test_rz_group_equals_product_of_single_qubit_rotations():
    """The 'rz' group (the R_z pre-layer of Sec. 2.2.1) is exp(-i theta
    sum_k Z_k / 2) = prod_k R_z(theta) on its modes, global phase included
    (checked against Kronecker products in the full space, on all modes and
    on a subset)."""
    lat = O.square_lattice(1, 3)
    m = O.make_model(lat, 1.0, 2.0)
    n = m.n_modes
    b = O.full_basis(m)
    rng = np.random.default_rng(9)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    th = 0.7311
    got = O.apply_group(m, b, O.Group("rz", tuple(range(n)), 0), th, psi)
    assert np.allclose(got, _kron_rz_product(n, th) @ psi, atol=1e-13)
    # a subset of modes: R_z on modes 1 and 4 only
    I2 = np.eye(2)
    rz = np.diag([np.exp(-0.5j * th), np.exp(0.5j * th)])
    M = np.ones((1, 1), dtype=complex)
    for k in range(n - 1, -1, -1):
        M = np.kron(M, rz if k in (1, 4) else I2)
    got = O.apply_group(m, b, O.Group("rz", (1, 4), 0), th, psi)
    assert np.allclose(got, M @ psi, atol=1e-13)


def test_energy_and_gradient_invariant_under_mode_order():
    """Blocked, interleaved (the paper's) and snake site orders describe the
    same fermions: E and the gradient agree."""
    th = np.random.default_rng(8).uniform(-np.pi, np.pi, 12)
    res = []
    for modes, order in [("blocked", "rowmajor"), ("interleaved", "rowmajor"), ("blocked", "snake")]:
        lat = O.square_lattice(2, 3, order)
        # physical coefficients keyed by coordinates, identical in every order
        rng = np.random.default_rng(21)
        tb = {}
        for x in range(2):
            for y in range(3):
                for (dx, dy) in [(0, 1), (1, 0)]:
                    if x + dx < 2 and y + dy < 3:
                        tb[((x, y), (x + dx, y + dy))] = 1 + 0.1 * rng.standard_normal()
        Uc = {(x, y): 4 + 0.3 * rng.standard_normal() for x in range(2) for y in range(3)}
        idx = {c: s for s, c in enumerate(lat.coords)}
        t = np.zeros((6, 6))
        for (a, c), v in tb.items():
            t[idx[a], idx[c]] = t[idx[c], idx[a]] = v
        U = np.array([Uc[lat.coords[s]] for s in range(6)])
        m = O.make_model(lat, t, U, V=0.3, n_up=3, n_dn=3, modes=modes)
        b = O.sector_basis(m)
        pu, pd, _ = O.orbitals(m)
        psi0 = O.slater_state(m, pu, pd)
        groups = O.hva_groups(lat, 2, ["U", "V", "h1", "v1", "h2", "v2"])
        res.append(O.energy_and_gradient(m, b, groups, th, psi0))
    for E, g in res[1:]:
        assert abs(E - res[0][0]) < 1e-11
        assert np.allclose(g, res[0][1], atol=1e-10)


def test_slater_energy_equals_hartree_fock_closed_form():
    lat, m = _model_2x3()
    b = O.sector_basis(m)
    pert = np.random.default_rng(6).standard_normal((6, 6))
    pu, pd, _ = O.orbitals(m, perturb=1e-3 * (pert + pert.T) / 2)
    psi0 = O.slater_state(m, pu, pd)
    assert abs(np.linalg.norm(psi0) - 1) < 1e-13
    H = O.hamiltonian(m, b)
    assert abs(np.vdot(psi0, H @ psi0).real - O.hartree_fock_energy(m, pu, pd)) < 1e-12
    # at U = V = 0 the Slater determinant of the lowest levels is the ground state
    m0 = O.make_model(lat, m.t, 0.0, n_up=3, n_dn=3)
    pu0, pd0, _ = O.orbitals(m0)
    psi00 = O.slater_state(m0, pu0, pd0)
    b0 = O.sector_basis(m0)
    assert abs(np.vdot(psi00, O.hamiltonian(m0, b0) @ psi00).real - O.u0_ground_energy(m0)) < 1e-12


def test_slater_amplitudes_are_determinants_in_blocked_order():
    """psi0(x) = det(Phi_up[occ_up]) det(Phi_dn[occ_dn]) when every up mode
    precedes every down mode (the creation order is already ascending)."""
    lat, m = _model_2x3()
    b = O.sector_basis(m)
    pu, pd, _ = O.orbitals(m)
    psi0 = O.slater_state(m, pu, pd)
    for k in range(0, len(b), 37):
        x = int(b[k])
        ou = [i for i in range(6) if (x >> int(m.up[i])) & 1]
        od = [i for i in range(6) if (x >> int(m.dn[i])) & 1]
        ref = np.linalg.det(pu[ou, :]) * np.linalg.det(pd[od, :])
        assert abs(psi0[k] - ref) < 1e-13


def test_neel_energy_closed_form():
    lat, m = _model_2x3()
    b = O.sector_basis(m)
    psi = O.neel_state(m, lat, b)
    H = O.hamiltonian(m, b)
    assert abs(np.vdot(psi, H @ psi).real - O.neel_energy(m)) < 1e-12


def test_mistakes_are_caught():
    """Plant plausible mistakes in oracle pieces and check a pin fails."""
    lat = O.square_lattice(2, 4)
    m = O.make_model(lat, 1.0, 0.0)
    b = O.sector_basis(m)
    E0 = O.u0_ground_energy(m)
    # (1) drop the Jordan-Wigner string: hop matrices without signs
    H = O.hamiltonian(m, b).tocoo()
    Hbad = H.copy()
    Hbad.data = np.where(Hbad.row != Hbad.col, -np.abs(Hbad.data), Hbad.data)
    e_bad, _ = O.lanczos_ground(Hbad.tocsr())
    assert abs(e_bad - E0) > 1e-3
    # (2) wrong sign of the hopping term leaves U=0 energies intact on a
    #     bipartite lattice, but the two-site U > 0 dimer still fixes E0
    #     through sqrt(U^2 + 16 t^2), and the gradient sign convention is
    #     fixed by FD (tests above).  A wrong factor does not survive:
    e_half, _ = O.lanczos_ground((0.5 * O.hamiltonian(m, b)).tocsr())
    assert abs(e_half - E0) > 1e-3
    # (3) coefficient slips in the generators of the diagonal groups and of
    #     the hops: each fails the layer-sum pin or the R_z pin
    lat2, m2 = _model_2x3()
    b2 = O.sector_basis(m2)
    rng = np.random.default_rng(22)
    vec = rng.standard_normal(len(b2)) + 1j * rng.standard_normal(len(b2))
    groups = O.hva_groups(lat2, 1, ["U", "V", "eps", "h1", "v1", "h2", "v2"])

    def slipped(kind, f):
        def terms(mm, bb, g):
            pieces = O.group_terms(mm, bb, g)
            if g.kind != kind:
                return pieces
            return [f(p) for p in pieces]
        return terms

    for kind, f in [("nn_v", lambda p: ("diag", 2.0 * p[1])),
                    ("eps", lambda p: ("diag", -p[1])),
                    ("onsite_u", lambda p: ("diag", 0.5 * p[1])),
                    ("hop", lambda p: ("hop", -p[1], p[2]))]:
        assert _generator_sum_residual(m2, b2, groups, vec, slipped(kind, f)) > 1e-3, kind
    assert _generator_sum_residual(m2, b2, groups, vec) < 1e-13
    # an R_z generator missing its constant 1/2, or with the wrong sign
    lat3 = O.square_lattice(1, 3)
    m3 = O.make_model(lat3, 1.0, 2.0)
    b3 = O.full_basis(m3)
    psi = rng.standard_normal(1 << 6) + 1j * rng.standard_normal(1 << 6)
    ref = _kron_rz_product(6, 0.7311) @ psi
    g = O.Group("rz", tuple(range(6)), 0)
    d = O.group_terms(m3, b3, g)[0][1]
    for bad in (d - 3.0, -d):              # constant dropped (sum of 6 halves), sign flipped
        got = np.exp(-1j * 0.7311 * bad) * psi
        assert not np.allclose(got, ref, atol=1e-6)


# ---------------------------------------------------------------------------
# overlap loss (Eq. 5), fidelity and spin correlations (Sec. 3)
# ---------------------------------------------------------------------------

def test_overlap_loss_two_site_closed_form():
    """One up electron on a two-site chain, one hop factor exp(-i theta G)
    with G = -(a+_0 a_1 + h.c.): psi = cos(theta)|0> + i sin(theta)|1> (up to
    the sign of the second amplitude), so with the reference on site 1,
    F = sin^2 theta, f = log10(cos^2 theta), df/dtheta = -2 tan(theta)/ln 10."""
    lat = O.square_lattice(1, 2)
    m = O.make_model(lat, 1.0, 0.0, n_up=1, n_dn=0)
    b = O.sector_basis(m)
    assert list(b) == [1, 2]
    psi0 = np.array([1.0 + 0j, 0.0])
    ref = np.array([0.0 + 0j, 1.0])
    groups = [O.Group("hop", ((0, 1),), 0)]
    for th in (0.3, -1.1, 0.77):
        F, f, g = O.overlap_loss_and_gradient(m, b, groups, np.array([th]), psi0, ref)
        assert abs(F - math.sin(th) ** 2) < 1e-15
        assert abs(f - math.log10(math.cos(th) ** 2)) < 1e-14
        assert abs(g[0] + 2 * math.tan(th) / math.log(10.0)) < 1e-13


def test_overlap_gradient_matches_central_differences():
    lat, m = _model_2x3()
    b = O.sector_basis(m)
    H = O.hamiltonian(m, b)
    _, ref = O.lanczos_ground(H)
    pu, pd, _ = O.orbitals(m)
    psi0 = O.slater_state(m, pu, pd)
    groups = O.hva_groups(lat, 2, ["U", "V", "eps", "h1", "v1", "h2"])
    th = np.random.default_rng(12).uniform(-1, 1, 12)
    F, f, g = O.overlap_loss_and_gradient(m, b, groups, th, psi0, ref)
    assert 0.0 < F < 1.0
    fd = O.overlap_fd_gradient(m, b, groups, th, psi0, ref, h=1e-5)
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(g)))
    # the reference taken as psi(theta') itself: F(theta') = 1 exactly
    ref2 = O.ansatz_state(m, b, groups, th, psi0)
    assert abs(O.fidelity(O.ansatz_state(m, b, groups, th, psi0), ref2) - 1.0) < 1e-13


def test_spin_correlation_closed_forms_and_sum_rule():
    """Two-site Hubbard ground state (one electron per spin): in the basis of
    the covalent and ionic singlets, H = [[0, -2t], [-2t, U]], so with E0 its
    lowest eigenvalue the covalent weight is w = 1 / (1 + E0^2 / (4 t^2)),
    <S^z_0 S^z_1> = -w / 4, <S^z_i> = 0 and C_00 = C_11 = w / 4.  On any
    state of a fixed (N_up, N_dn) sector S^z_total is a constant, so every
    row of C sums to zero; a product (Neel) state has C = 0."""
    lat = O.square_lattice(1, 2)
    for U in (4.0, 8.0):
        m = O.make_model(lat, 1.0, U, n_up=1, n_dn=1)
        b = O.sector_basis(m)
        e0, v = O.lanczos_ground(O.hamiltonian(m, b))
        assert abs(e0 - (U - math.sqrt(U * U + 16)) / 2) < 1e-12
        w = 1.0 / (1.0 + e0 * e0 / 4.0)
        C = O.spin_correlation(m, b, v)
        assert np.allclose(C, [[w / 4, -w / 4], [-w / 4, w / 4]], atol=1e-12)
    lat, m = _model_2x3()
    b = O.sector_basis(m)
    rng = np.random.default_rng(13)
    v = rng.standard_normal(len(b)) + 1j * rng.standard_normal(len(b))
    v /= np.linalg.norm(v)
    C = O.spin_correlation(m, b, v)
    assert np.allclose(C, C.T, atol=1e-14)
    assert np.max(np.abs(C.sum(axis=1))) < 1e-13
    psi = O.neel_state(m, lat, b)
    assert np.max(np.abs(O.spin_correlation(m, b, psi))) < 1e-15


def test_overlap_and_correlation_mistakes_are_caught():
    """Planted mistakes: the adjoint vector not scaled by the overlap
    (lambda_K = psi_ref) fails the finite differences; charge instead of
    spin in C fails the two-site closed form."""
    lat, m = _model_2x3()
    b = O.sector_basis(m)
    _, ref = O.lanczos_ground(O.hamiltonian(m, b))
    pu, pd, _ = O.orbitals(m)
    psi0 = O.slater_state(m, pu, pd)
    groups = O.hva_groups(lat, 1, ["U", "h1", "v1", "h2"])
    th = np.random.default_rng(14).uniform(-1, 1, 4)
    F, _, _ = O.overlap_loss_and_gradient(m, b, groups, th, psi0, ref)
    psi = O.ansatz_state(m, b, groups, th, psi0)
    lam = ref.copy()                               # missing the factor <ref|psi_K>
    dF = np.zeros(4)
    for g in reversed(groups):
        dF[g.param] += 2.0 * float(np.imag(np.vdot(lam, O.apply_generator(m, b, g, psi))))
        psi = O.apply_group(m, b, g, th[g.param], psi, inverse=True)
        lam = O.apply_group(m, b, g, th[g.param], lam, inverse=True)
    bad = -dF / ((1.0 - F) * math.log(10.0))
    fd = O.overlap_fd_gradient(m, b, groups, th, psi0, ref)
    assert np.max(np.abs(bad - fd)) > 1e-3
    lat2 = O.square_lattice(1, 2)
    m2 = O.make_model(lat2, 1.0, 4.0, n_up=1, n_dn=1)
    b2 = O.sector_basis(m2)
    e0, v = O.lanczos_ground(O.hamiltonian(m2, b2))
    nu, nd = O.hubbard._site_occ(m2, b2)
    ch = 0.5 * (nu + nd)
    p = np.abs(v) ** 2
    Cbad = (ch * p) @ ch.T - np.outer(ch @ p, ch @ p)
    w = 1.0 / (1.0 + e0 * e0 / 4.0)
    assert abs(Cbad[0, 1] + w / 4) > 1e-2


# ---------------------------------------------------------------------------
# NP ansatz (Sec. 2.2.1, Eq. 8) and EP ansatz (Sec. 2.2.2, Eq. 10)
# ---------------------------------------------------------------------------

def _gate_of_groups(groups, thetas, n=2):
    """4x4 matrix of a product of oracle groups on a two-mode full space
    (basis order |00>, |01>, |10>, |11> with bit 0 = mode 0)."""
    lat = O.square_lattice(1, 1)
    m = O.make_model(lat, 0.0, 0.0, n_up=0, n_dn=0, modes=(np.array([0]), np.array([1])))
    basis = np.arange(1 << n, dtype=np.uint64)
    cols = []
    for k in range(1 << n):
        e = np.zeros(1 << n, dtype=complex)
        e[k] = 1
        for g in groups:
            e = O.apply_group(m, basis, g, thetas[g.param], e)
        cols.append(e)
    return np.array(cols).T


def test_np_and_ep_gates_from_groups_match_the_printed_matrices():
    th, ph = 0.43, -0.87
    np_groups = [O.Group("givens", ((0, 1),), 0), O.Group("cphase", ((0, 1),), 1)]
    assert np.allclose(_gate_of_groups(np_groups, [th, ph]), _paper_gates(th, ph)["NP"], atol=1e-14)
    # Eq. 10: U_EP(theta, phi) = givens(-theta/2) cphase(-phi)
    assert np.allclose(_gate_of_groups(np_groups, [-th / 2, -ph]), _paper_gates(th, ph)["EP"], atol=1e-14)


def test_np_and_ep_parameter_counts():
    """The paper prints 1,568 parameters for 12 NP layers on the 4x4 lattice
    (Sec. 3); the builders give the paper's counts for other sizes too."""
    lat = O.square_lattice(4, 4)
    m = O.make_model(lat, 1.0, 2.0)
    g = O.np_groups(lat, m, 12)
    assert max(x.param for x in g) + 1 == 1568 == O.np_param_count(4, 4, 12)
    for (nx, ny, layers) in [(2, 3, 1), (2, 3, 5), (3, 3, 13), (1, 6, 4)]:
        lat = O.square_lattice(nx, ny)
        m = O.make_model(lat, 1.0, 2.0)
        assert max(x.param for x in O.np_groups(lat, m, layers)) + 1 == O.np_param_count(nx, ny, layers)
        assert max(x.param for x in O.ep_groups(2 * nx * ny, layers)) + 1 == O.ep_param_count(nx, ny, layers)


def test_np_ansatz_conserves_total_number_and_mixes_spins():
    """The on-site NP gate's theta part moves an electron between the two
    spin modes of a site: N_up + N_dn is conserved, N_up alone is not.  The
    adjoint gradient in the total-N basis agrees with central differences."""
    lat = O.square_lattice(2, 2)
    m = O.make_model(lat, 1.0, 4.0, n_up=2, n_dn=2, modes="interleaved")
    b = O.number_basis(m, 4)
    sec = set(int(x) for x in O.sector_basis(m))
    pu, pd, _ = O.orbitals(m, perturb=np.diag(1e-3 * np.arange(4)))
    psi0_s = O.slater_state(m, pu, pd)
    psi0 = np.zeros(len(b), dtype=complex)
    idx = {int(x): i for i, x in enumerate(b)}
    for x, v in zip(O.sector_basis(m), psi0_s):
        psi0[idx[int(x)]] = v
    groups = O.np_groups(lat, m, 2)
    P = max(x.param for x in groups) + 1
    th = np.random.default_rng(31).uniform(-1, 1, P)
    psi = O.ansatz_state(m, b, groups, th, psi0)
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-13
    outside = sum(abs(psi[i]) ** 2 for i, x in enumerate(b) if int(x) not in sec)
    assert outside > 1e-3
    Hm = O.hamiltonian(m, b)
    E, g = O.energy_and_gradient(m, b, groups, th, psi0, Hm)
    fd = O.fd_gradient(m, b, groups, th, psi0, h=1e-5, H=Hm)
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(g)))
    # without the on-site theta (set to zero) the sector is kept exactly
    th2 = th.copy()
    for x in groups:
        if x.kind == "givens" and x.terms[0][1] - x.terms[0][0] == 1 and x.terms[0][0] % 2 == 0:
            th2[x.param] = 0.0
    psi2 = O.ansatz_state(m, b, groups, th2, psi0)
    assert sum(abs(psi2[i]) ** 2 for i, x in enumerate(b) if int(x) not in sec) < 1e-28
