/*
 * hubsv.h -- C ABI of the GB300 statevector engine for Hubbard-model VQE.
 *
 * The library applies the layered Hamiltonian variational ansatz (HVA) of
 * Eq. 7 (the PQC of Eq. 3) to a dense 2^n amplitude vector of the
 * Jordan-Wigner-mapped Fermi-Hubbard model (Eqs. 1, 2, 15, 16; one qubit per
 * spin-orbital, Sec. 2.2.1), and evaluates the energy of Eq. 4 and its
 * parameter gradient by the adjoint recursion of Sec. 2.1.  n <= 32 qubits.
 *
 * Conventions (fixed here because the paper leaves them open):
 *  - Qubit k of the amplitude index x is fermionic mode k.  a_k|x> =
 *    (-1)^popcount(x & (2^k - 1)) |x ^ 2^k> for occupied k; |x> = a+_{k1}
 *    a+_{k2}..|vac> with k1 < k2 < ...  The site -> mode maps are inputs
 *    (default: up spin of site i on mode i, down spin on mode L + i).
 *  - H = -sum_sigma sum_{i != j} t_ij a+_{i sigma} a_{j sigma}
 *        - sum_{i,sigma} t_ii n_{i sigma} + sum_i U_i n_{i up} n_{i dn}
 *        + sum_{i<j} V_ij n_i n_j,            n_i = n_{i up} + n_{i dn}.
 *    The hopping sum runs over both orders of each pair; the diagonal of t is
 *    the on-site potential of Eq. 15; each V pair is counted once.
 *  - Each ansatz group g applies U_g = exp(-i theta_p G_g) (the sign of the
 *    exponent is read as -i; Eq. 7 writes +i, which mirrors the landscape).
 *    G_g is the group's Hamiltonian terms with coefficients and signs:
 *      HUB_G_HOP     -sum_{(i,j) in terms} t_ij sum_sigma (a+_i a_j + h.c.)
 *      HUB_G_ONSITE  sum_{i in terms} U_i n_{i up} n_{i dn}
 *      HUB_G_NN_V    sum_{(i,j) in terms} V_ij n_i n_j
 *      HUB_G_POT     -sum_{i in terms} t_ii (n_{i up} + n_{i dn})
 *      HUB_G_RZ      sum_{k in terms} (1/2 - n_k)  (= Z_k / 2, modes k)
 *      HUB_G_GIVENS  -sum_{(p,q) in terms} (a+_p a_q + a+_q a_p)  (mode pairs)
 *      HUB_G_CPHASE  -sum_{(p,q) in terms} n_p n_q                (mode pairs)
 *    GIVENS and CPHASE build the number-preserving gate of Eq. 8 term by
 *    term (U_NP(theta, phi) on modes p, q = the GIVENS factor with theta
 *    times the CPHASE factor with phi; the NP ansatz of Sec. 2.2.1) and the
 *    gate of Eq. 10 (U_EP(theta, phi) = GIVENS(-theta/2) CPHASE(-phi); the
 *    EP ansatz of Sec. 2.2.2).  A GIVENS pair may join an up and a down mode
 *    (the on-site NP gate); then only N_up + N_dn is conserved and every
 *    call runs as dense sweeps over all tiles.
 *    The terms of one group must commute: hop bonds of a group touch
 *    disjoint sites, Givens pairs of a group disjoint modes.
 *  - Gradient: dE/dtheta_p = sum over groups g with parameter p of
 *    2 Im <lambda_g| G_g |psi_g>, psi_g the state after group g and
 *    lambda_g = U_{g+1}^+ ... U_K^+ H psi_K (Sec. 2.1, standard form of the
 *    recursion).
 *
 * Memory and streams: the caller owns every amplitude, parameter and output
 * buffer (device pointers unless stated).  The library owns its handles and
 * small device tables (gate lists, coefficient tables, Slater-determinant
 * tables, reduction scratch), which the destroy calls free.  Compute calls
 * are asynchronous on the given stream and never synchronise the device;
 * host-side argument checks return an error status before anything is
 * launched.  Launch errors are reported by the call; errors raised later by
 * the device are reported by the next call or by hub_sync.  The library
 * never aborts and never prints.  Amplitudes: HUB_C64 = interleaved float
 * (re, im), HUB_C128 = interleaved double; batch b occupies amplitudes
 * [b * 2^n, (b+1) * 2^n).  Amplitude buffers are aligned to their element
 * size (8 bytes for HUB_C64, 16 for HUB_C128; any device allocation is);
 * calls given one that is not return HUB_EINVAL before launching anything.
 * theta, energies and gradients are double in both
 * precisions; reductions accumulate in double.
 */
#ifndef HUBSV_H
#define HUBSV_H

#include <stdint.h>

#if defined(__GNUC__)
#define HUB_API __attribute__((visibility("default")))
#else
#define HUB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hub_model* hub_t;
typedef struct hub_ansatz* ans_t;
typedef struct CUstream_st* hub_stream_t;   /* == cudaStream_t; NULL = default */

typedef enum {
  HUB_OK = 0,
  HUB_EINVAL = 1,        /* bad argument: null pointer, size, index, group */
  HUB_EUNSUPPORTED = 2,  /* valid but outside what this build supports     */
  HUB_ENOMEM = 3,        /* a library-owned allocation failed              */
  HUB_ECUDA = 4,         /* a CUDA call or kernel launch failed            */
  HUB_ETIMEOUT = 5       /* reserved: a bounded device wait ran out (no    */
                         /* kernel of this build waits on another)         */
} hub_status;

typedef enum { HUB_C64 = 0, HUB_C128 = 1 } hub_dtype;

typedef enum {
  HUB_G_HOP = 0, HUB_G_ONSITE = 1, HUB_G_NN_V = 2, HUB_G_POT = 3, HUB_G_RZ = 4,
  HUB_G_GIVENS = 5, HUB_G_CPHASE = 6
} hub_gkind;

typedef enum { HUB_PREP_SLATER = 0, HUB_PREP_NEEL = 1 } hub_prep;

/* Flags of energy / energy_grad. */
#define HUB_FLAG_PREP_FUSED 1u   /* psi is workspace: the initial state is the
                                    one set by the last state_prepare call
                                    and is generated inside the first sweep   */
#define HUB_FLAG_KEEP_STATE 2u   /* energy: leave the final state psi_K in psi */
#define HUB_FLAG_SWEEPS     4u   /* run as HBM sweeps of the dense vector even
                                    where another engine applies (energy_grad) */
#define HUB_FLAG_ROWS       8u   /* skip the on-chip engine: run on the row
                                    engine where it applies (energy_grad)      */
#define HUB_FLAG_ROW_CLUSTER 16u /* row engine: stage each row of psi and its
                                    row of lam on a cluster of two CTAs, one
                                    row each, even where one CTA would hold
                                    both (the staging it uses for rows too
                                    large for one SM; for tests and tuning)  */

/* Lattice: sites 0..n_sites-1, undirected bonds (pairs of sites).  mode_up /
 * mode_dn map a site to its two qubits; both NULL = blocked order (up i -> i,
 * dn i -> n_sites + i).  Every mode in [0, 2 n_sites) must be used once.  */
typedef struct {
  int32_t n_sites;
  int32_t n_bonds;
  const int32_t* bonds;     /* [n_bonds][2], host */
  const int32_t* mode_up;   /* [n_sites] or NULL, host */
  const int32_t* mode_dn;   /* [n_sites] or NULL, host */
} hub_lattice;

/* One ansatz group (one factor of Eq. 7).  terms (host): bond indices of the
 * lattice for HOP and NN_V, site indices for ONSITE and POT, mode indices for
 * RZ; for GIVENS and CPHASE n_terms mode pairs, terms holding 2 * n_terms
 * ints (p0, q0, p1, q1, ...; at most 16 pairs in a CPHASE group).  param
 * indexes theta; groups may share a parameter.                              */
typedef struct {
  int32_t kind;             /* hub_gkind */
  int32_t n_terms;
  const int32_t* terms;
  int32_t param;
} hub_group;

/* Open nx x ny square lattice (Sec. 3: open boundary conditions) and its HVA
 * bond classes (Eq. 7).  Rows x = 0..nx-1, columns y = 0..ny-1; site number
 * x*ny + y (order 0, row-major as in Sec. 2.2.1) or with odd rows reversed
 * (order 1, "snake").  Bonds: all horizontal bonds in row order, then all
 * vertical ones; each stored with the smaller site first.  bond_class (may be
 * NULL): 0 = h1 (horizontal, even y), 1 = h2 (horizontal, odd y), 2 = v1
 * (vertical, even x), 3 = v2 (vertical, odd x).  bonds must hold
 * 2 * (nx*(ny-1) + ny*(nx-1)) ints; *n_bonds receives the count.            */
HUB_API hub_status hub_square_lattice(int32_t nx, int32_t ny, int32_t order,
                              int32_t* bonds, int32_t* bond_class,
                              int32_t* n_bonds);

/* Hamiltonian (Eqs. 1, 2, 15, 16).  t_ij: [L*L] host, symmetric, t_ij != 0
 * only on lattice bonds off the diagonal; its diagonal is the on-site
 * potential.  U_i: [L] host or NULL (= 0).  V_ij: [L*L] host or NULL,
 * symmetric, nonzero only on bonds.  n_up, n_dn: particle numbers of the
 * sector.  Requires 2 <= 2L <= 32.                                            */
HUB_API hub_status hub_create(const hub_lattice* lat, const double* t_ij,
                      const double* U_i, const double* V_ij,
                      int32_t n_up, int32_t n_dn, hub_t* out);
HUB_API void hub_destroy(hub_t model);

/* Ansatz: n_layers * groups_per_layer groups applied in array order.
 * ans_create takes one model; ans_create_multi takes several instances that
 * share lattice, mode maps and particle numbers; they may
 * differ in t, U, V.  Batch element b of every compute call uses instance
 * b % n_models.  The ansatz keeps pointers to the models, which must
 * outlive it.                                                               */
HUB_API hub_status ans_create(hub_t model, int32_t n_layers, int32_t groups_per_layer,
                      const hub_group* groups, ans_t* out);
HUB_API hub_status ans_create_multi(const hub_t* models, int32_t n_models,
                            int32_t n_layers, int32_t groups_per_layer,
                            const hub_group* groups, ans_t* out);
HUB_API void ans_destroy(ans_t ans);
HUB_API int32_t ans_num_params(ans_t ans);   /* -1 for a NULL handle */
HUB_API int32_t ans_num_qubits(ans_t ans);   /* -1 for a NULL handle */

/* Initial state |psi_0>.  HUB_PREP_SLATER: the U = 0 Slater determinant of
 * each instance: the lowest n_up / n_dn eigenvectors Phi of h = -t + P
 * (P = orb_perturb, [L*L] host symmetric, or NULL), FP64, each eigenvector's
 * largest-magnitude entry (lowest index on a tie) made positive; psi_0 =
 * prod_m b+_{m,up} prod_m b+_{m,dn} |vac>, b+_m = sum_i Phi_im a+_{mode(i)},
 * i.e. det(Phi_up[occ_up]) det(Phi_dn[occ_dn]) times the sign of ordering
 * the creators by mode.  Where the n_up-th and (n_up+1)-th levels (or those
 * of n_dn) coincide to 1e-9 relative, the determinant is not unique and the
 * call returns HUB_EINVAL (pass an orb_perturb that splits the levels).
 * HUB_PREP_NEEL: the checkerboard state of Sec. 2.1,
 * up on site i when neel_up[i] != 0 (host [L]) and down otherwise.
 * Writes batch * 2^n amplitudes to psi (may be NULL: only the tables used by
 * HUB_FLAG_PREP_FUSED are set).                                               */
HUB_API hub_status state_prepare(ans_t ans, int32_t kind, const double* orb_perturb,
                         const int32_t* neel_up, void* psi, int32_t dtype,
                         int64_t batch, hub_stream_t stream);

/* Energy E(theta) = <psi|H|psi> of Eq. 4 for each batch element.
 * theta: device double [batch][P].  psi: device [batch][2^n] amplitudes; on
 * entry the initial state (unless HUB_FLAG_PREP_FUSED), on return clobbered.
 * With HUB_FLAG_PREP_FUSED psi is workspace only and needs just the bytes
 * ans_workspace_bytes reports for the call.
 * E: device double [batch].  The sum over H's terms is fused into the last
 * sweeps; H|psi> is never written.                                          */
HUB_API hub_status energy(ans_t ans, const double* theta, void* psi, double* E,
                  int32_t dtype, int64_t batch, uint32_t flags,
                  hub_stream_t stream);

/* Energy and adjoint gradient (Sec. 2.1).  lam: device workspace of the same
 * size as psi.  ckpt: NULL, or device workspace of the same size as psi for
 * one mid-circuit checkpoint of psi (bounds the rounding drift of the
 * backward un-computation).  grad: device double [batch][P], overwritten.
 * psi and lam are clobbered.
 *
 * Engines (energy and energy_grad alike).  With HUB_FLAG_PREP_FUSED and
 * without HUB_FLAG_KEEP_STATE / HUB_FLAG_SWEEPS, only the (N_up, N_dn)
 * sector's C = C(L, N_up) * C(L, N_dn) amplitudes can be nonzero, and the
 * call runs (1) on chip, one CTA per batch element, when psi and lam of
 * that size fit one CTA's shared memory (not with HUB_FLAG_ROWS); else
 * (2) on the row engine, when a row of the C_dn x C_up sector matrix (with
 * lam where the call builds it) fits shared memory, or a row of psi and its
 * row of lam fit the shared memory of a two-CTA cluster (one each; complex128
 * at 32 qubits), and 2 C <= 2^n: the
 * sector matrices and their transposes then live in the first
 * 2 * batch * C amplitudes of each of psi and lam, and ckpt is unused;
 * else (3) as HBM sweeps over the dense psi (and lam, ckpt).  Results agree
 * across engines to the rounding of the dtype; the contents of psi, lam and
 * ckpt on return are unspecified in every case.                            */
HUB_API hub_status energy_grad(ans_t ans, const double* theta, void* psi, void* lam,
                       void* ckpt, double* E, double* grad, int32_t dtype,
                       int64_t batch, uint32_t flags, hub_stream_t stream);

/* Device workspace of a call (0 = energy, 1 = energy_grad) with these
 * flags and batch: *bytes receives the bytes that psi and lam must each
 * hold (not part of the paper: buffer sizing).  The engine the call runs on
 * (*engine, may be NULL: 0 on chip, 1 rows, 2 dense sweeps) decides it:
 * on chip the state lives in shared memory and psi and lam are not touched
 * (0 bytes); the row engine keeps the sector matrix and its transpose,
 * 2 * batch * C(L, N_up) * C(L, N_dn) amplitudes (32 qubits, N = 8 + 8,
 * complex64: 2.65 GB instead of the 34.4 GB of a dense vector); the dense
 * sweeps need batch * 2^n amplitudes, as does a checkpoint buffer.  The
 * engine choice reads the device's shared-memory limit: query with the
 * device that will run the call current.                                   */
HUB_API hub_status ans_workspace_bytes(ans_t ans, int32_t which, int32_t dtype, uint32_t flags,
                                       int64_t batch, uint64_t* bytes, int32_t* engine);

/* energy() for callers that cannot allocate device memory.  (The paper has
 * no counterpart: this is an interface addition.)  Some callers cannot call
 * cudaMalloc while they compute -- their framework's allocator already owns
 * the free device memory, or an allocation would synchronise a
 * latency-critical loop.  energy() allocates
 * its per-call scratch (coefficient and phase tables, FP64 accumulators) and
 * its static tables on first use; energy_noalloc allocates nothing: it puts
 * every table and all scratch in one static device array of
 * HUB_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the library
 * holds until the process exits.  Arguments and results are those of
 * energy().  Problems whose tables do not fit return HUB_EINVAL with the
 * size needed.  The first call on a device looks up the array's device
 * address (with that device current); later calls reuse it.  Make that
 * first call on each device before any stream capture begins.  Every
 * call shares the array (it clears the accumulators it uses), so calls that
 * overlap on the GPU -- on different streams or threads -- race.  The
 * initial-state tables come from the last state_prepare call, which, being
 * a set-up call, may allocate.                                              */
#define HUB_NOALLOC_SCRATCH_BYTES (8u << 20)
HUB_API hub_status energy_noalloc(ans_t ans, const double* theta, void* psi, double* E,
                                  int32_t dtype, int64_t batch, uint32_t flags,
                                  hub_stream_t stream);

/* lam = H psi for each batch element (Eq. 4's operator; used by tests and
 * by callers that need the residual).  psi is read only.                    */
HUB_API hub_status hub_apply_h(ans_t ans, const void* psi, void* lam, int32_t dtype,
                       int64_t batch, hub_stream_t stream);

/* The overlap loss of Eq. 5 and the fidelity (Sec. 3): for each batch
 * element, F = |<psi_ref|psi(theta)>|^2 and f = log10(1 - F), with psi(theta)
 * the ansatz state of energy(), and (grad != NULL) df/dtheta by the adjoint
 * recursion of Sec. 2.1 with the projector |psi_ref><psi_ref| in place of
 * H: lam_K = psi_ref <psi_ref|psi_K>, dF/dtheta_p = sum over the groups of
 * p of 2 Im <lam_g|G_g|psi_g>, df/dtheta = -dF/dtheta / ((1 - F) ln 10).
 * psi_ref: device [ref_batch][2^n] amplitudes of the call's dtype,
 * normalised (ref_batch = 1: one reference for every batch element, or
 * batch).  psi: as energy() (initial state unless HUB_FLAG_PREP_FUSED;
 * clobbered).  lam: device workspace of psi's size, or NULL when grad is
 * NULL.  F, f: device double [batch] or NULL; grad: device double [batch][P]
 * or NULL.  With HUB_FLAG_PREP_FUSED and factors that conserve N_up and
 * N_dn, the passes run on the row engine (the overlap and lam_K formed on
 * the sector amplitudes, psi_ref read at the sector's indices only); else,
 * or with HUB_FLAG_SWEEPS, as dense sweeps.  f is -inf when F = 1.         */
HUB_API hub_status overlap_grad(ans_t ans, const double* theta, const void* psi_ref,
                                int64_t ref_batch, void* psi, void* lam, double* F,
                                double* f, double* grad, int32_t dtype, int64_t batch,
                                uint32_t flags, hub_stream_t stream);

/* Spin correlation of Sec. 3 for each batch element of the state psi
 * (device [batch][2^n] amplitudes, normalised, read only):
 * C[b][i][j] = <S^z_i S^z_j> - <S^z_i><S^z_j>, S^z_i = (n_{i up} - n_{i dn})/2,
 * for all site pairs (C: device double [batch][L][L]).  Reductions in FP64.
 * Obtain the ansatz state with energy(..., HUB_FLAG_KEEP_STATE, ...).      */
HUB_API hub_status spin_correlation(ans_t ans, const void* psi, double* C, int32_t dtype,
                                    int64_t batch, hub_stream_t stream);

/* Plan statistics for the last-planned configuration of a call kind (0 =
 * energy, 1 = energy_grad): number of sweeps and HBM bytes moved per batch
 * element (reads + writes of amplitude vectors) of the dense-sweep plan
 * that the call runs with these flags and no checkpoint buffer
 * (HUB_FLAG_SWEEPS does not change it).  With HUB_FLAG_ROWS in
 * flags: the row engine's schedule instead (n_sweeps = its row-sweep and
 * transpose launches), whether or not a call would run on it.              */
HUB_API hub_status ans_plan_stats(ans_t ans, int32_t which, int32_t dtype,
                          uint32_t flags, int32_t* n_sweeps,
                          double* bytes_per_state);

/* Schedule of a call kind (0 energy, 1 energy_grad, 2 apply_h) for checking
 * by tests: buf receives [n_sweeps, then per sweep: tile-bit mask, sweep
 * flags (bits 0-15) | register phases (bits 16-31), n_ops, the sequence
 * index of each op in execution order].  The
 * sequence is: the ansatz factors in order (one per hop term and spin, one
 * per diagonal group); then the H terms (one per bond and spin, bonds in
 * lattice order, up before down) and H's diagonal; then (energy_grad) for
 * each factor in reverse order its gradient step followed by its inverse.
 * With HUB_FLAG_ROWS in flags (energy and energy_grad): the row engine's
 * segments instead, each as [mask of the modes of its spin, orientation
 * (0 up, 1 down), n_ops, sequence indices].
 * With buf == NULL only *len is set.                                        */
HUB_API hub_status ans_plan_describe(ans_t ans, int32_t which, int32_t dtype,
                                     uint32_t flags, int64_t* buf, int32_t cap,
                                     int32_t* len);

/* Per-launch timing: with profiling enabled every sweep launch is bracketed
 * by CUDA events on its stream.  ans_profile_read waits for the recorded
 * events, writes 4 doubles per launch [vectors in the tile (1 = psi,
 * 2 = psi and lam), dtype, amplitude bytes moved (vector reads + writes),
 * milliseconds] and clears the record; out == NULL sets only *n.          */
HUB_API hub_status ans_profile(ans_t ans, int32_t enable);
HUB_API hub_status ans_profile_read(ans_t ans, double* out, int32_t cap,
                                    int32_t* n);

/* Tile size override (log2 amplitudes per tile, 6..14; 0 = automatic: 12 for
 * c64, 10 for c128; capped at 13 for c64 and 12 for c128 by the register
 * budget).  Used by the autotuner.                                          */
HUB_API hub_status ans_set_tile(ans_t ans, int32_t dtype, int32_t log2_tile);

/* Run length override (log2 of the contiguous amplitudes that a warp moves
 * between HBM and registers as one piece; the lowest log2_run index bits are
 * in every tile).  0 = automatic (c64: 3, 64-byte runs; c128: 1, 32-byte); else
 * 1..5.  Shorter runs leave more tile bits free for the operations (fewer
 * sweeps) at the cost of less contiguous HBM traffic.                       */
HUB_API hub_status ans_set_runs(ans_t ans, int32_t dtype, int32_t log2_run);

/* Threads per CTA override of a sector engine (used by the autotuner).
 * engine HUB_ENGINE_ONCHIP: 256 or 512 (0 = automatic: 512); engine
 * HUB_ENGINE_ROWS: 256, 512 or 1024 (0 = automatic: 256 where three CTAs fit
 * an SM, 1024 for a complex64 CTA alone on its SM, else 512; a row sweep
 * that the override cannot stage, or that runs on a two-CTA cluster, keeps
 * the automatic choice).  HUB_EINVAL for other values.                     */
#define HUB_ENGINE_ONCHIP 0
#define HUB_ENGINE_ROWS 1
HUB_API hub_status ans_set_threads(ans_t ans, int32_t dtype, int32_t engine, int32_t threads);

/* Wait for the stream and report any asynchronous device error.            */
HUB_API hub_status hub_sync(hub_stream_t stream);

/* Message of the last error on the calling thread ("" if none).             */
HUB_API const char* hub_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HUBSV_H */
