// Internal data structures shared by the host side (planner hubsv_plan.cpp,
// API hubsv_api.cpp, hubsv_noalloc.cu) and the sm_103a kernels
// (hubsv_sweep.cuh, hubsv_tables.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hubsv {

constexpr int kMaxQubits = 32;
constexpr int kMaxTileBits = 14;
constexpr int kLaneBits = 5;        // lanes of a warp <-> 5 tile bits
constexpr int kMaxRegBits = 5;      // amplitudes per thread = 2^r, r <= 5
constexpr int kMaxWarpBits = 5;
constexpr int kMaxModePairs = 16;   // mode-pair products in one diagonal operator

// One operation applied to a tile.  Operations are the factors of the ansatz
// (Eq. 7), the terms of H (Eqs. 1, 2, 15, 16) and the adjoint steps of
// Sec. 2.1, each restricted to what one tile holds.
enum OpKind : uint8_t {
  OP_GIV = 0,        // Givens factor exp(-i theta G_term) of one hop term
  OP_DIAG = 1,       // diagonal factor exp(-i theta G_diag)
  OP_MEAS_HOP = 2,   // E += <psi| h_term |psi>
  OP_MEAS_DIAG = 3,  // E += sum_x D(x) |psi_x|^2, N += |psi_x|^2
  OP_LAM_HOP = 4,    // lam += h_term psi, E += <psi| h_term |psi>
  OP_LAM_DIAG = 5,   // lam += D psi, E += ..., N += ...
  OP_GRAD_HOP = 6,   // acc[slot] += 2 Im <lam| G_term |psi>
  OP_GRAD_DIAG = 7,  // acc[slot] += 2 Im <lam| G_diag |psi>
  OP_GRADINV_HOP = 8,   // OP_GRAD_HOP then the inverse factor on psi and lam
  OP_GRADINV_DIAG = 9,  // OP_GRAD_DIAG then the inverse factor on psi and lam
};

enum OpFlag : uint8_t {
  OPF_INV = 1,   // apply the inverse factor
  OPF_LAM = 2,   // apply the factor to lam as well as psi
};

// An operation inside a register phase.  Hop-type operations act on the
// register slots a < b (bit a / b of the per-thread element index e).  The
// Jordan-Wigner string is split three ways: slots (bm_slots, over e), the
// thread's other tile bits (bm_local, over the tile-local index) and the
// non-tile bits (bm_global, over the state index).
struct alignas(16) OpDev {      // 32 bytes: read as two 16-byte words
  uint8_t kind, flags, a, b;
  uint32_t sgn;                 // bit e = parity(e & JW string on the slots)
  uint32_t bm_local;            // JW string on the thread's other tile bits
  uint32_t bm_global;           // JW string on the non-tile bits (state index)
  int32_t idx;                  // OP_GIV / OP_GRADINV_HOP: coefficient column;
                                // other hop ops: column of the -t table;
                                // diagonal ops: DiagOp
  int32_t slot;                 // OP_GRAD*: accumulator slot (parameter)
  int32_t idx2;                 // OP_GRADINV_HOP: column of the -t table
  int32_t pad;
};

// A register phase: each thread holds the 2^r amplitudes whose tile-local
// index is base(thread) | dep[e], dep[e] = the tile bits of the slots set in
// e; base takes the lane bits from the lane index and the warp bits from the
// warp index.  Per slot j the plan keeps the state-index bit (so[j]) and the
// swizzled exchange index (ss[j]) of its tile bit; both maps are linear, so
// an element's offsets are XORs of slot values and the thread's base part.
struct PhaseDev {
  int32_t op_begin, op_end;
  uint8_t lane[kLaneBits];
  uint8_t nwarp;
  uint8_t warp[kMaxWarpBits + 1];
  uint8_t pad[4];
  uint32_t so[kMaxRegBits + 1];
  uint32_t ss[kMaxRegBits + 1];
  // a thread's base part, looked up by lane and by warp index: tile-local
  // bits (bl, bw) and state-index bits (gl, gw)
  uint32_t bl[32], gl[32];
  uint32_t bw[16], gw[16];
};

// A diagonal operator d(x) = sum_bytes X[byte of x] + sum_bytes Y[byte of y]
//                            + sum_bonds v_b n_i n_j,
// with y = x & (x >> s) & upmask (bit up(i) of y set iff site i is doubly
// occupied).  Real values (per instance) are used for energies and
// gradients; phase tables exp(-i theta d) are generated per batch element.
struct DiagOpDev {
  int32_t has_x, has_y;          // number of x / y byte tables in use (0..4)
  int32_t n_vb;                  // bonds with V terms
  int32_t v_uniform;             // 1: all v_b equal -> phase from K = sum n_i n_j
  int32_t real_off;              // offset of the real tables (per instance)
  int32_t phase_off;             // offset of the phase tables (per batch elem)
  int32_t param;                 // theta column for phases; -1 for H's diagonal
  int32_t vb_up[64];             // up-mode of bond end i
  int32_t vb_up2[64];            // up-mode of bond end j
  // v_uniform: the bonds grouped by the distance of their up-modes, for
  // K = sum_g sum_{P,Q in (O1,O2)} popc(mask_g & P & (Q >> shift_g)), with
  // O1 / O2 the sites holding at least one / two electrons (at their
  // up-mode positions): n_i n_j = (O1_i + O2_i)(O1_j + O2_j).  n_vs = -1:
  // use the bond list (a bond given twice).
  int32_t n_vs;
  int32_t vs_shift[32];
  uint32_t vs_mask[32];          // bit u: a bond from up-mode u to u + shift
  // mode-pair products sum_m c_m n_p(m) n_q(m) (controlled phases of the NP
  // and EP gates, Eqs. 8 and 10): real values at real_off + mp_roff, phases
  // at phase_off + mp_poff, one per pair
  int32_t n_mp, mp_roff, mp_poff;
  int32_t mp_p[kMaxModePairs];
  int32_t mp_q[kMaxModePairs];
};
// Real table layout at real_off: [4][256] X, [4][256] Y, [n_vb] v_b,
// [n_mp] c_m.  Phase table layout at phase_off: [4][256] X, [4][256] Y,
// then either [4*n_vb+1] K-table (v_uniform) or [n_vb][5] per-bond powers,
// then [n_mp] mode-pair phases.

enum SweepFlag : uint32_t {
  SW_PREP = 1u,        // generate psi_0 instead of reading psi
  SW_READ_PSI = 2u,
  SW_WRITE_PSI = 4u,
  SW_HAS_LAM = 8u,     // the tile carries lam
  SW_READ_LAM = 16u,   // else lam starts at zero in the tile
  SW_WRITE_LAM = 32u,
  SW_CKPT_WRITE = 64u, // also store psi to the checkpoint buffer
  SW_CKPT_READ = 128u, // read psi from the checkpoint buffer
  SW_VPOP = 256u,      // a diagonal operation has uniform V terms or is a single
                       // controlled phase: the kernel variant with their fast
                       // paths (V counted with popcounts; the phase of one mode
                       // pair read once per operation) is used
};

struct SweepDev {
  int32_t phase_begin, phase_end;
  int32_t op_begin, op_end;       // operations of all its phases
  int32_t k;                      // log2 tile size
  int32_t r;                      // register bits per thread
  int32_t w;                      // warp bits (threads = 32 << w)
  uint32_t flags;
  int8_t tbits[kMaxTileBits];     // tile bit positions, ascending
  int8_t nbits[kMaxQubits];       // non-tile bit positions, ascending
  int32_t n_nontile;
  // Sector tiles: every operation conserves the numbers of up and down
  // electrons, so when the initial state is generated in the (N_up, N_dn)
  // sector, a tile whose non-tile bits hold too many or too few electrons
  // of either spin for the sector is zero throughout the call.  With sector
  // = 1 the sweep visits only the other tiles ("live" tiles).  The non-tile
  // bits are split by spin into part a (the spin holding the lowest
  // non-tile bit) and part b; live tile j of a state has part-a pattern
  // j % cnt_a and part-b pattern j / cnt_a, each ranked by electron count
  // (from lo_a / lo_b up) and then in colex order, so that consecutive live
  // tiles differ first in low index bits and lie close together in HBM.
  int32_t sector;
  int32_t na, nb;                 // non-tile bits of part a / b
  int32_t lo_a, lo_b;             // fewest electrons a live pattern holds
  int32_t hi_a, hi_b;             // most electrons a live pattern holds
  uint32_t cnt_a;                 // live part-a patterns
  uint32_t live;                  // live tiles per state
  int8_t pa[kMaxQubits];          // part-a bit positions, ascending
  int8_t pb[kMaxQubits];          // part-b bit positions, ascending
  // Accumulator slots the sweep adds to, numbered locally (its operations'
  // slot fields are local): local slot i is global slot
  // slot_map[lslot_off + i]; lslot_E / lslot_N hold the energy and norm
  // (-1 when the sweep measures nothing).  The CTA keeps rows for these
  // slots only, so an ansatz with thousands of parameters costs shared
  // memory in proportion to one sweep's parameters.
  int32_t n_lslot, lslot_off, lslot_E, lslot_N;
};

// Binomial coefficients C(n, k), n, k <= 32 (C(32, 16) < 2^32).
struct BinomTable {
  uint32_t c[kMaxQubits + 1][kMaxQubits + 1];
};
constexpr BinomTable make_binom_table() {
  BinomTable t{};
  for (int n = 0; n <= kMaxQubits; ++n) {
    t.c[n][0] = 1;
    for (int k = 1; k <= n; ++k) t.c[n][k] = t.c[n - 1][k - 1] + t.c[n - 1][k];
  }
  return t;
}

struct PrepDev {
  int32_t kind;            // 0 Slater, 1 Neel
  int32_t L, s;            // sites, dn-mode offset (dn(i) = up(i) + s)
  int32_t layout;          // 0 blocked (s == L), 1 interleaved (s == 1)
  uint64_t neel_x0;
  const double* sd;        // [n_inst][2][2^L] determinant tables
  const float* sd32;       // the same in FP32 (complex64 path)
};

struct KernelArgs {
  void* psi;
  void* lam;
  void* ckpt;
  const OpDev* ops;
  const PhaseDev* phases;
  const DiagOpDev* diag_ops;
  const double* theta;
  int32_t P;                       // parameters per batch element
  const void* coef;                // [batch][n_gates] (cos, sin), R2
  int32_t n_gates;
  const double* hcoef;             // [n_inst][n_hterms]: -t of each hop term
  int32_t n_hterms;
  const double* real_tabs;         // [n_inst][real_stride]
  const float* real_tabs32;        // the same in FP32 (complex64 path)
  int32_t real_stride;
  const void* phase_tabs;          // [batch][phase_stride] R2
  int32_t phase_stride;
  int32_t n_inst;
  int32_t n;                       // qubits
  int32_t s;                       // dn-mode offset
  uint64_t upmask;
  int64_t batch;
  uint64_t n_tiles;
  double* acc;                     // [batch][n_slots]
  int32_t n_slots;
  int32_t slot_E, slot_N;
  const int32_t* slot_map;         // local -> global accumulator slots (SweepDev)
  PrepDev prep;
};

// A sweep's operations as the kernel reads them from shared memory: OpDev
// with its table lookups done for the current batch element (coefficients,
// table offsets) and one dense case code, so that an operation costs three
// 16-byte shared loads and one indirect branch.
//   w0 = {code | aux << 8 | slot << 16, sgn, bm_local, bm_global}
//   hop ops, c64:  w1 = {c, s, c_lo, s_lo}, w2 = {tc, 0, 0, 0} (FP32)
//   hop ops, c128: w1 = {c, s}, w2 = {tc, 0} (FP64)
//   diagonal ops:  w1 = {phase-table offset, real-table offset, DiagOp, mode pair (RA_MP)}
// c, s: the factor's cos / sin (s negated for an inverse factor; in c64 as
// FP32 pairs hi + lo, see GC); tc: -t of the matching Hamiltonian term.
constexpr int kMaxSlots = 65535;     // slot is stored in 16 bits
inline int res_words(int /*dtype*/) { return 3; }
enum ResCode : int {
  RC_NOP = 0,
  RC_GIV = 1,          // + pair index (0..9): factor on psi
  RC_GIV_L = 11,       // + pair index: factor on psi and lam
  RC_GRADINV = 21,     // + pair index: OP_GRADINV_HOP
  RC_MEAS = 31,        // + pair index: OP_MEAS_HOP
  RC_LAM = 41,         // + pair index: OP_LAM_HOP
  RC_GRAD = 51,        // + pair index: OP_GRAD_HOP
  RC_DIAG = 61,
  RC_GRADINV_DIAG = 62,
  RC_MEAS_DIAG = 63,
  RC_LAM_DIAG = 64,
  RC_GRAD_DIAG = 65,
};
enum ResAux : int {
  RA_NY = 3,       // diagonal ops: number of y tables when only on-site terms (1, 2), else 0
  RA_INV = 4,      // diagonal factor: inverse
  RA_LAM = 8,      // diagonal factor: also on lam
  RA_MP = 16,      // diagonal ops: a single mode-pair product c n_p n_q (p | q << 8 in w1.w;
                   // real value at real offset + 2048, phase at phase offset + 2048)
  RA_GRAD = 128,   // reduces into the accumulator slot
};
// Register slot pair (a < b) -> dense index 0..9.
__host__ __device__ inline int pair_index(int a, int b) { return b * (b - 1) / 2 + a; }

// Shared-memory layout of a sweep: exchange buffer(s) for the tile (none
// when the sweep has a single phase), the CTA accumulators, copies of the
// sweep's phases, and its resolved operations plus one spare record (the
// kernel loads one operation ahead).
inline size_t sweep_smem_bytes(int dtype, int nv, int k, int n_slots, int n_phases, int n_ops, int threads) {
  const size_t amp = dtype == 0 ? 8 : 16;
  const int nbuf = n_phases > 1 ? nv : 0;
  const size_t rows = dtype == 0 ? (size_t)threads / 32 : 1;   // accumulator rows (8-byte entries)
  size_t s = (size_t)nbuf * (amp << k) + 8 * rows * (size_t)n_slots + sizeof(PhaseDev) * (size_t)n_phases;
  s = (s + 15) & ~(size_t)15;                  // operations are read as 16-byte words
  return s + 16 * (size_t)res_words(dtype) * (size_t)(n_ops + 1);
}

// Swizzle of tile-local indices in the exchange buffer: XOR the low bits
// with a fold of the higher nibbles, so that register phases whose lanes
// run over high tile bits still hit distinct banks.
__host__ __device__ inline uint32_t swz(uint32_t l, int dtype) {
  const uint32_t f = (l >> 4) ^ (l >> 8) ^ (l >> 12);
  return l ^ (f & (dtype == 0 ? 15u : 7u));
}

}  // namespace hubsv

// Launchers implemented in hubsv_tables.cu (C++ linkage, internal).
namespace hubsv {
cudaError_t launch_sweep(int dtype, const SweepDev& sw, const KernelArgs& a,
                         int grid, size_t smem, cudaStream_t st);
cudaError_t launch_coef(int dtype, const double* theta, int P, const int32_t* gate_param,
                        const double* gate_t, int n_gates, void* coef,
                        const int32_t* tab_param, const double* tab_val,
                        int n_tab, const int32_t* tab_live, int n_live, void* phase_tabs,
                        int64_t batch, int n_inst, cudaStream_t st);
cudaError_t launch_zero(double* p, int64_t n, cudaStream_t st);
cudaError_t launch_finalize(const double* acc, int n_slots, int P, int slot_E,
                            double* E, double* grad, int64_t batch, cudaStream_t st);
// Overlap loss and spin correlations (hubsv_overlap.cu).
cudaError_t launch_overlap(int dtype, const void* psi, const void* ref, int64_t ref_batch, int n, int64_t batch,
                           double* a, cudaStream_t st);
cudaError_t launch_scale_ref(int dtype, const void* ref, int64_t ref_batch, void* lam, int n, int64_t batch,
                             const double* a, cudaStream_t st);
// The overlap and lam_K = a psi_ref on the row engine's sector matrices
// (element (r, c) has the full index xrow[r] | xin[c]).
cudaError_t launch_sector_overlap(int dtype, const void* mat, const uint32_t* xrow, const uint32_t* xin, int n_rows,
                                  int row_len, const void* ref, int64_t ref_batch, int n, int64_t batch, double* a,
                                  cudaStream_t st);
cudaError_t launch_sector_scale_ref(int dtype, const void* ref, int64_t ref_batch, const uint32_t* xrow,
                                    const uint32_t* xin, int n_rows, int row_len, int n, int64_t batch,
                                    const double* a, void* lam, cudaStream_t st);
cudaError_t launch_overlap_finalize(const double* acc, int n_slots, int P, const double* a, double* F, double* f,
                                    double* grad, int64_t batch, cudaStream_t st);
cudaError_t launch_occ_corr(int dtype, const void* psi, int n, int64_t batch, double* M, cudaStream_t st);
cudaError_t launch_spin_corr(const double* M, int n, const int32_t* up, const int32_t* dn, int L, double* C,
                             int64_t batch, cudaStream_t st);
int sweep_max_smem_optin();
cudaError_t sweep_set_smem(int dtype, int nv, int r, int threads, bool vp, size_t smem);
int sweep_regs(int dtype, int nv, int r, int threads, bool vp);
int device_sm_count();
// Register bits the kernels are compiled for: r in [1, max_r(dtype, nv)].
inline int max_reg_bits(int dtype, int nv) {
  (void)nv;
  return dtype == 0 ? 4 : 3;
}
}  // namespace hubsv
