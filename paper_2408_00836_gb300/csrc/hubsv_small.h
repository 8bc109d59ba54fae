// Device-side types and launchers of the on-chip path for small sectors
// (hubsv_small.cu).  The state of one batch element is kept as its sector
// amplitudes only, C_up x C_dn of them (element e = r_dn * ld + r_up with
// ld = C_up | 1, r_up / r_dn = index of the up / down occupation pattern
// among the sector's patterns, ascending), in one CTA's shared memory; the
// call's operation sequence runs on it op by op.
#pragma once

#include "hubsv_internal.h"

namespace hubsv {

struct alignas(16) SmallOpDev {   // 32 bytes
  uint8_t kind, flags;            // OpKind, OpFlag
  uint8_t spin;                   // hop ops: 0 = pairs of up patterns, 1 = of down patterns
  uint8_t pad;
  int32_t a;                      // hop ops: offset of the pair list; diagonal ops: DiagOp
  int32_t b;                      // hop ops: number of pattern pairs
  uint32_t between;               // hop ops: Jordan-Wigner string (index bits strictly between p, q)
  int32_t gate, hterm, slot;      // coefficient column, -t column, accumulator slot
  int32_t pad2;
};

struct SmallArgs {
  const SmallOpDev* ops;
  int32_t n_ops;
  const uint32_t* xup;             // [C_up] index bits of each up pattern
  const uint32_t* xdn;             // [C_dn] index bits of each down pattern
  int32_t cup, cdn;
  int32_t ld;                      // row pitch of the element matrix: cup | 1
  uint32_t m_cup, m_cdn;           // small_magic(cup), small_magic(cdn)
  const uint32_t* pairs;           // pattern-rank pairs r | r' << 16 (r: bit p clear, q set),
                                   // bit 31: parity of the pattern r on the modes between p, q
  int32_t n_pairs;
  const DiagOpDev* diag_ops;
  const void* coef;                // [batch][n_gates] (cos, sin), R2
  int32_t n_gates;
  const double* hcoef;             // [n_inst][n_hterms]
  int32_t n_hterms;
  const double* real_tabs;
  const float* real_tabs32;
  int32_t real_stride;
  const void* phase_tabs;          // [batch][phase_stride] R2
  int32_t phase_stride;
  int32_t n_inst;
  int32_t s;
  uint64_t upmask;
  int64_t batch;
  double* acc;                     // [batch][n_slots]
  int32_t n_slots, slot_E, slot_N;
  PrepDev prep;
};

// Shared memory of one CTA: psi and lam (ld x C_dn each), the element's
// Givens coefficients, the accumulators, the -t of its instance, and the
// pattern and pair tables.
size_t small_smem_bytes(int dtype, int cup, int cdn, int n_pairs, int n_slots, int n_gates, int n_hterms,
                        int threads);
// Threads per CTA of the on-chip kernel: 512, or 256 (ans_set_threads).
constexpr int kSmallThreadsDefault = 512;
// ceil(2^32 / d) for d > 1, 0 for d = 1: the multiplier of the kernel's
// division n / d, exact for n * d < 2^32.
uint32_t small_magic(int d);
cudaError_t launch_small(int dtype, const SmallArgs& a, int threads, int grid, size_t smem, cudaStream_t st);
int small_max_ctas_per_sm(int dtype, int threads, size_t smem);

// ---------------------------------------------------------------------------
// Row engine (hubsv_rows.cu): the sector amplitudes of each batch element
// stored in HBM as a C_dn x C_up matrix (orientation 0: row r_dn holds the
// C_up amplitudes of that down pattern, in up-pattern order) or its
// transpose (orientation 1).  Up-spin hops pair elements of one row in
// orientation 0, down-spin hops in orientation 1; diagonal operations act
// element by element in either.  A row sweep stages whole rows in shared
// memory and runs a segment of the operation sequence on them; the matrix
// is transposed between segments of different orientation.
// ---------------------------------------------------------------------------

enum RowSegFlag : uint32_t {
  RS_PREP = 1u,        // generate psi_0 instead of reading psi
  RS_WRITE_PSI = 2u,   // the segment changes psi
  RS_HAS_LAM = 4u,     // rows carry lam
  RS_READ_LAM = 8u,    // else lam starts at zero
  RS_WRITE_LAM = 16u,
  RS_MEAS = 32u,       // the segment adds to E and N
};

struct RowArgs {
  const SmallOpDev* ops;           // the call's operation sequence
  int32_t op_begin, op_end;        // this segment's operations
  uint32_t flags;                  // RowSegFlag
  void* psi;                       // [batch][n_rows][row_len] amplitudes, R2
  void* lam;                       // the same for lam (RS_HAS_LAM)
  int32_t n_rows, row_len;         // C_dn, C_up (orientation 0) or C_up, C_dn
  const uint32_t* xrow;            // [n_rows] index bits of each row's pattern
  const uint32_t* xin;             // [row_len] index bits of each in-row pattern
  const uint32_t* pairs;           // pattern-rank pairs as SmallArgs::pairs (in-row ranks)
  const DiagOpDev* diag_ops;
  const void* coef;                // [batch][n_gates] (cos, sin), R2
  int32_t n_gates;
  const double* hcoef;             // [n_inst][n_hterms]
  int32_t n_hterms;
  const double* real_tabs;
  const float* real_tabs32;
  int32_t real_stride;
  const void* phase_tabs;          // [batch][phase_stride] R2
  int32_t phase_stride;
  int32_t n_inst;
  int32_t s;
  uint64_t upmask;
  int64_t batch;
  double* acc;                     // [batch][n_slots], added to atomically
  int32_t n_slots, slot_E, slot_N;
  PrepDev prep;
};

// Shared memory of a row sweep that stages rr rows: the rows of psi (and
// lam), the segment's operation records, the element's Givens
// coefficients, the accumulator rows and the -t values.
size_t rows_smem_bytes(int dtype, int nv, int row_len, int n_slots, int n_gates, int n_hterms, int threads,
                       int n_ops, int rr);
// Launch shape of a row sweep: rows staged together (2 for short complex64
// rows where two fit one CTA, else 1), threads per CTA (256 where three
// such CTAs fit an SM, 1024 for a c64 CTA alone on its SM, else 512) and
// shared memory.
// Where a row of psi and its row of lam do not fit one CTA, a cluster of
// two CTAs (cl = 2) stages them, one row each, in 512-thread CTAs.
struct RowLaunch {
  int threads = 0, rr = 1, cl = 1;
  size_t smem = 0;   // per CTA
};
// threads: a CTA size to use instead of the automatic one (0: automatic).
RowLaunch rows_launch(int dtype, int nv, int row_len, int n_rows, int n_slots, int n_gates, int n_hterms,
                      int n_ops, bool force_cluster = false, int threads = 0);
cudaError_t launch_rows(int dtype, const RowArgs& a, const RowLaunch& L, int grid, cudaStream_t st);
int rows_max_ctas_per_sm(int dtype, const RowLaunch& L);
int rows_max_clusters(int dtype, const RowLaunch& L);
// out[b][c][r] = in[b][r][c] for a [batch][n_r][n_c] matrix of amplitudes.
cudaError_t launch_transpose(int dtype, const void* in, void* out, int64_t batch, int n_r, int n_c,
                             cudaStream_t st);

}  // namespace hubsv
