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
  const uint32_t* pairs;           // pattern-rank pairs r | r' << 16 (r: bit p clear, q set)
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
size_t small_smem_bytes(int dtype, int cup, int cdn, int n_pairs, int n_slots, int n_gates, int n_hterms);
// ceil(2^32 / d) for d > 1, 0 for d = 1: the multiplier of the kernel's
// division n / d, exact for n * d < 2^32.
uint32_t small_magic(int d);
cudaError_t launch_small(int dtype, const SmallArgs& a, int grid, size_t smem, cudaStream_t st);
int small_max_ctas_per_sm(int dtype, size_t smem);

}  // namespace hubsv
