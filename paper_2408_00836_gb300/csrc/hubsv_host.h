// Host-side internal types of the Hubbard VQE statevector engine: handles,
// the operation sequence handed to the planner, and plans.
#pragma once
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "hubsv.h"
#include "hubsv_internal.h"
#include "hubsv_small.h"

namespace hubsv {

// Internal plan flag (beside HUB_FLAG_PREP_FUSED / HUB_FLAG_KEEP_STATE):
// energy_grad with a checkpoint buffer.
constexpr uint32_t kPlanCkpt = 4u;

hub_status fail(hub_status s, const std::string& m);
hub_status cuda_fail(cudaError_t e, const char* what);

#define HUB_CUDA(call, what)                             \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return ::hubsv::cuda_fail(e_, what); \
  } while (0)

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { if (p) cudaFree(p); }
  hub_status ensure(size_t n, const char* what);
  template <typename T>
  hub_status upload(const std::vector<T>& v, const char* what) {
    hub_status s = ensure(std::max<size_t>(v.size() * sizeof(T), 16), what);
    if (s != HUB_OK) return s;
    if (!v.empty()) HUB_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), what);
    return HUB_OK;
  }
};

// Host-level operation before tiling.
struct SeqOp {
  uint8_t kind = 0, flags = 0;
  int p = -1, q = -1;       // modes (hop-type), p < q
  int gate = -1, hterm = -1, slot = -1, diag = -1;
  uint64_t support = 0;     // modes the operation reads or changes
  bool diagonal = false;
  int cls = 0;              // 0 forward, 1 measure, 2 lam, 3 backward
};

struct Plan {
  std::vector<SweepDev> sweeps;
  std::vector<int> nvec;                  // 1 or 2 per sweep
  std::vector<OpDev> hops;                // operations of all phases
  std::vector<PhaseDev> hphases;          // phases of all sweeps
  std::vector<uint64_t> tiles;
  std::vector<std::vector<int>> seq_ids;  // sequence index of each op, per sweep
  std::vector<int32_t> slot_map;          // local -> global accumulator slots of all sweeps
  bool uploaded = false;
  DevBuf ops, phases, slots;
  int k = 0;
  bool sector = false;                    // sweeps visit live (sector) tiles only
  bool prep = false;                      // the first sweep generates psi_0
  double bytes_per_state = 0;             // amplitude bytes moved per state
};

// On-chip plan of a call kind (see SmallOpDev).
struct RowSegHost {
  int op_begin = 0, op_end = 0;   // operations of the segment (SmallPlan::ops)
  int orient = 0;                 // 0: rows = down patterns, 1: rows = up patterns
  uint32_t flags = 0;             // RowSegFlag
};

// The row engine's schedule of a call kind (hubsv_rows.cu): the on-chip
// plan's operations reordered into segments, each a contiguous range of ops.
struct RowPlan {
  std::vector<RowSegHost> segs;
  std::vector<SmallOpDev> ops;
  DevBuf d_ops;
  bool uploaded = false;
};

// Sequence indices of a row segment and its orientation.
struct RowSched {
  int orient;
  std::vector<int> ops;
};

struct SmallPlan {
  int cup = 0, cdn = 0;
  std::vector<uint32_t> xup, xdn, pairs;
  std::vector<SmallOpDev> ops;
  double accesses = 0;   // shared-memory amplitude loads + stores of one evaluation
  DevBuf d_ops, d_xup, d_xdn, d_pairs;
  bool uploaded = false;
};

}  // namespace hubsv

struct hub_model {
  int L = 0, n = 0, s = 0, layout = 0;
  std::vector<int> up, dn;
  std::vector<std::pair<int, int>> bonds;
  std::vector<double> t, U, V;
  int n_up = 0, n_dn = 0;
};

struct hub_ansatz {
  std::vector<hub_model*> models;
  int n_inst = 0, L = 0, n = 0, P = 0, s = 0, layout = 0;
  int small_threads[2] = {0, 0};         // ans_set_threads overrides per dtype (0 = automatic)
  int row_threads[2] = {0, 0};
  uint64_t upmask = 0;
  std::vector<hubsv::SeqOp> fwd;         // forward factors in order
  std::vector<int> layer_begin;          // index in fwd of each layer's first factor
  int n_layers = 0;
  struct HTerm { int p, q; };
  std::vector<HTerm> hterms;             // H hop terms: 2*bond + spin
  int h_diag = -1;                       // DiagOp index of H's diagonal
  std::vector<hubsv::DiagOpDev> diag_ops;
  std::vector<int32_t> gate_param;
  std::vector<uint8_t> gate_unit;        // 1: a HUB_G_GIVENS factor (unit generator)
  int n_hcol = 0;                        // columns of hcoef: H hop terms + 1 unit column
  bool spin_mix = false;                 // a Givens factor couples an up and a down mode
  std::vector<double> gate_t;            // [n_inst][n_gates]
  std::vector<int32_t> tab_param;        // [n_tab]
  std::vector<double> tab_val;           // [n_inst][n_tab]
  std::vector<int32_t> tab_live;         // entries of the phase tables that kernels read
  std::vector<double> hcoef;             // [n_inst][n_hcol]
  std::vector<double> real_tabs;         // [n_inst][real_stride]
  int n_gates = 0, n_tab = 0, real_stride = 0;
  hubsv::DevBuf d_gate_param, d_gate_t, d_tab_param, d_tab_val, d_tab_live, d_hcoef, d_real, d_diag;
  hubsv::DevBuf d_real32;                // FP32 copy of real_tabs
  hubsv::DevBuf d_sd, d_sd32;            // Slater determinant tables (FP64, FP32)
  std::vector<double> sd_host;           // host copy of the determinant tables
  int prep_kind = -1;
  uint64_t neel_x0 = 0;
  hubsv::DevBuf d_coef[2], d_phase[2], d_acc;
  hubsv::DevBuf d_ovl;                   // overlaps <psi_ref|psi_K> [batch][2]
  hubsv::DevBuf d_occ;                   // occupation correlations [batch][n][n]
  hubsv::DevBuf d_modes;                 // site -> mode maps (up, then dn) for C_ij
  std::map<int, hubsv::Plan*> plans;     // key = which*16 + dtype*4 + flags
  std::map<int, hubsv::SmallPlan*> small_plans;   // key = which
  std::map<int, hubsv::RowPlan*> row_plans;       // key = which
  int tile_override[2] = {0, 0};
  int run_override[2] = {0, 0};         // log2 contiguous amplitudes per run (0 = default)
  bool dev_ready = false;
  struct ProfRec { cudaEvent_t e0, e1; int nv, dtype; double bytes; };
  bool prof = false;
  std::vector<ProfRec> prof_recs;
  void prof_clear();
  ~hub_ansatz();
};

namespace hubsv {
// Default tile and run bits (log2 of the amplitudes per tile, and of the
// contiguous amplitudes a warp reads or writes as one piece), chosen by
// timing energy + gradient on GB300: c64 tiles of 2^13 from 28 qubits (one
// 512-thread CTA per SM: fewer sweeps; 32 qubits 1.00 vs 0.85 evals/s, 28
// qubits 10.2 vs 8.9) and 2^12 below (two CTAs of 256 threads per SM; 24
// qubits 250 vs 223), with 64-byte runs; c128 tiles of 2^10 (CTAs of 128
// threads) with 32-byte runs.  c128 is bound by FP64 arithmetic, so it
// gains most from the plan that visits the fewest live amplitudes.
inline int default_tile_bits(int dtype, int n) { return dtype == HUB_C64 ? (n >= 28 ? 13 : 12) : 10; }
inline int default_run_bits(int dtype) { return dtype == HUB_C64 ? 3 : 1; }
uint64_t diag_support(const hub_ansatz* a, int di);
hub_status make_plan(hub_ansatz* a, int which, int dtype, uint32_t flags, Plan*& out);
// The operation sequence of a call kind (0 energy, 1 energy + gradient, 2
// lam = H psi, 3 initial state only), before any tiling.
std::vector<SeqOp> op_sequence(const hub_ansatz* a, int which, uint32_t flags);
hub_status make_small_plan(hub_ansatz* a, int which, SmallPlan*& out);
hub_status make_row_plan(const hub_ansatz* a, int which, const SmallPlan* sp, RowPlan*& out);
std::vector<RowSched> row_schedule(const hub_ansatz* a, int which);
// HBM bytes per batch element and kernel launches of a row plan.
double row_plan_bytes(const SmallPlan* sp, const RowPlan* rp, int dtype, int* n_launches);
}  // namespace hubsv
