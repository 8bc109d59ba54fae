// Row engine of the Hubbard VQE statevector engine: sector amplitudes in HBM.
//
// Every operation of the ansatz (Eq. 7), of H (Eqs. 1, 2, 15, 16) and of the
// adjoint recursion (Sec. 2.1) conserves N_up and N_dn, so a state prepared
// in the sector is its C(L, N_up) * C(L, N_dn) sector amplitudes (at 32
// qubits, N = 8 + 8: 165.6 M of the 2^32).  They are stored per batch
// element as a matrix with one row per down pattern and one column per up
// pattern (orientation 0), or transposed (orientation 1).  A hop on two up
// modes pairs up patterns, i.e. elements of one row in orientation 0; a hop
// on two down modes pairs elements of one row in orientation 1; diagonal
// operations act on single elements.  So the call's operation sequence is
// cut into segments of one orientation, and each segment is one sweep over
// the rows: a CTA stages whole rows of psi (and lam) in shared memory, runs
// the segment's operations on them one at a time (a barrier between
// operations), and writes them back.  Between segments of different
// orientation the matrix is transposed.
//
// Element operations follow the on-chip engine: a pair of in-row ranks from
// the pair list of the hop's modes, the full index x = xrow[row] | xin[rank]
// for the Jordan-Wigner parity and the diagonal tables.
#include <algorithm>
#include <cstring>

#include <cooperative_groups.h>

#include "hubsv_host.h"
#include "hubsv_reduce.cuh"

namespace cg = cooperative_groups;

namespace hubsv {

namespace {
// Row kernels come in CTAs of 256 threads (three or four per SM, where the
// rows are short enough) and of 512 threads (two per SM, or one for the
// longest rows with lam): many small CTAs hide the barrier between
// operations best, but one or two CTAs on an SM need more warps each
// (measured: 256-thread CTAs everywhere are 19 % slower at 32 qubits and
// 19 % faster at 28).  A c64 CTA alone on its SM takes 1024 threads (2 %
// faster at 32 qubits; the c128 one at 28 qubits is 11 % slower so).
constexpr int kRowThreadsSmall = 256;
constexpr int kRowThreadsLarge = 512;
constexpr int kRowThreadsSolo = 1024;   // a c64 CTA alone on its SM (the longest rows with lam)
// complex64 rows shorter than this are staged two per CTA: a hop then has
// about one pair per thread, and staging two rows halves the per-operation
// work and barriers per row (24 qubits: 1319 -> 1463 evals/s; at 28 qubits,
// 3432 amplitudes a row, two rows per CTA measured 24 % slower, and c128
// slower at both sizes).
constexpr int kRowPairLen = 1024;
}  // namespace

// The row segments of a call kind: the operations of the on-chip plan
// (one per sequence entry) in the order of row_schedule, with what each
// segment reads and writes.
hub_status make_row_plan(const hub_ansatz* a, int which, const SmallPlan* sp, RowPlan*& out) {
  const std::vector<RowSched> sched = row_schedule(a, which);
  for (const RowSched& rs : sched)
    if (rs.orient < 0) return fail(HUB_EUNSUPPORTED, "row engine: no schedule");
  RowPlan* rp = new RowPlan();
  // call kind 5 (the backward pass of the overlap loss) starts from psi and
  // lam in the caller's buffers; kind 4 (the forward pass alone) leaves
  // psi_K there
  bool lam_live = which == 5;
  for (const RowSched& rs : sched) {
    RowSegHost g;
    g.op_begin = (int)rp->ops.size();
    g.orient = rs.orient;
    bool mod_psi = false, mod_lam = false, makes_lam = false, meas = false;
    for (size_t j = 0; j < rs.ops.size(); ++j) {
      const SmallOpDev& op = sp->ops[rs.ops[j]];
      // a gradient term directly followed by the inverse of its own factor
      // on psi and lam runs as one operation (one pass over the pairs)
      if ((op.kind == OP_GRAD_HOP || op.kind == OP_GRAD_DIAG) && j + 1 < rs.ops.size()) {
        const SmallOpDev& nx = sp->ops[rs.ops[j + 1]];
        const bool same = op.kind == OP_GRAD_HOP
                              ? (nx.kind == OP_GIV && nx.a == op.a && nx.b == op.b && nx.between == op.between)
                              : (nx.kind == OP_DIAG && nx.a == op.a);
        if (same && (nx.flags & OPF_INV) && (nx.flags & OPF_LAM)) {
          SmallOpDev f = op;
          f.kind = op.kind == OP_GRAD_HOP ? OP_GRADINV_HOP : OP_GRADINV_DIAG;
          f.flags = nx.flags;
          f.gate = nx.gate;
          rp->ops.push_back(f);
          mod_psi = mod_lam = true;
          ++j;
          continue;
        }
      }
      rp->ops.push_back(op);
      const bool lam_op = op.kind == OP_LAM_HOP || op.kind == OP_LAM_DIAG;
      mod_psi = mod_psi || op.kind == OP_GIV || op.kind == OP_DIAG;
      mod_lam = mod_lam || lam_op || ((op.kind == OP_GIV || op.kind == OP_DIAG) && (op.flags & OPF_LAM));
      makes_lam = makes_lam || lam_op;
      meas = meas || lam_op || op.kind == OP_MEAS_HOP || op.kind == OP_MEAS_DIAG;
    }
    g.op_end = (int)rp->ops.size();
    uint32_t f = 0;
    if (rp->segs.empty() && which != 5) f |= RS_PREP | RS_WRITE_PSI;
    if (mod_psi) f |= RS_WRITE_PSI;
    if (lam_live || makes_lam) f |= RS_HAS_LAM;
    if (lam_live) f |= RS_READ_LAM;
    if (mod_lam) f |= RS_WRITE_LAM;
    if (meas) f |= RS_MEAS;
    lam_live = lam_live || makes_lam;
    g.flags = f;
    rp->segs.push_back(g);
  }
  if (rp->segs.empty()) {   // no operations: prepare psi_0 only (E = 0)
    RowSegHost g;
    g.flags = RS_PREP;
    rp->segs.push_back(g);
  }
  if (rp->ops.empty()) rp->ops.push_back(SmallOpDev{});
  if (which != 4) rp->segs.back().flags &= ~(uint32_t)(RS_WRITE_PSI | RS_WRITE_LAM);   // nothing reads them
  out = rp;
  return HUB_OK;
}

double row_plan_bytes(const SmallPlan* sp, const RowPlan* rp, int dtype, int* n_launches) {
  const double m = (double)sp->cup * (double)sp->cdn * (dtype == 0 ? 8.0 : 16.0);
  double bytes = 0.0;
  int launches = 0, orient = rp->segs.empty() ? 0 : rp->segs[0].orient;
  bool lam_live = false;
  for (const RowSegHost& g : rp->segs) {
    if (g.orient != orient) {   // transposes: read + write of psi (and lam)
      bytes += 2.0 * m * (lam_live ? 2.0 : 1.0);
      launches += lam_live ? 2 : 1;
      orient = g.orient;
    }
    const bool has_lam = (g.flags & RS_HAS_LAM) != 0;
    const int io = ((g.flags & RS_PREP) ? 0 : 1) + ((g.flags & RS_WRITE_PSI) ? 1 : 0) +
                   ((g.flags & RS_READ_LAM) ? 1 : 0) + ((has_lam && (g.flags & RS_WRITE_LAM)) ? 1 : 0);
    bytes += (double)io * m;
    ++launches;
    lam_live = lam_live || (has_lam && (g.flags & RS_WRITE_LAM));
  }
  if (n_launches) *n_launches = launches;
  return bytes;
}

size_t rows_smem_bytes(int dtype, int nv, int row_len, int n_slots, int n_gates, int n_hterms, int threads,
                       int n_ops, int rr) {
  const size_t amp = dtype == 0 ? 8 : 16;
  size_t s = (size_t)rr * (size_t)nv * (size_t)row_len * amp;   // rows of psi (, lam)
  s = (s + 15) & ~(size_t)15;
  s += sizeof(SmallOpDev) * (size_t)n_ops;                  // the segment's operations
  s += 16 * (size_t)n_gates;                                // (cos, sin) of the element (see GC)
  s += 8 * (size_t)(threads / 32) * (size_t)n_slots;        // accumulator rows, one per warp
  s += amp / 2 * (size_t)n_hterms;                          // -t of the element's instance
  return (s + 15) & ~(size_t)15;
}

namespace {

enum { RH_GIV = 0, RH_MEAS = 1, RH_LAM = 2, RH_GRAD = 3, RH_GRADINV = 4 };

// One pair of a hop operation on a staged row (pair entry pr, as
// SmallArgs::pairs); returns its share of the measured or gradient term.
template <int K, bool DOL, typename R, typename T2>
__device__ __forceinline__ R row_pair(T2* __restrict__ prow, T2* __restrict__ lrow, uint32_t pr, uint32_t rpar,
                                      R c, R s, R cl, R sl, R tc) {
  const int e1 = (int)(pr & 0xffffu), e2 = (int)((pr >> 16) & 0x7fffu);
  const bool neg = ((pr >> 31) ^ rpar) != 0;
  T2 u = prow[e1], w = prow[e2];
  R part = 0;
  if constexpr (K == RH_GIV) {
    const R ss = neg ? -s : s, ssl = neg ? -sl : sl;
    rot(u, w, c, ss, cl, ssl);
    prow[e1] = u;
    prow[e2] = w;
    if constexpr (DOL) {
      T2 lu = lrow[e1], lw = lrow[e2];
      rot(lu, lw, c, ss, cl, ssl);
      lrow[e1] = lu;
      lrow[e2] = lw;
    }
  } else if constexpr (K == RH_GRAD || K == RH_GRADINV) {
    const R ts = neg ? -tc : tc;
    T2 lu = lrow[e1], lw = lrow[e2];
    part = ts * ((lu.x * w.y - lu.y * w.x) + (lw.x * u.y - lw.y * u.x));
    if constexpr (K == RH_GRADINV) {   // then the inverse factor on both
      const R ss = neg ? -s : s, ssl = neg ? -sl : sl;
      rot(u, w, c, ss, cl, ssl);
      prow[e1] = u;
      prow[e2] = w;
      rot(lu, lw, c, ss, cl, ssl);
      lrow[e1] = lu;
      lrow[e2] = lw;
    }
  } else {
    const R ts = neg ? -tc : tc;
    part = ts * (u.x * w.x + u.y * w.y);
    if constexpr (K == RH_LAM) {
      T2 lu = lrow[e1], lw = lrow[e2];
      lu.x += ts * w.x; lu.y += ts * w.y;
      lw.x += ts * u.x; lw.y += ts * u.y;
      lrow[e1] = lu;
      lrow[e2] = lw;
    }
  }
  return part;
}

// One hop operation on RR staged rows (row r at prow + r len, its lam at
// lrow + r len): thread tid takes entries tid, tid + nth, ... of the pair
// list (tid, nth: the thread's index and count over the CTAs sharing the
// rows), four loaded at a time, and applies each entry to every row (the
// rows differ only in the row part of the Jordan-Wigner parity, rpar[r]).
// Returns this thread's share of the measured or gradient term.  K and DOL
// are fixed per call site, so the loops carry no branches on the operation
// kind.
template <int K, bool DOL, int NT, int RR, typename R, typename T2>
__device__ __forceinline__ R row_hop(T2* __restrict__ prow, T2* __restrict__ lrow, int len,
                                     const uint32_t* __restrict__ pl, int nb, const uint32_t (&rpar)[RR], R c,
                                     R s, R cl, R sl, R tc, int tid, int nth) {
  // entries loaded at a time: eight for the complex64 psi-only rotations of
  // 512-thread CTAs (32 qubits: 3 432 pairs a row, one batch instead of two;
  // +0.4 %), four otherwise (eight cost 1.6 % where four cover the list)
  constexpr int NB = (K == RH_GIV && !DOL && sizeof(R) == 4 && NT == kRowThreadsLarge) ? 8 : 4;
  R part = 0;
  for (int it0 = tid; it0 < nb; it0 += NB * nth) {
    uint32_t prs[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      const int it = it0 + k * nth;
      prs[k] = it < nb ? __ldg(pl + it) : 0u;
    }
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      if (it0 + k * nth >= nb) break;
#pragma unroll
      for (int r = 0; r < RR; ++r)   // one pair entry for all staged rows
        part += row_pair<K, DOL>(prow + r * len, lrow + r * len, prs[k], rpar[r], c, s, cl, sl, tc);
    }
  }
  return part;
}

// Row staging: n elements from global memory into shared memory with
// cp.async (the copies take no registers, so all of a thread's copies are
// in flight at once; a CTA alone on its SM otherwise waits out the HBM
// latency several times per row).  16-byte copies where both addresses are
// 16-byte aligned (the last complex64 element of an odd count: 8 bytes),
// else 8-byte copies (element arrays are at least 8-byte aligned).
// Completed by stage_wait() in every thread, then a barrier.
template <typename T2>
__device__ __forceinline__ void stage_async(T2* dst, const T2* src, int n, int tid, int nth) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const size_t g = __cvta_generic_to_global(src);
  const size_t bytes = (size_t)n * sizeof(T2);   // a multiple of 8
  if (((d | g) & 15u) == 0) {
    const int n16 = (int)(bytes >> 4);
    for (int i = tid; i < n16; i += nth)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16u * (uint32_t)i), "l"(g + 16 * (size_t)i)
                   : "memory");
    if ((bytes & 8) && tid == 0)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d + (uint32_t)(bytes - 8)), "l"(g + bytes - 8)
                   : "memory");
  } else {
    const int n8 = (int)(bytes >> 3);
    for (int i = tid; i < n8; i += nth)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d + 8u * (uint32_t)i), "l"(g + 8 * (size_t)i)
                   : "memory");
  }
}
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// RR: rows staged together (1 or 2, consecutive rows of one batch
// element): every operation runs on all of them between two barriers, so
// its per-operation work and the pair-list loads are shared.
// CL = 2: a row of psi and its row of lam too large for one SM's shared
// memory (complex128 at 32 qubits: 2 x 206 KB) are staged by a cluster of
// two CTAs, psi in rank 0's shared memory and lam in rank 1's; both CTAs
// work on every operation (entries and elements split between them) and
// reach the other's row through distributed shared memory, with a cluster
// barrier wherever one CTA would synchronise.
template <typename R, int NT, int RR, int CL>
__global__ void __launch_bounds__(NT, CL == 2 ? 1
                                            : (NT == kRowThreadsSmall ? 4
                                                                      : (NT == kRowThreadsLarge ? (sizeof(R) == 8 ? 1 : 2) : 1)))
    rows_kernel(const RowArgs a) {
  constexpr int kRowWarps = NT / 32;
  using T2 = typename CT<R>::T2;
  constexpr int DT = CT<R>::DT;
  using AccT = typename std::conditional<DT == 0, float2, double>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const bool has_lam = (a.flags & RS_HAS_LAM) != 0;
  const int len = a.row_len;
  T2* const mine = reinterpret_cast<T2*>(smem_raw);   // the rows this CTA stages
  T2* prow = mine;                                     // [RR][len]
  T2* lrow = prow + RR * len;                          // [RR][len]
  int rank = 0;
  if constexpr (CL == 2) {
    cg::cluster_group cluster = cg::this_cluster();
    rank = (int)cluster.block_rank();
    prow = cluster.map_shared_rank(mine, 0);
    lrow = cluster.map_shared_rank(mine, 1);
  }
  auto row_sync = [&]() {
    if constexpr (CL == 2) cg::this_cluster().sync();
    else __syncthreads();
  };
  const size_t rows_b =
      (((size_t)RR * (has_lam && CL == 1 ? 2 : 1) * (size_t)len * sizeof(T2)) + 15) & ~(size_t)15;
  SmallOpDev* sops = reinterpret_cast<SmallOpDev*>(smem_raw + rows_b);
  const int n_ops = a.op_end - a.op_begin;
  using GT = typename GC<R>::T;
  GT* cs = reinterpret_cast<GT*>(sops + n_ops);
  AccT* acc = reinterpret_cast<AccT*>(cs + a.n_gates);   // [kRowWarps][n_slots]
  R* hc = reinterpret_cast<R*>(acc + kRowWarps * a.n_slots);
  // The launch has exactly NT threads (launch_rows checks it).  Complex64
  // takes the loop strides as compile-time constants (immediate offsets, no
  // stride arithmetic); complex128 keeps them in registers, which spills
  // less in its 64-register variants.
  const int tid = threadIdx.x, nth = sizeof(R) == 4 ? NT : (int)blockDim.x;
  const int wtid = tid + rank * nth, wnth = CL * nth;   // work split over the cluster
  const R* rtabs = reinterpret_cast<const R*>(DT == 0 ? (const void*)a.real_tabs32 : (const void*)a.real_tabs);
  const T2* ptabs = reinterpret_cast<const T2*>(a.phase_tabs);
  const GT* coef = reinterpret_cast<const GT*>(a.coef);
  const R* sdt = reinterpret_cast<const R*>(DT == 0 ? (const void*)a.prep.sd32 : (const void*)a.prep.sd);
  const uint32_t upm = (uint32_t)a.upmask;
  T2* psi = reinterpret_cast<T2*>(a.psi);
  T2* lam = reinterpret_cast<T2*>(a.lam);
  const bool meas = (a.flags & RS_MEAS) != 0;

  {   // the segment's operation records, read by every thread for every row
    const int4* src = reinterpret_cast<const int4*>(a.ops + a.op_begin);
    int4* dst = reinterpret_cast<int4*>(sops);
    const int nw = n_ops * (int)(sizeof(SmallOpDev) / sizeof(int4));
    for (int i = tid; i < nw; i += nth) dst[i] = src[i];
  }
  const int n_grp = (a.n_rows + RR - 1) / RR;   // row groups per batch element
  const int64_t total = a.batch * (int64_t)n_grp;
  int64_t cur_b = -1;
  for (int64_t g = blockIdx.x / CL; g < total; g += gridDim.x / CL) {
    const int64_t b = g / n_grp;
    const int rr0 = (int)(g - b * n_grp) * RR;
    const int inst = (int)(b % a.n_inst);
    row_sync();   // the previous rows are stored
    if (b != cur_b) {
      if (cur_b >= 0) {   // read out the previous element's accumulators
        for (int i = tid; i < a.n_slots; i += nth) {
          double x = 0.0;
          for (int w = 0; w < kRowWarps; ++w) x += row_value(acc[w * a.n_slots + i]);
          if (x != 0.0) atomicAdd(&a.acc[(size_t)cur_b * a.n_slots + i], x);
        }
        __syncthreads();
      }
      for (int i = tid; i < kRowWarps * a.n_slots; i += nth) acc[i] = AccT{};
      for (int i = tid; i < a.n_gates; i += nth) cs[i] = coef[b * a.n_gates + i];
      for (int i = tid; i < a.n_hterms; i += nth) hc[i] = (R)a.hcoef[(size_t)inst * a.n_hterms + i];
      cur_b = b;
    }
    // rows of the group; a missing last row (odd row count) is staged as
    // zeros with the first row's pattern, and not stored
    uint32_t xr[RR];
    bool live[RR];
    size_t base[RR];
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      live[r] = rr0 + r < a.n_rows;
      const int row = live[r] ? rr0 + r : rr0;
      xr[r] = a.xrow[row];
      base[r] = ((size_t)b * (size_t)a.n_rows + (size_t)row) * (size_t)len;
    }
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      if constexpr (CL == 2) {   // rank 0 stages the psi row, rank 1 the lam row
        if (rank == 0) {
          stage_async(mine, psi + base[r], len, tid, nth);
        } else if (a.flags & RS_READ_LAM) {
          stage_async(mine, lam + base[r], len, tid, nth);
        } else {
          for (int i = tid; i < len; i += nth) mine[i] = mk<T2, R>((R)0, (R)0);
        }
        continue;
      }
      T2* pr = prow + r * len;
      T2* lr = lrow + r * len;
      if (!live[r]) {
        for (int i = tid; i < len; i += nth) pr[i] = mk<T2, R>((R)0, (R)0);
      } else if (a.flags & RS_PREP) {
        for (int i = tid; i < len; i += nth) pr[i] = mk<T2, R>(prep_amp<R>(a.prep, sdt, xr[r] | a.xin[i], inst), (R)0);
      } else if constexpr (sizeof(R) == 4) {
        stage_async(pr, psi + base[r], len, tid, nth);
      } else {   // (complex128 CTAs share their SM with others: plain loads, fewer spills)
        for (int i = tid; i < len; i += nth) pr[i] = psi[base[r] + i];
      }
      if (has_lam) {
        if (live[r] && (a.flags & RS_READ_LAM)) {
          if constexpr (sizeof(R) == 4) stage_async(lr, lam + base[r], len, tid, nth);
          else for (int i = tid; i < len; i += nth) lr[i] = lam[base[r] + i];
        } else {
          for (int i = tid; i < len; i += nth) lr[i] = mk<T2, R>((R)0, (R)0);
        }
      }
    }
    stage_wait();
    row_sync();
    Tot<R> eacc, nacc;
    // gradient terms of consecutive operations with one accumulator slot
    // (the factors of one parameter) are summed per thread and reduced once
    R racc = 0;
    int rslot = -1;
    auto add_slot = [&](int slot, R v) {
      if (slot != rslot) {
        if (rslot >= 0) row_add(acc, a.n_slots, rslot, racc);
        racc = 0;
        rslot = slot;
      }
      racc += v;
    };
    for (int oi = 0; oi < n_ops; ++oi) {
      const SmallOpDev op = sops[oi];
      R part = 0, npart = 0;
      static_assert(OP_GIV % 2 == 0 && OP_MEAS_HOP % 2 == 0 && OP_LAM_HOP % 2 == 0 && OP_GRAD_HOP % 2 == 0 &&
                        OP_GRADINV_HOP % 2 == 0 && OP_DIAG % 2 == 1 && OP_MEAS_DIAG % 2 == 1 &&
                        OP_LAM_DIAG % 2 == 1 && OP_GRAD_DIAG % 2 == 1 && OP_GRADINV_DIAG % 2 == 1,
                    "hop kinds are even, diagonal kinds odd");
      // (complex128 keeps the five comparisons: its 64-register variants
      // spill less that way)
      const bool hop = sizeof(R) == 4 ? (op.kind & 1) == 0
                                      : (op.kind == OP_GIV || op.kind == OP_MEAS_HOP || op.kind == OP_LAM_HOP ||
                                         op.kind == OP_GRAD_HOP || op.kind == OP_GRADINV_HOP);
      if (hop) {   // hop operations
        R c = 0, s = 0, cl = 0, sl = 0, tc = 0;
        if (op.kind == OP_GIV || op.kind == OP_GRADINV_HOP) {
          const GT gq = cs[op.gate];
          c = gq.x;
          s = (op.flags & OPF_INV) ? -gq.y : gq.y;
          cl = GC<R>::cl(gq);
          sl = (op.flags & OPF_INV) ? -GC<R>::sl(gq) : GC<R>::sl(gq);
        }
        if (op.kind != OP_GIV) tc = hc[op.hterm];
        const bool dol = (op.flags & OPF_LAM) != 0;
        // the rows' part of the Jordan-Wigner parity (the in-row part is
        // bit 31 of the pair entry)
        uint32_t rpar[RR];
#pragma unroll
        for (int r = 0; r < RR; ++r) rpar[r] = (uint32_t)__popc(xr[r] & op.between) & 1u;
        const uint32_t* pl = a.pairs + op.a;
#define HUB_HOP(K, D) row_hop<K, D, NT, RR>(prow, lrow, len, pl, op.b, rpar, c, s, cl, sl, tc, wtid, wnth)
        switch (op.kind) {
          case OP_GIV:
            if (dol) HUB_HOP(RH_GIV, true);
            else HUB_HOP(RH_GIV, false);
            break;
          case OP_MEAS_HOP: part = HUB_HOP(RH_MEAS, false); break;
          case OP_LAM_HOP: part = HUB_HOP(RH_LAM, false); break;
          case OP_GRADINV_HOP: part = HUB_HOP(RH_GRADINV, true); break;
          default: part = HUB_HOP(RH_GRAD, false); break;
        }
#undef HUB_HOP
        if (op.kind == OP_GRAD_HOP || op.kind == OP_GRADINV_HOP) add_slot(op.slot, (R)2 * part);
        else if (op.kind != OP_GIV) eacc.add((R)2 * part);
      } else {   // diagonal operations
        const DiagOpDev* dp = a.diag_ops + op.a;
        const int hx = __ldg(&dp->has_x), hy = __ldg(&dp->has_y), nvb = __ldg(&dp->n_vb), nmp = __ldg(&dp->n_mp);
        const DiagVal<R, T2> dv{dp, (hx == 0 && nvb == 0 && nmp == 0 && (hy == 1 || hy == 2)) ? hy : 0};
        const T2* ptab = ptabs + (size_t)b * a.phase_stride + __ldg(&dp->phase_off);
        const R* rtab = rtabs + (size_t)inst * a.real_stride + __ldg(&dp->real_off);
        const bool inv = (op.flags & OPF_INV) != 0, dol = (op.flags & OPF_LAM) != 0;
        const uint32_t* __restrict__ xin = a.xin;
        switch (op.kind) {
          case OP_DIAG:
            for (int e = wtid; e < len; e += wnth) {
              const uint32_t xi = __ldg(xin + e);
#pragma unroll
              for (int r = 0; r < RR; ++r) {
                T2 p = dv.phase(ptab, xr[r] | xi, a.s, upm);
                if (inv) p.y = -p.y;
                prow[r * len + e] = cmul(prow[r * len + e], p);
                if (dol) lrow[r * len + e] = cmul(lrow[r * len + e], p);
              }
            }
            break;
          case OP_GRAD_DIAG:
            for (int e = wtid; e < len; e += wnth) {
              const uint32_t xi = __ldg(xin + e);
#pragma unroll
              for (int r = 0; r < RR; ++r) {
                const R v = dv.real(rtab, xr[r] | xi, a.s, upm);
                const T2 u = prow[r * len + e], l = lrow[r * len + e];
                part += v * (l.x * u.y - l.y * u.x);
              }
            }
            break;
          case OP_GRADINV_DIAG:   // the gradient term, then the inverse phase on both
            for (int e = wtid; e < len; e += wnth) {
              const uint32_t xi = __ldg(xin + e);
#pragma unroll
              for (int r = 0; r < RR; ++r) {
                const uint32_t x = xr[r] | xi;
                const R v = dv.real(rtab, x, a.s, upm);
                T2 p = dv.phase(ptab, x, a.s, upm);
                if (inv) p.y = -p.y;
                const T2 u = prow[r * len + e], l = lrow[r * len + e];
                part += v * (l.x * u.y - l.y * u.x);
                prow[r * len + e] = cmul(u, p);
                lrow[r * len + e] = cmul(l, p);
              }
            }
            break;
          case OP_LAM_DIAG:
            for (int e = wtid; e < len; e += wnth) {
              const uint32_t xi = __ldg(xin + e);
#pragma unroll
              for (int r = 0; r < RR; ++r) {
                const R v = dv.real(rtab, xr[r] | xi, a.s, upm);
                const T2 u = prow[r * len + e];
                const R m2 = u.x * u.x + u.y * u.y;
                part += v * m2;
                npart += m2;
                T2 l = lrow[r * len + e];
                l.x += v * u.x;
                l.y += v * u.y;
                lrow[r * len + e] = l;
              }
            }
            break;
          default:   // OP_MEAS_DIAG
            for (int e = wtid; e < len; e += wnth) {
              const uint32_t xi = __ldg(xin + e);
#pragma unroll
              for (int r = 0; r < RR; ++r) {
                const R v = dv.real(rtab, xr[r] | xi, a.s, upm);
                const T2 u = prow[r * len + e];
                const R m2 = u.x * u.x + u.y * u.y;
                part += v * m2;
                npart += m2;
              }
            }
            break;
        }
        if (op.kind == OP_GRAD_DIAG || op.kind == OP_GRADINV_DIAG) {
          add_slot(op.slot, (R)2 * part);
        } else if (op.kind != OP_DIAG) {
          eacc.add(part);
          nacc.add(npart);
        }
      }
      row_sync();
    }
    if (rslot >= 0) row_add(acc, a.n_slots, rslot, racc);
    if (meas) {
      row_add_tot(acc, a.n_slots, a.slot_E, eacc);
      row_add_tot(acc, a.n_slots, a.slot_N, nacc);
    }
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      if constexpr (CL == 2) {
        if (rank == 0 && (a.flags & RS_WRITE_PSI))
          for (int i = tid; i < len; i += nth) psi[base[r] + i] = mine[i];
        if (rank == 1 && (a.flags & RS_WRITE_LAM))
          for (int i = tid; i < len; i += nth) lam[base[r] + i] = mine[i];
        continue;
      }
      if (!live[r]) continue;
      if (a.flags & RS_WRITE_PSI)
        for (int i = tid; i < len; i += nth) psi[base[r] + i] = prow[r * len + i];
      if (has_lam && (a.flags & RS_WRITE_LAM))
        for (int i = tid; i < len; i += nth) lam[base[r] + i] = lrow[r * len + i];
    }
  }
  row_sync();   // (cluster: no CTA leaves while the other may read its row)
  if (cur_b >= 0) {
    for (int i = tid; i < a.n_slots; i += nth) {
      double x = 0.0;
      for (int w = 0; w < kRowWarps; ++w) x += row_value(acc[w * a.n_slots + i]);
      if (x != 0.0) atomicAdd(&a.acc[(size_t)cur_b * a.n_slots + i], x);
    }
  }
}

// out[b][c][r] = in[b][r][c], TS x TS tiles through shared memory (one
// padding column keeps the column reads free of bank conflicts); 32 x 8
// threads, each moving TS / 32 x TS / 8 elements, all loads issued before
// the first shared-memory store.
template <typename T2, int TS>
__global__ void __launch_bounds__(256) transpose_kernel(const T2* __restrict__ in, T2* __restrict__ out,
                                                        int64_t batch, int n_r, int n_c) {
  __shared__ T2 tile[TS][TS + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  const int c0 = blockIdx.x * TS, r0 = blockIdx.y * TS;
  const size_t mat = (size_t)n_r * (size_t)n_c;
  for (int64_t b = blockIdx.z; b < batch; b += gridDim.z) {
    const T2* src = in + (size_t)b * mat;
    T2* dst = out + (size_t)b * mat;
    T2 v[TS / 8][TS / 32];
#pragma unroll
    for (int j = 0; j < TS / 8; ++j)
#pragma unroll
      for (int i = 0; i < TS / 32; ++i) {
        const int r = r0 + ty + 8 * j, c = c0 + tx + 32 * i;
        if (r < n_r && c < n_c) v[j][i] = src[(size_t)r * n_c + c];
      }
#pragma unroll
    for (int j = 0; j < TS / 8; ++j)
#pragma unroll
      for (int i = 0; i < TS / 32; ++i) tile[ty + 8 * j][tx + 32 * i] = v[j][i];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < TS / 8; ++j)
#pragma unroll
      for (int i = 0; i < TS / 32; ++i) {
        const int c = c0 + ty + 8 * j, r = r0 + tx + 32 * i;
        if (r < n_r && c < n_c) dst[(size_t)c * n_r + r] = tile[tx + 32 * i][ty + 8 * j];
      }
    __syncthreads();
  }
}

// complex64 tiles of 64 x 64 (33 KB of shared memory), complex128 32 x 32
constexpr int kTransposeTile64 = 64;

}  // namespace

namespace {
template <int NT, int RR>
const void* rows_fn_nt(int dtype) {
  return dtype == 0 ? (const void*)rows_kernel<float, NT, RR, 1> : (const void*)rows_kernel<double, NT, RR, 1>;
}
template <int RR>
const void* rows_fn_rr(int dtype, int threads) {
  if (threads == kRowThreadsSolo) return rows_fn_nt<kRowThreadsSolo, RR>(dtype);
  if (threads == kRowThreadsSmall) return rows_fn_nt<kRowThreadsSmall, RR>(dtype);
  return rows_fn_nt<kRowThreadsLarge, RR>(dtype);
}
const void* rows_fn(int dtype, const RowLaunch& L) {
  if (L.cl == 2)
    return dtype == 0 ? (const void*)rows_kernel<float, kRowThreadsLarge, 1, 2>
                      : (const void*)rows_kernel<double, kRowThreadsLarge, 1, 2>;
  return L.rr == 2 ? rows_fn_rr<2>(dtype, L.threads) : rows_fn_rr<1>(dtype, L.threads);
}
// Threads per CTA for a row sweep of smem(threads) bytes: 256 where three
// such CTAs fit an SM, 512 where two fit (and for c128), else 1024.
template <typename F>
int pick_threads(int dtype, F smem) {
  if (3 * (smem(kRowThreadsSmall) + 1024) <= (size_t)228 * 1024) return kRowThreadsSmall;
  if (2 * (smem(kRowThreadsLarge) + 1024) <= (size_t)228 * 1024 || dtype != 0) return kRowThreadsLarge;
  return kRowThreadsSolo;
}
cudaLaunchConfig_t rows_config(const RowLaunch& L, int grid, cudaStream_t st, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)L.threads);
  cfg.dynamicSmemBytes = L.smem;
  cfg.stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)L.cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}
}  // namespace

RowLaunch rows_launch(int dtype, int nv, int row_len, int n_rows, int n_slots, int n_gates, int n_hterms,
                      int n_ops, bool force_cluster, int threads) {
  RowLaunch L;
  for (int rr = (n_rows >= 2 && dtype == 0 && row_len < kRowPairLen) ? 2 : 1; rr >= 1 && !(force_cluster && nv == 2);
       --rr) {
    auto smem = [&](int nt) { return rows_smem_bytes(dtype, nv, row_len, n_slots, n_gates, n_hterms, nt, n_ops, rr); };
    const int nt = threads ? threads : pick_threads(dtype, smem);
    L.threads = nt;
    L.rr = rr;
    L.smem = smem(nt);
    if (L.smem + 1024 <= (size_t)228 * 1024) return L;   // two rows fit one CTA, else one
  }
  L = RowLaunch();   // smem = 0: no launch shape fits
  if (nv == 2) {   // psi and lam rows on a cluster of two CTAs, one row each
    const size_t s1 = rows_smem_bytes(dtype, 1, row_len, n_slots, n_gates, n_hterms, kRowThreadsLarge, n_ops, 1);
    if (s1 + 1024 <= (size_t)228 * 1024) {
      L.threads = kRowThreadsLarge;
      L.rr = 1;
      L.cl = 2;
      L.smem = s1;
    }
  }
  return L;
}

cudaError_t launch_rows(int dtype, const RowArgs& a, const RowLaunch& L, int grid, cudaStream_t st) {
  // the kernel's loops assume blockDim.x == its NT
  const bool nt_ok = L.cl == 2 ? L.threads == kRowThreadsLarge
                               : (L.threads == kRowThreadsSolo || L.threads == kRowThreadsSmall ||
                                  L.threads == kRowThreadsLarge);
  if (!nt_ok) return cudaErrorInvalidValue;
  const void* f = rows_fn(dtype, L);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
  if (e != cudaSuccess) return e;
  RowArgs ac = a;
  void* args[] = {(void*)&ac};
  if (L.cl == 1) return cudaLaunchKernel(f, dim3(grid), dim3(L.threads), args, L.smem, st);
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = rows_config(L, grid, st, at);
  return cudaLaunchKernelExC(&cfg, f, args);
}

// CTAs of one launch that run at the same time per SM (cluster launches:
// per SM on average, from the number of clusters that fit the device).
int rows_max_ctas_per_sm(int dtype, const RowLaunch& L) {
  const void* f = rows_fn(dtype, L);
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem) != cudaSuccess) return 0;
  int n = 0;
  if (L.cl == 1) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, L.threads, L.smem) != cudaSuccess) return 0;
    return n;
  }
  return 1;
}

// Clusters of a cluster launch that can be resident at once (0 if none).
int rows_max_clusters(int dtype, const RowLaunch& L) {
  const void* f = rows_fn(dtype, L);
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem) != cudaSuccess) return 0;
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = rows_config(L, 2 * L.cl, nullptr, at);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, f, &cfg) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_transpose(int dtype, const void* in, void* out, int64_t batch, int n_r, int n_c,
                             cudaStream_t st) {
  if (batch <= 0 || n_r <= 0 || n_c <= 0) return cudaSuccess;
  const int ts = dtype == 0 ? kTransposeTile64 : 32;
  const dim3 grid((unsigned)((n_c + ts - 1) / ts), (unsigned)((n_r + ts - 1) / ts),
                  (unsigned)std::min<int64_t>(batch, 1024));
  if (dtype == 0) {
    if (ts == 64)
      transpose_kernel<float2, 64><<<grid, dim3(32, 8), 0, st>>>((const float2*)in, (float2*)out, batch, n_r, n_c);
    else
      transpose_kernel<float2, 32><<<grid, dim3(32, 8), 0, st>>>((const float2*)in, (float2*)out, batch, n_r, n_c);
  } else {
    transpose_kernel<double2, 32><<<grid, dim3(32, 8), 0, st>>>((const double2*)in, (double2*)out, batch, n_r, n_c);
  }
  return cudaGetLastError();
}

}  // namespace hubsv
