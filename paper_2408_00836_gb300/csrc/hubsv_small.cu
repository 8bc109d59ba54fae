// On-chip path of the Hubbard VQE statevector engine for small sectors.
//
// Every operation of the ansatz (Eq. 7), of H (Eqs. 1, 2, 15, 16) and of the
// adjoint recursion (Sec. 2.1) conserves the numbers of up and down
// electrons, so a state generated in the (N_up, N_dn) sector stays there and
// is fully described by its C(L, N_up) x C(L, N_down) sector amplitudes.  When
// that many amplitudes of psi and lam fit in one CTA's shared memory (4900
// for a 2x4 lattice at half filling: 78 KB in c64), a whole evaluation runs
// on chip: one CTA per batch element prepares psi_0, applies the call's
// operation sequence one operation at a time, and writes only E and the
// gradient.  Nothing of the state touches HBM.
//
// Element e = r_dn * ld + r_up (ld = C_up | 1), with r_up / r_dn the
// position of the up / down occupation pattern among the sector's patterns
// in ascending order.
// A hop term on up modes (p, q) pairs the up patterns that differ in p and q
// (one of the two occupied), for every down pattern; the Jordan-Wigner sign
// of a pair is the parity of the full index on the modes strictly between p
// and q, with the full index x = xup[r_up] | xdn[r_dn].  Diagonal factors
// and terms use the same per-byte tables as the sweep kernel, on x.
#include <algorithm>
#include <cstring>
#include <map>
#include <type_traits>

#include "hubsv_host.h"
#include "hubsv_reduce.cuh"

namespace hubsv {

// ---------------------------------------------------------------------------
// host: the on-chip plan of a call kind
// ---------------------------------------------------------------------------

namespace {

// Order a hop's pair list so that the row kernel's half-warps meet no
// shared-memory bank conflicts where possible.  Lane i of a warp takes
// entry 32 w + i of the list (per pass), and an 8-byte access of 16 lanes
// is conflict-free when their element indices are distinct modulo 16 (one
// bank pair each).  The pairs of one hop are independent, so any order is
// valid: groups of 16 are formed as perfect matchings between the classes
// e1 mod 16 and e2 mod 16 (augmenting paths over the remaining pairs);
// pairs left when no perfect matching remains follow in their old order.
void order_pairs_for_banks(std::vector<uint32_t>& pl) {
  const size_t n = pl.size();
  if (n < 32) return;
  std::vector<std::vector<int>> bucket(256);   // (e1 % 16) * 16 + e2 % 16 -> entries
  for (size_t i = 0; i < n; ++i) {
    const uint32_t e1 = pl[i] & 0xffffu, e2 = (pl[i] >> 16) & 0x7fffu;
    bucket[(e1 & 15u) * 16 + (e2 & 15u)].push_back((int)i);
  }
  for (auto& b : bucket) std::reverse(b.begin(), b.end());   // pop from the back = old order
  std::vector<uint32_t> out;
  out.reserve(n);
  std::vector<char> used(n, 0);
  while (true) {
    int match_col[16];   // e2 class -> e1 class
    for (int c = 0; c < 16; ++c) match_col[c] = -1;
    bool ok = true;
    for (int r = 0; r < 16 && ok; ++r) {
      // augmenting path from e1 class r (breadth first over the classes)
      int from_r[16], seen[16] = {0};
      for (int c = 0; c < 16; ++c) from_r[c] = -1;
      std::vector<int> queue = {r};
      int found = -1;
      for (size_t qi = 0; qi < queue.size() && found < 0; ++qi) {
        const int rr = queue[qi];
        for (int c = 0; c < 16 && found < 0; ++c) {
          if (seen[c] || bucket[rr * 16 + c].empty()) continue;
          seen[c] = 1;
          from_r[c] = rr;
          if (match_col[c] < 0) found = c;
          else queue.push_back(match_col[c]);
        }
      }
      if (found < 0) { ok = false; break; }
      // flip the path back to r
      for (int c = found;;) {
        const int rr = from_r[c];
        int prev = -1;
        for (int cc = 0; cc < 16; ++cc)
          if (match_col[cc] == rr) prev = cc;
        match_col[c] = rr;
        if (rr == r) break;
        c = prev;
      }
    }
    if (!ok) break;
    for (int c = 0; c < 16; ++c) {
      auto& b = bucket[match_col[c] * 16 + c];
      const int idx = b.back();
      b.pop_back();
      used[idx] = 1;
      out.push_back(pl[idx]);
    }
  }
  for (size_t i = 0; i < n; ++i)
    if (!used[i]) out.push_back(pl[i]);
  pl.swap(out);
}

std::vector<uint32_t> patterns(const std::vector<int>& modes, int N) {
  std::vector<uint32_t> out;
  const int L = (int)modes.size();
  for (uint32_t y = 0; y < (1u << L); ++y) {
    if (__builtin_popcount(y) != N) continue;
    uint32_t x = 0;
    for (int i = 0; i < L; ++i)
      if (y >> i & 1u) x |= 1u << modes[i];
    out.push_back(x);
  }
  std::sort(out.begin(), out.end());
  return out;
}

}  // namespace

hub_status make_small_plan(hub_ansatz* a, int which, SmallPlan*& out) {
  const hub_model* m = a->models[0];
  if (a->n > 32) return fail(HUB_EUNSUPPORTED, "on-chip path: more than 32 qubits");
  // the sector layout needs N_up and N_dn conserved separately
  if (a->spin_mix) return fail(HUB_EUNSUPPORTED, "sector engines: a Givens factor mixes the spins");
  SmallPlan* sp = new SmallPlan();
  sp->xup = patterns(m->up, m->n_up);
  sp->xdn = patterns(m->dn, m->n_dn);
  sp->cup = (int)sp->xup.size();
  sp->cdn = (int)sp->xdn.size();
  if (sp->cup >= 65536 || sp->cdn >= 65536) {
    delete sp;
    return fail(HUB_EUNSUPPORTED, "on-chip path: sector too large");
  }
  std::map<uint32_t, int> rank_up, rank_dn;
  for (int i = 0; i < sp->cup; ++i) rank_up[sp->xup[i]] = i;
  for (int i = 0; i < sp->cdn; ++i) rank_dn[sp->xdn[i]] = i;
  std::map<std::pair<int, int>, std::pair<int, int>> lists;   // (p, q) -> (offset, count)
  const std::vector<SeqOp> seq = op_sequence(a, which, HUB_FLAG_PREP_FUSED);
  for (const SeqOp& op : seq) {
    SmallOpDev d;
    std::memset(&d, 0, sizeof(d));
    d.kind = op.kind;
    d.flags = op.flags;
    d.gate = op.gate;
    d.hterm = op.hterm;
    d.slot = op.slot;
    if (op.diagonal) {
      d.a = op.diag;
    } else {
      const int p = op.p, q = op.q;
      const bool up = (a->upmask >> p) & 1ull;
      d.spin = up ? 0 : 1;
      d.between = (uint32_t)(((1ull << q) - 1ull) & ~((1ull << (p + 1)) - 1ull));
      auto it = lists.find({p, q});
      if (it == lists.end()) {
        const std::vector<uint32_t>& xs = up ? sp->xup : sp->xdn;
        std::map<uint32_t, int>& rk = up ? rank_up : rank_dn;
        const int off = (int)sp->pairs.size();
        for (size_t r = 0; r < xs.size(); ++r) {
          const uint32_t x = xs[r];
          if ((x >> p & 1u) == 0 && (x >> q & 1u) == 1) {
            const uint32_t x2 = x ^ (1u << p) ^ (1u << q);
            const uint32_t par = (uint32_t)__builtin_popcount(x & d.between) & 1u;
            sp->pairs.push_back((uint32_t)r | ((uint32_t)rk.at(x2) << 16) | (par << 31));
          }
        }
        std::vector<uint32_t> pl(sp->pairs.begin() + off, sp->pairs.end());
        order_pairs_for_banks(pl);
        std::copy(pl.begin(), pl.end(), sp->pairs.begin() + off);
        it = lists.emplace(std::make_pair(p, q), std::make_pair(off, (int)sp->pairs.size() - off)).first;
      }
      d.a = it->second.first;
      d.b = it->second.second;
    }
    sp->ops.push_back(d);
    // shared-memory amplitude loads + stores per item of the operation
    const bool lam = (op.flags & OPF_LAM) != 0;
    const double C = (double)sp->cup * (double)sp->cdn;
    const double items = op.diagonal ? C : (double)d.b * (d.spin == 0 ? sp->cdn : sp->cup);
    double per = 0;
    switch (op.kind) {
      case OP_GIV: per = lam ? 8 : 4; break;
      case OP_MEAS_HOP: per = 2; break;
      case OP_LAM_HOP: per = 6; break;
      case OP_GRAD_HOP: per = 4; break;
      case OP_DIAG: per = lam ? 4 : 2; break;
      case OP_MEAS_DIAG: per = 1; break;
      case OP_LAM_DIAG: per = 3; break;
      case OP_GRAD_DIAG: per = 2; break;
      default: break;
    }
    sp->accesses += per * items;
  }
  sp->accesses += 2.0 * (double)sp->cup * (double)sp->cdn;   // psi_0 and lam = 0
  if (sp->pairs.empty()) sp->pairs.push_back(0u);
  if (sp->ops.empty()) sp->ops.push_back(SmallOpDev{});
  out = sp;
  return HUB_OK;
}

uint32_t small_magic(int d) { return d <= 1 ? 0u : (uint32_t)((((uint64_t)1 << 32) + (uint64_t)d - 1) / (uint64_t)d); }

size_t small_smem_bytes(int dtype, int cup, int cdn, int n_pairs, int n_slots, int n_gates, int n_hterms,
                        int threads) {
  const int warps = threads / 32;
  const size_t amp = dtype == 0 ? 8 : 16;
  const size_t c = (size_t)(cup | 1) * (size_t)cdn;       // rows of odd pitch
  size_t s = 2 * c * amp;                                   // psi, lam
  s += 16 * (size_t)n_gates;                                // (cos, sin) of the element (see GC)
  s += 8 * (size_t)warps * (size_t)n_slots;                // accumulators, one row per warp
  s += amp / 2 * (size_t)n_hterms;                          // -t of the element's instance
  s += 4 * ((size_t)cup + (size_t)cdn + (size_t)n_pairs);   // patterns, pair lists
  return (s + 15) & ~(size_t)15;
}

// ---------------------------------------------------------------------------
// device
// ---------------------------------------------------------------------------

namespace {

// n / d for the n < 2^32 / d met here, with m = ceil(2^32 / d) from
// small_magic (0 for d = 1): one high multiply instead of a division.
__device__ __forceinline__ uint32_t div_magic(uint32_t n, uint32_t m) { return m ? __umulhi(n, m) : n; }

// Every loop runs flat over the CTA's threads: sector elements (prep and
// diagonal operations), or (pair, other-spin pattern) items of a hop.
// Consecutive threads take consecutive patterns of the other spin, so a
// warp touches a row (down hops) or a column (up hops) of the element
// matrix; the odd row pitch ld keeps the column accesses free of bank
// conflicts.
template <typename R, int NT>
__global__ void __launch_bounds__(NT, (sizeof(R) == 4 ? 2 : 1) * (512 / NT)) small_kernel(const SmallArgs a) {
  constexpr int kSmallWarps = NT / 32;
  using T2 = typename CT<R>::T2;
  constexpr int DT = CT<R>::DT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int C = a.cup * a.cdn, ld = a.ld;
  using GT = typename GC<R>::T;
  T2* psi = reinterpret_cast<T2*>(smem_raw);
  T2* lam = psi + (size_t)ld * a.cdn;
  GT* cs = reinterpret_cast<GT*>(lam + (size_t)ld * a.cdn);
  using AccT = typename std::conditional<DT == 0, float2, double>::type;
  AccT* acc = reinterpret_cast<AccT*>(cs + a.n_gates);   // [kSmallWarps][n_slots]
  R* hc = reinterpret_cast<R*>(acc + kSmallWarps * a.n_slots);
  uint32_t* xup = reinterpret_cast<uint32_t*>(hc + a.n_hterms);
  uint32_t* xdn = xup + a.cup;
  uint32_t* pairs = xdn + a.cdn;
  const int tid = threadIdx.x, nth = blockDim.x;
  const R* rtabs = reinterpret_cast<const R*>(DT == 0 ? (const void*)a.real_tabs32 : (const void*)a.real_tabs);
  const T2* ptabs = reinterpret_cast<const T2*>(a.phase_tabs);
  const GT* coef = reinterpret_cast<const GT*>(a.coef);
  const R* sdt = reinterpret_cast<const R*>(DT == 0 ? (const void*)a.prep.sd32 : (const void*)a.prep.sd);
  const uint32_t upm = (uint32_t)a.upmask;

  for (int i = tid; i < a.cup; i += nth) xup[i] = a.xup[i];
  for (int i = tid; i < a.cdn; i += nth) xdn[i] = a.xdn[i];
  for (int i = tid; i < a.n_pairs; i += nth) pairs[i] = a.pairs[i];

  for (int64_t b = blockIdx.x; b < a.batch; b += gridDim.x) {
    const int inst = (int)(b % a.n_inst);
    __syncthreads();   // tables copied; the previous element's read-out done
    for (int i = tid; i < kSmallWarps * a.n_slots; i += nth) acc[i] = AccT{};
    for (int i = tid; i < a.n_gates; i += nth) cs[i] = coef[b * a.n_gates + i];
    for (int i = tid; i < a.n_hterms; i += nth) hc[i] = (R)a.hcoef[(size_t)inst * a.n_hterms + i];
    for (int f = tid; f < C; f += nth) {
      const int rd = (int)div_magic((uint32_t)f, a.m_cup), ru = f - rd * a.cup;
      const int e = rd * ld + ru;
      psi[e] = mk<T2, R>(prep_amp<R>(a.prep, sdt, xup[ru] | xdn[rd], inst), (R)0);
      lam[e] = mk<T2, R>((R)0, (R)0);
    }
    __syncthreads();
    Tot<R> eacc, nacc;   // this thread's share, over all operations
    SmallOpDev nxt = a.ops[0];
    for (int oi = 0; oi < a.n_ops; ++oi) {
      const SmallOpDev op = nxt;
      if (oi + 1 < a.n_ops) nxt = a.ops[oi + 1];   // in flight during this operation
      R part = 0, npart = 0;   // this thread's share of one operation
      if (op.kind == OP_GIV || op.kind == OP_MEAS_HOP || op.kind == OP_LAM_HOP || op.kind == OP_GRAD_HOP) {
        R c = 0, s = 0, cl = 0, sl = 0, tc = 0;
        if (op.kind == OP_GIV) {
          const GT g = cs[op.gate];
          c = g.x;
          s = (op.flags & OPF_INV) ? -g.y : g.y;
          cl = GC<R>::cl(g);
          sl = (op.flags & OPF_INV) ? -GC<R>::sl(g) : GC<R>::sl(g);
        } else {
          tc = hc[op.hterm];
        }
        const bool dol = (op.flags & OPF_LAM) != 0;
        const bool upair = op.spin == 0;
        const int other = upair ? a.cdn : a.cup;
        const uint32_t mo = upair ? a.m_cdn : a.m_cup;
        const int items = op.b * other;
        for (int it = tid; it < items; it += nth) {
          const int pi = (int)div_magic((uint32_t)it, mo), ro = it - pi * other;
          const uint32_t pr = pairs[op.a + pi];
          const int r1 = (int)(pr & 0xffffu), r2 = (int)((pr >> 16) & 0x7fffu);
          int e1, e2;
          uint32_t x;
          if (upair) {
            e1 = ro * ld + r1;
            e2 = ro * ld + r2;
            x = xup[r1] | xdn[ro];
          } else {
            e1 = r1 * ld + ro;
            e2 = r2 * ld + ro;
            x = xup[ro] | xdn[r1];
          }
          const bool neg = (__popc(x & op.between) & 1) != 0;
          T2 u = psi[e1], w = psi[e2];
          if (op.kind == OP_GIV) {
            const R ss = neg ? -s : s, ssl = neg ? -sl : sl;
            rot(u, w, c, ss, cl, ssl);
            psi[e1] = u;
            psi[e2] = w;
            if (dol) {
              T2 lu = lam[e1], lw = lam[e2];
              rot(lu, lw, c, ss, cl, ssl);
              lam[e1] = lu;
              lam[e2] = lw;
            }
          } else {
            const R ts = neg ? -tc : tc;
            if (op.kind == OP_GRAD_HOP) {
              const T2 lu = lam[e1], lw = lam[e2];
              part += ts * ((lu.x * w.y - lu.y * w.x) + (lw.x * u.y - lw.y * u.x));
            } else {
              part += ts * (u.x * w.x + u.y * w.y);
              if (op.kind == OP_LAM_HOP) {
                T2 lu = lam[e1], lw = lam[e2];
                lu.x += ts * w.x; lu.y += ts * w.y;
                lw.x += ts * u.x; lw.y += ts * u.y;
                lam[e1] = lu;
                lam[e2] = lw;
              }
            }
          }
        }
        if (op.kind == OP_GRAD_HOP) row_add(acc, a.n_slots, op.slot, (R)2 * part);
        else if (op.kind != OP_GIV) eacc.add((R)2 * part);
      } else {   // diagonal operations
        const DiagOpDev& d = a.diag_ops[op.a];
        const T2* ptab = ptabs + (size_t)b * a.phase_stride + d.phase_off;
        const R* rtab = rtabs + (size_t)inst * a.real_stride + d.real_off;
        const bool inv = (op.flags & OPF_INV) != 0, dol = (op.flags & OPF_LAM) != 0;
        for (int f = tid; f < C; f += nth) {
          const int rd = (int)div_magic((uint32_t)f, a.m_cup), ru = f - rd * a.cup;
          const int e = rd * ld + ru;
          const uint32_t x = xup[ru] | xdn[rd];
          if (op.kind == OP_DIAG) {
            T2 p = diag_phase<T2>(d, ptab, x, a.s, upm);
            if (inv) p.y = -p.y;
            psi[e] = cmul(psi[e], p);
            if (dol) lam[e] = cmul(lam[e], p);
          } else {
            const R dv = diag_real<R>(d, rtab, x, a.s, upm);
            const T2 u = psi[e];
            if (op.kind == OP_GRAD_DIAG) {
              const T2 l = lam[e];
              part += dv * (l.x * u.y - l.y * u.x);
            } else {
              const R m2 = u.x * u.x + u.y * u.y;
              part += dv * m2;
              npart += m2;
              if (op.kind == OP_LAM_DIAG) {
                T2 l = lam[e];
                l.x += dv * u.x;
                l.y += dv * u.y;
                lam[e] = l;
              }
            }
          }
        }
        if (op.kind == OP_GRAD_DIAG) {
          row_add(acc, a.n_slots, op.slot, (R)2 * part);
        } else if (op.kind != OP_DIAG) {
          eacc.add(part);
          nacc.add(npart);
        }
      }
      __syncthreads();
    }
    row_add_tot(acc, a.n_slots, a.slot_E, eacc);
    row_add_tot(acc, a.n_slots, a.slot_N, nacc);
    __syncthreads();
    for (int i = tid; i < a.n_slots; i += nth) {
      double x = 0.0;
      for (int w = 0; w < kSmallWarps; ++w) x += row_value(acc[w * a.n_slots + i]);
      a.acc[(size_t)b * a.n_slots + i] = x;
    }
  }
}

}  // namespace

namespace {
const void* small_fn(int dtype, int threads) {
  if (threads == 256) return dtype == 0 ? (const void*)small_kernel<float, 256> : (const void*)small_kernel<double, 256>;
  return dtype == 0 ? (const void*)small_kernel<float, 512> : (const void*)small_kernel<double, 512>;
}
}  // namespace

cudaError_t launch_small(int dtype, const SmallArgs& a, int threads, int grid, size_t smem, cudaStream_t st) {
  const void* f = small_fn(dtype, threads);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  SmallArgs ac = a;
  void* args[] = {(void*)&ac};
  return cudaLaunchKernel(f, dim3(grid), dim3(threads), args, smem, st);
}

int small_max_ctas_per_sm(int dtype, int threads, size_t smem) {
  const void* f = small_fn(dtype, threads);
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, threads, smem) != cudaSuccess) return 0;
  return n;
}

}  // namespace hubsv
