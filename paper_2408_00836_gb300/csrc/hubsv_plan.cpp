// Planner of the Hubbard VQE statevector engine.
//
// The work of one call is a sequence of operations on amplitude vectors:
// the ansatz factors of Eq. 7 in order, then the terms of H (energy of
// Eq. 4, or lam = H psi), then for the gradient each factor's reduction
// 2 Im <lam|G|psi> and its inverse, in reverse order (Sec. 2.1).  Two
// operations commute when they act on disjoint modes (fermionic bilinears on
// disjoint modes commute) or when both are diagonal.  The planner reorders
// the sequence within those rules into
//
//   sweeps  -- passes over the vector; a sweep holds a tile of k index bits
//              (always including the c lowest, the run bits) and runs every
//              operation whose modes lie in the tile;
//   phases  -- within a sweep, groups of operations whose modes are r of the
//              tile bits, run in registers (one thread holds 2^r amplitudes).
//
// Both levels use the same greedy scan: take operations in sequence order,
// run one if it commutes with everything skipped before it and fits, skip it
// otherwise.  For sweeps several candidate tiles are scanned and the one that
// runs the most operations wins.
#include <algorithm>
#include <cstring>
#include <map>

#include "hubsv_host.h"

namespace hubsv {

namespace {

inline int popc64(uint64_t x) { return __builtin_popcountll(x); }

uint64_t between_mask(int p, int q) {  // bits strictly between p < q
  return ((1ull << q) - 1ull) & ~((1ull << (p + 1)) - 1ull);
}

// Checkpoint markers (host only, never sent to the device): barriers that
// make a sweep store psi to the checkpoint buffer at its end (SAVE) or load
// psi from it at its start (LOAD).
constexpr uint8_t MARK_SAVE = 100, MARK_LOAD = 101;
constexpr int CLS_MARK = 4;

SeqOp marker(uint8_t kind) {
  SeqOp m;
  m.kind = kind;
  m.support = ~0ull;
  m.cls = CLS_MARK;
  return m;
}

// Call kinds: 0 energy, 1 energy + gradient, 2 lam = H psi, 3 initial state
// only (no operations), 4 the forward circuit only (psi_K kept), 5 the
// backward pass only (gradient steps and inverse factors in reverse order,
// from psi_K and a given lam_K: the overlap gradient).  With a checkpoint
// (energy + gradient), psi is saved after the first half of the layers and
// reloaded when the backward pass has undone the second half.
std::vector<SeqOp> build_sequence(const hub_ansatz* a, int which, uint32_t flags) {
  std::vector<SeqOp> seq;
  if (which == 3) return seq;
  if (which == 4) return a->fwd;
  if (which == 5) {
    for (int i = (int)a->fwd.size() - 1; i >= 0; --i) {
      SeqOp g = a->fwd[i];
      g.kind = g.kind == OP_GIV ? OP_GRAD_HOP : OP_GRAD_DIAG;
      g.cls = 3;
      seq.push_back(g);
      SeqOp v = a->fwd[i];
      v.flags = OPF_INV | OPF_LAM;
      v.cls = 3;
      seq.push_back(v);
    }
    return seq;
  }
  const bool ck = which == 1 && (flags & kPlanCkpt) && a->n_layers >= 2 &&
                  (int)a->layer_begin.size() == a->n_layers;
  const int split = ck ? a->layer_begin[a->n_layers / 2] : -1;
  if (which != 2) {
    for (int i = 0; i < (int)a->fwd.size(); ++i) {
      if (i == split) seq.push_back(marker(MARK_SAVE));
      seq.push_back(a->fwd[i]);
    }
  }
  const uint64_t hsup = diag_support(a, a->h_diag);
  for (size_t t = 0; t < a->hterms.size(); ++t) {
    SeqOp op;
    op.kind = which == 0 ? OP_MEAS_HOP : OP_LAM_HOP;
    op.p = a->hterms[t].p;
    op.q = a->hterms[t].q;
    op.hterm = (int)t;
    op.support = (1ull << op.p) | (1ull << op.q);
    op.cls = which == 0 ? 1 : 2;
    seq.push_back(op);
  }
  {
    SeqOp op;
    op.kind = which == 0 ? OP_MEAS_DIAG : OP_LAM_DIAG;
    op.diag = a->h_diag;
    op.diagonal = true;
    op.support = hsup;
    op.cls = which == 0 ? 1 : 2;
    seq.push_back(op);
  }
  if (which == 1) {
    for (int i = (int)a->fwd.size() - 1; i >= 0; --i) {
      SeqOp g = a->fwd[i];
      g.kind = g.kind == OP_GIV ? OP_GRAD_HOP : OP_GRAD_DIAG;
      g.cls = 3;
      seq.push_back(g);
      SeqOp v = a->fwd[i];
      v.flags = OPF_INV | OPF_LAM;
      v.cls = 3;
      seq.push_back(v);
      if (i == split) seq.push_back(marker(MARK_LOAD));
    }
  }
  return seq;
}

bool modifies_psi(const SeqOp& op) { return op.kind == OP_GIV || op.kind == OP_DIAG; }
bool uses_lam(const SeqOp& op) {
  return op.kind == OP_LAM_HOP || op.kind == OP_LAM_DIAG || op.kind == OP_GRAD_HOP ||
         op.kind == OP_GRAD_DIAG || (op.flags & OPF_LAM);
}
bool modifies_lam(const SeqOp& op) {
  return op.kind == OP_LAM_HOP || op.kind == OP_LAM_DIAG || (modifies_psi(op) && (op.flags & OPF_LAM));
}

struct Scan {
  uint64_t tile = 0;
  std::vector<int> exec, rest;
};

// One greedy scan.  need(op) gives the bits an operation needs (0 for
// diagonal ones); the tile starts at init and may grow to `cap` bits using
// only `allowed` bits.  Lam-building operations wait for the whole forward
// circuit.
template <typename NeedFn>
Scan scan(const std::vector<SeqOp>& seq, const std::vector<int>& order, uint64_t init, uint64_t allowed,
          int cap, NeedFn need) {
  Scan s;
  s.tile = init;
  uint64_t s_any = 0, s_diag = 0;
  bool fwd_skipped = false;
  for (size_t oi = 0; oi < order.size(); ++oi) {
    const int idx = order[oi];
    const SeqOp& op = seq[idx];
    bool ok = !((op.support & s_any) || (!op.diagonal && (op.support & s_diag)));
    if (op.cls == 2 && fwd_skipped) ok = false;
    if (op.cls == CLS_MARK) {
      if (op.kind == MARK_LOAD && !s.exec.empty()) ok = false;   // a load opens its sweep
      if (ok) {
        s.exec.push_back(idx);
        if (op.kind == MARK_SAVE) {   // a save closes its sweep
          s.rest.insert(s.rest.end(), order.begin() + oi + 1, order.end());
          return s;
        }
        continue;
      }
    }
    if (ok) {
      const uint64_t nd = need(op);
      if (nd & ~allowed) ok = false;
      else {
        const uint64_t nt = s.tile | nd;
        if (popc64(nt) <= cap) s.tile = nt;
        else ok = false;
      }
    }
    if (ok) {
      s.exec.push_back(idx);
    } else {
      s.rest.push_back(idx);
      if (op.diagonal) s_diag |= op.support; else s_any |= op.support;
      if (op.cls == 0) fwd_skipped = true;
    }
  }
  return s;
}

// GF(2) rank of up to 5 columns of 4-bit values.
int rank_gf2(std::vector<uint32_t> cols) {
  int r = 0;
  for (int bit = 3; bit >= 0; --bit) {
    int piv = -1;
    for (size_t i = 0; i < cols.size(); ++i)
      if (cols[i] >> bit & 1) { piv = (int)i; break; }
    if (piv < 0) continue;
    const uint32_t pv = cols[piv];
    cols.erase(cols.begin() + piv);
    for (auto& c : cols)
      if (c >> bit & 1) c ^= pv;
    ++r;
  }
  return r;
}

// Lane bits of a phase: 5 of the free tile bits, including the `required`
// ones (the run bits, in the first and last phase, so that a warp's global
// accesses are whole runs), ordered so that the first 4 (c64) or 3 (c128)
// columns of the swizzle map are independent: a warp's shared-memory
// accesses then hit distinct banks.
void choose_lanes(uint32_t free_bits, uint32_t required, int dtype, uint8_t* lanes, uint8_t* warps,
                  int& nwarp) {
  std::vector<int> req, fb;
  for (int b = 0; b < 32; ++b) {
    if (required >> b & 1) req.push_back(b);
    else if (free_bits >> b & 1) fb.push_back(b);
  }
  const int need = dtype == 0 ? 4 : 3;
  const uint32_t m = dtype == 0 ? 15u : 7u;
  const int nsel = kLaneBits - (int)req.size();
  std::vector<int> best(req);
  best.insert(best.end(), fb.begin(), fb.begin() + nsel);
  const int nfb = (int)fb.size();
  bool found = false;
  // combinations of nsel of the other free bits; orderings checked for rank
  std::vector<int> idx(nsel);
  for (int i = 0; i < nsel; ++i) idx[i] = i;
  while (!found) {
    std::vector<int> perm(req);
    for (int i : idx) perm.push_back(fb[i]);
    std::sort(perm.begin(), perm.end());
    do {
      std::vector<uint32_t> cols;
      for (int j = 0; j < need; ++j) cols.push_back(swz(1u << perm[j], dtype) & m);
      if (rank_gf2(cols) == need) { best = perm; found = true; break; }
    } while (std::next_permutation(perm.begin(), perm.end()));
    // next combination
    int i = nsel - 1;
    while (i >= 0 && idx[i] == nfb - nsel + i) --i;
    if (i < 0) break;
    ++idx[i];
    for (int j = i + 1; j < nsel; ++j) idx[j] = idx[j - 1] + 1;
  }
  uint32_t used = 0;
  for (int j = 0; j < kLaneBits; ++j) { lanes[j] = (uint8_t)best[j]; used |= 1u << best[j]; }
  nwarp = 0;
  for (int b = 0; b < 32; ++b)
    if ((free_bits >> b & 1) && !(used >> b & 1)) warps[nwarp++] = (uint8_t)b;
}

}  // namespace

// Row-engine schedule: segments of the fused-preparation sequence, each run
// in one orientation (0: all up modes in a row, 1: all down modes), found
// by the same greedy scan as the sweeps with the up modes or the down modes
// as the tile (diagonal operations fit either); each step takes the
// orientation that runs more operations, the current one on a tie.
std::vector<RowSched> row_schedule(const hub_ansatz* a, int which) {
  const std::vector<SeqOp> seq = build_sequence(a, which, HUB_FLAG_PREP_FUSED);
  uint64_t upm = 0, dnm = 0;
  for (int i = 0; i < a->L; ++i) {
    upm |= 1ull << a->models[0]->up[i];
    dnm |= 1ull << a->models[0]->dn[i];
  }
  auto need = [](const SeqOp& op) -> uint64_t {
    return op.diagonal ? 0ull : ((1ull << op.p) | (1ull << op.q));
  };
  std::vector<int> rem(seq.size());
  for (size_t i = 0; i < seq.size(); ++i) rem[i] = (int)i;
  std::vector<RowSched> out;
  int orient = 0;
  while (!rem.empty()) {
    Scan s0 = scan(seq, rem, 0ull, upm, 64, need);
    Scan s1 = scan(seq, rem, 0ull, dnm, 64, need);
    int pick = orient;
    if (s0.exec.size() != s1.exec.size()) pick = s0.exec.size() > s1.exec.size() ? 0 : 1;
    Scan& sp = pick == 0 ? s0 : s1;
    if (sp.exec.empty()) return {RowSched{-1, {}}};   // no progress: not schedulable by rows
    out.push_back({pick, sp.exec});
    rem.swap(sp.rest);
    orient = pick;
  }
  return out;
}

std::vector<SeqOp> op_sequence(const hub_ansatz* a, int which, uint32_t flags) {
  return build_sequence(a, which, flags);
}

hub_status make_plan(hub_ansatz* a, int which, int dtype, uint32_t flags, Plan*& out) {
  const int n = a->n;
  if (n < kLaneBits + 1) return fail(HUB_EUNSUPPORTED, "need at least 6 qubits (3 sites)");
  int k = a->tile_override[dtype] ? a->tile_override[dtype] : default_tile_bits(dtype, n);
  // threads = 32 << (k - 5 - r) must stay <= 512 for every sweep
  k = std::min(k, kLaneBits + 4 + std::min(max_reg_bits(dtype, 1), max_reg_bits(dtype, 2)));
  k = std::min(k, n);
  // run bits: the lowest index bits, always in the tile, so that global
  // accesses come in runs of 2^c contiguous amplitudes
  const int c = std::min(k, a->run_override[dtype] ? a->run_override[dtype] : default_run_bits(dtype));
  const uint64_t cmask = (1ull << c) - 1ull;
  const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1ull);
  uint64_t upm = 0, dnm = 0;
  for (int i = 0; i < a->L; ++i) {
    upm |= 1ull << a->models[0]->up[i];
    dnm |= 1ull << a->models[0]->dn[i];
  }
  std::vector<SeqOp> seq = build_sequence(a, which, flags);
  std::vector<int> remaining(seq.size());
  for (size_t i = 0; i < seq.size(); ++i) remaining[i] = (int)i;
  auto need_modes = [](const SeqOp& op) -> uint64_t {
    return op.diagonal ? 0ull : ((1ull << op.p) | (1ull << op.q));
  };
  // candidate tiles: windows of consecutive modes, and of consecutive modes of one spin
  std::vector<uint64_t> windows;
  for (int s0 = 0; s0 < n; ++s0) {
    uint64_t t = cmask;
    for (int b = s0; b < n && popc64(t) < k; ++b) t |= 1ull << b;
    windows.push_back(t);
  }
  for (uint64_t sm : {upm, dnm}) {
    std::vector<int> ms;
    for (int b = 0; b < n; ++b)
      if (sm >> b & 1) ms.push_back(b);
    for (size_t s0 = 0; s0 < ms.size(); ++s0) {
      uint64_t t = cmask;
      for (size_t j = s0; j < ms.size() && popc64(t) < k; ++j) t |= 1ull << ms[j];
      windows.push_back(t);
    }
  }
  // An initial state generated here lies in the (N_up, N_dn) sector and
  // every operation keeps it there: sweeps then visit only the tiles that
  // meet the sector (see SweepDev), and a candidate tile is worth the
  // operations it runs per live fraction of the vector it moves.
  // (with a factor that mixes the spins only N_up + N_dn is conserved: every
  // tile is visited)
  const bool sector = (which == 3 || (flags & HUB_FLAG_PREP_FUSED) != 0) && which != 2 && !a->spin_mix;
  const BinomTable binom = make_binom_table();
  auto pad_tile = [&](uint64_t t) {
    for (int b = 0; b < n && popc64(t) < k; ++b) t |= 1ull << b;   // pad with low bits
    return t;
  };
  auto live_frac = [&](uint64_t t) {
    double f = 1.0;
    for (int sp = 0; sp < 2; ++sp) {
      const uint64_t m = sp == 0 ? upm : dnm;
      const int N = sp == 0 ? a->models[0]->n_up : a->models[0]->n_dn;
      const int in = popc64(t & m), fr = popc64(m) - in;
      double c = 0.0;
      for (int e = std::max(0, N - in); e <= std::min(N, fr); ++e) c += binom.c[fr][e];
      f *= c / (double)(1ull << fr);
    }
    return f;
  };
  auto worth = [&](const Scan& s) {
    if (!sector) return (double)s.exec.size();
    return (double)s.exec.size() / (live_frac(pad_tile(s.tile)) + 0.05);
  };
  auto candidates = [&](const std::vector<int>& rem) {
    std::vector<Scan> cs;
    cs.push_back(scan(seq, rem, cmask, all, k, need_modes));
    cs.push_back(scan(seq, rem, cmask, cmask | upm, k, need_modes));
    cs.push_back(scan(seq, rem, cmask, cmask | dnm, k, need_modes));
    for (uint64_t t : windows) cs.push_back(scan(seq, rem, t, t, k, need_modes));
    return cs;
  };
  auto lf_of = [&](const Scan& s) { return sector ? live_frac(pad_tile(s.tile)) : 1.0; };
  // Sweep selection.  Sector mode looks one sweep ahead: of the best `width`
  // candidates by worth, take the one whose pair (it, then the best next
  // sweep) runs the most operations per live fraction moved.  The outcome
  // of such greedy rules varies with the width in no regular way, so
  // several widths are planned (planning is cheap next to one sweep) and the
  // plan that moves the fewest vector bytes is kept (cost: live fraction x
  // vectors a sweep reads and writes: 2, 3 with lam being built, 4 with the
  // gradient).
  struct PS { uint64_t tile; std::vector<int> ops; };
  auto select_sweeps = [&](int width, std::vector<PS>& out, double& cost) -> bool {
    std::vector<int> rem = remaining;
    cost = 0.0;
    while (!rem.empty()) {
      std::vector<Scan> cs = candidates(rem);
      std::vector<int> order(cs.size());
      for (size_t i = 0; i < cs.size(); ++i) order[i] = (int)i;
      std::stable_sort(order.begin(), order.end(),
                       [&](int x, int y) { return worth(cs[x]) > worth(cs[y]); });
      if (cs[order[0]].exec.empty()) return false;
      int pick = order[0];
      if (sector && width > 1) {
        double best_v = -1.0;
        for (int i = 0; i < width && i < (int)order.size(); ++i) {
          const Scan& s1 = cs[order[i]];
          if (s1.exec.empty()) break;
          double n2 = 0.0, l2 = 0.0;
          if (!s1.rest.empty()) {
            std::vector<Scan> c2 = candidates(s1.rest);
            const Scan* b2 = nullptr;
            for (const Scan& t : c2)
              if (!b2 || worth(t) > worth(*b2)) b2 = &t;
            n2 = (double)b2->exec.size();
            l2 = lf_of(*b2);
          }
          const double v = ((double)s1.exec.size() + n2) / (lf_of(s1) + l2 + 0.1);
          if (v > best_v) { best_v = v; pick = order[i]; }
        }
      }
      int nvec = 2;
      for (int idx : cs[pick].exec) nvec = std::max(nvec, seq[idx].cls == 3 ? 4 : (seq[idx].cls == 2 ? 3 : 2));
      cost += lf_of(cs[pick]) * nvec;
      out.push_back({pad_tile(cs[pick].tile), cs[pick].exec});
      std::vector<int> rest = cs[pick].rest;
      rem.swap(rest);
    }
    return true;
  };
  std::vector<PS> sweeps;
  {
    double best_cost = 0.0;
    for (int width : {1, 2, 3, 4, 6}) {
      if (!sector && width > 1) break;
      std::vector<PS> sw;
      double cost = 0.0;
      if (!select_sweeps(width, sw, cost)) return fail(HUB_EUNSUPPORTED, "planner made no progress");
      if (sweeps.empty() || cost < best_cost) { sweeps.swap(sw); best_cost = cost; }
    }
  }
  if (sweeps.empty()) sweeps.push_back({(1ull << k) - 1ull, {}});   // initial state only

  Plan* pl = new Plan();
  pl->k = k;
  // the backward-only pass reads psi_K and lam_K (in the sector when the
  // forward pass generated the initial state)
  const bool prep = (which == 3 || (flags & HUB_FLAG_PREP_FUSED) != 0) && which != 5;
  pl->sector = sector;
  pl->prep = prep;
  const bool keep = which == 3 || (flags & HUB_FLAG_KEEP_STATE) != 0;
  bool lam_live = which == 5;
  const double amp = dtype == HUB_C64 ? 8.0 : 16.0;
  double bytes = 0.0;
  for (size_t si = 0; si < sweeps.size(); ++si) {
    const PS& ps = sweeps[si];
    // sweep flags; checkpoint markers become flags and leave the op list
    bool mod_psi = false, use_lam = false, mod_lam = false, ck_save = false, ck_load = false;
    std::vector<int> sweep_ops;
    for (int idx : ps.ops) {
      if (seq[idx].cls == CLS_MARK) {
        ck_save = ck_save || seq[idx].kind == MARK_SAVE;
        ck_load = ck_load || seq[idx].kind == MARK_LOAD;
        continue;
      }
      sweep_ops.push_back(idx);
      mod_psi = mod_psi || modifies_psi(seq[idx]);
      use_lam = use_lam || uses_lam(seq[idx]);
      mod_lam = mod_lam || modifies_lam(seq[idx]);
    }
    const bool first = si == 0, last = si + 1 == sweeps.size();
    uint32_t f = 0;
    if (first && prep && which != 2) f |= SW_PREP; else f |= SW_READ_PSI;
    if (ck_load) f |= SW_CKPT_READ;          // psi comes from the checkpoint
    if (ck_save) f |= SW_CKPT_WRITE;         // and a copy goes to it
    if ((!last || keep) && (mod_psi || (f & (SW_PREP | SW_CKPT_READ))) && which != 2) f |= SW_WRITE_PSI;
    if (use_lam || (lam_live && mod_lam)) {
      f |= SW_HAS_LAM;
      if (lam_live) f |= SW_READ_LAM;
      if (mod_lam && (!last || which == 2)) f |= SW_WRITE_LAM;
      lam_live = true;
    }
    const int nv = (f & SW_HAS_LAM) ? 2 : 1;
    const int r = std::min(max_reg_bits(dtype, nv), k - kLaneBits);
    SweepDev sw;
    std::memset(&sw, 0, sizeof(sw));
    sw.k = k;
    sw.r = r;
    sw.w = k - kLaneBits - r;
    sw.flags = f;
    int nt = 0, nn = 0;
    int localpos[64];
    for (int b = 0; b < n; ++b) {
      if (ps.tile >> b & 1) { localpos[b] = nt; sw.tbits[nt++] = (int8_t)b; }
      else { localpos[b] = -1; sw.nbits[nn++] = (int8_t)b; }
    }
    sw.n_nontile = nn;
    uint64_t tiles_per_state = 1ull << (n - k);
    if (pl->sector) {
      const int n_up = a->models[0]->n_up, n_dn = a->models[0]->n_dn;
      int tu = 0, td = 0, nu = 0, nd = 0;
      int8_t upos[kMaxQubits], dpos[kMaxQubits];
      for (int b = 0; b < n; ++b) {
        const bool isup = upm >> b & 1;
        if (ps.tile >> b & 1) (isup ? tu : td)++;
        else if (isup) upos[nu++] = (int8_t)b;
        else dpos[nd++] = (int8_t)b;
      }
      const int lo_u = std::max(0, n_up - tu), hi_u = std::min(n_up, nu);
      const int lo_d = std::max(0, n_dn - td), hi_d = std::min(n_dn, nd);
      uint64_t cu = 0, cd = 0;
      for (int e = lo_u; e <= hi_u; ++e) cu += binom.c[nu][e];
      for (int e = lo_d; e <= hi_d; ++e) cd += binom.c[nd][e];
      // part a: the spin that holds the lowest non-tile bit
      const bool up_a = nd == 0 || (nu > 0 && upos[0] < dpos[0]);
      sw.sector = 1;
      sw.na = up_a ? nu : nd;
      sw.nb = up_a ? nd : nu;
      sw.lo_a = up_a ? lo_u : lo_d;
      sw.lo_b = up_a ? lo_d : lo_u;
      sw.hi_a = up_a ? hi_u : hi_d;
      sw.hi_b = up_a ? hi_d : hi_u;
      sw.cnt_a = (uint32_t)(up_a ? cu : cd);
      for (int i = 0; i < sw.na; ++i) sw.pa[i] = up_a ? upos[i] : dpos[i];
      for (int i = 0; i < sw.nb; ++i) sw.pb[i] = up_a ? dpos[i] : upos[i];
      sw.live = (uint32_t)(cu * cd);   // <= 2^(n-k)
      tiles_per_state = sw.live;
    }
    // ---- register phases ----
    const uint32_t low = (uint32_t)cmask;   // tile-local bits 0..c-1 are the run bits
    const uint32_t tmask = (k >= 32) ? ~0u : ((1u << k) - 1u);
    auto need_local = [&](const SeqOp& op) -> uint64_t {
      return op.diagonal ? 0ull : ((1ull << localpos[op.p]) | (1ull << localpos[op.q]));
    };
    struct PH { uint32_t S; std::vector<int> ops; };
    std::vector<PH> phs;
    std::vector<int> rem = sweep_ops;
    while (!rem.empty()) {
      const uint32_t allowed = phs.empty() ? (tmask & ~low) : tmask;
      Scan s = scan(seq, rem, 0, allowed, r, need_local);
      // also try register sets seeded with each of the next operations' bits
      int tried = 0;
      for (size_t j = 0; j < rem.size() && tried < 16; ++j) {
        const SeqOp& op = seq[rem[j]];
        if (op.diagonal) continue;
        const uint64_t sd = need_local(op);
        if (sd & ~(uint64_t)allowed) continue;
        ++tried;
        Scan c = scan(seq, rem, sd, allowed, r, need_local);
        if (c.exec.size() > s.exec.size()) s = std::move(c);
      }
      if (s.exec.empty()) {
        if (phs.empty()) { phs.push_back({0u, {}}); continue; }   // first phase keeps the lanes low
        delete pl;
        return fail(HUB_EUNSUPPORTED, "phase planner made no progress");
      }
      phs.push_back({(uint32_t)s.tile, s.exec});
      rem.swap(s.rest);
    }
    if (phs.empty()) phs.push_back({0u, {}});
    if (phs.back().S & low) phs.push_back({0u, {}});
    sw.phase_begin = (int)pl->hphases.size();
    sw.op_begin = (int)pl->hops.size();
    std::vector<int> exec_order;
    for (const PH& P : phs) exec_order.insert(exec_order.end(), P.ops.begin(), P.ops.end());
    for (size_t pi = 0; pi < phs.size(); ++pi) {
      PH& P = phs[pi];
      const bool edge = pi == 0 || pi + 1 == phs.size();
      // pad the register set to r bits (never with the low bits in edge phases)
      for (int bit = k - 1; bit >= 0 && popc64(P.S) < r; --bit)
        if (!(P.S >> bit & 1) && !(edge && (low >> bit & 1))) P.S |= 1u << bit;
      for (int bit = 0; bit < k && popc64(P.S) < r; ++bit) P.S |= 1u << bit;
      PhaseDev pd;
      std::memset(&pd, 0, sizeof(pd));
      int slot_of[32];
      int ns = 0;
      std::vector<int> sb;
      for (int bit = 0; bit < k; ++bit) {
        slot_of[bit] = -1;
        if (P.S >> bit & 1) { slot_of[bit] = ns++; sb.push_back(bit); }
      }
      for (int j = 0; j < r; ++j) {
        pd.so[j] = 1u << sw.tbits[sb[j]];
        pd.ss[j] = swz(1u << sb[j], dtype);
      }
      const uint32_t freeb = tmask & ~P.S;
      int nw = 0;
      choose_lanes(freeb, (edge && !(P.S & low)) ? low : 0u, dtype, pd.lane, pd.warp, nw);
      pd.nwarp = (uint8_t)nw;
      for (int v = 0; v < 32; ++v)
        for (int j = 0; j < kLaneBits; ++j)
          if (v >> j & 1) {
            pd.bl[v] |= 1u << pd.lane[j];
            pd.gl[v] |= 1u << sw.tbits[pd.lane[j]];
          }
      for (int v = 0; v < 16; ++v)
        for (int j = 0; j < nw; ++j)
          if (v >> j & 1) {
            pd.bw[v] |= 1u << pd.warp[j];
            pd.gw[v] |= 1u << sw.tbits[pd.warp[j]];
          }
      pd.op_begin = (int)pl->hops.size();
      for (size_t oj = 0; oj < P.ops.size(); ++oj) {
        const int idx = P.ops[oj];
        const SeqOp& op = seq[idx];
        OpDev d;
        std::memset(&d, 0, sizeof(d));
        d.kind = op.kind;
        d.flags = op.flags;
        d.idx = op.kind == OP_GIV ? op.gate : (op.diagonal ? op.diag : op.hterm);
        d.slot = op.slot;
        // a gradient step directly followed by its own inverse factor: fuse
        if ((op.kind == OP_GRAD_HOP || op.kind == OP_GRAD_DIAG) && oj + 1 < P.ops.size()) {
          const SeqOp& nx = seq[P.ops[oj + 1]];
          const bool same = (op.kind == OP_GRAD_HOP) ? (nx.kind == OP_GIV && nx.gate == op.gate)
                                                     : (nx.kind == OP_DIAG && nx.diag == op.diag);
          if (same && (nx.flags & OPF_INV) && (nx.flags & OPF_LAM)) {
            if (op.kind == OP_GRAD_HOP) {
              d.kind = OP_GRADINV_HOP;
              d.idx = op.gate;
              d.idx2 = op.hterm;
            } else {
              d.kind = OP_GRADINV_DIAG;
            }
            d.flags = nx.flags;
            ++oj;   // the inverse is folded into this operation
          }
        }
        if (!op.diagonal) {
          const int lp = localpos[op.p], lq = localpos[op.q];
          d.a = (uint8_t)slot_of[lp];
          d.b = (uint8_t)slot_of[lq];
          const uint64_t bm = between_mask(op.p, op.q);
          uint32_t bs = 0, bl = 0;
          for (int b = 0; b < n; ++b) {
            if (!(bm >> b & 1) || localpos[b] < 0) continue;
            const int lb = localpos[b];
            if (slot_of[lb] >= 0) bs |= 1u << slot_of[lb];
            else bl |= 1u << lb;
          }
          d.bm_local = bl;
          uint32_t sg = 0;
          for (int e = 0; e < (1 << r); ++e)
            if (__builtin_popcount((uint32_t)e & bs) & 1) sg |= 1u << e;
          d.sgn = sg;
          d.bm_global = (uint32_t)(bm & ~ps.tile);
        }
        pl->hops.push_back(d);
      }
      pd.op_end = (int)pl->hops.size();
      pl->hphases.push_back(pd);
    }
    sw.phase_end = (int)pl->hphases.size();
    sw.op_end = (int)pl->hops.size();
    // local accumulator slots: the parameters of the sweep's gradient
    // steps, then the energy and norm if it measures
    {
      std::map<int, int> loc;
      bool measures = false;
      sw.lslot_off = (int)pl->slot_map.size();
      for (int oi = sw.op_begin; oi < sw.op_end; ++oi) {
        OpDev& d = pl->hops[oi];
        if (d.kind == OP_GRAD_HOP || d.kind == OP_GRAD_DIAG || d.kind == OP_GRADINV_HOP ||
            d.kind == OP_GRADINV_DIAG) {
          auto it = loc.find(d.slot);
          if (it == loc.end()) {
            it = loc.emplace(d.slot, (int)loc.size()).first;
            pl->slot_map.push_back(d.slot);
          }
          d.slot = it->second;
        }
        measures = measures || d.kind == OP_MEAS_HOP || d.kind == OP_MEAS_DIAG || d.kind == OP_LAM_HOP ||
                   d.kind == OP_LAM_DIAG;
      }
      sw.lslot_E = sw.lslot_N = -1;
      if (measures) {
        sw.lslot_E = (int)loc.size();
        sw.lslot_N = sw.lslot_E + 1;
        pl->slot_map.push_back(a->P);
        pl->slot_map.push_back(a->P + 1);
      }
      sw.n_lslot = (int)pl->slot_map.size() - sw.lslot_off;
    }
    for (int oi = sw.op_begin; oi < sw.op_end; ++oi) {
      const OpDev& d = pl->hops[oi];
      const bool diag = d.kind == OP_DIAG || d.kind == OP_MEAS_DIAG || d.kind == OP_LAM_DIAG ||
                        d.kind == OP_GRAD_DIAG || d.kind == OP_GRADINV_DIAG;
      if (!diag) continue;
      const DiagOpDev& g = a->diag_ops[d.idx];
      if (g.n_vb > 0 && g.v_uniform && g.n_vs >= 0) sw.flags |= SW_VPOP;
      if (g.has_x == 0 && g.has_y == 0 && g.n_vb == 0 && g.n_mp == 1) sw.flags |= SW_VPOP;
    }
    bytes += amp * (double)tiles_per_state * (double)(1ull << k) *
             (((f & SW_READ_PSI) ? 1 : 0) + ((f & SW_WRITE_PSI) ? 1 : 0) +
              ((f & SW_READ_LAM) ? 1 : 0) + ((f & SW_WRITE_LAM) ? 1 : 0) +
              ((f & SW_CKPT_WRITE) ? 1 : 0));
    pl->sweeps.push_back(sw);
    pl->nvec.push_back(nv);
    pl->tiles.push_back(ps.tile);
    pl->seq_ids.push_back(exec_order);
  }
  pl->bytes_per_state = bytes;
  out = pl;
  return HUB_OK;
}

}  // namespace hubsv
