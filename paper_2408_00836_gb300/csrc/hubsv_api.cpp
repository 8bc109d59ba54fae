// C-ABI entry points of the Hubbard VQE statevector engine (hubsv.h): model
// and ansatz handles with their coefficient tables, the FP64 one-body
// diagonalisation and determinant tables of the Slater-determinant initial
// state, plan execution and the profiling hooks.  The planner lives in
// hubsv_plan.cpp, the kernels in hubsv_sweep.cuh and hubsv_tables.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <string>
#include <vector>

#include "hubsv_host.h"

using namespace hubsv;

namespace {
thread_local std::string g_err;
inline int popc64(uint64_t x) { return __builtin_popcountll(x); }
}  // namespace

namespace hubsv {

hub_status fail(hub_status s, const std::string& m) {
  g_err = m;
  return s;
}

hub_status cuda_fail(cudaError_t e, const char* what) {
  return fail(HUB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

hub_status DevBuf::ensure(size_t n, const char* what) {
  if (n <= bytes && p) return HUB_OK;
  if (p) { cudaFree(p); p = nullptr; bytes = 0; }
  if (n == 0) n = 16;
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    p = nullptr;
    // an allocation failure is not sticky: clear it so that the next call's
    // check for earlier asynchronous errors does not report it again
    (void)cudaGetLastError();
    return fail(HUB_ENOMEM, std::string("cudaMalloc failed for ") + what);
  }
  bytes = n;
  return HUB_OK;
}

}  // namespace hubsv

void hub_ansatz::prof_clear() {
  for (auto& r : prof_recs) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
  prof_recs.clear();
}

hub_ansatz::~hub_ansatz() {
  prof_clear();
  for (auto& kv : plans) delete kv.second;
  for (auto& kv : small_plans) delete kv.second;
  for (auto& kv : row_plans) delete kv.second;
}

// ---------------------------------------------------------------------------
// FP64 symmetric eigensolver (cyclic Jacobi) and determinants
// ---------------------------------------------------------------------------

namespace {

void jacobi_eigh(int n, std::vector<double> a, std::vector<double>& w, std::vector<double>& v) {
  v.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += a[(size_t)i * n + j] * a[(size_t)i * n + j];
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = c * akp - s * akq;
          a[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = c * apk - s * aqk;
          a[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
          v[(size_t)k * n + p] = c * vkp - s * vkq;
          v[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a[(size_t)i * n + i];
  // sort ascending (stable, with the eigenvector columns)
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return w[x] < w[y]; });
  std::vector<double> w2(n), v2((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w2[j] = w[idx[j]];
    for (int i = 0; i < n; ++i) v2[(size_t)i * n + j] = v[(size_t)i * n + idx[j]];
  }
  // gauge: largest-magnitude entry positive (lowest index on a tie)
  for (int j = 0; j < n; ++j) {
    double mx = 0.0;
    for (int i = 0; i < n; ++i) mx = std::max(mx, std::fabs(v2[(size_t)i * n + j]));
    int im = 0;
    for (int i = 0; i < n; ++i)
      if (std::fabs(v2[(size_t)i * n + j]) >= mx - 1e-12) { im = i; break; }
    if (v2[(size_t)im * n + j] < 0)
      for (int i = 0; i < n; ++i) v2[(size_t)i * n + j] = -v2[(size_t)i * n + j];
  }
  w = w2;
  v = v2;
}

double det_lu(int n, std::vector<double> m) {
  double d = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(m[(size_t)r * n + c]) > std::fabs(m[(size_t)piv * n + c])) piv = r;
    if (m[(size_t)piv * n + c] == 0.0) return 0.0;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(m[(size_t)c * n + k], m[(size_t)piv * n + k]);
      d = -d;
    }
    const double p = m[(size_t)c * n + c];
    d *= p;
    for (int r = c + 1; r < n; ++r) {
      const double f = m[(size_t)r * n + c] / p;
      for (int k = c; k < n; ++k) m[(size_t)r * n + k] -= f * m[(size_t)c * n + k];
    }
  }
  return d;
}
}  // namespace

// ---------------------------------------------------------------------------
// lattice helper and model
// ---------------------------------------------------------------------------

extern "C" hub_status hub_square_lattice(int32_t nx, int32_t ny, int32_t order, int32_t* bonds,
                                         int32_t* bond_class, int32_t* n_bonds) {
  if (nx < 1 || ny < 1 || nx * ny > 16) return fail(HUB_EINVAL, "hub_square_lattice: need 1 <= nx*ny <= 16");
  if (order != 0 && order != 1) return fail(HUB_EINVAL, "hub_square_lattice: order must be 0 or 1");
  if (!n_bonds) return fail(HUB_EINVAL, "hub_square_lattice: n_bonds is NULL");
  auto site = [&](int x, int y) { return x * ny + ((order == 1 && (x & 1)) ? ny - 1 - y : y); };
  int nb = 0;
  auto add = [&](int i, int j, int cls) {
    if (bonds) { bonds[2 * nb] = std::min(i, j); bonds[2 * nb + 1] = std::max(i, j); }
    if (bond_class) bond_class[nb] = cls;
    ++nb;
  };
  for (int x = 0; x < nx; ++x)
    for (int y = 0; y + 1 < ny; ++y) add(site(x, y), site(x, y + 1), (y & 1) ? 1 : 0);
  for (int x = 0; x + 1 < nx; ++x)
    for (int y = 0; y < ny; ++y) add(site(x, y), site(x + 1, y), (x & 1) ? 3 : 2);
  *n_bonds = nb;
  return HUB_OK;
}

extern "C" hub_status hub_create(const hub_lattice* lat, const double* t_ij, const double* U_i,
                                 const double* V_ij, int32_t n_up, int32_t n_dn, hub_t* out) {
  if (!lat || !t_ij || !out) return fail(HUB_EINVAL, "hub_create: NULL argument");
  *out = nullptr;
  const int L = lat->n_sites;
  if (L < 1 || 2 * L > kMaxQubits) return fail(HUB_EINVAL, "hub_create: need 1 <= n_sites <= 16");
  if (lat->n_bonds < 0 || (lat->n_bonds > 0 && !lat->bonds)) return fail(HUB_EINVAL, "hub_create: bad bond list");
  if (n_up < 0 || n_up > L || n_dn < 0 || n_dn > L) return fail(HUB_EINVAL, "hub_create: particle numbers out of range");
  auto m = new hub_model();
  m->L = L;
  m->n = 2 * L;
  m->n_up = n_up;
  m->n_dn = n_dn;
  m->up.resize(L);
  m->dn.resize(L);
  if ((lat->mode_up == nullptr) != (lat->mode_dn == nullptr)) {
    delete m;
    return fail(HUB_EINVAL, "hub_create: give both mode maps or neither");
  }
  std::vector<int> used(2 * L, 0);
  for (int i = 0; i < L; ++i) {
    m->up[i] = lat->mode_up ? lat->mode_up[i] : i;
    m->dn[i] = lat->mode_dn ? lat->mode_dn[i] : L + i;
    for (int md : {m->up[i], m->dn[i]}) {
      if (md < 0 || md >= 2 * L || used[md]++) {
        delete m;
        return fail(HUB_EINVAL, "hub_create: mode maps are not a permutation of 0..2L-1");
      }
    }
  }
  bool blocked = true, inter = true;
  for (int i = 0; i < L; ++i) {
    blocked = blocked && m->up[i] == i && m->dn[i] == L + i;
    inter = inter && m->up[i] == 2 * i && m->dn[i] == 2 * i + 1;
  }
  if (blocked) { m->layout = 0; m->s = L; }
  else if (inter) { m->layout = 1; m->s = 1; }
  else {
    delete m;
    return fail(HUB_EUNSUPPORTED, "hub_create: mode maps must be blocked (up i -> i, dn i -> L+i) or interleaved (up i -> 2i, dn i -> 2i+1)");
  }
  std::vector<std::vector<int>> isbond(L, std::vector<int>(L, 0));
  for (int b = 0; b < lat->n_bonds; ++b) {
    const int i = lat->bonds[2 * b], j = lat->bonds[2 * b + 1];
    if (i < 0 || j < 0 || i >= L || j >= L || i == j || isbond[i][j]) {
      delete m;
      return fail(HUB_EINVAL, "hub_create: bond " + std::to_string(b) + " is invalid or repeated");
    }
    isbond[i][j] = isbond[j][i] = 1;
    m->bonds.push_back({std::min(i, j), std::max(i, j)});
  }
  m->t.assign(t_ij, t_ij + (size_t)L * L);
  m->U.assign(L, 0.0);
  if (U_i) m->U.assign(U_i, U_i + L);
  m->V.assign((size_t)L * L, 0.0);
  if (V_ij) m->V.assign(V_ij, V_ij + (size_t)L * L);
  for (int i = 0; i < L; ++i) {
    if (!std::isfinite(m->U[i])) { delete m; return fail(HUB_EINVAL, "hub_create: U not finite"); }
    for (int j = 0; j < L; ++j) {
      const double a = m->t[(size_t)i * L + j], b = m->t[(size_t)j * L + i];
      const double va = m->V[(size_t)i * L + j], vb = m->V[(size_t)j * L + i];
      if (!std::isfinite(a) || !std::isfinite(va)) { delete m; return fail(HUB_EINVAL, "hub_create: t or V not finite"); }
      if (std::fabs(a - b) > 1e-12 * (1.0 + std::fabs(a)) || std::fabs(va - vb) > 1e-12 * (1.0 + std::fabs(va))) {
        delete m;
        return fail(HUB_EINVAL, "hub_create: t and V must be symmetric");
      }
      if (i != j && !isbond[i][j] && (a != 0.0 || va != 0.0)) {
        delete m;
        return fail(HUB_EINVAL, "hub_create: t_ij or V_ij nonzero off the bond list");
      }
      if (i == j && va != 0.0) { delete m; return fail(HUB_EINVAL, "hub_create: V has a nonzero diagonal"); }
    }
  }
  *out = m;
  return HUB_OK;
}

extern "C" void hub_destroy(hub_t m) { delete m; }

// ---------------------------------------------------------------------------
// ansatz construction: gates, H terms, diagonal operators and their tables
// ---------------------------------------------------------------------------

namespace {

int add_diag_op(hub_ansatz* a, const std::vector<std::vector<double>>& xcoef,
                const std::vector<double>& xconst,
                const std::vector<std::vector<double>>& ycoef,
                const std::vector<std::pair<int, int>>& vbonds,
                const std::vector<std::vector<double>>& vval,
                const std::vector<std::pair<int, int>>& mpairs,
                const std::vector<std::vector<double>>& mval, int param) {
  DiagOpDev d;
  std::memset(&d, 0, sizeof(d));
  bool any_x = false, any_y = false;
  for (int r = 0; r < a->n_inst; ++r) {
    for (double v : xcoef[r]) any_x = any_x || v != 0.0;
    any_x = any_x || xconst[r] != 0.0;
    for (double v : ycoef[r]) any_y = any_y || v != 0.0;
  }
  d.has_x = any_x ? (a->n + 7) / 8 : 0;
  int maxup = 0;
  for (int i = 0; i < a->L; ++i) maxup = std::max(maxup, a->models[0]->up[i]);
  d.has_y = any_y ? (maxup + 8) / 8 : 0;
  d.n_vb = (int)vbonds.size();
  d.v_uniform = 1;
  for (int r = 0; r < a->n_inst; ++r)
    for (int b = 1; b < d.n_vb; ++b) d.v_uniform = d.v_uniform && vval[r][b] == vval[r][0];
  for (int b = 0; b < d.n_vb; ++b) {
    d.vb_up[b] = a->models[0]->up[vbonds[b].first];
    d.vb_up2[b] = a->models[0]->up[vbonds[b].second];
  }
  d.n_vs = 0;
  for (int b = 0; b < d.n_vb && d.n_vs >= 0; ++b) {
    const int u1 = std::min(d.vb_up[b], d.vb_up2[b]), u2 = std::max(d.vb_up[b], d.vb_up2[b]);
    int g = 0;
    while (g < d.n_vs && d.vs_shift[g] != u2 - u1) ++g;
    if (g == d.n_vs) {
      if (g == 32) { d.n_vs = -1; break; }
      d.vs_shift[g] = u2 - u1;
      d.vs_mask[g] = 0u;
      ++d.n_vs;
    }
    if (u1 == u2 || (d.vs_mask[g] >> u1 & 1u)) d.n_vs = -1;   // not a plain bond list
    else d.vs_mask[g] |= 1u << u1;
  }
  d.n_mp = (int)mpairs.size();
  for (int m = 0; m < d.n_mp; ++m) {
    d.mp_p[m] = mpairs[m].first;
    d.mp_q[m] = mpairs[m].second;
  }
  d.mp_roff = 2048 + d.n_vb;
  d.param = param;
  d.real_off = a->real_stride;
  const int real_len = 2048 + d.n_vb + d.n_mp;
  // real tables per instance (appended; real_stride grows)
  std::vector<std::vector<double>> rt(a->n_inst, std::vector<double>(real_len, 0.0));
  for (int r = 0; r < a->n_inst; ++r) {
    for (int byte = 0; byte < 4; ++byte)
      for (int j = 0; j < 256; ++j) {
        double vx = (byte == 0) ? xconst[r] : 0.0, vy = 0.0;
        for (int bit = 0; bit < 8; ++bit) {
          const int mode = 8 * byte + bit;
          if (!((j >> bit) & 1) || mode >= a->n) continue;
          vx += xcoef[r][mode];
          vy += ycoef[r][mode];
        }
        rt[r][byte * 256 + j] = vx;
        rt[r][1024 + byte * 256 + j] = vy;
      }
    for (int b = 0; b < d.n_vb; ++b) rt[r][2048 + b] = vval[r][b];
    for (int m = 0; m < d.n_mp; ++m) rt[r][d.mp_roff + m] = mval[r][m];
  }
  const int old = a->real_stride;
  std::vector<double> nr((size_t)a->n_inst * (old + real_len));
  for (int r = 0; r < a->n_inst; ++r) {
    std::copy(a->real_tabs.begin() + (size_t)r * old, a->real_tabs.begin() + (size_t)(r + 1) * old,
              nr.begin() + (size_t)r * (old + real_len));
    std::copy(rt[r].begin(), rt[r].end(), nr.begin() + (size_t)r * (old + real_len) + old);
  }
  a->real_tabs.swap(nr);
  a->real_stride = old + real_len;
  // phase table entries (generator values; phases made per batch element)
  if (param >= 0) {
    d.phase_off = a->n_tab;
    const int vlen = d.n_vb == 0 ? 0 : (d.v_uniform ? 4 * d.n_vb + 1 : 5 * d.n_vb);
    d.mp_poff = 2048 + vlen;
    const int len = 2048 + vlen + d.n_mp;
    std::vector<double> nv((size_t)a->n_inst * (a->n_tab + len));
    for (int r = 0; r < a->n_inst; ++r) {
      std::copy(a->tab_val.begin() + (size_t)r * a->n_tab, a->tab_val.begin() + (size_t)(r + 1) * a->n_tab,
                nv.begin() + (size_t)r * (a->n_tab + len));
      double* dst = nv.data() + (size_t)r * (a->n_tab + len) + a->n_tab;
      std::copy(rt[r].begin(), rt[r].begin() + 2048, dst);
      if (d.n_vb > 0) {
        if (d.v_uniform)
          for (int K = 0; K <= 4 * d.n_vb; ++K) dst[2048 + K] = vval[r][0] * K;
        else
          for (int b = 0; b < d.n_vb; ++b)
            for (int e = 0; e < 5; ++e) dst[2048 + 5 * b + e] = vval[r][b] * e;
      }
      for (int m = 0; m < d.n_mp; ++m) dst[d.mp_poff + m] = mval[r][m];
    }
    a->tab_val.swap(nv);
    for (int e = 0; e < len; ++e) a->tab_param.push_back(param);
    for (int i = 0; i < d.has_x; ++i)
      for (int j = 0; j < 256; ++j) a->tab_live.push_back(a->n_tab + i * 256 + j);
    for (int i = 0; i < d.has_y; ++i)
      for (int j = 0; j < 256; ++j) a->tab_live.push_back(a->n_tab + 1024 + i * 256 + j);
    for (int e = 0; e < vlen + d.n_mp; ++e) a->tab_live.push_back(a->n_tab + 2048 + e);
    a->n_tab += len;
  } else {
    d.phase_off = -1;
  }
  a->diag_ops.push_back(d);
  return (int)a->diag_ops.size() - 1;
}
}  // namespace

namespace hubsv {

uint64_t diag_support(const hub_ansatz* a, int di) {
  // modes that the diagonal operator reads
  const DiagOpDev& d = a->diag_ops[di];
  uint64_t m = 0;
  for (int r = 0; r < a->n_inst; ++r) {
    const double* rt = a->real_tabs.data() + (size_t)r * a->real_stride + d.real_off;
    for (int mode = 0; mode < a->n; ++mode) {
      const int byte = mode / 8, bit = mode % 8;
      if (rt[byte * 256 + (1 << bit)] != rt[byte * 256]) m |= 1ull << mode;
      if (d.has_y && rt[1024 + byte * 256 + (1 << bit)] != 0.0) m |= (1ull << mode) | (1ull << (mode + a->s));
    }
  }
  for (int b = 0; b < d.n_vb; ++b) {
    m |= 1ull << d.vb_up[b];
    m |= 1ull << (d.vb_up[b] + a->s);
    m |= 1ull << d.vb_up2[b];
    m |= 1ull << (d.vb_up2[b] + a->s);
  }
  for (int k = 0; k < d.n_mp; ++k) m |= (1ull << d.mp_p[k]) | (1ull << d.mp_q[k]);
  return m;
}

}  // namespace hubsv

extern "C" hub_status ans_create_multi(const hub_t* models, int32_t n_models, int32_t n_layers,
                                       int32_t groups_per_layer, const hub_group* groups, ans_t* out) {
  if (!models || !out || n_models < 1 || n_layers < 0 || groups_per_layer < 0 ||
      (n_layers * groups_per_layer > 0 && !groups))
    return fail(HUB_EINVAL, "ans_create: bad arguments");
  *out = nullptr;
  for (int r = 0; r < n_models; ++r)
    if (!models[r]) return fail(HUB_EINVAL, "ans_create: NULL model");
  const hub_model* m0 = models[0];
  for (int r = 1; r < n_models; ++r) {
    const hub_model* m = models[r];
    if (m->L != m0->L || m->up != m0->up || m->dn != m0->dn || m->bonds != m0->bonds ||
        m->n_up != m0->n_up || m->n_dn != m0->n_dn)
      return fail(HUB_EINVAL, "ans_create: instances must share lattice, modes and particle numbers");
  }
  auto a = new hub_ansatz();
  a->models.assign(models, models + n_models);
  a->n_inst = n_models;
  a->L = m0->L;
  a->n = m0->n;
  a->s = m0->s;
  a->layout = m0->layout;
  for (int i = 0; i < a->L; ++i) a->upmask |= 1ull << m0->up[i];
  const int L = a->L, R = n_models, nb = (int)m0->bonds.size();
  int P = 0;
  const int G = n_layers * groups_per_layer;
  auto bad = [&](const std::string& msg) { delete a; return fail(HUB_EINVAL, "ans_create: " + msg); };
  for (int g = 0; g < G; ++g) {
    const hub_group& gr = groups[g];
    if (gr.param < 0) return bad("negative parameter index");
    if (gr.n_terms < 0 || (gr.n_terms > 0 && !gr.terms)) return bad("bad term list");
    P = std::max(P, gr.param + 1);
    const bool hop = gr.kind == HUB_G_HOP;
    if (gr.kind < 0 || gr.kind > HUB_G_CPHASE) return bad("unknown group kind");
    if (gr.kind == HUB_G_GIVENS || gr.kind == HUB_G_CPHASE) {
      // terms: n_terms mode pairs (p, q); Givens pairs of one group touch
      // disjoint modes, so that its factors commute
      if (gr.kind == HUB_G_CPHASE && gr.n_terms > kMaxModePairs) return bad("too many mode pairs in a CPHASE group");
      uint64_t used = 0;
      for (int k = 0; k < gr.n_terms; ++k) {
        const int p = gr.terms[2 * k], q = gr.terms[2 * k + 1];
        if (p < 0 || q < 0 || p >= a->n || q >= a->n || p == q) return bad("mode pair out of range");
        if (gr.kind == HUB_G_GIVENS) {
          if ((used >> p & 1) || (used >> q & 1)) return bad("Givens pairs of one group must touch disjoint modes");
          used |= (1ull << p) | (1ull << q);
          if (((a->upmask >> p) & 1) != ((a->upmask >> q) & 1)) a->spin_mix = true;
        }
      }
      continue;
    }
    uint64_t seen = 0;
    for (int k = 0; k < gr.n_terms; ++k) {
      const int tm = gr.terms[k];
      if (gr.kind == HUB_G_HOP || gr.kind == HUB_G_NN_V) {
        if (tm < 0 || tm >= nb) return bad("bond index out of range");
        if (hop) {
          const int i = m0->bonds[tm].first, j = m0->bonds[tm].second;
          if ((seen >> i & 1) || (seen >> j & 1)) return bad("hop terms of one group must touch disjoint sites");
          seen |= (1ull << i) | (1ull << j);
        }
      } else if (gr.kind == HUB_G_RZ) {
        if (tm < 0 || tm >= a->n) return bad("mode index out of range");
      } else {
        if (tm < 0 || tm >= L) return bad("site index out of range");
      }
    }
  }
  if (P + 2 > kMaxSlots) return bad("too many parameters (accumulator slots are 16-bit)");
  a->P = P;
  // H hop terms: every bond, both spins; term index 2*bond + spin
  for (int b = 0; b < nb; ++b)
    for (int sp = 0; sp < 2; ++sp) {
      const auto& mm = sp == 0 ? m0->up : m0->dn;
      int p = mm[m0->bonds[b].first], q = mm[m0->bonds[b].second];
      if (p > q) std::swap(p, q);
      a->hterms.push_back({p, q});
    }
  // columns of the -t table: one per H hop term, then one column of -1 for
  // the unit generators -(a+_p a_q + h.c.) of HUB_G_GIVENS factors
  const int unit_col = (int)a->hterms.size();
  a->n_hcol = unit_col + 1;
  a->hcoef.assign((size_t)R * a->n_hcol, 0.0);
  for (int r = 0; r < R; ++r) {
    for (int b = 0; b < nb; ++b)
      for (int sp = 0; sp < 2; ++sp) {
        const auto& bd = m0->bonds[b];
        a->hcoef[(size_t)r * a->n_hcol + 2 * b + sp] = -models[r]->t[(size_t)bd.first * L + bd.second];
      }
    a->hcoef[(size_t)r * a->n_hcol + unit_col] = -1.0;
  }
  // H diagonal: potential -t_ii on both modes of site i, U_i on double occupancy, V bonds
  {
    std::vector<std::vector<double>> xc(R, std::vector<double>(a->n, 0.0)), yc(R, std::vector<double>(a->n, 0.0)), vv(R);
    std::vector<double> xk(R, 0.0);
    std::vector<std::pair<int, int>> vb;
    for (int b = 0; b < nb; ++b) {
      bool any = false;
      for (int r = 0; r < R; ++r) any = any || models[r]->V[(size_t)m0->bonds[b].first * L + m0->bonds[b].second] != 0.0;
      if (any) vb.push_back(m0->bonds[b]);
    }
    if (vb.size() > 64) return bad("too many V bonds");
    for (int r = 0; r < R; ++r) {
      for (int i = 0; i < L; ++i) {
        xc[r][m0->up[i]] += -models[r]->t[(size_t)i * L + i];
        xc[r][m0->dn[i]] += -models[r]->t[(size_t)i * L + i];
        yc[r][m0->up[i]] += models[r]->U[i];
      }
      for (auto& bd : vb) vv[r].push_back(models[r]->V[(size_t)bd.first * L + bd.second]);
    }
    a->h_diag = add_diag_op(a, xc, xk, yc, vb, vv, {}, {}, -1);
  }
  // forward sequence
  a->n_layers = n_layers;
  for (int g = 0; g < G; ++g) {
    const hub_group& gr = groups[g];
    if (groups_per_layer > 0 && g % groups_per_layer == 0) a->layer_begin.push_back((int)a->fwd.size());
    if (gr.kind == HUB_G_HOP) {
      for (int k = 0; k < gr.n_terms; ++k) {
        const int b = gr.terms[k];
        for (int sp = 0; sp < 2; ++sp) {
          SeqOp op;
          op.kind = OP_GIV;
          op.hterm = 2 * b + sp;
          op.p = a->hterms[op.hterm].p;
          op.q = a->hterms[op.hterm].q;
          op.gate = a->n_gates++;
          op.slot = gr.param;
          op.support = (1ull << op.p) | (1ull << op.q);
          op.cls = 0;
          a->gate_param.push_back(gr.param);
          a->gate_unit.push_back(0);
          a->fwd.push_back(op);
        }
      }
    } else if (gr.kind == HUB_G_GIVENS) {
      for (int k = 0; k < gr.n_terms; ++k) {
        SeqOp op;
        op.kind = OP_GIV;
        op.hterm = unit_col;
        op.p = std::min(gr.terms[2 * k], gr.terms[2 * k + 1]);
        op.q = std::max(gr.terms[2 * k], gr.terms[2 * k + 1]);
        op.gate = a->n_gates++;
        op.slot = gr.param;
        op.support = (1ull << op.p) | (1ull << op.q);
        op.cls = 0;
        a->gate_param.push_back(gr.param);
        a->gate_unit.push_back(1);
        a->fwd.push_back(op);
      }
    } else {
      std::vector<std::vector<double>> xc(R, std::vector<double>(a->n, 0.0)), yc(R, std::vector<double>(a->n, 0.0)), vv(R);
      std::vector<double> xk(R, 0.0);
      std::vector<std::pair<int, int>> vb, mp;
      std::vector<std::vector<double>> mv(R);
      for (int k = 0; k < gr.n_terms && gr.kind == HUB_G_CPHASE; ++k) {
        // generator -n_p n_q: exp(-i phi G) puts exp(+i phi) on |11> (Eq. 8)
        mp.push_back({gr.terms[2 * k], gr.terms[2 * k + 1]});
        for (int r = 0; r < R; ++r) mv[r].push_back(-1.0);
      }
      for (int k = 0; k < gr.n_terms && gr.kind != HUB_G_CPHASE; ++k) {
        const int tm = gr.terms[k];
        for (int r = 0; r < R; ++r) {
          const hub_model* m = models[r];
          if (gr.kind == HUB_G_ONSITE) yc[r][m0->up[tm]] += m->U[tm];
          else if (gr.kind == HUB_G_POT) {
            xc[r][m0->up[tm]] += -m->t[(size_t)tm * L + tm];
            xc[r][m0->dn[tm]] += -m->t[(size_t)tm * L + tm];
          } else if (gr.kind == HUB_G_RZ) {
            xc[r][tm] += -1.0;
            xk[r] += 0.5;
          } else if (gr.kind == HUB_G_NN_V) {
            vv[r].push_back(m->V[(size_t)m0->bonds[tm].first * L + m0->bonds[tm].second]);
          }
        }
        if (gr.kind == HUB_G_NN_V) vb.push_back(m0->bonds[tm]);
      }
      if (vb.size() > 64) return bad("too many V bonds in a group");
      SeqOp op;
      op.kind = OP_DIAG;
      op.diag = add_diag_op(a, xc, xk, yc, vb, vv, mp, mv, gr.param);
      op.slot = gr.param;
      op.diagonal = true;
      op.support = diag_support(a, op.diag);
      op.cls = 0;
      a->fwd.push_back(op);
    }
  }
  a->gate_t.resize((size_t)R * a->n_gates);
  for (int r = 0; r < R; ++r) {
    int gi = 0;
    for (const SeqOp& op : a->fwd)
      if (op.kind == OP_GIV) {
        if (a->gate_unit[gi]) {
          a->gate_t[(size_t)r * a->n_gates + gi++] = 1.0;
        } else {
          const auto& bd = m0->bonds[op.hterm / 2];
          a->gate_t[(size_t)r * a->n_gates + gi++] = models[r]->t[(size_t)bd.first * L + bd.second];
        }
      }
  }
  *out = a;
  return HUB_OK;
}

extern "C" hub_status ans_create(hub_t model, int32_t n_layers, int32_t groups_per_layer,
                                 const hub_group* groups, ans_t* out) {
  return ans_create_multi(&model, 1, n_layers, groups_per_layer, groups, out);
}

extern "C" void ans_destroy(ans_t a) { delete a; }
extern "C" int32_t ans_num_params(ans_t a) { return a ? a->P : -1; }
extern "C" int32_t ans_num_qubits(ans_t a) { return a ? a->n : -1; }

extern "C" hub_status ans_set_tile(ans_t a, int32_t dtype, int32_t log2_tile) {
  if (!a || (dtype != HUB_C64 && dtype != HUB_C128)) return fail(HUB_EINVAL, "ans_set_tile: bad arguments");
  if (log2_tile != 0 && (log2_tile < 6 || log2_tile > kMaxTileBits))
    return fail(HUB_EINVAL, "ans_set_tile: log2_tile must be 0 or in [6, 14]");
  a->tile_override[dtype] = log2_tile;
  for (auto& kv : a->plans) delete kv.second;
  a->plans.clear();
  return HUB_OK;
}

extern "C" hub_status ans_set_threads(ans_t a, int32_t dtype, int32_t engine, int32_t threads) {
  if (!a || (dtype != HUB_C64 && dtype != HUB_C128)) return fail(HUB_EINVAL, "ans_set_threads: bad arguments");
  if (engine == HUB_ENGINE_ONCHIP) {
    if (threads != 0 && threads != 256 && threads != 512)
      return fail(HUB_EINVAL, "ans_set_threads: on-chip threads must be 0, 256 or 512");
    a->small_threads[dtype] = threads;
    return HUB_OK;
  }
  if (engine == HUB_ENGINE_ROWS) {
    if (threads != 0 && threads != 256 && threads != 512 && threads != 1024)
      return fail(HUB_EINVAL, "ans_set_threads: row threads must be 0, 256, 512 or 1024");
    a->row_threads[dtype] = threads;
    return HUB_OK;
  }
  return fail(HUB_EINVAL, "ans_set_threads: engine must be HUB_ENGINE_ONCHIP or HUB_ENGINE_ROWS");
}

extern "C" hub_status ans_set_runs(ans_t a, int32_t dtype, int32_t log2_run) {
  if (!a || (dtype != HUB_C64 && dtype != HUB_C128)) return fail(HUB_EINVAL, "ans_set_runs: bad arguments");
  if (log2_run != 0 && (log2_run < 1 || log2_run > 5))
    return fail(HUB_EINVAL, "ans_set_runs: log2_run must be 0 or in [1, 5]");
  a->run_override[dtype] = log2_run;
  for (auto& kv : a->plans) delete kv.second;
  a->plans.clear();
  return HUB_OK;
}

namespace {

hub_status ensure_device(hub_ansatz* a) {
  if (a->dev_ready) return HUB_OK;
  hub_status st;
  if ((st = a->d_gate_param.upload(a->gate_param, "gate params")) != HUB_OK ||
      (st = a->d_gate_t.upload(a->gate_t, "gate coefficients")) != HUB_OK ||
      (st = a->d_tab_param.upload(a->tab_param, "phase params")) != HUB_OK ||
      (st = a->d_tab_val.upload(a->tab_val, "phase values")) != HUB_OK ||
      (st = a->d_tab_live.upload(a->tab_live.empty() ? std::vector<int32_t>(1) : a->tab_live,
                                 "phase entries")) != HUB_OK ||
      (st = a->d_hcoef.upload(a->hcoef, "hop coefficients")) != HUB_OK ||
      (st = a->d_real.upload(a->real_tabs, "diagonal tables")) != HUB_OK ||
      (st = a->d_real32.upload(std::vector<float>(a->real_tabs.begin(), a->real_tabs.end()),
                               "diagonal tables (FP32)")) != HUB_OK ||
      (st = a->d_diag.upload(a->diag_ops, "diagonal operators")) != HUB_OK)
    return st;
  a->dev_ready = true;
  return HUB_OK;
}
hub_status get_plan(hub_ansatz* a, int which, int dtype, uint32_t flags, Plan*& pl) {
  // flags: PREP_FUSED | KEEP_STATE | internal checkpoint bit (4)
  const int key = which * 16 + dtype * 8 + (int)(flags & 7u);
  auto it = a->plans.find(key);
  if (it != a->plans.end()) { pl = it->second; return HUB_OK; }
  hub_status st = make_plan(a, which, dtype, flags, pl);
  if (st != HUB_OK) return st;
  a->plans[key] = pl;
  return HUB_OK;
}

hub_status run_plan(hub_ansatz* a, Plan* pl, int dtype, const double* theta, void* psi, void* lam,
                    void* ckpt, int64_t batch, double* E, double* grad, cudaStream_t st) {
  const int n = a->n;
  const int n_slots = a->P + 2;
  hub_status s;
  if ((s = ensure_device(a)) != HUB_OK) return s;
  if (!pl->uploaded) {
    if ((s = pl->ops.upload(pl->hops.empty() ? std::vector<OpDev>(1) : pl->hops, "sweep ops")) != HUB_OK) return s;
    if ((s = pl->phases.upload(pl->hphases, "sweep phases")) != HUB_OK) return s;
    if ((s = pl->slots.upload(pl->slot_map.empty() ? std::vector<int32_t>(1) : pl->slot_map, "sweep slots")) != HUB_OK)
      return s;
    pl->uploaded = true;
  }
  const size_t r2 = dtype == HUB_C64 ? 8 : 16;
  if ((s = a->d_coef[dtype].ensure(16 * std::max<int64_t>(1, batch * a->n_gates), "coefficients")) != HUB_OK) return s;
  if ((s = a->d_phase[dtype].ensure(r2 * std::max<int64_t>(1, batch * a->n_tab), "phase tables")) != HUB_OK) return s;
  if ((s = a->d_acc.ensure(8 * (size_t)batch * n_slots, "accumulators")) != HUB_OK) return s;
  HUB_CUDA(launch_zero((double*)a->d_acc.p, batch * n_slots, st), "zero accumulators");
  if (theta) {
    HUB_CUDA(launch_coef(dtype, theta, a->P, (const int32_t*)a->d_gate_param.p, (const double*)a->d_gate_t.p,
                         a->n_gates, a->d_coef[dtype].p, (const int32_t*)a->d_tab_param.p,
                         (const double*)a->d_tab_val.p, a->n_tab, (const int32_t*)a->d_tab_live.p,
                         (int)a->tab_live.size(), a->d_phase[dtype].p, batch,
                         a->n_inst, st),
             "coefficient kernel");
  }
  if (pl->sector && pl->prep) {
    // sweeps visit only the tiles that meet the sector; the amplitudes
    // outside it, which those tiles also hold, must read as zero (a
    // backward-only pass reads a psi that its forward pass left so)
    const size_t vb = (size_t)batch * ((size_t)1 << n) * (dtype == HUB_C64 ? 8 : 16);
    HUB_CUDA(cudaMemsetAsync(psi, 0, vb, st), "clear psi");
    if (lam) HUB_CUDA(cudaMemsetAsync(lam, 0, vb, st), "clear lam");
    if (ckpt) HUB_CUDA(cudaMemsetAsync(ckpt, 0, vb, st), "clear checkpoint");
  }
  KernelArgs ka;
  std::memset(&ka, 0, sizeof(ka));
  ka.psi = psi;
  ka.lam = lam;
  ka.ckpt = ckpt;
  ka.ops = (const OpDev*)pl->ops.p;
  ka.phases = (const PhaseDev*)pl->phases.p;
  ka.diag_ops = (const DiagOpDev*)a->d_diag.p;
  ka.theta = theta;
  ka.P = a->P;
  ka.coef = a->d_coef[dtype].p;
  ka.n_gates = a->n_gates;
  ka.hcoef = (const double*)a->d_hcoef.p;
  ka.n_hterms = a->n_hcol;
  ka.real_tabs = (const double*)a->d_real.p;
  ka.real_tabs32 = (const float*)a->d_real32.p;
  ka.real_stride = a->real_stride;
  ka.phase_tabs = a->d_phase[dtype].p;
  ka.phase_stride = a->n_tab;
  ka.n_inst = a->n_inst;
  ka.n = n;
  ka.s = a->s;
  ka.upmask = a->upmask;
  ka.batch = batch;
  ka.n_tiles = ((uint64_t)batch) << (n - pl->k);
  if (ka.n_tiles >= (1ull << 31)) return fail(HUB_EUNSUPPORTED, "batch too large for one launch (2^31 tiles)");
  if ((uint64_t)batch * (uint64_t)a->n_tab >= (1ull << 31) ||
      (uint64_t)a->n_inst * (uint64_t)a->real_stride >= (1ull << 31))
    return fail(HUB_EUNSUPPORTED, "batch too large for one launch (32-bit table offsets)");
  ka.acc = (double*)a->d_acc.p;
  ka.n_slots = n_slots;
  ka.slot_E = a->P;
  ka.slot_N = a->P + 1;
  ka.slot_map = (const int32_t*)pl->slots.p;
  ka.prep.kind = a->prep_kind < 0 ? 0 : a->prep_kind;
  ka.prep.L = a->L;
  ka.prep.s = a->s;
  ka.prep.layout = a->layout;
  ka.prep.neel_x0 = a->neel_x0;
  ka.prep.sd = (const double*)a->d_sd.p;
  ka.prep.sd32 = (const float*)a->d_sd32.p;
  const int sms = device_sm_count();
  if (sms <= 0) return fail(HUB_ECUDA, "no CUDA device");
  const int optin = sweep_max_smem_optin();
  for (size_t i = 0; i < pl->sweeps.size(); ++i) {
    const SweepDev& sw = pl->sweeps[i];
    const int nv = pl->nvec[i];
    const int nph = sw.phase_end - sw.phase_begin;
    const size_t smem = sweep_smem_bytes(dtype, nv, sw.k, sw.n_lslot, nph, sw.op_end - sw.op_begin, 32 << sw.w);
    if ((int)smem > optin) return fail(HUB_EUNSUPPORTED, "tile does not fit in shared memory");
    HUB_CUDA(sweep_set_smem(dtype, nv, sw.r, 32 << sw.w, (sw.flags & SW_VPOP) != 0, smem), "cudaFuncSetAttribute");
    const int threads = 32 << sw.w;
    const int regs = std::max(1, sweep_regs(dtype, nv, sw.r, 32 << sw.w, (sw.flags & SW_VPOP) != 0));
    int per_sm = (int)((size_t)(228 * 1024) / (smem + 1024));
    per_sm = std::min(per_sm, 2048 / threads);
    per_sm = std::min(per_sm, 65536 / (regs * threads));
    per_sm = std::max(per_sm, 1);
    uint64_t grid = (uint64_t)sms * per_sm;
    const uint64_t sweep_tiles = sw.sector ? (uint64_t)batch * sw.live : ka.n_tiles;
    grid = std::min<uint64_t>(grid, std::max<uint64_t>(1, sweep_tiles));
    hub_ansatz::ProfRec rec{};
    if (a->prof) {
      HUB_CUDA(cudaEventCreate(&rec.e0), "cudaEventCreate");
      HUB_CUDA(cudaEventCreate(&rec.e1), "cudaEventCreate");
      HUB_CUDA(cudaEventRecord(rec.e0, st), "cudaEventRecord");
    }
    HUB_CUDA(launch_sweep(dtype, sw, ka, (int)grid, smem, st), "sweep kernel launch");
    if (a->prof) {
      HUB_CUDA(cudaEventRecord(rec.e1, st), "cudaEventRecord");
      const uint32_t f = sw.flags;
      const int nvec_io = ((f & SW_READ_PSI) ? 1 : 0) + ((f & SW_WRITE_PSI) ? 1 : 0) +
                          ((f & SW_READ_LAM) ? 1 : 0) + ((f & SW_WRITE_LAM) ? 1 : 0) +
                          ((f & SW_CKPT_WRITE) ? 1 : 0) + ((f & SW_CKPT_READ) ? 1 : 0);
      rec.nv = nv;
      rec.dtype = dtype;
      rec.bytes = (double)nvec_io * (double)(dtype == HUB_C64 ? 8 : 16) * (double)batch *
                  (sw.sector ? (double)sw.live * (double)(1ull << sw.k) : (double)(1ull << n));
      a->prof_recs.push_back(rec);
    }
  }
  HUB_CUDA(launch_finalize((const double*)a->d_acc.p, n_slots, a->P, a->P, E, grad, batch, st), "finalize kernel");
  return HUB_OK;
}

// The on-chip path (hubsv_small.cu) for a call, or nullptr when the call
// must run as sweeps: the state is caller-given or must be kept, the caller
// asked for sweeps, or the sector does not fit in one CTA's shared memory.
// The sector plan of a call kind (patterns, pair lists, operation sequence),
// shared by the on-chip and row engines; nullptr where none can be made.
SmallPlan* get_small_plan(hub_ansatz* a, int which) {
  auto it = a->small_plans.find(which);
  if (it != a->small_plans.end()) return it->second;
  SmallPlan* sp = nullptr;
  if (make_small_plan(a, which, sp) != HUB_OK) sp = nullptr;
  a->small_plans[which] = sp;   // a failed build is remembered as nullptr
  return sp;
}

SmallPlan* small_plan_for(hub_ansatz* a, int which, int dtype, uint32_t flags, size_t& smem) {
  if (!(flags & HUB_FLAG_PREP_FUSED) || (flags & (HUB_FLAG_KEEP_STATE | HUB_FLAG_SWEEPS | HUB_FLAG_ROWS)))
    return nullptr;
  SmallPlan* sp = get_small_plan(a, which);
  if (!sp) return nullptr;
  // the kernel's multiply-high division is exact for n * d < 2^32
  const uint64_t C = (uint64_t)sp->cup * (uint64_t)sp->cdn;
  if (C * (uint64_t)std::max(sp->cup, sp->cdn) >= (1ull << 32)) return nullptr;
  smem = small_smem_bytes(dtype, sp->cup, sp->cdn, (int)sp->pairs.size(), a->P + 2, a->n_gates,
                          a->n_hcol, a->small_threads[dtype] ? a->small_threads[dtype] : kSmallThreadsDefault);
  if ((int)smem > sweep_max_smem_optin()) return nullptr;
  return sp;
}

hub_status run_small(hub_ansatz* a, SmallPlan* sp, size_t smem, int dtype, const double* theta, int64_t batch,
                     double* E, double* grad, cudaStream_t st) {
  const int n_slots = a->P + 2;
  hub_status s;
  if ((s = ensure_device(a)) != HUB_OK) return s;
  if (!sp->uploaded) {
    if ((s = sp->d_ops.upload(sp->ops, "on-chip ops")) != HUB_OK ||
        (s = sp->d_xup.upload(sp->xup, "up patterns")) != HUB_OK ||
        (s = sp->d_xdn.upload(sp->xdn, "down patterns")) != HUB_OK ||
        (s = sp->d_pairs.upload(sp->pairs, "pattern pairs")) != HUB_OK)
      return s;
    sp->uploaded = true;
  }
  const size_t r2 = dtype == HUB_C64 ? 8 : 16;
  if ((s = a->d_coef[dtype].ensure(16 * std::max<int64_t>(1, batch * a->n_gates), "coefficients")) != HUB_OK) return s;
  if ((s = a->d_phase[dtype].ensure(r2 * std::max<int64_t>(1, batch * a->n_tab), "phase tables")) != HUB_OK) return s;
  if ((s = a->d_acc.ensure(8 * (size_t)batch * n_slots, "accumulators")) != HUB_OK) return s;
  if (theta) {
    HUB_CUDA(launch_coef(dtype, theta, a->P, (const int32_t*)a->d_gate_param.p, (const double*)a->d_gate_t.p,
                         a->n_gates, a->d_coef[dtype].p, (const int32_t*)a->d_tab_param.p,
                         (const double*)a->d_tab_val.p, a->n_tab, (const int32_t*)a->d_tab_live.p,
                         (int)a->tab_live.size(), a->d_phase[dtype].p, batch,
                         a->n_inst, st),
             "coefficient kernel");
  }
  SmallArgs ka;
  std::memset(&ka, 0, sizeof(ka));
  ka.ops = (const SmallOpDev*)sp->d_ops.p;
  ka.n_ops = (int)sp->ops.size();
  ka.xup = (const uint32_t*)sp->d_xup.p;
  ka.xdn = (const uint32_t*)sp->d_xdn.p;
  ka.cup = sp->cup;
  ka.cdn = sp->cdn;
  ka.ld = sp->cup | 1;
  ka.m_cup = small_magic(sp->cup);
  ka.m_cdn = small_magic(sp->cdn);
  ka.pairs = (const uint32_t*)sp->d_pairs.p;
  ka.n_pairs = (int)sp->pairs.size();
  ka.diag_ops = (const DiagOpDev*)a->d_diag.p;
  ka.coef = a->d_coef[dtype].p;
  ka.n_gates = a->n_gates;
  ka.hcoef = (const double*)a->d_hcoef.p;
  ka.n_hterms = a->n_hcol;
  ka.real_tabs = (const double*)a->d_real.p;
  ka.real_tabs32 = (const float*)a->d_real32.p;
  ka.real_stride = a->real_stride;
  ka.phase_tabs = a->d_phase[dtype].p;
  ka.phase_stride = a->n_tab;
  ka.n_inst = a->n_inst;
  ka.s = a->s;
  ka.upmask = a->upmask;
  ka.batch = batch;
  ka.acc = (double*)a->d_acc.p;
  ka.n_slots = n_slots;
  ka.slot_E = a->P;
  ka.slot_N = a->P + 1;
  ka.prep.kind = a->prep_kind;
  ka.prep.L = a->L;
  ka.prep.s = a->s;
  ka.prep.layout = a->layout;
  ka.prep.neel_x0 = a->neel_x0;
  ka.prep.sd = (const double*)a->d_sd.p;
  ka.prep.sd32 = (const float*)a->d_sd32.p;
  const int sms = device_sm_count();
  if (sms <= 0) return fail(HUB_ECUDA, "no CUDA device");
  const int nt = a->small_threads[dtype] ? a->small_threads[dtype] : kSmallThreadsDefault;
  const int per_sm = std::max(1, small_max_ctas_per_sm(dtype, nt, smem));
  const int64_t grid = std::min<int64_t>(batch, (int64_t)sms * per_sm);
  hub_ansatz::ProfRec rec{};
  if (a->prof) {
    HUB_CUDA(cudaEventCreate(&rec.e0), "cudaEventCreate");
    HUB_CUDA(cudaEventCreate(&rec.e1), "cudaEventCreate");
    HUB_CUDA(cudaEventRecord(rec.e0, st), "cudaEventRecord");
  }
  HUB_CUDA(launch_small(dtype, ka, nt, (int)grid, smem, st), "on-chip kernel launch");
  if (a->prof) {
    HUB_CUDA(cudaEventRecord(rec.e1, st), "cudaEventRecord");
    rec.nv = 0;   // on-chip: shared-memory amplitude traffic, no vector in HBM
    rec.dtype = dtype;
    rec.bytes = (double)sp->accesses * (double)(dtype == HUB_C64 ? 8 : 16) * (double)batch;
    a->prof_recs.push_back(rec);
  }
  HUB_CUDA(launch_finalize((const double*)a->d_acc.p, n_slots, a->P, a->P, E, grad, batch, st), "finalize kernel");
  return HUB_OK;
}

// The row engine (hubsv_rows.cu) for a call, or nullptr: the state is
// caller-given or must be kept, the caller asked for sweeps, a row (with
// lam, where the call builds it) does not fit in shared memory, or the
// compressed matrix and its transpose do not fit in the caller's psi buffer.
RowPlan* row_plan_for(hub_ansatz* a, int which, int dtype, uint32_t flags, SmallPlan*& sp_out) {
  if (!(flags & HUB_FLAG_PREP_FUSED) || (flags & (HUB_FLAG_KEEP_STATE | HUB_FLAG_SWEEPS))) return nullptr;
  SmallPlan* sp = get_small_plan(a, which);
  if (!sp) return nullptr;
  const uint64_t C = (uint64_t)sp->cup * (uint64_t)sp->cdn;
  if (2 * C > (1ull << a->n)) return nullptr;
  RowPlan* rp = nullptr;
  auto it = a->row_plans.find(which);
  if (it != a->row_plans.end()) {
    rp = it->second;
  } else {
    if (make_row_plan(a, which, sp, rp) != HUB_OK) rp = nullptr;
    a->row_plans[which] = rp;
  }
  if (!rp) return nullptr;
  const int optin = sweep_max_smem_optin();
  for (const RowSegHost& g : rp->segs) {
    const int nv = (g.flags & RS_HAS_LAM) ? 2 : 1;
    const int len = g.orient == 0 ? sp->cup : sp->cdn;
    const int nr = g.orient == 0 ? sp->cdn : sp->cup;
    const int no = g.op_end - g.op_begin;
    const RowLaunch rl =
        rows_launch(dtype, nv, len, nr, a->P + 2, a->n_gates, a->n_hcol, no, (flags & HUB_FLAG_ROW_CLUSTER) != 0,
                    a->row_threads[dtype]);
    if ((int)rl.smem > optin || rl.smem == 0) return nullptr;
  }
  sp_out = sp;
  return rp;
}

// Where the sector matrices are between row-engine calls of one evaluation
// (the overlap loss runs a forward and a backward plan): the region of
// psi / lam that holds them, their orientation (-1: none yet), and whether
// lam holds data.
struct RowRun {
  int cur = 0, orient = -1;
  bool lam_live = false;
};

hub_status run_rows(hub_ansatz* a, SmallPlan* sp, RowPlan* rp, int dtype, const double* theta, void* psi,
                    void* lam, int64_t batch, double* E, double* grad, uint32_t flags, cudaStream_t st,
                    RowRun* state = nullptr, bool finalize = true) {
  const bool force_cluster = (flags & HUB_FLAG_ROW_CLUSTER) != 0;
  const int n_slots = a->P + 2;
  hub_status s;
  if ((s = ensure_device(a)) != HUB_OK) return s;
  if (!sp->uploaded) {
    if ((s = sp->d_ops.upload(sp->ops, "on-chip ops")) != HUB_OK ||
        (s = sp->d_xup.upload(sp->xup, "up patterns")) != HUB_OK ||
        (s = sp->d_xdn.upload(sp->xdn, "down patterns")) != HUB_OK ||
        (s = sp->d_pairs.upload(sp->pairs, "pattern pairs")) != HUB_OK)
      return s;
    sp->uploaded = true;
  }
  if (!rp->uploaded) {
    if ((s = rp->d_ops.upload(rp->ops, "row ops")) != HUB_OK) return s;
    rp->uploaded = true;
  }
  const size_t r2 = dtype == HUB_C64 ? 8 : 16;
  if ((s = a->d_coef[dtype].ensure(16 * std::max<int64_t>(1, batch * a->n_gates), "coefficients")) != HUB_OK) return s;
  if ((s = a->d_phase[dtype].ensure(r2 * std::max<int64_t>(1, batch * a->n_tab), "phase tables")) != HUB_OK) return s;
  if ((s = a->d_acc.ensure(8 * (size_t)batch * n_slots, "accumulators")) != HUB_OK) return s;
  HUB_CUDA(launch_zero((double*)a->d_acc.p, batch * n_slots, st), "zero accumulators");
  if (theta) {
    HUB_CUDA(launch_coef(dtype, theta, a->P, (const int32_t*)a->d_gate_param.p, (const double*)a->d_gate_t.p,
                         a->n_gates, a->d_coef[dtype].p, (const int32_t*)a->d_tab_param.p,
                         (const double*)a->d_tab_val.p, a->n_tab, (const int32_t*)a->d_tab_live.p,
                         (int)a->tab_live.size(), a->d_phase[dtype].p, batch,
                         a->n_inst, st),
             "coefficient kernel");
  }
  // the compressed matrix (region 0) and its transpose (region 1) of psi,
  // likewise of lam, inside the caller's buffers
  const size_t mat = (size_t)batch * (size_t)sp->cup * (size_t)sp->cdn;   // amplitudes
  unsigned char* preg[2] = {(unsigned char*)psi, (unsigned char*)psi + mat * r2};
  unsigned char* lreg[2] = {(unsigned char*)lam, lam ? (unsigned char*)lam + mat * r2 : nullptr};
  int cur = state ? state->cur : 0;
  int orient = (state && state->orient >= 0) ? state->orient : (rp->segs.empty() ? 0 : rp->segs[0].orient);
  bool lam_live = state ? state->lam_live : false;
  const int sms = device_sm_count();
  if (sms <= 0) return fail(HUB_ECUDA, "no CUDA device");
  auto record = [&](hub_ansatz::ProfRec& rec, bool start) -> cudaError_t {
    if (!a->prof) return cudaSuccess;
    if (start) {
      cudaError_t e = cudaEventCreate(&rec.e0);
      if (e == cudaSuccess) e = cudaEventCreate(&rec.e1);
      if (e == cudaSuccess) e = cudaEventRecord(rec.e0, st);
      return e;
    }
    cudaError_t e = cudaEventRecord(rec.e1, st);
    a->prof_recs.push_back(rec);
    return e;
  };
  for (const RowSegHost& g : rp->segs) {
    if (g.orient != orient) {   // transpose psi (and lam) into the other region
      const int n_r = orient == 0 ? sp->cdn : sp->cup, n_c = orient == 0 ? sp->cup : sp->cdn;
      for (int v = 0; v < (lam_live ? 2 : 1); ++v) {
        unsigned char* const* reg = v == 0 ? preg : lreg;
        hub_ansatz::ProfRec rec{};
        HUB_CUDA(record(rec, true), "cudaEventRecord");
        HUB_CUDA(launch_transpose(dtype, reg[cur], reg[cur ^ 1], batch, n_r, n_c, st), "transpose");
        rec.nv = 4;
        rec.dtype = dtype;
        rec.bytes = 2.0 * (double)mat * (double)r2;
        HUB_CUDA(record(rec, false), "cudaEventRecord");
      }
      cur ^= 1;
      orient = g.orient;
    }
    const bool has_lam = (g.flags & RS_HAS_LAM) != 0;
    if (has_lam && !lam) return fail(HUB_EINVAL, "row engine: lam buffer needed");
    RowArgs ka;
    std::memset(&ka, 0, sizeof(ka));
    ka.ops = (const SmallOpDev*)rp->d_ops.p;
    ka.op_begin = g.op_begin;
    ka.op_end = g.op_end;
    ka.flags = g.flags;
    ka.psi = preg[cur];
    ka.lam = has_lam ? lreg[cur] : nullptr;
    ka.n_rows = orient == 0 ? sp->cdn : sp->cup;
    ka.row_len = orient == 0 ? sp->cup : sp->cdn;
    ka.xrow = (const uint32_t*)(orient == 0 ? sp->d_xdn.p : sp->d_xup.p);
    ka.xin = (const uint32_t*)(orient == 0 ? sp->d_xup.p : sp->d_xdn.p);
    ka.pairs = (const uint32_t*)sp->d_pairs.p;
    ka.diag_ops = (const DiagOpDev*)a->d_diag.p;
    ka.coef = a->d_coef[dtype].p;
    ka.n_gates = a->n_gates;
    ka.hcoef = (const double*)a->d_hcoef.p;
    ka.n_hterms = a->n_hcol;
    ka.real_tabs = (const double*)a->d_real.p;
    ka.real_tabs32 = (const float*)a->d_real32.p;
    ka.real_stride = a->real_stride;
    ka.phase_tabs = a->d_phase[dtype].p;
    ka.phase_stride = a->n_tab;
    ka.n_inst = a->n_inst;
    ka.s = a->s;
    ka.upmask = a->upmask;
    ka.batch = batch;
    ka.acc = (double*)a->d_acc.p;
    ka.n_slots = n_slots;
    ka.slot_E = a->P;
    ka.slot_N = a->P + 1;
    ka.prep.kind = a->prep_kind;
    ka.prep.L = a->L;
    ka.prep.s = a->s;
    ka.prep.layout = a->layout;
    ka.prep.neel_x0 = a->neel_x0;
    ka.prep.sd = (const double*)a->d_sd.p;
    ka.prep.sd32 = (const float*)a->d_sd32.p;
    const int nv = has_lam ? 2 : 1;
    const int no = g.op_end - g.op_begin;
    const RowLaunch rl =
        rows_launch(dtype, nv, ka.row_len, ka.n_rows, n_slots, a->n_gates, ka.n_hterms, no, force_cluster,
                    a->row_threads[dtype]);
    const int64_t groups = batch * (int64_t)((ka.n_rows + rl.rr - 1) / rl.rr);
    int64_t grid;
    if (rl.cl == 1) {
      const int per_sm = std::max(1, rows_max_ctas_per_sm(dtype, rl));
      grid = std::min<int64_t>(groups, (int64_t)sms * per_sm);
    } else {   // whole clusters, as many as can be resident
      const int ncl = rows_max_clusters(dtype, rl);
      if (ncl <= 0) return fail(HUB_EUNSUPPORTED, "row engine: no cluster of two CTAs fits");
      grid = (int64_t)rl.cl * std::min<int64_t>(groups, ncl);
    }
    hub_ansatz::ProfRec rec{};
    HUB_CUDA(record(rec, true), "cudaEventRecord");
    HUB_CUDA(launch_rows(dtype, ka, rl, (int)grid, st), "row kernel launch");
    rec.nv = 3;
    rec.dtype = dtype;
    const int io = ((g.flags & RS_PREP) ? 0 : 1) + ((g.flags & RS_WRITE_PSI) ? 1 : 0) +
                   ((g.flags & RS_READ_LAM) ? 1 : 0) + ((has_lam && (g.flags & RS_WRITE_LAM)) ? 1 : 0);
    rec.bytes = (double)io * (double)mat * (double)r2;
    HUB_CUDA(record(rec, false), "cudaEventRecord");
    lam_live = lam_live || (has_lam && (g.flags & RS_WRITE_LAM));
  }
  if (state) {
    state->cur = cur;
    state->orient = orient;
    state->lam_live = lam_live;
  }
  if (finalize)
    HUB_CUDA(launch_finalize((const double*)a->d_acc.p, n_slots, a->P, a->P, E, grad, batch, st), "finalize kernel");
  return HUB_OK;
}

// amps: the call's amplitude buffers (NULL entries are checked by the
// caller), each of which must be aligned to its element size (8 bytes for
// complex64, 16 for complex128): the kernels access whole elements.
hub_status check_call(hub_ansatz* a, int32_t dtype, int64_t batch, std::initializer_list<const void*> amps = {}) {
  if (!a) return fail(HUB_EINVAL, "NULL ansatz");
  if (dtype != HUB_C64 && dtype != HUB_C128) return fail(HUB_EINVAL, "dtype must be HUB_C64 or HUB_C128");
  if (batch < 1) return fail(HUB_EINVAL, "batch must be >= 1");
  if (a->n + 63 - __builtin_clzll((unsigned long long)batch) > 62) return fail(HUB_EINVAL, "batch too large");
  const uintptr_t align = dtype == HUB_C64 ? 8 : 16;
  for (const void* p : amps)
    if (((uintptr_t)p & (align - 1)) != 0)
      return fail(HUB_EINVAL, dtype == HUB_C64 ? "amplitude buffers must be 8-byte aligned (complex64)"
                                               : "amplitude buffers must be 16-byte aligned (complex128)");
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "earlier asynchronous error");
  return HUB_OK;
}

}  // namespace

extern "C" hub_status state_prepare(ans_t a, int32_t kind, const double* orb_perturb, const int32_t* neel_up,
                                    void* psi, int32_t dtype, int64_t batch, hub_stream_t stream) {
  hub_status s = check_call(a, dtype, batch, {psi});
  if (s != HUB_OK) return s;
  const int L = a->L;
  const hub_model* m0 = a->models[0];
  if (kind == HUB_PREP_NEEL) {
    if (!neel_up) return fail(HUB_EINVAL, "state_prepare: neel_up is NULL");
    uint64_t x0 = 0;
    int nu = 0, nd = 0;
    for (int i = 0; i < L; ++i) {
      if (neel_up[i]) { x0 |= 1ull << m0->up[i]; ++nu; }
      else { x0 |= 1ull << m0->dn[i]; ++nd; }
    }
    if (nu != m0->n_up || nd != m0->n_dn)
      return fail(HUB_EINVAL, "state_prepare: Neel pattern does not match the particle numbers");
    a->neel_x0 = x0;
    a->prep_kind = 1;
  } else if (kind == HUB_PREP_SLATER) {
    const size_t tl = (size_t)1 << L;
    std::vector<double> sd((size_t)a->n_inst * 2 * tl, 0.0);
    for (int r = 0; r < a->n_inst; ++r) {
      const hub_model* m = a->models[r];
      std::vector<double> h((size_t)L * L);
      for (int i = 0; i < L * L; ++i) h[i] = -m->t[i] + (orb_perturb ? orb_perturb[i] : 0.0);
      for (int i = 0; i < L; ++i)
        for (int j = 0; j < i; ++j)
          if (std::fabs(h[(size_t)i * L + j] - h[(size_t)j * L + i]) > 1e-12)
            return fail(HUB_EINVAL, "state_prepare: orb_perturb must be symmetric");
      std::vector<double> w, v;
      jacobi_eigh(L, h, w, v);
      // a degenerate Fermi level (the N-th and (N+1)-th levels equal) leaves
      // the Slater determinant undetermined: any basis of the degenerate
      // levels is as good, so refuse rather than pick one
      for (int sp = 0; sp < 2; ++sp) {
        const int N = sp == 0 ? m->n_up : m->n_dn;
        if (N > 0 && N < L) {
          const double gap = w[N] - w[N - 1];
          const double scale = std::max(1.0, std::max(std::fabs(w[N]), std::fabs(w[N - 1])));
          if (gap < 1e-9 * scale)
            return fail(HUB_EINVAL, "state_prepare: degenerate Fermi level (levels " + std::to_string(N - 1) +
                                        " and " + std::to_string(N) +
                                        " coincide): the Slater determinant is not unique; pass orb_perturb");
        }
      }
      for (int sp = 0; sp < 2; ++sp) {
        const int N = sp == 0 ? m->n_up : m->n_dn;
        for (uint32_t y = 0; y < tl; ++y) {
          if (__builtin_popcount(y) != N) continue;
          std::vector<double> mat((size_t)N * N);
          int row = 0;
          for (int i = 0; i < L; ++i)
            if (y >> i & 1) {
              for (int col = 0; col < N; ++col) mat[(size_t)row * N + col] = v[(size_t)i * L + col];
              ++row;
            }
          sd[(size_t)r * 2 * tl + sp * tl + y] = N == 0 ? 1.0 : det_lu(N, mat);
        }
      }
    }
    a->sd_host = sd;
    if ((s = a->d_sd.upload(sd, "determinant tables")) != HUB_OK) return s;
    if ((s = a->d_sd32.upload(std::vector<float>(sd.begin(), sd.end()), "determinant tables (FP32)")) != HUB_OK)
      return s;
    a->prep_kind = 0;
  } else {
    return fail(HUB_EINVAL, "state_prepare: unknown kind");
  }
  if (!psi) return HUB_OK;
  // one sweep with no operations: generate and store psi_0
  Plan* pl;
  if ((s = get_plan(a, 3, dtype, 0, pl)) != HUB_OK) return s;
  return run_plan(a, pl, dtype, nullptr, psi, nullptr, nullptr, batch, nullptr, nullptr, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// compute calls
// ---------------------------------------------------------------------------
extern "C" hub_status energy(ans_t a, const double* theta, void* psi, double* E, int32_t dtype, int64_t batch,
                             uint32_t flags, hub_stream_t stream) {
  hub_status s = check_call(a, dtype, batch, {psi});
  if (s != HUB_OK) return s;
  if (!psi || !E || (a->P > 0 && !theta)) return fail(HUB_EINVAL, "energy: NULL buffer");
  if ((flags & HUB_FLAG_PREP_FUSED) && a->prep_kind < 0)
    return fail(HUB_EINVAL, "energy: HUB_FLAG_PREP_FUSED needs a prior state_prepare");
  size_t smem = 0;
  if (SmallPlan* sp = small_plan_for(a, 0, dtype, flags, smem))
    return run_small(a, sp, smem, dtype, theta, batch, E, nullptr, (cudaStream_t)stream);
  SmallPlan* rsp = nullptr;
  if (RowPlan* rp = row_plan_for(a, 0, dtype, flags, rsp))
    return run_rows(a, rsp, rp, dtype, theta, psi, nullptr, batch, E, nullptr, flags, (cudaStream_t)stream);
  Plan* pl;
  if ((s = get_plan(a, 0, dtype, flags & 3u, pl)) != HUB_OK) return s;
  return run_plan(a, pl, dtype, theta, psi, nullptr, nullptr, batch, E, nullptr, (cudaStream_t)stream);
}

extern "C" hub_status energy_grad(ans_t a, const double* theta, void* psi, void* lam, void* ckpt, double* E,
                                  double* grad, int32_t dtype, int64_t batch, uint32_t flags,
                                  hub_stream_t stream) {
  hub_status s = check_call(a, dtype, batch, {psi, lam, ckpt});
  if (s != HUB_OK) return s;
  if (!psi || !lam || !E || !grad || (a->P > 0 && !theta)) return fail(HUB_EINVAL, "energy_grad: NULL buffer");
  if (psi == lam) return fail(HUB_EINVAL, "energy_grad: psi and lam must be distinct");
  if ((flags & HUB_FLAG_PREP_FUSED) && a->prep_kind < 0)
    return fail(HUB_EINVAL, "energy_grad: HUB_FLAG_PREP_FUSED needs a prior state_prepare");
  if (ckpt && (ckpt == psi || ckpt == lam)) return fail(HUB_EINVAL, "energy_grad: ckpt must be a third buffer");
  size_t smem = 0;
  if (SmallPlan* sp = small_plan_for(a, 1, dtype, flags, smem))
    return run_small(a, sp, smem, dtype, theta, batch, E, grad, (cudaStream_t)stream);
  SmallPlan* rsp = nullptr;
  if (RowPlan* rp = row_plan_for(a, 1, dtype, flags, rsp))
    return run_rows(a, rsp, rp, dtype, theta, psi, lam, batch, E, grad, flags, (cudaStream_t)stream);
  const uint32_t pf = (flags & 3u) | (ckpt ? kPlanCkpt : 0u);
  Plan* pl;
  if ((s = get_plan(a, 1, dtype, pf, pl)) != HUB_OK) return s;
  return run_plan(a, pl, dtype, theta, psi, lam, ckpt, batch, E, grad, (cudaStream_t)stream);
}

extern "C" hub_status hub_apply_h(ans_t a, const void* psi, void* lam, int32_t dtype, int64_t batch,
                                  hub_stream_t stream) {
  hub_status s = check_call(a, dtype, batch, {psi, lam});
  if (s != HUB_OK) return s;
  if (!psi || !lam || psi == lam) return fail(HUB_EINVAL, "hub_apply_h: bad buffers");
  Plan* pl;
  if ((s = get_plan(a, 2, dtype, 0, pl)) != HUB_OK) return s;
  return run_plan(a, pl, dtype, nullptr, const_cast<void*>(psi), lam, nullptr, batch, nullptr, nullptr,
                  (cudaStream_t)stream);
}

extern "C" hub_status ans_workspace_bytes(ans_t a, int32_t which, int32_t dtype, uint32_t flags, int64_t batch,
                                           uint64_t* bytes, int32_t* engine) {
  if (!a || !bytes || which < 0 || which > 1 || (dtype != HUB_C64 && dtype != HUB_C128) || batch < 1)
    return fail(HUB_EINVAL, "ans_workspace_bytes: bad arguments");
  const uint64_t amp = dtype == HUB_C64 ? 8 : 16;
  size_t smem = 0;
  if (small_plan_for(a, which, dtype, flags, smem)) {
    *bytes = 0;   // the state lives in shared memory only
    if (engine) *engine = 0;
    return HUB_OK;
  }
  SmallPlan* sp = nullptr;
  if (row_plan_for(a, which, dtype, flags, sp)) {
    // the sector matrix and its transpose
    *bytes = 2ull * (uint64_t)batch * (uint64_t)sp->cup * (uint64_t)sp->cdn * amp;
    if (engine) *engine = 1;
    return HUB_OK;
  }
  *bytes = (uint64_t)batch * (1ull << a->n) * amp;
  if (engine) *engine = 2;
  return HUB_OK;
}

extern "C" hub_status overlap_grad(ans_t a, const double* theta, const void* psi_ref, int64_t ref_batch,
                                   void* psi, void* lam, double* F, double* f, double* grad, int32_t dtype,
                                   int64_t batch, uint32_t flags, hub_stream_t stream) {
  hub_status s = check_call(a, dtype, batch, {psi_ref, psi, lam});
  if (s != HUB_OK) return s;
  if (!psi_ref || !psi || (a->P > 0 && !theta)) return fail(HUB_EINVAL, "overlap_grad: NULL buffer");
  if (grad && !lam) return fail(HUB_EINVAL, "overlap_grad: the gradient needs lam");
  if (lam && (lam == psi || lam == psi_ref)) return fail(HUB_EINVAL, "overlap_grad: lam must be a separate buffer");
  if (psi == psi_ref) return fail(HUB_EINVAL, "overlap_grad: psi and psi_ref must be distinct");
  if (ref_batch != 1 && ref_batch != batch) return fail(HUB_EINVAL, "overlap_grad: ref_batch must be 1 or batch");
  if (flags & ~(uint32_t)(HUB_FLAG_PREP_FUSED | HUB_FLAG_SWEEPS))
    return fail(HUB_EINVAL, "overlap_grad: unknown flags");
  const bool fused = (flags & HUB_FLAG_PREP_FUSED) != 0;
  if (fused && a->prep_kind < 0)
    return fail(HUB_EINVAL, "overlap_grad: HUB_FLAG_PREP_FUSED needs a prior state_prepare");
  cudaStream_t st = (cudaStream_t)stream;
  // the row engine, where both passes have a row plan (a prepared state,
  // N_up and N_dn conserved): the forward pass leaves the sector matrices
  // of psi_K in psi, the overlap and lam_K = a psi_ref are formed on them,
  // and the backward pass starts from there
  if (fused && !(flags & HUB_FLAG_SWEEPS)) {
    SmallPlan *spf = nullptr, *spb = nullptr;
    RowPlan* rpf = row_plan_for(a, 4, dtype, HUB_FLAG_PREP_FUSED, spf);
    RowPlan* rpb = (rpf && grad) ? row_plan_for(a, 5, dtype, HUB_FLAG_PREP_FUSED, spb) : nullptr;
    if (rpf && (!grad || rpb)) {
      RowRun rr;
      if ((s = run_rows(a, spf, rpf, dtype, theta, psi, nullptr, batch, nullptr, nullptr, 0u, st, &rr, false)) !=
          HUB_OK)
        return s;
      if ((s = a->d_ovl.ensure(16 * (size_t)batch, "overlaps")) != HUB_OK) return s;
      double* ov = (double*)a->d_ovl.p;
      HUB_CUDA(launch_zero(ov, 2 * batch, st), "zero overlaps");
      const size_t r2 = dtype == HUB_C64 ? 8 : 16;
      const size_t off = (size_t)rr.cur * (size_t)batch * (size_t)spf->cup * (size_t)spf->cdn * r2;
      const uint32_t* xrow = (const uint32_t*)(rr.orient == 0 ? spf->d_xdn.p : spf->d_xup.p);
      const uint32_t* xin = (const uint32_t*)(rr.orient == 0 ? spf->d_xup.p : spf->d_xdn.p);
      const int n_rows = rr.orient == 0 ? spf->cdn : spf->cup, row_len = rr.orient == 0 ? spf->cup : spf->cdn;
      HUB_CUDA(launch_sector_overlap(dtype, (const unsigned char*)psi + off, xrow, xin, n_rows, row_len, psi_ref,
                                     ref_batch, a->n, batch, ov, st),
               "sector overlap kernel");
      const double* acc = nullptr;
      if (grad) {
        HUB_CUDA(launch_sector_scale_ref(dtype, psi_ref, ref_batch, xrow, xin, n_rows, row_len, a->n, batch, ov,
                                         (unsigned char*)lam + off, st),
                 "sector reference scaling kernel");
        rr.lam_live = true;
        if ((s = run_rows(a, spb, rpb, dtype, theta, psi, lam, batch, nullptr, nullptr, 0u, st, &rr, false)) !=
            HUB_OK)
          return s;
        acc = (const double*)a->d_acc.p;
      }
      HUB_CUDA(launch_overlap_finalize(acc, a->P + 2, a->P, ov, F, f, grad, batch, st), "overlap finalize kernel");
      return HUB_OK;
    }
  }
  // forward circuit, psi_K kept in psi
  Plan* pf;
  if ((s = get_plan(a, 4, dtype, (fused ? HUB_FLAG_PREP_FUSED : 0u) | HUB_FLAG_KEEP_STATE, pf)) != HUB_OK) return s;
  if ((s = run_plan(a, pf, dtype, theta, psi, nullptr, nullptr, batch, nullptr, nullptr, st)) != HUB_OK) return s;
  // a = <psi_ref|psi_K>
  if ((s = a->d_ovl.ensure(16 * (size_t)batch, "overlaps")) != HUB_OK) return s;
  double* ov = (double*)a->d_ovl.p;
  HUB_CUDA(launch_zero(ov, 2 * batch, st), "zero overlaps");
  HUB_CUDA(launch_overlap(dtype, psi, psi_ref, ref_batch, a->n, batch, ov, st), "overlap kernel");
  const double* acc = nullptr;
  if (grad) {
    // lam_K = psi_ref a, then the backward pass accumulates dF/dtheta
    HUB_CUDA(launch_scale_ref(dtype, psi_ref, ref_batch, lam, a->n, batch, ov, st), "reference scaling kernel");
    Plan* pb;
    if ((s = get_plan(a, 5, dtype, fused ? HUB_FLAG_PREP_FUSED : 0u, pb)) != HUB_OK) return s;
    if ((s = run_plan(a, pb, dtype, theta, psi, lam, nullptr, batch, nullptr, nullptr, st)) != HUB_OK) return s;
    acc = (const double*)a->d_acc.p;
  }
  HUB_CUDA(launch_overlap_finalize(acc, a->P + 2, a->P, ov, F, f, grad, batch, st), "overlap finalize kernel");
  return HUB_OK;
}

extern "C" hub_status spin_correlation(ans_t a, const void* psi, double* C, int32_t dtype, int64_t batch,
                                       hub_stream_t stream) {
  hub_status s = check_call(a, dtype, batch, {psi});
  if (s != HUB_OK) return s;
  if (!psi || !C) return fail(HUB_EINVAL, "spin_correlation: NULL buffer");
  const int n = a->n, L = a->L;
  cudaStream_t st = (cudaStream_t)stream;
  if (!a->d_modes.p) {
    std::vector<int32_t> md(a->models[0]->up);
    md.insert(md.end(), a->models[0]->dn.begin(), a->models[0]->dn.end());
    if ((s = a->d_modes.upload(md, "mode maps")) != HUB_OK) return s;
  }
  if ((s = a->d_occ.ensure(8 * (size_t)batch * n * n, "occupation correlations")) != HUB_OK) return s;
  double* M = (double*)a->d_occ.p;
  HUB_CUDA(launch_zero(M, batch * n * n, st), "zero correlations");
  HUB_CUDA(launch_occ_corr(dtype, psi, n, batch, M, st), "occupation correlation kernel");
  const int32_t* md = (const int32_t*)a->d_modes.p;
  HUB_CUDA(launch_spin_corr(M, n, md, md + L, L, C, batch, st), "spin correlation kernel");
  return HUB_OK;
}

extern "C" hub_status ans_plan_stats(ans_t a, int32_t which, int32_t dtype, uint32_t flags, int32_t* n_sweeps,
                                     double* bytes_per_state) {
  if (!a || which < 0 || which > 2 || (dtype != HUB_C64 && dtype != HUB_C128))
    return fail(HUB_EINVAL, "ans_plan_stats: bad arguments");
  if (flags & HUB_FLAG_ROWS) {   // the row engine's schedule (energy or energy_grad)
    if (which > 1) return fail(HUB_EINVAL, "ans_plan_stats: the row engine runs energy and energy_grad only");
    SmallPlan* sp = get_small_plan(a, which);
    if (!sp) return fail(HUB_EUNSUPPORTED, "ans_plan_stats: no sector plan");
    RowPlan* rp = nullptr;
    auto it = a->row_plans.find(which);
    if (it != a->row_plans.end()) {
      rp = it->second;
    } else {
      if (make_row_plan(a, which, sp, rp) != HUB_OK) rp = nullptr;
      a->row_plans[which] = rp;
    }
    if (!rp) return fail(HUB_EUNSUPPORTED, "ans_plan_stats: no row schedule");
    int launches = 0;
    const double by = row_plan_bytes(sp, rp, dtype, &launches);
    if (n_sweeps) *n_sweeps = launches;
    if (bytes_per_state) *bytes_per_state = by;
    return HUB_OK;
  }
  // the plan energy / energy_grad run for these flags (without a checkpoint;
  // HUB_FLAG_SWEEPS selects the engine, not a different sweep plan)
  Plan* pl;
  hub_status s = get_plan(a, which, dtype, flags & 3u, pl);
  if (s != HUB_OK) return s;
  if (n_sweeps) *n_sweeps = (int32_t)pl->sweeps.size();
  if (bytes_per_state) *bytes_per_state = pl->bytes_per_state;
  return HUB_OK;
}

extern "C" hub_status ans_plan_describe(ans_t a, int32_t which, int32_t dtype, uint32_t flags, int64_t* buf,
                                        int32_t cap, int32_t* len) {
  if (!a || !len || which < 0 || which > 2 || (dtype != HUB_C64 && dtype != HUB_C128))
    return fail(HUB_EINVAL, "ans_plan_describe: bad arguments");
  std::vector<int64_t> out;
  if (flags & HUB_FLAG_ROWS) {   // the row engine's segments: tile = the modes of one spin
    if (which > 1) return fail(HUB_EINVAL, "ans_plan_describe: the row engine runs energy and energy_grad only");
    uint64_t upm = 0, dnm = 0;
    for (int i = 0; i < a->L; ++i) {
      upm |= 1ull << a->models[0]->up[i];
      dnm |= 1ull << a->models[0]->dn[i];
    }
    const std::vector<RowSched> sched = row_schedule(a, which);
    out.push_back((int64_t)sched.size());
    for (const RowSched& rs : sched) {
      if (rs.orient < 0) return fail(HUB_EUNSUPPORTED, "ans_plan_describe: no row schedule");
      out.push_back((int64_t)(rs.orient == 0 ? upm : dnm));
      out.push_back((int64_t)rs.orient);
      out.push_back((int64_t)rs.ops.size());
      for (int id : rs.ops) out.push_back(id);
    }
    *len = (int32_t)out.size();
    if (buf) {
      if (cap < (int32_t)out.size()) return fail(HUB_EINVAL, "ans_plan_describe: buffer too small");
      std::copy(out.begin(), out.end(), buf);
    }
    return HUB_OK;
  }
  Plan* pl;
  hub_status s = get_plan(a, which, dtype, flags & 3u, pl);
  if (s != HUB_OK) return s;
  out.push_back((int64_t)pl->sweeps.size());
  for (size_t i = 0; i < pl->sweeps.size(); ++i) {
    out.push_back((int64_t)pl->tiles[i]);
    const int nph = pl->sweeps[i].phase_end - pl->sweeps[i].phase_begin;
    out.push_back((int64_t)pl->sweeps[i].flags | ((int64_t)nph << 16));
    out.push_back((int64_t)pl->seq_ids[i].size());
    for (int id : pl->seq_ids[i]) out.push_back(id);
  }
  *len = (int32_t)out.size();
  if (buf) {
    if (cap < (int32_t)out.size()) return fail(HUB_EINVAL, "ans_plan_describe: buffer too small");
    std::copy(out.begin(), out.end(), buf);
  }
  return HUB_OK;
}

extern "C" hub_status ans_profile(ans_t a, int32_t enable) {
  if (!a) return fail(HUB_EINVAL, "ans_profile: NULL ansatz");
  a->prof_clear();
  a->prof = enable != 0;
  return HUB_OK;
}

extern "C" hub_status ans_profile_read(ans_t a, double* out, int32_t cap, int32_t* n) {
  if (!a || !n) return fail(HUB_EINVAL, "ans_profile_read: bad arguments");
  *n = (int32_t)a->prof_recs.size();
  if (!out) return HUB_OK;
  if (cap < 4 * *n) return fail(HUB_EINVAL, "ans_profile_read: buffer too small");
  for (size_t i = 0; i < a->prof_recs.size(); ++i) {
    auto& r = a->prof_recs[i];
    float ms = 0.f;
    HUB_CUDA(cudaEventSynchronize(r.e1), "cudaEventSynchronize");
    HUB_CUDA(cudaEventElapsedTime(&ms, r.e0, r.e1), "cudaEventElapsedTime");
    out[4 * i + 0] = r.nv;
    out[4 * i + 1] = r.dtype;
    out[4 * i + 2] = r.bytes;
    out[4 * i + 3] = ms;
  }
  a->prof_clear();
  return HUB_OK;
}

extern "C" hub_status hub_sync(hub_stream_t stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "hub_sync");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "hub_sync");
  return HUB_OK;
}

extern "C" const char* hub_last_error(void) { return g_err.c_str(); }
