// Host side of the Hubbard VQE statevector engine: model and ansatz handles,
// the FP64 one-body diagonalisation for the Slater-determinant initial
// state, the sweep planner and the C-ABI entry points of hubsv.h.
#include "hubsv.h"
#include "hubsv_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

using namespace hubsv;

namespace {

thread_local std::string g_err;

hub_status fail(hub_status s, const std::string& m) {
  g_err = m;
  return s;
}

hub_status cuda_fail(cudaError_t e, const char* what) {
  return fail(HUB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define HUB_CUDA(call, what)                       \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

inline int popc64(uint64_t x) { return __builtin_popcountll(x); }

uint64_t between_mask(int p, int q) {  // bits strictly between p < q
  return ((1ull << q) - 1ull) & ~((1ull << (p + 1)) - 1ull);
}

// ---------------------------------------------------------------------------
// FP64 symmetric eigensolver (cyclic Jacobi) and determinants
// ---------------------------------------------------------------------------

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

// ---------------------------------------------------------------------------
// device buffer helper
// ---------------------------------------------------------------------------

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~DevBuf() { if (p) cudaFree(p); }
  hub_status ensure(size_t n, const char* what) {
    if (n <= bytes && p) return HUB_OK;
    if (p) { cudaFree(p); p = nullptr; bytes = 0; }
    if (n == 0) n = 16;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      p = nullptr;
      return fail(HUB_ENOMEM, std::string("cudaMalloc failed for ") + what);
    }
    bytes = n;
    return HUB_OK;
  }
  template <typename T>
  hub_status upload(const std::vector<T>& v, const char* what) {
    hub_status s = ensure(std::max<size_t>(v.size() * sizeof(T), 16), what);
    if (s != HUB_OK) return s;
    if (!v.empty()) HUB_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), what);
    return HUB_OK;
  }
};

}  // namespace

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------

struct hub_model {
  int L = 0, n = 0, s = 0, layout = 0;
  std::vector<int> up, dn;
  std::vector<std::pair<int, int>> bonds;
  std::vector<double> t, U, V;
  int n_up = 0, n_dn = 0;
};

namespace {

// Host-level operation before tiling.
struct SeqOp {
  uint8_t kind = 0, flags = 0;
  int p = -1, q = -1;       // modes (hop-type)
  int gate = -1, hterm = -1, slot = -1, diag = -1;
  uint64_t support = 0;
  bool diagonal = false;
  int cls = 0;              // 0 forward, 1 measure, 2 lam, 3 backward
};

struct Plan {
  std::vector<SweepDev> sweeps;
  std::vector<int> nvec;    // 1 or 2 per sweep
  std::vector<OpDev> hops;  // host copy of the operations
  std::vector<uint64_t> tiles;
  std::vector<std::vector<int>> seq_ids;   // sequence index of each op, per sweep
  bool uploaded = false;
  DevBuf ops;
  int k = 0, c = 0;
  double bytes_per_state = 0;
};

}  // namespace

struct hub_ansatz {
  std::vector<hub_model*> models;
  int n_inst = 0, L = 0, n = 0, P = 0, s = 0, layout = 0;
  uint64_t upmask = 0;
  // forward sequence and H terms
  std::vector<SeqOp> fwd;
  struct HTerm { int p, q; };
  std::vector<HTerm> hterms;
  int h_diag = -1;                       // DiagOp index of H's diagonal
  std::vector<DiagOpDev> diag_ops;
  // static device tables
  std::vector<int32_t> gate_param;
  std::vector<double> gate_t;            // [n_inst][n_gates]
  std::vector<int32_t> tab_param;        // [n_tab]
  std::vector<double> tab_val;           // [n_inst][n_tab]
  std::vector<double> hcoef;             // [n_inst][n_hterms]
  std::vector<double> real_tabs;         // [n_inst][real_stride]
  int n_gates = 0, n_tab = 0, real_stride = 0;
  DevBuf d_gate_param, d_gate_t, d_tab_param, d_tab_val, d_hcoef, d_real, d_diag;
  // initial state
  DevBuf d_sd;
  int prep_kind = -1;
  uint64_t neel_x0 = 0;
  // per-call scratch
  DevBuf d_coef[2], d_phase[2], d_acc;
  // plans: key = which*16 + dtype*4 + flags
  std::map<int, Plan*> plans;
  int tile_override[2] = {0, 0};
  bool dev_ready = false;
  // optional per-launch timing (CUDA events around every sweep launch)
  struct ProfRec { cudaEvent_t e0, e1; int nv, dtype; double bytes; };
  bool prof = false;
  std::vector<ProfRec> prof_recs;
  void prof_clear() {
    for (auto& r : prof_recs) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
    prof_recs.clear();
  }
  ~hub_ansatz() {
    prof_clear();
    for (auto& kv : plans) delete kv.second;
  }
};

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

// Register a diagonal operator given per-mode X coefficients (and a constant),
// per-site Y (double occupancy) coefficients and V bonds, each per instance.
int add_diag_op(hub_ansatz* a, const std::vector<std::vector<double>>& xcoef,
                const std::vector<double>& xconst,
                const std::vector<std::vector<double>>& ycoef,
                const std::vector<std::pair<int, int>>& vbonds,
                const std::vector<std::vector<double>>& vval, int param) {
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
  d.param = param;
  d.real_off = a->real_stride;
  const int real_len = 2048 + d.n_vb;
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
    const int len = 2048 + vlen;
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
    }
    a->tab_val.swap(nv);
    for (int e = 0; e < len; ++e) a->tab_param.push_back(param);
    a->n_tab += len;
  } else {
    d.phase_off = -1;
  }
  a->diag_ops.push_back(d);
  return (int)a->diag_ops.size() - 1;
}

uint64_t diag_support(hub_ansatz* a, int di) {
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
  return m;
}

}  // namespace

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
    if (gr.kind < 0 || gr.kind > HUB_G_RZ) return bad("unknown group kind");
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
  a->P = P;
  // H hop terms: every bond, both spins; term index 2*bond + spin
  for (int b = 0; b < nb; ++b)
    for (int sp = 0; sp < 2; ++sp) {
      const auto& mm = sp == 0 ? m0->up : m0->dn;
      int p = mm[m0->bonds[b].first], q = mm[m0->bonds[b].second];
      if (p > q) std::swap(p, q);
      a->hterms.push_back({p, q});
    }
  a->hcoef.resize((size_t)R * a->hterms.size());
  for (int r = 0; r < R; ++r)
    for (int b = 0; b < nb; ++b)
      for (int sp = 0; sp < 2; ++sp) {
        const auto& bd = m0->bonds[b];
        a->hcoef[(size_t)r * a->hterms.size() + 2 * b + sp] = -models[r]->t[(size_t)bd.first * L + bd.second];
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
    a->h_diag = add_diag_op(a, xc, xk, yc, vb, vv, -1);
  }
  // forward sequence
  for (int g = 0; g < G; ++g) {
    const hub_group& gr = groups[g];
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
          a->fwd.push_back(op);
        }
      }
    } else {
      std::vector<std::vector<double>> xc(R, std::vector<double>(a->n, 0.0)), yc(R, std::vector<double>(a->n, 0.0)), vv(R);
      std::vector<double> xk(R, 0.0);
      std::vector<std::pair<int, int>> vb;
      for (int k = 0; k < gr.n_terms; ++k) {
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
      op.diag = add_diag_op(a, xc, xk, yc, vb, vv, gr.param);
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
        const auto& bd = m0->bonds[op.hterm / 2];
        a->gate_t[(size_t)r * a->n_gates + gi++] = models[r]->t[(size_t)bd.first * L + bd.second];
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

// ---------------------------------------------------------------------------
// planner
// ---------------------------------------------------------------------------

namespace {

// Static tables go to the device on the first compute call (ans_create
// itself touches no GPU, so the host logic runs anywhere).
hub_status ensure_device(hub_ansatz* a) {
  if (a->dev_ready) return HUB_OK;
  hub_status st;
  if ((st = a->d_gate_param.upload(a->gate_param, "gate params")) != HUB_OK ||
      (st = a->d_gate_t.upload(a->gate_t, "gate coefficients")) != HUB_OK ||
      (st = a->d_tab_param.upload(a->tab_param, "phase params")) != HUB_OK ||
      (st = a->d_tab_val.upload(a->tab_val, "phase values")) != HUB_OK ||
      (st = a->d_hcoef.upload(a->hcoef, "hop coefficients")) != HUB_OK ||
      (st = a->d_real.upload(a->real_tabs, "diagonal tables")) != HUB_OK ||
      (st = a->d_diag.upload(a->diag_ops, "diagonal operators")) != HUB_OK)
    return st;
  a->dev_ready = true;
  return HUB_OK;
}

int default_tile_bits(int dtype) { return dtype == HUB_C64 ? 13 : 12; }
int coalesce_bits(int dtype) { return dtype == HUB_C64 ? 5 : 4; }   // 256-byte runs

// Build the operation sequence of a call kind: 0 energy, 1 energy + gradient,
// 2 apply H.
std::vector<SeqOp> build_sequence(hub_ansatz* a, int which) {
  std::vector<SeqOp> seq;
  if (which != 2) seq = a->fwd;
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

// Greedy sweep construction.  Operations are taken in sequence order; an
// operation runs in the current sweep when it commutes with every operation
// skipped before it in this sweep and its modes fit in the tile (diagonal
// operations need no tile bits).  Operations on disjoint modes commute;
// diagonal operations commute with each other.  Lam-building operations wait
// until the whole forward circuit has run.
hub_status make_plan(hub_ansatz* a, int which, int dtype, uint32_t flags, Plan*& out) {
  const int n = a->n;
  int k = a->tile_override[dtype] ? a->tile_override[dtype] : default_tile_bits(dtype);
  k = std::min(k, n);
  const int c = std::min(coalesce_bits(dtype), k);
  const uint64_t cmask = (1ull << c) - 1ull;
  std::vector<SeqOp> seq = build_sequence(a, which);
  std::vector<int> remaining(seq.size());
  for (size_t i = 0; i < seq.size(); ++i) remaining[i] = (int)i;
  struct PS { uint64_t tile; std::vector<int> ops; };
  std::vector<PS> sweeps;
  while (!remaining.empty()) {
    uint64_t tile = cmask;
    uint64_t s_any = 0, s_diag = 0;
    bool fwd_skipped = false;
    std::vector<int> exec, rest;
    for (int idx : remaining) {
      const SeqOp& op = seq[idx];
      bool conflict = (op.support & s_any) || (!op.diagonal && (op.support & s_diag));
      if (op.cls == 2 && fwd_skipped) conflict = true;
      bool ok = false;
      if (!conflict) {
        const uint64_t need = op.diagonal ? 0ull : ((1ull << op.p) | (1ull << op.q));
        const uint64_t nt = tile | need;
        if (popc64(nt) <= k) { tile = nt; ok = true; }
      }
      if (ok) {
        exec.push_back(idx);
      } else {
        rest.push_back(idx);
        if (op.diagonal) s_diag |= op.support; else s_any |= op.support;
        if (op.cls == 0) fwd_skipped = true;
      }
    }
    if (exec.empty()) return fail(HUB_EUNSUPPORTED, "planner made no progress");
    // pad the tile with the lowest unused bits
    for (int b = 0; b < n && popc64(tile) < k; ++b) tile |= 1ull << b;
    sweeps.push_back({tile, exec});
    remaining.swap(rest);
  }
  if (sweeps.empty()) {  // nothing to do (e.g. no H terms and no gates): one read sweep
    uint64_t tile = (k >= 64) ? ~0ull : ((1ull << k) - 1ull);
    sweeps.push_back({tile, {}});
  }
  // flags and device ops
  Plan* pl = new Plan();
  pl->k = k;
  pl->c = c;
  std::vector<OpDev> dops;
  const bool prep = (flags & HUB_FLAG_PREP_FUSED) != 0;
  const bool keep = (flags & HUB_FLAG_KEEP_STATE) != 0;
  bool lam_live = false;
  const double amp = dtype == HUB_C64 ? 8.0 : 16.0;
  double bytes = 0.0;
  for (size_t si = 0; si < sweeps.size(); ++si) {
    const PS& ps = sweeps[si];
    SweepDev sw;
    std::memset(&sw, 0, sizeof(sw));
    sw.k = k;
    sw.c = c;
    sw.h1 = (k - c + 1) / 2;
    int nt = 0, nn = 0;
    int localpos[64];
    for (int b = 0; b < n; ++b) {
      if (ps.tile >> b & 1) { localpos[b] = nt; sw.tbits[nt++] = (int8_t)b; }
      else { localpos[b] = -1; sw.nbits[nn++] = (int8_t)b; }
    }
    sw.n_nontile = nn;
    sw.op_begin = (int)dops.size();
    bool mod_psi = false, use_lam = false, mod_lam = false;
    for (int idx : ps.ops) {
      const SeqOp& op = seq[idx];
      OpDev d;
      std::memset(&d, 0, sizeof(d));
      d.kind = op.kind;
      d.flags = op.flags;
      d.gate = op.gate;
      d.hterm = op.hterm;
      d.slot = op.slot;
      d.diag = op.diag;
      if (!op.diagonal) {
        d.p = (uint8_t)localpos[op.p];
        d.q = (uint8_t)localpos[op.q];
        const uint64_t bm = between_mask(op.p, op.q);
        uint32_t bl = 0;
        for (int b = 0; b < n; ++b)
          if ((bm >> b & 1) && localpos[b] >= 0) bl |= 1u << localpos[b];
        d.bmask_local = bl;
        d.bmask_global = bm & ~ps.tile;
      }
      dops.push_back(d);
      mod_psi = mod_psi || modifies_psi(op);
      use_lam = use_lam || uses_lam(op);
      mod_lam = mod_lam || modifies_lam(op);
    }
    sw.op_end = (int)dops.size();
    const bool first = si == 0, last = si + 1 == sweeps.size();
    uint32_t f = 0;
    if (first && prep && which != 2) f |= SW_PREP; else f |= SW_READ_PSI;
    if ((!last || keep) && (mod_psi || (f & SW_PREP))) f |= SW_WRITE_PSI;
    if (which == 2 && !last) { /* psi is read only */ }
    if (use_lam || (lam_live && mod_lam)) {
      f |= SW_HAS_LAM;
      if (lam_live) f |= SW_READ_LAM;
      if (mod_lam && (!last || which == 2)) f |= SW_WRITE_LAM;
      lam_live = true;
    }
    if (which == 2) f &= ~SW_WRITE_PSI;
    sw.flags = f;
    bytes += amp * (double)(1ull << n) *
             (((f & SW_READ_PSI) ? 1 : 0) + ((f & SW_WRITE_PSI) ? 1 : 0) +
              ((f & SW_READ_LAM) ? 1 : 0) + ((f & SW_WRITE_LAM) ? 1 : 0));
    pl->sweeps.push_back(sw);
    pl->nvec.push_back((f & SW_HAS_LAM) ? 2 : 1);
    pl->tiles.push_back(ps.tile);
    pl->seq_ids.push_back(ps.ops);
  }
  pl->bytes_per_state = bytes;
  pl->hops = dops;
  out = pl;
  return HUB_OK;
}

hub_status get_plan(hub_ansatz* a, int which, int dtype, uint32_t flags, Plan*& pl) {
  const int key = which * 16 + dtype * 4 + (int)(flags & 3u);  // PREP_FUSED | KEEP_STATE
  auto it = a->plans.find(key);
  if (it != a->plans.end()) { pl = it->second; return HUB_OK; }
  hub_status st = make_plan(a, which, dtype, flags, pl);
  if (st != HUB_OK) return st;
  a->plans[key] = pl;
  return HUB_OK;
}

size_t sweep_smem(const Plan* pl, int nv, int dtype, int n_slots) {
  const int k = pl->k, c = pl->c, h1 = (k - c + 1) / 2, h2 = k - c - h1;
  const size_t amp = dtype == HUB_C64 ? 8 : 16;
  return (size_t)nv * (amp << k) + 8 * ((1u << h1) + (1u << h2)) + 8 * (size_t)n_slots;
}

hub_status run_plan(hub_ansatz* a, Plan* pl, int dtype, const double* theta, void* psi, void* lam,
                    void* ckpt, int64_t batch, double* E, double* grad, cudaStream_t st) {
  const int n = a->n;
  const int n_slots = a->P + 2;
  hub_status s;
  if ((s = ensure_device(a)) != HUB_OK) return s;
  if (!pl->uploaded) {
    if ((s = pl->ops.upload(pl->hops.empty() ? std::vector<OpDev>(1) : pl->hops, "sweep ops")) != HUB_OK) return s;
    pl->uploaded = true;
  }
  const size_t r2 = dtype == HUB_C64 ? 8 : 16;
  if ((s = a->d_coef[dtype].ensure(r2 * std::max<int64_t>(1, batch * a->n_gates), "coefficients")) != HUB_OK) return s;
  if ((s = a->d_phase[dtype].ensure(r2 * std::max<int64_t>(1, batch * a->n_tab), "phase tables")) != HUB_OK) return s;
  if ((s = a->d_acc.ensure(8 * (size_t)batch * n_slots, "accumulators")) != HUB_OK) return s;
  HUB_CUDA(launch_zero((double*)a->d_acc.p, batch * n_slots, st), "zero accumulators");
  if (theta) {
    HUB_CUDA(launch_coef(dtype, theta, a->P, (const int32_t*)a->d_gate_param.p, (const double*)a->d_gate_t.p,
                         a->n_gates, a->d_coef[dtype].p, (const int32_t*)a->d_tab_param.p,
                         (const double*)a->d_tab_val.p, a->n_tab, a->n_inst, a->d_phase[dtype].p, batch,
                         a->n_inst, st),
             "coefficient kernel");
  }
  KernelArgs ka;
  std::memset(&ka, 0, sizeof(ka));
  ka.psi = psi;
  ka.lam = lam;
  ka.ckpt = ckpt;
  ka.ops = (const OpDev*)pl->ops.p;
  ka.diag_ops = (const DiagOpDev*)a->d_diag.p;
  ka.theta = theta;
  ka.P = a->P;
  ka.coef = a->d_coef[dtype].p;
  ka.n_gates = a->n_gates;
  ka.hcoef = (const double*)a->d_hcoef.p;
  ka.n_hterms = (int)a->hterms.size();
  ka.real_tabs = (const double*)a->d_real.p;
  ka.real_stride = a->real_stride;
  ka.phase_tabs = a->d_phase[dtype].p;
  ka.phase_stride = a->n_tab;
  ka.n_inst = a->n_inst;
  ka.n = n;
  ka.s = a->s;
  ka.upmask = a->upmask;
  ka.batch = batch;
  ka.n_tiles = ((uint64_t)batch) << (n - pl->k);
  ka.acc = (double*)a->d_acc.p;
  ka.n_slots = n_slots;
  ka.slot_E = a->P;
  ka.slot_N = a->P + 1;
  ka.prep.kind = a->prep_kind < 0 ? 0 : a->prep_kind;
  ka.prep.L = a->L;
  ka.prep.s = a->s;
  ka.prep.layout = a->layout;
  ka.prep.neel_x0 = a->neel_x0;
  ka.prep.sd = (const double*)a->d_sd.p;
  const int sms = device_sm_count();
  if (sms <= 0) return fail(HUB_ECUDA, "no CUDA device");
  const int optin = sweep_max_smem_optin();
  for (size_t i = 0; i < pl->sweeps.size(); ++i) {
    const int nv = pl->nvec[i];
    const size_t smem = sweep_smem(pl, nv, dtype, n_slots);
    if ((int)smem > optin) return fail(HUB_EUNSUPPORTED, "tile does not fit in shared memory");
    HUB_CUDA(sweep_set_smem(dtype, nv, smem), "cudaFuncSetAttribute");
    int per_sm = (int)std::min<size_t>(8, (size_t)(228 * 1024) / (smem + 1024));
    per_sm = std::max(per_sm, 1);
    uint64_t grid = (uint64_t)sms * per_sm;
    grid = std::min<uint64_t>(grid, ka.n_tiles);
    hub_ansatz::ProfRec rec{};
    if (a->prof) {
      HUB_CUDA(cudaEventCreate(&rec.e0), "cudaEventCreate");
      HUB_CUDA(cudaEventCreate(&rec.e1), "cudaEventCreate");
      HUB_CUDA(cudaEventRecord(rec.e0, st), "cudaEventRecord");
    }
    HUB_CUDA(launch_sweep(dtype, pl->sweeps[i], ka, (int)grid, smem, st), "sweep kernel launch");
    if (a->prof) {
      HUB_CUDA(cudaEventRecord(rec.e1, st), "cudaEventRecord");
      const uint32_t f = pl->sweeps[i].flags;
      const int nvec_io = ((f & SW_READ_PSI) ? 1 : 0) + ((f & SW_WRITE_PSI) ? 1 : 0) +
                          ((f & SW_READ_LAM) ? 1 : 0) + ((f & SW_WRITE_LAM) ? 1 : 0) +
                          ((f & SW_CKPT_WRITE) ? 1 : 0) + ((f & SW_CKPT_READ) ? 1 : 0);
      rec.nv = nv;
      rec.dtype = dtype;
      rec.bytes = (double)nvec_io * (double)(dtype == HUB_C64 ? 8 : 16) * (double)(1ull << n) * (double)batch;
      a->prof_recs.push_back(rec);
    }
  }
  HUB_CUDA(launch_finalize((const double*)a->d_acc.p, n_slots, a->P, a->P, E, grad, batch, st), "finalize kernel");
  return HUB_OK;
}

hub_status check_call(hub_ansatz* a, int32_t dtype, int64_t batch) {
  if (!a) return fail(HUB_EINVAL, "NULL ansatz");
  if (dtype != HUB_C64 && dtype != HUB_C128) return fail(HUB_EINVAL, "dtype must be HUB_C64 or HUB_C128");
  if (batch < 1) return fail(HUB_EINVAL, "batch must be >= 1");
  if (a->n + 63 - __builtin_clzll((unsigned long long)batch) > 62) return fail(HUB_EINVAL, "batch too large");
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "earlier asynchronous error");
  return HUB_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// initial state
// ---------------------------------------------------------------------------

extern "C" hub_status state_prepare(ans_t a, int32_t kind, const double* orb_perturb, const int32_t* neel_up,
                                    void* psi, int32_t dtype, int64_t batch, hub_stream_t stream) {
  hub_status s = check_call(a, dtype, batch);
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
    if ((s = a->d_sd.upload(sd, "determinant tables")) != HUB_OK) return s;
    a->prep_kind = 0;
  } else {
    return fail(HUB_EINVAL, "state_prepare: unknown kind");
  }
  if (!psi) return HUB_OK;
  // one sweep with no operations: generate and store psi_0
  Plan pl;
  const int k = std::min(dtype == HUB_C64 ? 13 : 12, a->n);
  pl.k = k;
  pl.c = std::min(coalesce_bits(dtype), k);
  SweepDev sw;
  std::memset(&sw, 0, sizeof(sw));
  sw.k = k;
  sw.c = pl.c;
  sw.h1 = (k - pl.c + 1) / 2;
  for (int b = 0; b < k; ++b) sw.tbits[b] = (int8_t)b;
  for (int b = k; b < a->n; ++b) sw.nbits[b - k] = (int8_t)b;
  sw.n_nontile = a->n - k;
  sw.flags = SW_PREP | SW_WRITE_PSI;
  pl.sweeps.push_back(sw);
  pl.nvec.push_back(1);
  OpDev dummy;
  std::memset(&dummy, 0, sizeof(dummy));
  pl.hops.push_back(dummy);
  return run_plan(a, &pl, dtype, nullptr, psi, nullptr, nullptr, batch, nullptr, nullptr, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// compute calls
// ---------------------------------------------------------------------------

extern "C" hub_status energy(ans_t a, const double* theta, void* psi, double* E, int32_t dtype, int64_t batch,
                             uint32_t flags, hub_stream_t stream) {
  hub_status s = check_call(a, dtype, batch);
  if (s != HUB_OK) return s;
  if (!psi || !E || (a->P > 0 && !theta)) return fail(HUB_EINVAL, "energy: NULL buffer");
  if ((flags & HUB_FLAG_PREP_FUSED) && a->prep_kind < 0)
    return fail(HUB_EINVAL, "energy: HUB_FLAG_PREP_FUSED needs a prior state_prepare");
  Plan* pl;
  if ((s = get_plan(a, 0, dtype, flags, pl)) != HUB_OK) return s;
  return run_plan(a, pl, dtype, theta, psi, nullptr, nullptr, batch, E, nullptr, (cudaStream_t)stream);
}

extern "C" hub_status energy_grad(ans_t a, const double* theta, void* psi, void* lam, void* ckpt, double* E,
                                  double* grad, int32_t dtype, int64_t batch, uint32_t flags,
                                  hub_stream_t stream) {
  hub_status s = check_call(a, dtype, batch);
  if (s != HUB_OK) return s;
  if (!psi || !lam || !E || !grad || (a->P > 0 && !theta)) return fail(HUB_EINVAL, "energy_grad: NULL buffer");
  if (psi == lam) return fail(HUB_EINVAL, "energy_grad: psi and lam must be distinct");
  if ((flags & HUB_FLAG_PREP_FUSED) && a->prep_kind < 0)
    return fail(HUB_EINVAL, "energy_grad: HUB_FLAG_PREP_FUSED needs a prior state_prepare");
  (void)ckpt;
  Plan* pl;
  if ((s = get_plan(a, 1, dtype, flags, pl)) != HUB_OK) return s;
  return run_plan(a, pl, dtype, theta, psi, lam, nullptr, batch, E, grad, (cudaStream_t)stream);
}

extern "C" hub_status hub_apply_h(ans_t a, const void* psi, void* lam, int32_t dtype, int64_t batch,
                                  hub_stream_t stream) {
  hub_status s = check_call(a, dtype, batch);
  if (s != HUB_OK) return s;
  if (!psi || !lam || psi == lam) return fail(HUB_EINVAL, "hub_apply_h: bad buffers");
  Plan* pl;
  if ((s = get_plan(a, 2, dtype, 0, pl)) != HUB_OK) return s;
  return run_plan(a, pl, dtype, nullptr, const_cast<void*>(psi), lam, nullptr, batch, nullptr, nullptr,
                  (cudaStream_t)stream);
}

extern "C" hub_status ans_plan_stats(ans_t a, int32_t which, int32_t dtype, uint32_t flags, int32_t* n_sweeps,
                                     double* bytes_per_state) {
  if (!a || which < 0 || which > 2 || (dtype != HUB_C64 && dtype != HUB_C128))
    return fail(HUB_EINVAL, "ans_plan_stats: bad arguments");
  Plan* pl;
  hub_status s = get_plan(a, which, dtype, flags, pl);
  if (s != HUB_OK) return s;
  if (n_sweeps) *n_sweeps = (int32_t)pl->sweeps.size();
  if (bytes_per_state) *bytes_per_state = pl->bytes_per_state;
  return HUB_OK;
}

extern "C" hub_status ans_plan_describe(ans_t a, int32_t which, int32_t dtype, uint32_t flags, int64_t* buf,
                                        int32_t cap, int32_t* len) {
  if (!a || !len || which < 0 || which > 2 || (dtype != HUB_C64 && dtype != HUB_C128))
    return fail(HUB_EINVAL, "ans_plan_describe: bad arguments");
  Plan* pl;
  hub_status s = get_plan(a, which, dtype, flags, pl);
  if (s != HUB_OK) return s;
  std::vector<int64_t> out;
  out.push_back((int64_t)pl->sweeps.size());
  for (size_t i = 0; i < pl->sweeps.size(); ++i) {
    out.push_back((int64_t)pl->tiles[i]);
    out.push_back((int64_t)pl->sweeps[i].flags);
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
