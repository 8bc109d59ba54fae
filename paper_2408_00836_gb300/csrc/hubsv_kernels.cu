// sm_103a kernels of the Hubbard VQE statevector engine.
//
// One kernel, sweep_kernel, does all amplitude work.  A sweep streams the
// whole 2^n (x batch) amplitude vector through shared memory once, one tile
// of 2^k amplitudes at a time.  A tile holds every amplitude whose index
// agrees with the tile's base on the non-tile bits; the tile bits always
// include the c lowest bits, so global loads and stores are runs of 2^c
// contiguous amplitudes (>= 256 B).  Inside the tile the sweep applies an
// ordered list of operations chosen by the host planner:
//
//  * OP_GIV: the factor exp(-i theta G) of one hopping term of Eq. 7,
//    G = -t (a+_p a_q + h.c.).  On each pair (x, x') with b_p != b_q it is
//    the 2x2 rotation [c, i s sigma; i s sigma, c], c = cos(theta t),
//    sigma = sin(theta t), s = (-1)^popcount(x & bits strictly between p and
//    q) -- the Jordan-Wigner string, from one popcount per pair.
//  * OP_DIAG: the diagonal factors of Eq. 7 (on-site U, NN V, potential,
//    Rz) as a phase looked up from per-byte tables.
//  * OP_MEAS_* / OP_LAM_*: the energy of Eq. 4 term by term (and lam = H psi
//    for the adjoint pass) without ever materialising H psi in HBM unless
//    the gradient needs it.
//  * OP_GRAD_*: the per-parameter reductions 2 Im <lam|G|psi> of the
//    adjoint recursion of Sec. 2.1.
//
// Reductions accumulate per thread (FP32 within one operation for c64,
// FP64 otherwise), are reduced per warp in FP64 and summed per CTA in
// shared memory; each CTA adds its totals to the global FP64 accumulators
// once per batch element.
#include "hubsv_internal.h"

namespace hubsv {

template <typename R> struct CT;
template <> struct CT<float> {
  using T2 = float2;
  using V = float4;       // 16-byte vector = 2 amplitudes
  static constexpr int VEC = 2;
};
template <> struct CT<double> {
  using T2 = double2;
  using V = double2;      // 16-byte vector = 1 amplitude
  static constexpr int VEC = 1;
};

template <typename T2, typename R>
__device__ __forceinline__ T2 mk(R x, R y) { T2 r; r.x = x; r.y = y; return r; }

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  T2 r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

__device__ __forceinline__ uint32_t insert_zero(uint32_t j, int b) {
  return (j & ((1u << b) - 1u)) | ((j >> b) << (b + 1));
}

__device__ __forceinline__ uint64_t deposit_bits(uint64_t v, const int8_t* pos, int cnt) {
  uint64_t r = 0;
  for (int i = 0; i < cnt; ++i) r |= ((v >> i) & 1ull) << pos[i];
  return r;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Add a per-thread partial to acc[slot] (shared).  Called uniformly by the
// whole CTA.
__device__ __forceinline__ void cta_add(double* acc, int slot, double v) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&acc[slot], v);
}

// Real value of a diagonal operator at x (see DiagOpDev).
__device__ __forceinline__ double diag_real(const DiagOpDev& d, const double* tab,
                                           uint64_t x, int s, uint64_t upmask) {
  double v = 0.0;
  for (int i = 0; i < d.has_x; ++i) v += tab[i * 256 + ((x >> (8 * i)) & 255u)];
  const uint64_t y = x & (x >> s) & upmask;
  for (int i = 0; i < d.has_y; ++i) v += tab[1024 + i * 256 + ((y >> (8 * i)) & 255u)];
  const double* vb = tab + 2048;
  for (int b = 0; b < d.n_vb; ++b) {
    const int u1 = d.vb_up[b], u2 = d.vb_up2[b];
    const int ni = (int)((x >> u1) & 1u) + (int)((x >> (u1 + s)) & 1u);
    const int nj = (int)((x >> u2) & 1u) + (int)((x >> (u2 + s)) & 1u);
    v += vb[b] * (double)(ni * nj);
  }
  return v;
}

// Phase exp(-i theta d(x)) from the per-batch-element phase tables.
template <typename T2>
__device__ __forceinline__ T2 diag_phase(const DiagOpDev& d, const T2* tab, uint64_t x,
                                         int s, uint64_t upmask) {
  T2 ph; ph.x = 1; ph.y = 0;
  for (int i = 0; i < d.has_x; ++i) ph = cmul(ph, tab[i * 256 + ((x >> (8 * i)) & 255u)]);
  const uint64_t y = x & (x >> s) & upmask;
  for (int i = 0; i < d.has_y; ++i) ph = cmul(ph, tab[1024 + i * 256 + ((y >> (8 * i)) & 255u)]);
  if (d.n_vb > 0) {
    const T2* vt = tab + 2048;
    if (d.v_uniform) {
      int K = 0;
      for (int b = 0; b < d.n_vb; ++b) {
        const int u1 = d.vb_up[b], u2 = d.vb_up2[b];
        const int ni = (int)((x >> u1) & 1u) + (int)((x >> (u1 + s)) & 1u);
        const int nj = (int)((x >> u2) & 1u) + (int)((x >> (u2 + s)) & 1u);
        K += ni * nj;
      }
      ph = cmul(ph, vt[K]);
    } else {
      for (int b = 0; b < d.n_vb; ++b) {
        const int u1 = d.vb_up[b], u2 = d.vb_up2[b];
        const int ni = (int)((x >> u1) & 1u) + (int)((x >> (u1 + s)) & 1u);
        const int nj = (int)((x >> u2) & 1u) + (int)((x >> (u2 + s)) & 1u);
        const int e = ni * nj;
        if (e) ph = cmul(ph, vt[b * 5 + e]);
      }
    }
  }
  return ph;
}

// Compress the bits of x at positions 0, 2, 4, ... into consecutive bits.
__device__ __forceinline__ uint32_t compress_even(uint64_t x) {
  x &= 0x5555555555555555ull;
  x = (x | (x >> 1)) & 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x >> 4)) & 0x00ff00ff00ff00ffull;
  x = (x | (x >> 8)) & 0x0000ffff0000ffffull;
  x = (x | (x >> 16)) & 0x00000000ffffffffull;
  return (uint32_t)x;
}

// Initial state amplitude at x (state-local index) for instance inst.
__device__ __forceinline__ double prep_amp(const PrepDev& p, uint64_t x, int inst) {
  if (p.kind == 1) return x == p.neel_x0 ? 1.0 : 0.0;
  uint32_t oa, ob;
  int sign = 0;
  if (p.layout == 0) {
    oa = (uint32_t)(x & ((1ull << p.L) - 1));
    ob = (uint32_t)(x >> p.L);
  } else {
    oa = compress_even(x);
    ob = compress_even(x >> 1);
    // ordering the creators a+(up, ascending) a+(dn, ascending) by mode:
    // dn mode 2j+1 precedes up mode 2i iff j < i.
    for (uint32_t m = oa; m; m &= m - 1) {
      const int i = __ffs(m) - 1;
      sign += __popc(ob & ((1u << i) - 1u));
    }
  }
  const size_t tl = (size_t)1 << p.L;
  const double* sd = p.sd + (size_t)inst * 2 * tl;
  const double v = sd[oa] * sd[tl + ob];
  return (sign & 1) ? -v : v;
}

template <typename R, int NV>
__global__ void __launch_bounds__(kThreads)
sweep_kernel(const SweepDev sw, const KernelArgs a) {
  using T2 = typename CT<R>::T2;
  using VT = typename CT<R>::V;
  constexpr int VEC = CT<R>::VEC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = sw.k, c = sw.c, h1 = sw.h1, h2 = sw.k - sw.c - sw.h1;
  const uint32_t tsize = 1u << k;
  T2* tp = reinterpret_cast<T2*>(smem_raw);
  T2* tl = tp + (NV == 2 ? tsize : 0);
  uint64_t* off_lo = reinterpret_cast<uint64_t*>(tp + NV * tsize);
  uint64_t* off_hi = off_lo + (1u << h1);
  double* acc = reinterpret_cast<double*>(off_hi + (1u << h2));
  const int tid = threadIdx.x;

  for (uint32_t i = tid; i < (1u << h1); i += kThreads) off_lo[i] = deposit_bits(i, sw.tbits + c, h1);
  for (uint32_t i = tid; i < (1u << h2); i += kThreads) off_hi[i] = deposit_bits(i, sw.tbits + c + h1, h2);
  for (int i = tid; i < a.n_slots; i += kThreads) acc[i] = 0.0;
  __syncthreads();

  const uint64_t chunk = (a.n_tiles + gridDim.x - 1) / gridDim.x;
  const uint64_t t0 = (uint64_t)blockIdx.x * chunk;
  const uint64_t t1 = min(t0 + chunk, a.n_tiles);
  const uint64_t cmask = (1ull << c) - 1;
  const uint32_t lmask = (1u << h1) - 1;
  long long cur_b = -1;

  for (uint64_t tau = t0; tau < t1; ++tau) {
    const uint64_t tl_idx = tau & ((1ull << sw.n_nontile) - 1);
    const long long b = (long long)(tau >> sw.n_nontile);
    if (b != cur_b) {
      if (cur_b >= 0) {
        __syncthreads();
        for (int i = tid; i < a.n_slots; i += kThreads) {
          const double v = acc[i];
          if (v != 0.0) atomicAdd(&a.acc[cur_b * a.n_slots + i], v);
          acc[i] = 0.0;
        }
        __syncthreads();
      }
      cur_b = b;
    }
    const int inst = (int)(b % a.n_inst);
    const uint64_t sbase = deposit_bits(tl_idx, sw.nbits, sw.n_nontile);   // state-local
    const uint64_t gbase = ((uint64_t)b << a.n) | sbase;                      // global

    // ---- load (or generate) the tile ----
    for (uint32_t v = tid; v < tsize / VEC; v += kThreads) {
      const uint32_t l = v * VEC;
      const uint64_t off = (l & cmask) | off_lo[(l >> c) & lmask] | off_hi[l >> (c + h1)];
      if (sw.flags & SW_PREP) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          const double amp = prep_amp(a.prep, sbase | (off + e), inst);
          tp[l + e] = mk<T2, R>((R)amp, (R)0);
        }
      } else {
        const T2* src = reinterpret_cast<const T2*>((sw.flags & SW_CKPT_READ) ? a.ckpt : a.psi);
        const VT w = *reinterpret_cast<const VT*>(src + gbase + off);
        *reinterpret_cast<VT*>(tp + l) = w;
      }
      if (NV == 2) {
        if (sw.flags & SW_READ_LAM) {
          const T2* src = reinterpret_cast<const T2*>(a.lam);
          *reinterpret_cast<VT*>(tl + l) = *reinterpret_cast<const VT*>(src + gbase + off);
        } else {
#pragma unroll
          for (int e = 0; e < VEC; ++e) tl[l + e] = mk<T2, R>((R)0, (R)0);
        }
      }
    }
    __syncthreads();

    double eacc = 0.0, nacc = 0.0;
    double racc = 0.0;
    int rslot = -1;

    for (int oi = sw.op_begin; oi < sw.op_end; ++oi) {
      const OpDev op = a.ops[oi];
      if (op.kind == OP_GRAD_HOP || op.kind == OP_GRAD_DIAG) {
        if (op.slot != rslot) {
          if (rslot >= 0) cta_add(acc, rslot, racc);
          racc = 0.0;
          rslot = op.slot;
        }
      }
      const uint32_t mp = 1u << op.p, mq = 1u << op.q;
      const int tpar = __popcll(sbase & op.bmask_global) & 1;
      switch (op.kind) {
        case OP_GIV: {
          const T2 cs = reinterpret_cast<const T2*>(a.coef)[(size_t)b * a.n_gates + op.gate];
          const R cc = cs.x;
          const R sn = (op.flags & OPF_INV) ? -cs.y : cs.y;
          const bool dol = (NV == 2) && (op.flags & OPF_LAM);
          for (uint32_t j = tid; j < tsize / 4; j += kThreads) {
            const uint32_t l0 = insert_zero(insert_zero(j, op.p), op.q);
            const int par = (__popc(l0 & op.bmask_local) + tpar) & 1;
            const R ss = par ? -sn : sn;
            const uint32_t lx = l0 | mq, ly = l0 | mp;
            T2 u = tp[lx], w = tp[ly];
            tp[lx] = mk<T2, R>(cc * u.x - ss * w.y, cc * u.y + ss * w.x);
            tp[ly] = mk<T2, R>(cc * w.x - ss * u.y, cc * w.y + ss * u.x);
            if (dol) {
              u = tl[lx]; w = tl[ly];
              tl[lx] = mk<T2, R>(cc * u.x - ss * w.y, cc * u.y + ss * w.x);
              tl[ly] = mk<T2, R>(cc * w.x - ss * u.y, cc * w.y + ss * u.x);
            }
          }
          break;
        }
        case OP_MEAS_HOP:
        case OP_LAM_HOP:
        case OP_GRAD_HOP: {
          const R tc = (R)a.hcoef[(size_t)inst * a.n_hterms + op.hterm];
          R part = 0;
          for (uint32_t j = tid; j < tsize / 4; j += kThreads) {
            const uint32_t l0 = insert_zero(insert_zero(j, op.p), op.q);
            const int par = (__popc(l0 & op.bmask_local) + tpar) & 1;
            const R ts = par ? -tc : tc;
            const uint32_t lx = l0 | mq, ly = l0 | mp;
            const T2 u = tp[lx], w = tp[ly];
            if (op.kind == OP_GRAD_HOP) {
              if (NV == 2) {
                const T2 lu = tl[lx], lw = tl[ly];
                // Im(conj(lam_x) psi_x') + Im(conj(lam_x') psi_x)
                part += ts * ((lu.x * w.y - lu.y * w.x) + (lw.x * u.y - lw.y * u.x));
              }
            } else {
              part += ts * (u.x * w.x + u.y * w.y);
              if (NV == 2 && op.kind == OP_LAM_HOP) {
                T2 lu = tl[lx], lw = tl[ly];
                lu.x += ts * w.x; lu.y += ts * w.y;
                lw.x += ts * u.x; lw.y += ts * u.y;
                tl[lx] = lu; tl[ly] = lw;
              }
            }
          }
          if (op.kind == OP_GRAD_HOP) racc += 2.0 * (double)part;
          else eacc += 2.0 * (double)part;
          break;
        }
        case OP_DIAG: {
          const DiagOpDev& d = a.diag_ops[op.diag];
          const T2* ptab = reinterpret_cast<const T2*>(a.phase_tabs) + (size_t)b * a.phase_stride + d.phase_off;
          const bool inv = op.flags & OPF_INV;
          const bool dol = (NV == 2) && (op.flags & OPF_LAM);
          for (uint32_t l = tid; l < tsize; l += kThreads) {
            const uint64_t off = (l & cmask) | off_lo[(l >> c) & lmask] | off_hi[l >> (c + h1)];
            T2 ph = diag_phase<T2>(d, ptab, sbase | off, a.s, a.upmask);
            if (inv) ph.y = -ph.y;
            tp[l] = cmul(tp[l], ph);
            if (dol) tl[l] = cmul(tl[l], ph);
          }
          break;
        }
        case OP_MEAS_DIAG:
        case OP_LAM_DIAG:
        case OP_GRAD_DIAG: {
          const DiagOpDev& d = a.diag_ops[op.diag];
          const double* rtab = a.real_tabs + (size_t)inst * a.real_stride + d.real_off;
          double pe = 0.0, pn = 0.0;
          R pe32 = 0, pn32 = 0;
          for (uint32_t l = tid; l < tsize; l += kThreads) {
            const uint64_t off = (l & cmask) | off_lo[(l >> c) & lmask] | off_hi[l >> (c + h1)];
            const R dv = (R)diag_real(d, rtab, sbase | off, a.s, a.upmask);
            const T2 u = tp[l];
            if (op.kind == OP_GRAD_DIAG) {
              if (NV == 2) {
                const T2 lu = tl[l];
                pe32 += dv * (lu.x * u.y - lu.y * u.x);
              }
            } else {
              const R m2 = u.x * u.x + u.y * u.y;
              pe32 += dv * m2;
              pn32 += m2;
              if (NV == 2 && op.kind == OP_LAM_DIAG) {
                T2 lu = tl[l];
                lu.x += dv * u.x; lu.y += dv * u.y;
                tl[l] = lu;
              }
            }
          }
          pe += (double)pe32; pn += (double)pn32;
          if (op.kind == OP_GRAD_DIAG) racc += 2.0 * pe;
          else { eacc += pe; nacc += pn; }
          break;
        }
        default: break;
      }
      __syncthreads();
    }
    if (rslot >= 0) cta_add(acc, rslot, racc);
    cta_add(acc, a.slot_E, eacc);
    cta_add(acc, a.slot_N, nacc);

    // ---- store ----
    const bool wp = sw.flags & SW_WRITE_PSI, wc = sw.flags & SW_CKPT_WRITE;
    const bool wl = (NV == 2) && (sw.flags & SW_WRITE_LAM);
    if (wp || wc || wl) {
      for (uint32_t v = tid; v < tsize / VEC; v += kThreads) {
        const uint32_t l = v * VEC;
        const uint64_t off = (l & cmask) | off_lo[(l >> c) & lmask] | off_hi[l >> (c + h1)];
        const VT w = *reinterpret_cast<const VT*>(tp + l);
        if (wp) *reinterpret_cast<VT*>(reinterpret_cast<T2*>(a.psi) + gbase + off) = w;
        if (wc) *reinterpret_cast<VT*>(reinterpret_cast<T2*>(a.ckpt) + gbase + off) = w;
        if (wl) *reinterpret_cast<VT*>(reinterpret_cast<T2*>(a.lam) + gbase + off) = *reinterpret_cast<const VT*>(tl + l);
      }
    }
    __syncthreads();
  }
  __syncthreads();
  if (cur_b >= 0) {
    for (int i = tid; i < a.n_slots; i += kThreads) {
      const double v = acc[i];
      if (v != 0.0) atomicAdd(&a.acc[cur_b * a.n_slots + i], v);
    }
  }
}

// ---------------------------------------------------------------------------
// coefficient and phase tables (one thread per entry, FP64 trig)
// ---------------------------------------------------------------------------

// Round the unit complex number (c, s) to the precision of R.  For FP32 the
// pair is chosen among the neighbouring representable values as the one
// closest to the unit circle, so a rotation or phase with these entries
// changes norms by ~1e-8 instead of ~1e-7 (this drift would otherwise add
// up over the forward factors and their inverses in the adjoint pass).
template <typename R>
__device__ __forceinline__ typename CT<R>::T2 unit_round(double c, double s);
template <>
__device__ __forceinline__ double2 unit_round<double>(double c, double s) {
  return make_double2(c, s);
}
template <>
__device__ __forceinline__ float2 unit_round<float>(double c, double s) {
  const float c0 = (float)c, s0 = (float)s;
  float bc = c0, bs = s0;
  double be = fabs((double)c0 * c0 + (double)s0 * s0 - 1.0);
  const float cs[3] = {nextafterf(c0, -2.f), c0, nextafterf(c0, 2.f)};
  const float ss[3] = {nextafterf(s0, -2.f), s0, nextafterf(s0, 2.f)};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double e = fabs((double)cs[i] * cs[i] + (double)ss[j] * ss[j] - 1.0);
      if (e < be) { be = e; bc = cs[i]; bs = ss[j]; }
    }
  return make_float2(bc, bs);
}

template <typename R>
__global__ void coef_kernel(const double* __restrict__ theta, int P,
                            const int32_t* __restrict__ gate_param,
                            const double* __restrict__ gate_t, int n_gates,
                            typename CT<R>::T2* __restrict__ coef,
                            const int32_t* __restrict__ tab_param,
                            const double* __restrict__ tab_val, int n_tab,
                            typename CT<R>::T2* __restrict__ phase, int64_t batch, int n_inst) {
  using T2 = typename CT<R>::T2;
  const int64_t per = (int64_t)n_gates + n_tab;
  const int64_t total = per * batch;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / per;
    const int64_t j = i - b * per;
    const int inst = (int)(b % n_inst);
    if (j < n_gates) {
      const double al = theta[b * P + gate_param[j]] * gate_t[(int64_t)inst * n_gates + j];
      double s, c;
      sincos(al, &s, &c);
      coef[b * n_gates + j] = unit_round<R>(c, s);
    } else {
      const int64_t e = j - n_gates;
      const int pp = tab_param[e];
      const double th = pp >= 0 ? theta[b * P + pp] : 0.0;
      const double al = -th * tab_val[(int64_t)inst * n_tab + e];
      double s, c;
      sincos(al, &s, &c);
      phase[b * n_tab + e] = unit_round<R>(c, s);
    }
  }
}

__global__ void zero_kernel(double* p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0.0;
}

__global__ void finalize_kernel(const double* __restrict__ acc, int n_slots, int P, int slot_E,
                                double* __restrict__ E, double* __restrict__ grad, int64_t batch) {
  const int64_t total = batch * (P + 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / (P + 1);
    const int j = (int)(i - b * (P + 1));
    if (j == P) {
      if (E) E[b] = acc[b * n_slots + slot_E];
    } else if (grad) {
      grad[b * P + j] = acc[b * n_slots + j];
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

static int g_sm_count = 0;

int device_sm_count() {
  if (g_sm_count == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  }
  return g_sm_count;
}

int sweep_max_smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return v;
}

cudaError_t sweep_set_smem(int dtype, int nv, size_t smem) {
  const void* f;
  if (dtype == 0) f = nv == 2 ? (const void*)sweep_kernel<float, 2> : (const void*)sweep_kernel<float, 1>;
  else f = nv == 2 ? (const void*)sweep_kernel<double, 2> : (const void*)sweep_kernel<double, 1>;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_sweep(int dtype, const SweepDev& sw, const KernelArgs& a, int grid,
                         size_t smem, cudaStream_t st) {
  const bool two = sw.flags & SW_HAS_LAM;
  if (dtype == 0) {
    if (two) sweep_kernel<float, 2><<<grid, kThreads, smem, st>>>(sw, a);
    else sweep_kernel<float, 1><<<grid, kThreads, smem, st>>>(sw, a);
  } else {
    if (two) sweep_kernel<double, 2><<<grid, kThreads, smem, st>>>(sw, a);
    else sweep_kernel<double, 1><<<grid, kThreads, smem, st>>>(sw, a);
  }
  return cudaGetLastError();
}

cudaError_t launch_coef(int dtype, const double* theta, int P, const int32_t* gate_param,
                        const double* gate_t, int n_gates, void* coef,
                        const int32_t* tab_param, const double* tab_val, int n_tab,
                        int /*n_inst_tab*/, void* phase_tabs, int64_t batch, int n_inst,
                        cudaStream_t st) {
  const int64_t total = ((int64_t)n_gates + n_tab) * batch;
  if (total == 0) return cudaSuccess;
  int grid = (int)((total + 255) / 256);
  if (grid > 4096) grid = 4096;
  if (dtype == 0)
    coef_kernel<float><<<grid, 256, 0, st>>>(theta, P, gate_param, gate_t, n_gates,
                                             (float2*)coef, tab_param, tab_val, n_tab,
                                             (float2*)phase_tabs, batch, n_inst);
  else
    coef_kernel<double><<<grid, 256, 0, st>>>(theta, P, gate_param, gate_t, n_gates,
                                              (double2*)coef, tab_param, tab_val, n_tab,
                                              (double2*)phase_tabs, batch, n_inst);
  return cudaGetLastError();
}

cudaError_t launch_zero(double* p, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256);
  if (grid > 1024) grid = 1024;
  zero_kernel<<<grid, 256, 0, st>>>(p, n);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double* acc, int n_slots, int P, int slot_E, double* E,
                            double* grad, int64_t batch, cudaStream_t st) {
  const int64_t total = batch * (P + 1);
  int grid = (int)((total + 255) / 256);
  if (grid > 1024) grid = 1024;
  finalize_kernel<<<grid, 256, 0, st>>>(acc, n_slots, P, slot_E, E, grad, batch);
  return cudaGetLastError();
}

}  // namespace hubsv
