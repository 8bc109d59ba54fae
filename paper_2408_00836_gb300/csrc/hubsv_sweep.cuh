// The sweep kernel of the Hubbard VQE statevector engine (sm_103a),
// included by the four instantiation units hubsv_sweep_{f1,f2,d1,d2}.cu.
//
// One kernel, sweep_kernel, does all amplitude work.  A sweep streams the
// whole 2^n (x batch) amplitude vector once, one tile of 2^k amplitudes at a
// time.  A tile holds every amplitude whose index agrees with the tile's
// base on the non-tile bits; the tile bits always include the c lowest bits
// (the run bits), so a warp loads and stores whole runs of 2^c contiguous
// amplitudes (8 by default: 64 B in c64).  Fewer run bits leave more tile
// bits to the operations, and so fewer sweeps.  Every operation conserves
// the numbers of up and down electrons, so when the library generates the
// initial state (in the (N_up, N_dn) sector) a sweep visits only the tiles
// that meet the sector; the others are zero throughout (see SweepDev).
//
// Inside a tile the amplitudes live in registers: in a register phase each
// thread holds the 2^r amplitudes that differ in r chosen tile bits (its
// register slots), and every operation whose bits are register slots runs
// without touching memory.  Between phases the tile is exchanged through
// shared memory (XOR-swizzled against bank conflicts) to bring other bits
// into the register slots.  The first and last phase put the run bits on
// lanes, so global loads and stores go straight to and from registers.
//
// Operations (chosen and ordered by the host planner):
//  * OP_GIV: the factor exp(-i theta G) of one hopping term of Eq. 7,
//    G = -t (a+_p a_q + h.c.).  On each pair (x, x') with b_p != b_q it is
//    the 2x2 rotation [c, i s sigma; i s sigma, c], c = cos(theta t),
//    sigma = sin(theta t), s = (-1)^popcount(x & bits strictly between p and
//    q) -- the Jordan-Wigner string, from popcounts of masked indices.
//  * OP_DIAG: the diagonal factors of Eq. 7 (on-site U, NN V, potential,
//    Rz) as a phase looked up from per-byte tables.
//  * OP_MEAS_* / OP_LAM_*: the energy of Eq. 4 term by term (and lam = H psi
//    for the adjoint pass) without materialising H psi in HBM unless the
//    gradient needs it.
//  * OP_GRAD_*: the per-parameter reductions 2 Im <lam|G|psi> of the
//    adjoint recursion of Sec. 2.1.
//
// Reductions accumulate per thread in the working precision within one tile
// and are reduced per warp in that precision (c64: FP32 shuffles into
// per-warp float-pair rows updated with TwoSum; c128: FP64); the rows are
// summed in FP64 and each CTA adds its totals to the global FP64
// accumulators once per batch element.
#pragma once
#include <type_traits>

#include "hubsv_internal.h"

namespace hubsv {

template <typename R> struct CT;
template <> struct CT<float> { using T2 = float2; static constexpr int DT = 0; };
template <> struct CT<double> { using T2 = double2; static constexpr int DT = 1; };

// Givens coefficients of one factor, (cos, sin) of its angle, 16 bytes in
// both precisions.  complex64 keeps each as an FP32 pair hi + lo (GC<float>
// = {c, s, c_lo, s_lo}): rounding cos and sin to FP32 alone moves each
// rotation's angle by up to ~1e-7, the same shift on every factor of a
// shared parameter, and that coherent shift gave complex64 gradients
// errors of ~1e-6 relative; the pair keeps the angle exact to ~1e-14.
// complex128 keeps doubles (GC<double> = {c, s}).
template <typename R> struct GC;
template <> struct GC<float> {
  using T = float4;
  __device__ static float cl(const float4& g) { return g.z; }
  __device__ static float sl(const float4& g) { return g.w; }
};
template <> struct GC<double> {
  using T = double2;
  __device__ static double cl(const double2&) { return 0.0; }
  __device__ static double sl(const double2&) { return 0.0; }
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

__device__ __forceinline__ uint32_t deposit_bits(uint32_t v, const int8_t* pos, int cnt) {
  uint32_t r = 0;
  for (int i = 0; i < cnt; ++i) r |= ((v >> i) & 1u) << pos[i];
  return r;
}

static __constant__ BinomTable c_binom = make_binom_table();

// The r-th n-bit pattern among those with lo, lo+1, ... bits set, ordered by
// the number of set bits and then colexicographically (combinatorial number
// system: the highest set bit is the largest p with C(p, m) <= rank).  All
// threads of a CTA unrank the same r, so the table reads are uniform.
__device__ __forceinline__ uint32_t unrank_bits(uint32_t r, int n, int lo) {
  int m = lo;
  while (r >= c_binom.c[n][m]) { r -= c_binom.c[n][m]; ++m; }
  uint32_t x = 0;
  for (int p = n - 1; p >= 0 && m > 0; --p) {
    const uint32_t cnt = c_binom.c[p][m];
    if (r >= cnt) { x |= 1u << p; r -= cnt; --m; }
  }
  return x;
}

// Advance x to the next pattern in that order (n bits, at most hi set):
// the colex successor with the same number of set bits (Gosper's rule), else
// the smallest pattern with one more bit set.  Returns false when x was the
// last pattern.
__device__ __forceinline__ bool next_pattern(uint32_t& x, int n, int hi) {
  const int m = __popc(x);
  if (m > 0) {
    const uint32_t c = x & (0u - x);
    const uint32_t r = x + c;
    const uint32_t nx = r | (((r ^ x) >> 2) >> (__ffs(c) - 1));
    if (nx < (1u << n)) { x = nx; return true; }
  }
  if (m + 1 > hi) return false;
  x = (1u << (m + 1)) - 1u;
  return true;
}

// Bits of x moved to positions pos[i] (one step per set bit).
__device__ __forceinline__ uint32_t deposit_set(uint32_t x, const int8_t* pos) {
  uint32_t r = 0;
  for (; x; x &= x - 1u) r |= 1u << pos[__ffs(x) - 1];
  return r;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP64 arithmetic is a small fraction of FP32 throughput on this part, so
// the complex64 kernels reduce in FP32 and keep their running sums as
// unevaluated float pairs (hi + lo) updated with Knuth's TwoSum, which is
// exact: the sums carry about 48 bits although no FP64 instruction runs per
// tile.  The complex128 kernels reduce in FP64.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (h, l) += v, renormalised so that |l| <= ulp(h) / 2.
__device__ __forceinline__ void ff_add(float& h, float& l, float v) {
  float s, e;
  two_sum(h, v, s, e);
  e += l;
  h = s + e;
  l = e - (h - s);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of float pairs over the warp, into lane 0's (h, l): each level adds
// with TwoSum and carries the rounding error in l.
__device__ __forceinline__ void warp_sum_ff(float& h, float& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
    float s, e;
    two_sum(h, h2, s, e);
    e += l + l2;
    h = s + e;
    l = e - (h - s);
  }
}

__device__ __forceinline__ double row_value(const float2& v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ double row_value(double v) { return v; }

// Shared accumulators of a CTA.  complex64: one row of float pairs per warp
// (row w, slot i at acc[w * n_slots + i]), written by lane 0 of warp w only,
// so no atomics; complex128: one row of doubles, FP64 atomics.  Both are
// summed over rows in FP64 when they are flushed to global memory.
// cta_add adds a per-thread partial to slot; called uniformly by the CTA.
__device__ __forceinline__ void cta_add(float2* acc, int n_slots, int slot, float v) {
  v = warp_sum_f(v);
  if ((threadIdx.x & 31) == 0) {
    float2& t = acc[(threadIdx.x >> 5) * n_slots + slot];
    ff_add(t.x, t.y, v);
  }
}
__device__ __forceinline__ void cta_add(double* acc, int /*n_slots*/, int slot, double v) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&acc[slot], v);
}

// XOR of the slot values m[j] over the set bits j of e (e is a constant
// after unrolling, so this folds to at most a few logic operations).
template <int RB>
__device__ __forceinline__ uint32_t comb(const uint32_t (&m)[RB], int e) {
  uint32_t v = 0;
#pragma unroll
  for (int j = 0; j < RB; ++j)
    if ((e >> j) & 1) v ^= m[j];
  return v;
}

// K = sum over the bonds of n_i n_j at x, for uniform V (see DiagOpDev).
__device__ __forceinline__ int v_count(const DiagOpDev& d, uint32_t x, int s, uint32_t upmask) {
  int K = 0;
  if (d.n_vs >= 0) {
    const uint32_t A = x & upmask, B = (x >> s) & upmask;
    const uint32_t O1 = A | B, O2 = A & B;
    for (int g = 0; g < d.n_vs; ++g) {
      const int sh = d.vs_shift[g];
      const uint32_t m = d.vs_mask[g];
      const uint32_t p1 = O1 & m, p2 = O2 & m, q1 = O1 >> sh, q2 = O2 >> sh;
      K += __popc(p1 & q1) + __popc(p1 & q2) + __popc(p2 & q1) + __popc(p2 & q2);
    }
  } else {
    for (int b = 0; b < d.n_vb; ++b) {
      const int u1 = d.vb_up[b], u2 = d.vb_up2[b];
      const int ni = (int)((x >> u1) & 1u) + (int)((x >> (u1 + s)) & 1u);
      const int nj = (int)((x >> u2) & 1u) + (int)((x >> (u2 + s)) & 1u);
      K += ni * nj;
    }
  }
  return K;
}

// Real value of a diagonal operator at x (see DiagOpDev), in the working
// precision R (tables stored in R).
// VP: uniform V terms through v_count's popcounts (kernel variants for
// sweeps flagged SW_VPOP); otherwise bond by bond.
template <typename R, bool VP = false>
__device__ __forceinline__ R diag_real(const DiagOpDev& d, const R* tab, uint32_t x, int s,
                                      uint32_t upmask) {
  R v = 0;
  for (int i = 0; i < d.has_x; ++i) v += tab[i * 256 + ((x >> (8 * i)) & 255u)];
  const uint32_t y = x & (x >> s) & upmask;
  for (int i = 0; i < d.has_y; ++i) v += tab[1024 + i * 256 + ((y >> (8 * i)) & 255u)];
  const R* vb = tab + 2048;
  if (VP && d.n_vb > 0 && d.v_uniform) {
    v += vb[0] * (R)v_count(d, x, s, upmask);
  } else {
    for (int b = 0; b < d.n_vb; ++b) {
      const int u1 = d.vb_up[b], u2 = d.vb_up2[b];
      const int ni = (int)((x >> u1) & 1u) + (int)((x >> (u1 + s)) & 1u);
      const int nj = (int)((x >> u2) & 1u) + (int)((x >> (u2 + s)) & 1u);
      v += vb[b] * (R)(ni * nj);
    }
  }
  for (int m = 0; m < d.n_mp; ++m)
    if ((x >> d.mp_p[m]) & (x >> d.mp_q[m]) & 1u) v += tab[d.mp_roff + m];
  return v;
}

// Phase exp(-i theta d(x)) from the per-batch-element phase tables.
template <typename T2, bool VP = false>
__device__ __forceinline__ T2 diag_phase(const DiagOpDev& d, const T2* tab, uint32_t x, int s,
                                         uint32_t upmask) {
  T2 ph; ph.x = 1; ph.y = 0;
  for (int i = 0; i < d.has_x; ++i) ph = cmul(ph, tab[i * 256 + ((x >> (8 * i)) & 255u)]);
  const uint32_t y = x & (x >> s) & upmask;
  for (int i = 0; i < d.has_y; ++i) ph = cmul(ph, tab[1024 + i * 256 + ((y >> (8 * i)) & 255u)]);
  if (d.n_vb > 0) {
    const T2* vt = tab + 2048;
    if (VP && d.v_uniform) {
      ph = cmul(ph, vt[v_count(d, x, s, upmask)]);
    } else if (d.v_uniform) {
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
  for (int m = 0; m < d.n_mp; ++m)
    if ((x >> d.mp_p[m]) & (x >> d.mp_q[m]) & 1u) ph = cmul(ph, tab[d.mp_poff + m]);
  return ph;
}

// Compress the bits of x at positions 0, 2, 4, ... into consecutive bits.
__device__ __forceinline__ uint32_t compress_even(uint32_t x) {
  x &= 0x55555555u;
  x = (x | (x >> 1)) & 0x33333333u;
  x = (x | (x >> 2)) & 0x0f0f0f0fu;
  x = (x | (x >> 4)) & 0x00ff00ffu;
  x = (x | (x >> 8)) & 0x0000ffffu;
  return x;
}

// Initial state amplitude at x (state-local index) for instance inst, from
// the determinant tables stored in the working precision R.
template <typename R>
__device__ __forceinline__ R prep_amp(const PrepDev& p, const R* sdt, uint32_t x, int inst) {
  if (p.kind == 1) return x == (uint32_t)p.neel_x0 ? (R)1 : (R)0;
  uint32_t oa, ob;
  int sign = 0;
  if (p.layout == 0) {
    oa = x & ((1u << p.L) - 1u);
    ob = (uint32_t)((uint64_t)x >> p.L);
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
  const R* sd = sdt + (size_t)inst * 2 * tl;
  const R v = sd[oa] * sd[tl + ob];
  return (sign & 1) ? -v : v;
}

// ---------------------------------------------------------------------------
// register-slot pair operations (A < B compile-time slots)
// ---------------------------------------------------------------------------

template <typename T2, typename R>
__device__ __forceinline__ void rot(T2& u, T2& w, R c, R s) {
  const T2 u0 = u, w0 = w;
  u = mk<T2, R>(c * u0.x - s * w0.y, c * u0.y + s * w0.x);
  w = mk<T2, R>(c * w0.x - s * u0.y, c * w0.y + s * u0.x);
}

// The same rotation with (cos, sin) given as FP32 pairs c + cl, s + sl
// (complex64; see GC): the low parts enter as one more product each, so the
// rotation angle is exact to the pair's ~1e-14 while the amplitudes stay
// FP32.  For complex128 (cl = sl = 0) it is rot().
template <typename T2, typename R>
__device__ __forceinline__ void rot(T2& u, T2& w, R c, R s, R cl, R sl) {
  if constexpr (sizeof(R) == 4) {
    const T2 u0 = u, w0 = w;
    u = mk<T2, R>(fmaf(c, u0.x, fmaf(-s, w0.y, fmaf(cl, u0.x, -sl * w0.y))),
                  fmaf(c, u0.y, fmaf(s, w0.x, fmaf(cl, u0.y, sl * w0.x))));
    w = mk<T2, R>(fmaf(c, w0.x, fmaf(-s, u0.y, fmaf(cl, w0.x, -sl * u0.y))),
                  fmaf(c, w0.y, fmaf(s, u0.x, fmaf(cl, w0.y, sl * u0.x))));
  } else {
    rot(u, w, c, s);
  }
}

// Packed FP32 pair arithmetic: on sm_100-family GPUs fma.rn.f32x2 and
// mul.rn.f32x2 work on both halves of a 64-bit register pair in one
// instruction, each half rounded exactly as the scalar fmaf / multiply.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 splat2(float x) { return make_float2(x, x); }

// i * sigma * w as a float pair, sigma = -1 where m = 0x80000000, +1 where
// m = 0: (-sigma w.y, sigma w.x), two sign-bit logic ops.
__device__ __forceinline__ float2 iswap(float2 w, uint32_t m) {
  return make_float2(__int_as_float(__float_as_int(w.y) ^ (int)(m ^ 0x80000000u)),
                     __int_as_float(__float_as_int(w.x) ^ (int)m));
}
// sigma * w
__device__ __forceinline__ float2 sflip2(float2 w, uint32_t m) {
  return make_float2(__int_as_float(__float_as_int(w.x) ^ (int)m), __int_as_float(__float_as_int(w.y) ^ (int)m));
}

// The complex64 rotation of rot(u, w, c, sigma s, cl, sigma sl) in packed
// form: u' = c u + i sigma s w (+ the low parts), w' likewise; C, S, CL, SL
// hold each coefficient in both halves.  The same products and sums as the
// scalar form, so the results are bitwise equal.  su, sw (i sigma u,
// i sigma w of the inputs) are returned for a gradient term.
__device__ __forceinline__ void rot_pk(float2& u, float2& w, float2 C, float2 S, float2 CL, float2 SL,
                                       uint32_t m, float2& su, float2& sw) {
  sw = iswap(w, m);
  su = iswap(u, m);
  u = fma2(C, u, fma2(S, sw, fma2(CL, u, mul2(SL, sw))));
  w = fma2(C, w, fma2(S, su, fma2(CL, w, mul2(SL, su))));
}
__device__ __forceinline__ void rot_pk(float2& u, float2& w, float2 C, float2 S, float2 CL, float2 SL,
                                       uint32_t m) {
  float2 su, sw;
  rot_pk(u, w, C, S, CL, SL, m, su, sw);
}

// x with its sign flipped when bit e of m is set (m: per-op sign mask; e is
// a constant after unrolling, so this is a shift and two logic ops).
__device__ __forceinline__ float sflip(float x, uint32_t m, int e) {
  return __int_as_float(__float_as_int(x) ^ ((m << (31 - e)) & 0x80000000u));
}
__device__ __forceinline__ double sflip(double x, uint32_t m, int e) {
  return __hiloint2double(__double2hiint(x) ^ (int)((m << (31 - e)) & 0x80000000u), __double2loint(x));
}

// PKD: packed complex64 arithmetic (the kernel variants with the V and
// mode-pair fast paths keep the scalar form: the register pairs the packed
// instructions need made them spill).
template <int A, int B, bool PKD, int NE, typename T2, typename R>
__device__ __forceinline__ void pair_giv(T2 (&v)[NE], R c, R s, R cl, R sl, uint32_t sm) {
  if constexpr (PKD && sizeof(R) == 4) {   // complex64: packed pair arithmetic (see rot_pk)
    const float2 C2 = splat2(c), S2 = splat2(s), CL2 = splat2(cl), SL2 = splat2(sl);
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      if (((e >> A) & 1) == 0 && ((e >> B) & 1) == 1) {
        constexpr int F = (1 << A) | (1 << B);
        rot_pk(v[e], v[e ^ F], C2, S2, CL2, SL2, (sm << (31 - e)) & 0x80000000u);
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      if (((e >> A) & 1) == 0 && ((e >> B) & 1) == 1) {
        constexpr int F = (1 << A) | (1 << B);
        rot(v[e], v[e ^ F], c, sflip(s, sm, e), cl, sflip(sl, sm, e));
      }
    }
  }
}

// mode 0: energy term; 1: energy term + lam += h psi; 2: gradient term.
template <int A, int B, int MODE, int NE, typename T2, typename R>
__device__ __forceinline__ R pair_hop(T2 (&v)[NE], T2 (&l)[NE], R tc, uint32_t sm) {
  R part = 0;
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    if (((e >> A) & 1) == 0 && ((e >> B) & 1) == 1) {
      constexpr int F = (1 << A) | (1 << B);
      const R ts = sflip(tc, sm, e);
      const T2 u = v[e], w = v[e ^ F];
      if (MODE == 2) {
        const T2 lu = l[e], lw = l[e ^ F];
        part += ts * ((lu.x * w.y - lu.y * w.x) + (lw.x * u.y - lw.y * u.x));
      } else {
        part += ts * (u.x * w.x + u.y * w.y);
        if (MODE == 1) {
          l[e].x += ts * w.x; l[e].y += ts * w.y;
          l[e ^ F].x += ts * u.x; l[e ^ F].y += ts * u.y;
        }
      }
    }
  }
  return part;
}

// Gradient term 2 Im <lam|G_term|psi> of one hop term, then its inverse
// factor on psi and lam (the reduction uses the values before the inverse;
// the factor commutes with its own generator, so either order is exact).
template <int A, int B, bool PKD, int NE, typename T2, typename R>
__device__ __forceinline__ R pair_gradinv(T2 (&v)[NE], T2 (&l)[NE], R c, R s, R cl, R sl, R tc, uint32_t sm) {
  if constexpr (PKD && sizeof(R) == 4) {   // complex64: packed (see rot_pk and row_hop)
    const float2 C2 = splat2(c), S2 = splat2(s), CL2 = splat2(cl), SL2 = splat2(sl);
    float2 acc2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      if (((e >> A) & 1) == 0 && ((e >> B) & 1) == 1) {
        constexpr int F = (1 << A) | (1 << B);
        const uint32_t m = (sm << (31 - e)) & 0x80000000u;
        const T2 lu = l[e], lw = l[e ^ F];
        float2 su, sw;
        rot_pk(v[e], v[e ^ F], C2, S2, CL2, SL2, m, su, sw);
        acc2 = fma2(lu, sw, acc2);
        acc2 = fma2(lw, su, acc2);
        rot_pk(l[e], l[e ^ F], C2, S2, CL2, SL2, m);
      }
    }
    // (lu, i sigma w) + (lw, i sigma u) over both halves: -sigma (the term)
    return -tc * (acc2.x + acc2.y);
  } else {
    R part = 0;
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      if (((e >> A) & 1) == 0 && ((e >> B) & 1) == 1) {
        constexpr int F = (1 << A) | (1 << B);
        const T2 u = v[e], w = v[e ^ F], lu = l[e], lw = l[e ^ F];
        part += sflip(tc, sm, e) * ((lu.x * w.y - lu.y * w.x) + (lw.x * u.y - lw.y * u.x));
        const R ss = sflip(s, sm, e), ssl = sflip(sl, sm, e);
        rot(v[e], v[e ^ F], c, ss, cl, ssl);
        rot(l[e], l[e ^ F], c, ss, cl, ssl);
      }
    }
    return part;
  }
}

// Case labels of the ten register slot pairs (a, b), a < b, for one
// operation class starting at code BASE (see ResCode / pair_index).
#define HUB_PAIRS(BASE, CALL)                                       \
  case (BASE) + 0: { CALL(0, 1) } break;                            \
  case (BASE) + 1: if constexpr (RB > 2) { CALL(0, 2) } break;      \
  case (BASE) + 2: if constexpr (RB > 2) { CALL(1, 2) } break;      \
  case (BASE) + 3: if constexpr (RB > 3) { CALL(0, 3) } break;      \
  case (BASE) + 4: if constexpr (RB > 3) { CALL(1, 3) } break;      \
  case (BASE) + 5: if constexpr (RB > 3) { CALL(2, 3) } break;      \
  case (BASE) + 6: if constexpr (RB > 4) { CALL(0, 4) } break;      \
  case (BASE) + 7: if constexpr (RB > 4) { CALL(1, 4) } break;      \
  case (BASE) + 8: if constexpr (RB > 4) { CALL(2, 4) } break;      \
  case (BASE) + 9: if constexpr (RB > 4) { CALL(3, 4) } break;

__device__ __forceinline__ uint32_t f2u(float x) { return __float_as_uint(x); }

// Write the resolved form of the sweep's operations for batch element b
// (instance inst) into shared memory, plus one zero record at the end.
// Called by the whole CTA; the caller synchronises afterwards.
template <typename R>
__device__ void resolve_ops(const SweepDev& sw, const KernelArgs& a, uint4* sres, int b, int inst,
                            int* s_meas) {
  using GT = typename GC<R>::T;
  constexpr int DT = CT<R>::DT;
  constexpr int NW = 3;
  const int nops = sw.op_end - sw.op_begin;
  const GT* coef = reinterpret_cast<const GT*>(a.coef) + (size_t)b * a.n_gates;
  const double* hc = a.hcoef + (size_t)inst * a.n_hterms;
  for (int i = threadIdx.x; i <= nops; i += blockDim.x) {
    uint4 w[3];
    w[0] = w[1] = w[2] = make_uint4(0u, 0u, 0u, 0u);
    if (i < nops) {
      const OpDev o = a.ops[sw.op_begin + i];
      const int pidx = pair_index(o.a, o.b);
      int code = RC_NOP, aux = 0, slot = 0;
      bool hop = true;
      R c = 0, s = 0, cl = 0, sl = 0, tc = 0;
      switch (o.kind) {
        case OP_GIV: {
          const GT cs = coef[o.idx];
          c = cs.x;
          s = (o.flags & OPF_INV) ? -cs.y : cs.y;
          cl = GC<R>::cl(cs);
          sl = (o.flags & OPF_INV) ? -GC<R>::sl(cs) : GC<R>::sl(cs);
          code = ((o.flags & OPF_LAM) ? RC_GIV_L : RC_GIV) + pidx;
          break;
        }
        case OP_GRADINV_HOP: {
          const GT cs = coef[o.idx];
          c = cs.x;
          s = -cs.y;
          cl = GC<R>::cl(cs);
          sl = -GC<R>::sl(cs);
          tc = (R)hc[o.idx2];
          code = RC_GRADINV + pidx;
          aux = RA_GRAD;
          slot = o.slot;
          break;
        }
        case OP_MEAS_HOP: tc = (R)hc[o.idx]; code = RC_MEAS + pidx; break;
        case OP_LAM_HOP: tc = (R)hc[o.idx]; code = RC_LAM + pidx; break;
        case OP_GRAD_HOP: tc = (R)hc[o.idx]; code = RC_GRAD + pidx; aux = RA_GRAD; slot = o.slot; break;
        default: {
          hop = false;
          const DiagOpDev& d = a.diag_ops[o.idx];
          const bool onsite = d.has_x == 0 && d.n_vb == 0 && d.n_mp == 0 && (d.has_y == 1 || d.has_y == 2);
          const bool mp1 = d.has_x == 0 && d.has_y == 0 && d.n_vb == 0 && d.n_mp == 1;
          aux = onsite ? d.has_y : (mp1 ? RA_MP : 0);
          switch (o.kind) {
            case OP_DIAG:
              code = RC_DIAG;
              aux |= ((o.flags & OPF_INV) ? RA_INV : 0) | ((o.flags & OPF_LAM) ? RA_LAM : 0);
              break;
            case OP_GRADINV_DIAG: code = RC_GRADINV_DIAG; aux |= RA_GRAD; slot = o.slot; break;
            case OP_MEAS_DIAG: code = RC_MEAS_DIAG; break;
            case OP_LAM_DIAG: code = RC_LAM_DIAG; break;
            case OP_GRAD_DIAG: code = RC_GRAD_DIAG; aux |= RA_GRAD; slot = o.slot; break;
            default: code = RC_NOP; break;
          }
          w[1] = make_uint4((uint32_t)((size_t)b * a.phase_stride + d.phase_off),
                            (uint32_t)((size_t)inst * a.real_stride + d.real_off), (uint32_t)o.idx,
                            mp1 ? (uint32_t)d.mp_p[0] | ((uint32_t)d.mp_q[0] << 8) : 0u);
          break;
        }
      }
      if (o.kind == OP_MEAS_HOP || o.kind == OP_LAM_HOP || o.kind == OP_MEAS_DIAG || o.kind == OP_LAM_DIAG)
        *s_meas = 1;
      w[0] = make_uint4((uint32_t)code | ((uint32_t)aux << 8) | ((uint32_t)slot << 16), o.sgn, o.bm_local,
                        o.bm_global);
      if (hop) {
        if constexpr (DT == 0) {
          w[1] = make_uint4(f2u((float)c), f2u((float)s), f2u((float)cl), f2u((float)sl));
          w[2] = make_uint4(f2u((float)tc), 0u, 0u, 0u);
        } else {
          w[1] = make_uint4((uint32_t)__double2loint((double)c), (uint32_t)__double2hiint((double)c),
                            (uint32_t)__double2loint((double)s), (uint32_t)__double2hiint((double)s));
          w[2] = make_uint4((uint32_t)__double2loint((double)tc), (uint32_t)__double2hiint((double)tc), 0u, 0u);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NW; ++j) sres[(size_t)NW * i + j] = w[j];
  }
}

// Global load of one amplitude of a run, with the L2 told to fetch 64 bytes
// for a miss (the default fetched the whole 128-byte line, doubling DRAM
// reads where a run is 64 bytes long and the rest of the line belongs to a
// tile processed at another time).
__device__ __forceinline__ float2 ldg_run(const float2* p) {
  float2 r;
  asm volatile("ld.global.L2::64B.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p) : "memory");
  return r;
}
__device__ __forceinline__ double2 ldg_run(const double2* p) {
  double2 r;
  asm volatile("ld.global.L2::64B.v2.f64 {%0, %1}, [%2];" : "=d"(r.x), "=d"(r.y) : "l"(p) : "memory");
  return r;
}

// ---------------------------------------------------------------------------
// the sweep kernel
// ---------------------------------------------------------------------------

// MINB = 1: up to 512 threads, one CTA per SM guaranteed (128 registers a
// thread); MINB = 4: at most 256 threads and four CTAs per SM (64
// registers), used for psi-only c64 sweeps of 256-thread tiles, where the
// extra CTAs hide the tile loads.
template <typename R, int NV, int RB, int MINB = 1, bool VP = false>
__global__ void __launch_bounds__(MINB == 1 ? 512 : 256, MINB)
sweep_kernel(const SweepDev sw, const KernelArgs a) {
  using T2 = typename CT<R>::T2;
  constexpr int DT = CT<R>::DT;
  constexpr int NE = 1 << RB;
  constexpr int NW = 3;   // resolved words per operation (see res_words)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nph = sw.phase_end - sw.phase_begin;
  const uint32_t tsize = 1u << sw.k;
  const int nbuf = nph > 1 ? NV : 0;
  T2* xb = reinterpret_cast<T2*>(smem_raw);
  T2* xl = xb + tsize;
  using AccT = typename std::conditional<DT == 0, float2, double>::type;
  const int n_rows = DT == 0 ? (int)(blockDim.x >> 5) : 1;
  const int nls = sw.n_lslot;   // local accumulator slots (see SweepDev)
  AccT* acc = reinterpret_cast<AccT*>(smem_raw + (size_t)nbuf * tsize * sizeof(T2));
  PhaseDev* phs = reinterpret_cast<PhaseDev*>(acc + n_rows * nls);
  const size_t op_off = ((size_t)(reinterpret_cast<unsigned char*>(phs + nph) - smem_raw) + 15) & ~(size_t)15;
  uint4* sres = reinterpret_cast<uint4*>(smem_raw + op_off);   // indexed by local op index
  __shared__ int8_t s_nbits[kMaxQubits];
  __shared__ int8_t s_pa[kMaxQubits];
  __shared__ int8_t s_pb[kMaxQubits];
  __shared__ int8_t s_tbits[kMaxTileBits];
  __shared__ int s_meas;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nth = blockDim.x;
  const R* rtabs = reinterpret_cast<const R*>(DT == 0 ? (const void*)a.real_tabs32 : (const void*)a.real_tabs);
  const T2* ptabs = reinterpret_cast<const T2*>(a.phase_tabs);
  const R* sdt = reinterpret_cast<const R*>(DT == 0 ? (const void*)a.prep.sd32 : (const void*)a.prep.sd);
  const uint32_t upm = (uint32_t)a.upmask;

  if (tid == 0) {   // constant indices: no local copy of the parameter block
#pragma unroll
    for (int i = 0; i < kMaxQubits; ++i) s_nbits[i] = sw.nbits[i];
#pragma unroll
    for (int i = 0; i < kMaxQubits; ++i) s_pa[i] = sw.pa[i];
#pragma unroll
    for (int i = 0; i < kMaxQubits; ++i) s_pb[i] = sw.pb[i];
#pragma unroll
    for (int i = 0; i < kMaxTileBits; ++i) s_tbits[i] = sw.tbits[i];
    s_meas = 0;
  }
  for (int i = tid; i < n_rows * nls; i += nth) acc[i] = AccT{};
  {
    const int* src = reinterpret_cast<const int*>(a.phases + sw.phase_begin);
    int* dst = reinterpret_cast<int*>(phs);
    const int nw = nph * (int)(sizeof(PhaseDev) / sizeof(int));
    for (int i = tid; i < nw; i += nth) dst[i] = src[i];
  }
  __syncthreads();

  // tiles of this sweep: all 2^(n-k) per state, or the live ones (sector);
  // each CTA takes a contiguous chunk.  (Handing out tiles round-robin,
  // which keeps the tiles in flight next to each other in HBM, measured
  // slower on GB300 for sweeps that carry psi and lam.)
  const uint32_t n_tiles = sw.sector ? (uint32_t)a.batch * sw.live : (uint32_t)a.n_tiles;
  const uint32_t chunk = (n_tiles + gridDim.x - 1) / gridDim.x;
  const uint32_t t0 = blockIdx.x * chunk;
  const uint32_t t1 = min(t0 + chunk, n_tiles);
  const uint32_t tl_mask = (uint32_t)((1ull << sw.n_nontile) - 1ull);
  int cur_b = -1;
  T2 v[NE];
  T2 l[NE];
  // Sector tiles: thread 0 unranks the CTA's first live tile and then steps
  // the two patterns (part a fastest), one tile ahead, into a double buffer
  // in shared memory (so that they hold no registers during the operations);
  // the barrier at the top of each tile publishes them.
  __shared__ uint32_t s_tile[2][3];   // pattern a, pattern b, batch element
  if (sw.sector && t0 < t1 && tid == 0) {
    const uint32_t b0 = t0 / sw.live;
    const uint32_t j = t0 - b0 * sw.live;
    const uint32_t jb = j / sw.cnt_a, ja = j - jb * sw.cnt_a;
    s_tile[0][0] = unrank_bits(ja, sw.na, sw.lo_a);
    s_tile[0][1] = unrank_bits(jb, sw.nb, sw.lo_b);
    s_tile[0][2] = b0;
  }

  for (uint32_t tau = t0; tau < t1; ++tau) {
    // batch element and non-tile bits of the tile (state-local indices fit
    // in 32 bits, n <= 32)
    int b;
    uint32_t sbase;
    if (sw.sector) {
      __syncthreads();
      const uint32_t* cur = s_tile[(tau - t0) & 1u];
      uint32_t pat_a = cur[0], pat_b = cur[1];
      b = (int)cur[2];
      sbase = deposit_set(pat_a, s_pa) | deposit_set(pat_b, s_pb);
      if (tid == 0 && tau + 1 < t1) {
        uint32_t bn = (uint32_t)b;
        if (!next_pattern(pat_a, sw.na, sw.hi_a)) {
          pat_a = (1u << sw.lo_a) - 1u;
          if (!next_pattern(pat_b, sw.nb, sw.hi_b)) {
            pat_b = (1u << sw.lo_b) - 1u;
            ++bn;
          }
        }
        uint32_t* nxt = s_tile[(tau + 1 - t0) & 1u];
        nxt[0] = pat_a;
        nxt[1] = pat_b;
        nxt[2] = bn;
      }
    } else {
      b = (int)(tau >> sw.n_nontile);
      sbase = deposit_bits(tau & tl_mask, s_nbits, sw.n_nontile);
    }
    const int inst = b % a.n_inst;
    if (b != cur_b) {
      if (cur_b >= 0) {
        __syncthreads();
        for (int i = tid; i < nls; i += nth) {
          double x = 0.0;
          for (int w = 0; w < n_rows; ++w) {
            x += row_value(acc[w * nls + i]);
            acc[w * nls + i] = AccT{};
          }
          if (x != 0.0) atomicAdd(&a.acc[(size_t)cur_b * a.n_slots + a.slot_map[sw.lslot_off + i]], x);
        }
        __syncthreads();
      }
      resolve_ops<R>(sw, a, sres, b, inst, &s_meas);
      __syncthreads();
      cur_b = b;
    }
    R eacc = 0, nacc = 0, racc = 0;
    int rslot = -1;
    uint32_t base = 0;      // thread's tile-local base index in this phase
    uint32_t sbw = 0;       // its swizzled exchange index
    uint32_t gob = 0;       // its state-index bits
    // The per-slot state-index bits (so) and exchange indices (ss) of a
    // phase are read from shared memory where they are used, so that they
    // hold no registers during the operations.
    // operation words, loaded one operation ahead (the records of the
    // sweep's phases are consecutive; a zero record follows the last)
    // (c128: the third word, tc, is read when the operation runs)
    uint4 n0 = sres[0], n1 = sres[1];
    const uint4* onext = sres + NW;

    for (int pi = 0; pi < nph; ++pi) {
      const PhaseDev& ph = phs[pi];
      if (pi > 0) {  // exchange through shared memory: old mapping out
        uint32_t ss[RB];
#pragma unroll
        for (int j = 0; j < RB; ++j) ss[j] = phs[pi - 1].ss[j];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < NE; ++e) {
          const uint32_t loc = sbw ^ comb<RB>(ss, e);
          xb[loc] = v[e];
          if (NV == 2) xl[loc] = l[e];
        }
        __syncthreads();
      }
      base = ph.bl[lane] | ph.bw[warp];
      gob = ph.gl[lane] | ph.gw[warp];
      sbw = swz(base, DT);
      if (pi == 0) {  // global load (the run bits are on lanes)
        const uint64_t gbase = ((uint64_t)b << a.n) | sbase;
        uint32_t so[RB];
#pragma unroll
        for (int j = 0; j < RB; ++j) so[j] = ph.so[j];
        const T2* src = reinterpret_cast<const T2*>((sw.flags & SW_CKPT_READ) ? a.ckpt : a.psi);
#pragma unroll
        for (int e = 0; e < NE; ++e) {
          const uint32_t off = gob | comb<RB>(so, e);
          if (sw.flags & SW_PREP) {
            v[e] = mk<T2, R>(prep_amp<R>(a.prep, sdt, sbase | off, inst), (R)0);
          } else {
            v[e] = ldg_run(src + gbase + off);
          }
          if (NV == 2) {
            if (sw.flags & SW_READ_LAM) l[e] = ldg_run(reinterpret_cast<const T2*>(a.lam) + gbase + off);
            else l[e] = mk<T2, R>((R)0, (R)0);
          }
        }
      } else {        // new mapping in
        uint32_t ss[RB];
#pragma unroll
        for (int j = 0; j < RB; ++j) ss[j] = ph.ss[j];
#pragma unroll
        for (int e = 0; e < NE; ++e) {
          const uint32_t loc = sbw ^ comb<RB>(ss, e);
          v[e] = xb[loc];
          if (NV == 2) l[e] = xl[loc];
        }
      }

      const int nops_ph = ph.op_end - ph.op_begin;
      for (int oi = 0; oi < nops_ph; ++oi) {
        const uint4 w0 = n0, w1 = n1;
        uint4 w2;
        if constexpr (NW == 3) w2 = onext[2 - NW];
        n0 = onext[0];
        n1 = onext[1];
        onext += NW;
        const int code = (int)(w0.x & 255u), aux = (int)((w0.x >> 8) & 255u);
        if (aux & RA_GRAD) {
          const int slot = (int)(w0.x >> 16);
          if (slot != rslot) {
            if (rslot >= 0) cta_add(acc, nls, rslot, racc);
            racc = 0;
            rslot = slot;
          }
        }
        // sign mask of the pairs: slot part from the plan, the rest from
        // the thread's other tile bits and the tile's non-tile bits
        const int tpar = (__popc(base & w0.z) + __popc(sbase & w0.w)) & 1;
        const uint32_t sm = w0.y ^ (tpar ? 0xffffffffu : 0u);
        R c, s, cl, sl, tc;
        if constexpr (DT == 0) {
          c = __uint_as_float(w1.x);
          s = __uint_as_float(w1.y);
          cl = __uint_as_float(w1.z);
          sl = __uint_as_float(w1.w);
          tc = __uint_as_float(w2.x);
        } else {
          c = __hiloint2double((int)w1.y, (int)w1.x);
          s = __hiloint2double((int)w1.w, (int)w1.z);
          cl = sl = 0.0;
          tc = __hiloint2double((int)w2.y, (int)w2.x);
        }
#define HUB_GIV1(A, B) pair_giv<A, B, !VP>(v, c, s, cl, sl, sm);
#define HUB_GIV2(A, B)                                  \
  pair_giv<A, B, !VP>(v, c, s, cl, sl, sm);             \
  if constexpr (NV == 2) pair_giv<A, B, !VP>(l, c, s, cl, sl, sm);
#define HUB_GI(A, B) \
  if constexpr (NV == 2) racc += (R)2 * pair_gradinv<A, B, !VP>(v, l, c, s, cl, sl, tc, sm);
#define HUB_M0(A, B) eacc += (R)2 * pair_hop<A, B, 0>(v, l, tc, sm);
#define HUB_M1(A, B) \
  if constexpr (NV == 2) eacc += (R)2 * pair_hop<A, B, 1>(v, l, tc, sm);
#define HUB_M2(A, B) \
  if constexpr (NV == 2) racc += (R)2 * pair_hop<A, B, 2>(v, l, tc, sm);
        switch (code) {
          HUB_PAIRS(RC_GIV, HUB_GIV1)
          HUB_PAIRS(RC_GIV_L, HUB_GIV2)
          HUB_PAIRS(RC_GRADINV, HUB_GI)
          HUB_PAIRS(RC_MEAS, HUB_M0)
          HUB_PAIRS(RC_LAM, HUB_M1)
          HUB_PAIRS(RC_GRAD, HUB_M2)
          case RC_DIAG: {
            const T2* ptab = ptabs + w1.x;
            uint32_t so[RB];
#pragma unroll
            for (int j = 0; j < RB; ++j) so[j] = ph.so[j];
            const bool inv = aux & RA_INV;
            const bool dol = (NV == 2) && (aux & RA_LAM);
            const uint32_t xb0 = sbase | gob;
            const int ny = aux & RA_NY;
            if (VP && (aux & RA_MP)) {
              // one controlled phase (NP / EP gate): exp(i phi) where both modes are occupied
              T2 pv = ptab[2048];
              if (inv) pv.y = -pv.y;
              const uint32_t mp = w1.w & 255u, mq = (w1.w >> 8) & 255u;
#pragma unroll
              for (int e = 0; e < NE; ++e) {
                const uint32_t x = xb0 | comb<RB>(so, e);
                if ((x >> mp) & (x >> mq) & 1u) {
                  v[e] = cmul(v[e], pv);
                  if (dol) l[e] = cmul(l[e], pv);
                }
              }
              break;
            }
            if (ny) {
              // on-site factor only: phase of the double-occupancy pattern
              const T2* ty = ptab + 1024;
#pragma unroll
              for (int e = 0; e < NE; ++e) {
                const uint32_t x = xb0 | comb<RB>(so, e);
                const uint32_t y = x & (x >> a.s) & upm;
                T2 p = ty[y & 255u];
                if (ny == 2) p = cmul(p, ty[256 + ((y >> 8) & 255u)]);
                if (inv) p.y = -p.y;
                v[e] = cmul(v[e], p);
                if (dol) l[e] = cmul(l[e], p);
              }
              break;
            }
            const DiagOpDev& d = a.diag_ops[w1.z];
#pragma unroll
            for (int e = 0; e < NE; ++e) {
              T2 p = diag_phase<T2, VP>(d, ptab, xb0 | comb<RB>(so, e), a.s, upm);
              if (inv) p.y = -p.y;
              v[e] = cmul(v[e], p);
              if (dol) l[e] = cmul(l[e], p);
            }
            break;
          }
          case RC_GRADINV_DIAG: {
            if constexpr (NV == 2) {
              const T2* ptab = ptabs + w1.x;
            uint32_t so[RB];
#pragma unroll
            for (int j = 0; j < RB; ++j) so[j] = ph.so[j];
              const R* rtab = rtabs + w1.y;
              const int ny = aux & RA_NY;
              const uint32_t xb0 = sbase | gob;
              R pe = 0;
              if (VP && (aux & RA_MP)) {
                const R dv0 = rtab[2048];
                T2 pv = ptab[2048];
                pv.y = -pv.y;
                const uint32_t mp = w1.w & 255u, mq = (w1.w >> 8) & 255u;
#pragma unroll
                for (int e = 0; e < NE; ++e) {
                  const uint32_t x = xb0 | comb<RB>(so, e);
                  if ((x >> mp) & (x >> mq) & 1u) {
                    pe += dv0 * (l[e].x * v[e].y - l[e].y * v[e].x);
                    v[e] = cmul(v[e], pv);
                    l[e] = cmul(l[e], pv);
                  }
                }
                racc += (R)2 * pe;
                break;
              }
              const DiagOpDev* dp = ny ? nullptr : &a.diag_ops[w1.z];
#pragma unroll
              for (int e = 0; e < NE; ++e) {
                const uint32_t x = xb0 | comb<RB>(so, e);
                R dv;
                T2 p;
                if (ny) {
                  const uint32_t y = x & (x >> a.s) & upm;
                  dv = rtab[1024 + (y & 255u)];
                  p = ptab[1024 + (y & 255u)];
                  if (ny == 2) {
                    dv += rtab[1280 + ((y >> 8) & 255u)];
                    p = cmul(p, ptab[1280 + ((y >> 8) & 255u)]);
                  }
                } else {
                  dv = diag_real<R, VP>(*dp, rtab, x, a.s, upm);
                  p = diag_phase<T2, VP>(*dp, ptab, x, a.s, upm);
                }
                pe += dv * (l[e].x * v[e].y - l[e].y * v[e].x);
                p.y = -p.y;
                v[e] = cmul(v[e], p);
                l[e] = cmul(l[e], p);
              }
              racc += (R)2 * pe;
            }
            break;
          }
          case RC_MEAS_DIAG:
          case RC_LAM_DIAG:
          case RC_GRAD_DIAG: {
            const R* rtab = rtabs + w1.y;
            uint32_t so[RB];
#pragma unroll
            for (int j = 0; j < RB; ++j) so[j] = ph.so[j];
            const int ny = aux & RA_NY;
            R pe = 0, pn = 0;
            const uint32_t xb0 = sbase | gob;
            if (VP && (aux & RA_MP) && code == RC_GRAD_DIAG) {
              if constexpr (NV == 2) {
                const R dv0 = rtab[2048];
                const uint32_t mp = w1.w & 255u, mq = (w1.w >> 8) & 255u;
#pragma unroll
                for (int e = 0; e < NE; ++e) {
                  const uint32_t x = xb0 | comb<RB>(so, e);
                  if ((x >> mp) & (x >> mq) & 1u) pe += dv0 * (l[e].x * v[e].y - l[e].y * v[e].x);
                }
                racc += (R)2 * pe;
              }
              break;
            }
            const DiagOpDev* dp = ny ? nullptr : &a.diag_ops[w1.z];
#pragma unroll
            for (int e = 0; e < NE; ++e) {
              const uint32_t x = xb0 | comb<RB>(so, e);
              R dv;
              if (ny) {   // on-site terms only
                const uint32_t y = x & (x >> a.s) & upm;
                dv = rtab[1024 + (y & 255u)];
                if (ny == 2) dv += rtab[1280 + ((y >> 8) & 255u)];
              } else {
                dv = diag_real<R, VP>(*dp, rtab, x, a.s, upm);
              }
              const T2 u = v[e];
              if (code == RC_GRAD_DIAG) {
                if (NV == 2) pe += dv * (l[e].x * u.y - l[e].y * u.x);
              } else {
                const R m2 = u.x * u.x + u.y * u.y;
                pe += dv * m2;
                pn += m2;
                if (NV == 2 && code == RC_LAM_DIAG) {
                  l[e].x += dv * u.x;
                  l[e].y += dv * u.y;
                }
              }
            }
            if (code == RC_GRAD_DIAG) racc += (R)2 * pe;
            else { eacc += pe; nacc += pn; }
            break;
          }
          default: break;
        }
#undef HUB_GIV1
#undef HUB_GIV2
#undef HUB_GI
#undef HUB_M0
#undef HUB_M1
#undef HUB_M2
      }
    }
    if (rslot >= 0) cta_add(acc, nls, rslot, racc);
    if (s_meas) {
      cta_add(acc, nls, sw.lslot_E, eacc);
      cta_add(acc, nls, sw.lslot_N, nacc);
    }

    // ---- store from registers (the last phase has the run bits on lanes) ----
    const bool wp = sw.flags & SW_WRITE_PSI, wc = sw.flags & SW_CKPT_WRITE;
    const bool wl = (NV == 2) && (sw.flags & SW_WRITE_LAM);
    if (wp || wc || wl) {
      const uint64_t gbase = ((uint64_t)b << a.n) | sbase;
      uint32_t so[RB];
#pragma unroll
      for (int j = 0; j < RB; ++j) so[j] = phs[nph - 1].so[j];
#pragma unroll
      for (int e = 0; e < NE; ++e) {
        const uint64_t g = gbase + (gob | comb<RB>(so, e));
        if (wp) reinterpret_cast<T2*>(a.psi)[g] = v[e];
        if (wc) reinterpret_cast<T2*>(a.ckpt)[g] = v[e];
        if (wl) reinterpret_cast<T2*>(a.lam)[g] = l[e];
      }
    }
  }
  __syncthreads();
  if (cur_b >= 0) {
    for (int i = tid; i < nls; i += nth) {
      double x = 0.0;
      for (int w = 0; w < n_rows; ++w) x += row_value(acc[w * nls + i]);
      if (x != 0.0) atomicAdd(&a.acc[(size_t)cur_b * a.n_slots + a.slot_map[sw.lslot_off + i]], x);
    }
  }
}

}  // namespace hubsv
