// Block reductions shared by the on-chip and row kernels (device code).
#pragma once

#include "hubsv_sweep.cuh"

namespace hubsv {

// The complex64 kernels reduce in FP32 and keep their running totals as
// float pairs (two_sum, ff_add, warp_sum_ff from the sweep kernel's header);
// the complex128 kernels reduce in FP64.

// Running totals of one thread (R = float: float pairs; double: FP64).
template <typename R> struct Tot;
template <> struct Tot<float> {
  float h = 0.f, l = 0.f;
  __device__ __forceinline__ void add(float v) { ff_add(h, l, v); }
};
template <> struct Tot<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
};

// Per-warp accumulator rows: row w, slot i at acc[w * n_slots + i], float
// pairs (c64) or doubles (c128); lane 0 of warp w alone writes row w, so no
// atomics are needed, and the rows are summed in FP64 when they are read out.
// Adds the warp's sum of v to its row's slot (every lane calls).
__device__ __forceinline__ void row_add(float2* acc, int n_slots, int slot, float v) {
  v = warp_sum_f(v);
  if ((threadIdx.x & 31) == 0) {
    float2& t = acc[(threadIdx.x >> 5) * n_slots + slot];
    ff_add(t.x, t.y, v);
  }
}
__device__ __forceinline__ void row_add(double* acc, int n_slots, int slot, double v) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) acc[(threadIdx.x >> 5) * n_slots + slot] += v;
}
// Adds the warp's sum of the lanes' running totals to its row (every lane calls).
__device__ __forceinline__ void row_add_tot(float2* acc, int n_slots, int slot, Tot<float> t) {
  warp_sum_ff(t.h, t.l);
  if ((threadIdx.x & 31) == 0) {
    float2& r = acc[(threadIdx.x >> 5) * n_slots + slot];
    ff_add(r.x, r.y, t.h);
    ff_add(r.x, r.y, t.l);
  }
}
__device__ __forceinline__ void row_add_tot(double* acc, int n_slots, int slot, Tot<double> t) {
  row_add(acc, n_slots, slot, t.v);
}

// Diagonal value (real, or phase) of an element: on-site terms only (ny =
// 1 or 2 byte tables of the double-occupancy pattern), or the general form.
template <typename R, typename T2>
struct DiagVal {
  const DiagOpDev* d;
  int ny;
  __device__ __forceinline__ R real(const R* rtab, uint32_t x, int s, uint32_t upm) const {
    if (ny) {
      const uint32_t y = x & (x >> s) & upm;
      R v = rtab[1024 + (y & 255u)];
      if (ny == 2) v += rtab[1280 + ((y >> 8) & 255u)];
      return v;
    }
    return diag_real<R, true>(*d, rtab, x, s, upm);
  }
  __device__ __forceinline__ T2 phase(const T2* ptab, uint32_t x, int s, uint32_t upm) const {
    if (ny) {
      const uint32_t y = x & (x >> s) & upm;
      T2 p = ptab[1024 + (y & 255u)];
      if (ny == 2) p = cmul(p, ptab[1280 + ((y >> 8) & 255u)]);
      return p;
    }
    return diag_phase<T2, true>(*d, ptab, x, s, upm);
  }
};

}  // namespace hubsv
