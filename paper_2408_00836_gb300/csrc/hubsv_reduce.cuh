// Block reductions shared by the on-chip and row kernels (device code).
#pragma once

#include "hubsv_sweep.cuh"

namespace hubsv {

// The complex64 kernels reduce in FP32 and keep their running totals as
// float pairs (two_sum, ff_add, warp_sum_f from the sweep kernel's header);
// the complex128 kernels reduce in FP64.

// Sum of float pairs over the warp, into lane 0's (h, l).
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

}  // namespace hubsv
