// Small kernels of the Hubbard VQE statevector engine (coefficient and
// phase tables, accumulator reset and read-out) and the launchers.
#include <algorithm>

#include "hubsv_internal.h"

namespace hubsv {

template <typename R> struct CT;
template <> struct CT<float> { using T2 = float2; using G = float4; };
template <> struct CT<double> { using T2 = double2; using G = double2; };

// Givens coefficients (c, s): complex128 as doubles; complex64 as FP32 pairs
// {c_hi, s_hi, c_lo, s_lo} with c_hi = fl32(c), c_lo = fl32(c - c_hi), so
// that the rotation angle is exact to ~1e-14 (see GC in the sweep header).
template <typename R>
__device__ __forceinline__ typename CT<R>::G giv_coef(double c, double s);
template <>
__device__ __forceinline__ double2 giv_coef<double>(double c, double s) {
  return make_double2(c, s);
}
template <>
__device__ __forceinline__ float4 giv_coef<float>(double c, double s) {
  const float ch = (float)c, sh = (float)s;
  return make_float4(ch, sh, (float)(c - (double)ch), (float)(s - (double)sh));
}

// ---------------------------------------------------------------------------
// coefficient and phase tables (one thread per entry, FP64 trig)
// ---------------------------------------------------------------------------

// Round the unit complex number (c, s) of a diagonal phase to the
// precision of R.  For FP32 the pair is chosen among the neighbouring
// representable values as the one closest to the unit circle, so a phase
// with these entries changes norms by ~1e-8 instead of ~1e-7 (this drift
// would otherwise add up over the forward factors and their inverses in
// the adjoint pass).
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

// Batch elements along y, entries along x.  Only the phase-table entries
// in tab_live (those some kernel reads: the byte tables a diagonal operator
// uses) are made.
template <typename R>
__global__ void coef_kernel(const double* __restrict__ theta, int P,
                            const int32_t* __restrict__ gate_param,
                            const double* __restrict__ gate_t, int n_gates,
                            typename CT<R>::G* __restrict__ coef,
                            const int32_t* __restrict__ tab_param,
                            const double* __restrict__ tab_val, int n_tab,
                            const int32_t* __restrict__ tab_live, int n_live,
                            typename CT<R>::T2* __restrict__ phase, int64_t batch, int n_inst) {
  const int per = n_gates + n_live;
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const int inst = (int)(b % n_inst);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < per; j += gridDim.x * blockDim.x) {
      if (j < n_gates) {
        const double al = theta[b * P + gate_param[j]] * gate_t[(int64_t)inst * n_gates + j];
        double s, c;
        sincos(al, &s, &c);
        coef[b * n_gates + j] = giv_coef<R>(c, s);
      } else {
        const int e = tab_live[j - n_gates];
        const int pp = tab_param[e];
        const double th = pp >= 0 ? theta[b * P + pp] : 0.0;
        const double al = -th * tab_val[(int64_t)inst * n_tab + e];
        double s, c;
        sincos(al, &s, &c);
        phase[b * n_tab + e] = unit_round<R>(c, s);
      }
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

const void* sweep_ptr_f1(int r);
const void* sweep_ptr_f2(int r);
const void* sweep_ptr_d1(int r);
const void* sweep_ptr_d2(int r);
const void* sweep_ptr_f1_narrow(int r);
const void* sweep_ptr_fv(int nv, int r, int threads);
const void* sweep_ptr_dv(int nv, int r, int threads);

namespace {
int g_sm_count = 0;

// vp: the sweep has uniform V terms (SW_VPOP); the popcount variant is
// taken where one is compiled, else the plain kernel (bond by bond).
const void* kernel_for(int dtype, int nv, int r, int threads, bool vp) {
  if (r < 1 || r > max_reg_bits(dtype, nv)) return nullptr;
  if (vp) {
    if (const void* f = dtype == 0 ? sweep_ptr_fv(nv, r, threads) : sweep_ptr_dv(nv, r, threads)) return f;
  }
  if (dtype == 0 && nv == 1 && threads <= 256) {
    if (const void* f = sweep_ptr_f1_narrow(r)) return f;
  }
  if (dtype == 0) return nv == 2 ? sweep_ptr_f2(r) : sweep_ptr_f1(r);
  return nv == 2 ? sweep_ptr_d2(r) : sweep_ptr_d1(r);
}
}  // namespace

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

cudaError_t sweep_set_smem(int dtype, int nv, int r, int threads, bool vp, size_t smem) {
  const void* f = kernel_for(dtype, nv, r, threads, vp);
  if (!f) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int sweep_regs(int dtype, int nv, int r, int threads, bool vp) {
  const void* f = kernel_for(dtype, nv, r, threads, vp);
  cudaFuncAttributes at;
  if (!f || cudaFuncGetAttributes(&at, f) != cudaSuccess) return 0;
  return at.numRegs;
}

cudaError_t launch_sweep(int dtype, const SweepDev& sw, const KernelArgs& a, int grid, size_t smem,
                         cudaStream_t st) {
  const int nv = (sw.flags & SW_HAS_LAM) ? 2 : 1;
  const int threads = 32 << sw.w;
  const void* f = kernel_for(dtype, nv, sw.r, threads, (sw.flags & SW_VPOP) != 0);
  if (!f) return cudaErrorInvalidValue;
  SweepDev swc = sw;
  KernelArgs ac = a;
  void* args[] = {(void*)&swc, (void*)&ac};
  return cudaLaunchKernel(f, dim3(grid), dim3(threads), args, smem, st);
}

cudaError_t launch_coef(int dtype, const double* theta, int P, const int32_t* gate_param,
                        const double* gate_t, int n_gates, void* coef,
                        const int32_t* tab_param, const double* tab_val, int n_tab,
                        const int32_t* tab_live, int n_live, void* phase_tabs, int64_t batch,
                        int n_inst, cudaStream_t st) {
  const int per = n_gates + n_live;
  if (per == 0 || batch <= 0) return cudaSuccess;
  const int gx = std::min((per + 255) / 256, 64);
  const int gy = (int)std::min<int64_t>(batch, std::max(1, 8192 / gx));
  const dim3 grid(gx, gy);
  if (dtype == 0)
    coef_kernel<float><<<grid, 256, 0, st>>>(theta, P, gate_param, gate_t, n_gates,
                                             (float4*)coef, tab_param, tab_val, n_tab, tab_live,
                                             n_live, (float2*)phase_tabs, batch, n_inst);
  else
    coef_kernel<double><<<grid, 256, 0, st>>>(theta, P, gate_param, gate_t, n_gates,
                                              (double2*)coef, tab_param, tab_val, n_tab, tab_live,
                                              n_live, (double2*)phase_tabs, batch, n_inst);
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
