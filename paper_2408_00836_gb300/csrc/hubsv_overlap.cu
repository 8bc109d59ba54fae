// Overlap loss, fidelity and spin correlations (device side).
//
// The overlap loss of Eq. 5, f = log10(1 - F) with F = |<psi(theta)|
// psi_ref>|^2, and its gradient run on the dense sweeps: the forward circuit
// leaves psi_K in psi; overlap_kernel reduces a = <psi_ref|psi_K>;
// scale_ref_kernel writes lam_K = a psi_ref, the projector
// |psi_ref><psi_ref| applied to psi_K; the backward sweeps of the adjoint
// recursion (Sec. 2.1) then accumulate dF/dtheta_k = 2 Im <lam_k|G_k|psi_k>
// exactly as they accumulate the energy gradient from lam_K = H psi_K; and
// overlap_finalize_kernel forms F, f and df/dtheta = -dF/dtheta / ((1 - F)
// ln 10).
//
// The spin correlation C_ij = <S^z_i S^z_j> - <S^z_i><S^z_j> (Sec. 3) of a
// state comes from the occupation correlations M_kl = <n_k n_l> of all mode
// pairs: occ_corr_kernel walks runs of 2^8 contiguous amplitudes (the high
// index bits fixed within a run), accumulates the run's weight and its
// low-bit moments in registers, and adds them to a per-CTA matrix in shared
// memory through the run's high bits; spin_corr_kernel combines M into C.
#include <algorithm>

#include "hubsv_internal.h"

namespace hubsv {

namespace {

template <typename R> struct OT;
template <> struct OT<float> { using T2 = float2; };
template <> struct OT<double> { using T2 = double2; };

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// a[b] += sum_x conj(ref[b % ref_batch][x]) psi[b][x]; blocks along x, batch
// along y.  Products in the working precision, partial sums per thread in
// FP64 (one FP64 add per amplitude and component), one FP64 atomic per
// block and component.
template <typename R>
__global__ void __launch_bounds__(256) overlap_kernel(const typename OT<R>::T2* __restrict__ psi,
                                                      const typename OT<R>::T2* __restrict__ ref,
                                                      int64_t ref_batch, uint64_t len, int64_t batch,
                                                      double* __restrict__ a) {
  __shared__ double sre[8], sim[8];
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const typename OT<R>::T2* p = psi + (uint64_t)b * len;
    const typename OT<R>::T2* r = ref + (uint64_t)(b % ref_batch) * len;
    double re = 0.0, im = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (uint64_t)gridDim.x * blockDim.x) {
      const typename OT<R>::T2 u = p[i], w = r[i];
      re += (double)(w.x * u.x + w.y * u.y);
      im += (double)(w.x * u.y - w.y * u.x);
    }
    re = warp_sum_d(re);
    im = warp_sum_d(im);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sre[wid] = re; sim[wid] = im; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tr = 0.0, ti = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tr += sre[w]; ti += sim[w]; }
      atomicAdd(&a[2 * b], tr);
      atomicAdd(&a[2 * b + 1], ti);
    }
    __syncthreads();
  }
}

// lam[b][x] = a_b ref[b % ref_batch][x].
template <typename R>
__global__ void __launch_bounds__(256) scale_ref_kernel(const typename OT<R>::T2* __restrict__ ref,
                                                        int64_t ref_batch, typename OT<R>::T2* __restrict__ lam,
                                                        uint64_t len, int64_t batch,
                                                        const double* __restrict__ a) {
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const R ar = (R)a[2 * b], ai = (R)a[2 * b + 1];
    const typename OT<R>::T2* r = ref + (uint64_t)(b % ref_batch) * len;
    typename OT<R>::T2* l = lam + (uint64_t)b * len;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (uint64_t)gridDim.x * blockDim.x) {
      const typename OT<R>::T2 w = r[i];
      typename OT<R>::T2 o;
      o.x = ar * w.x - ai * w.y;
      o.y = ar * w.y + ai * w.x;
      l[i] = o;
    }
  }
}

__global__ void overlap_finalize_kernel(const double* __restrict__ acc, int n_slots, int P,
                                        const double* __restrict__ a, double* __restrict__ F,
                                        double* __restrict__ f, double* __restrict__ grad, int64_t batch) {
  const int64_t total = batch * (P + 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / (P + 1);
    const int j = (int)(i - b * (P + 1));
    const double Fb = a[2 * b] * a[2 * b] + a[2 * b + 1] * a[2 * b + 1];
    if (j == P) {
      if (F) F[b] = Fb;
      if (f) f[b] = log10(1.0 - Fb);
    } else if (grad) {
      grad[b * P + j] = -acc[b * n_slots + j] / ((1.0 - Fb) * 2.302585092994045684);
    }
  }
}

// The overlap on the row engine's sector matrices: mat[b][r][c] is the
// amplitude of the full index x = xrow[r] | xin[c] (rows and columns in
// either orientation).  a[b] += sum conj(ref[b % ref_batch][x]) mat[b][r][c]
// (blocks along the elements, batch along y; the reference is read at the
// sector's indices only), and lam[b][r][c] = a_b ref[b % ref_batch][x].
template <typename R>
__global__ void __launch_bounds__(256) sector_overlap_kernel(const typename OT<R>::T2* __restrict__ mat,
                                                             const uint32_t* __restrict__ xrow,
                                                             const uint32_t* __restrict__ xin, int n_rows,
                                                             int row_len, const typename OT<R>::T2* __restrict__ ref,
                                                             int64_t ref_batch, int n, int64_t batch,
                                                             double* __restrict__ a) {
  __shared__ double sre[8], sim[8];
  const uint64_t C = (uint64_t)n_rows * (uint64_t)row_len;
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const typename OT<R>::T2* p = mat + (uint64_t)b * C;
    const typename OT<R>::T2* r = ref + ((uint64_t)(b % ref_batch) << n);
    double re = 0.0, im = 0.0;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < C; e += (uint64_t)gridDim.x * blockDim.x) {
      const uint64_t row = e / (uint64_t)row_len;
      const uint32_t x = __ldg(xrow + row) | __ldg(xin + (e - row * (uint64_t)row_len));
      const typename OT<R>::T2 u = p[e], w = r[x];
      re += (double)(w.x * u.x + w.y * u.y);
      im += (double)(w.x * u.y - w.y * u.x);
    }
    re = warp_sum_d(re);
    im = warp_sum_d(im);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sre[wid] = re; sim[wid] = im; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tr = 0.0, ti = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tr += sre[w]; ti += sim[w]; }
      atomicAdd(&a[2 * b], tr);
      atomicAdd(&a[2 * b + 1], ti);
    }
    __syncthreads();
  }
}

template <typename R>
__global__ void __launch_bounds__(256) sector_scale_ref_kernel(const typename OT<R>::T2* __restrict__ ref,
                                                               int64_t ref_batch, const uint32_t* __restrict__ xrow,
                                                               const uint32_t* __restrict__ xin, int n_rows,
                                                               int row_len, int n, int64_t batch,
                                                               const double* __restrict__ a,
                                                               typename OT<R>::T2* __restrict__ lam) {
  const uint64_t C = (uint64_t)n_rows * (uint64_t)row_len;
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const typename OT<R>::T2* r = ref + ((uint64_t)(b % ref_batch) << n);
    const R ar = (R)a[2 * b], ai = (R)a[2 * b + 1];
    typename OT<R>::T2* l = lam + (uint64_t)b * C;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < C; e += (uint64_t)gridDim.x * blockDim.x) {
      const uint64_t row = e / (uint64_t)row_len;
      const uint32_t x = __ldg(xrow + row) | __ldg(xin + (e - row * (uint64_t)row_len));
      const typename OT<R>::T2 w = r[x];
      typename OT<R>::T2 v;
      v.x = ar * w.x - ai * w.y;
      v.y = ar * w.y + ai * w.x;
      l[e] = v;
    }
  }
}

// M[b][k][l] (k <= l) += sum_x |psi[b][x]|^2 n_k(x) n_l(x).  Runs of 2^KR
// amplitudes share their high bits h; per run the thread keeps s = sum p,
// m_j = sum p bit_j and q_jk = sum p bit_j bit_k over the KR low bits in
// FP64 registers, then adds s to M[a][b] for set high bits a <= b, m_j to
// M[a][j] for set high bits a, and m, q to the low block.
constexpr int KR = 8;

template <typename R>
__global__ void __launch_bounds__(128) occ_corr_kernel(const typename OT<R>::T2* __restrict__ psi, int n,
                                                       int64_t batch, double* __restrict__ M) {
  __shared__ double sm[kMaxQubits * kMaxQubits];
  const int kr = n < KR ? n : KR;
  const uint64_t len = 1ull << n;
  const uint64_t runs = len >> kr;
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) sm[i] = 0.0;
    __syncthreads();
    const typename OT<R>::T2* p = psi + (uint64_t)b * len;
    for (uint64_t run = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; run < runs;
         run += (uint64_t)gridDim.x * blockDim.x) {
      double s = 0.0, m[KR], q[KR * (KR - 1) / 2];
#pragma unroll
      for (int j = 0; j < KR; ++j) m[j] = 0.0;
#pragma unroll
      for (int j = 0; j < KR * (KR - 1) / 2; ++j) q[j] = 0.0;
      const typename OT<R>::T2* pr = p + (run << kr);
      for (int l = 0; l < (1 << kr); ++l) {
        const typename OT<R>::T2 u = pr[l];
        const double w = (double)u.x * (double)u.x + (double)u.y * (double)u.y;
        s += w;
        int t = 0;
#pragma unroll
        for (int j = 0; j < KR; ++j) {
          const double wj = ((l >> j) & 1) ? w : 0.0;
          m[j] += wj;
#pragma unroll
          for (int k = j + 1; k < KR; ++k) q[t++] += ((l >> k) & 1) ? wj : 0.0;
        }
      }
      if (s == 0.0) continue;
      const uint64_t h = run << kr;   // the run's high bits at their index positions
      int t = 0;
#pragma unroll
      for (int j = 0; j < KR; ++j) {
        if (j < kr) atomicAdd(&sm[j * n + j], m[j]);
#pragma unroll
        for (int k = j + 1; k < KR; ++k, ++t)
          if (k < kr) atomicAdd(&sm[j * n + k], q[t]);
      }
      for (uint64_t ha = h; ha; ha &= ha - 1) {
        const int a = __ffsll((long long)ha) - 1;
        atomicAdd(&sm[a * n + a], s);
#pragma unroll
        for (int j = 0; j < KR; ++j)
          if (j < kr) atomicAdd(&sm[j * n + a], m[j]);
        for (uint64_t hb = ha & (ha - 1); hb; hb &= hb - 1) atomicAdd(&sm[a * n + (__ffsll((long long)hb) - 1)], s);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n * n; i += blockDim.x)
      if (sm[i] != 0.0) atomicAdd(&M[(uint64_t)b * n * n + i], sm[i]);
    __syncthreads();
  }
}

// The same M for n >= KW, one warp per run of 2^KW = 1024 contiguous
// amplitudes: lane = index bits 0-4, register slot r = bits 5-9, so each
// load instruction of the warp reads 32 consecutive amplitudes.  Per lane,
// the sums over its 32 slots whose slot bits are set are unrolled (the bit
// pattern of r is a constant), in the working precision.  Moments that involve only the
// low 10 bits are kept per lane across all of the warp's runs and reduced
// once; per run, the weight S and the ten low-bit moments m_j are reduced
// over the warp and added, by the lanes in parallel, to M[j][a] and
// M[a][b] for the run's set high bits a < b.
constexpr int KW = 10;

__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename R>
__global__ void __launch_bounds__(256) occ_corr_warp_kernel(const typename OT<R>::T2* __restrict__ psi, int n,
                                                            int64_t batch, double* __restrict__ M) {
  __shared__ double sm[kMaxQubits * kMaxQubits];
  const int lane = threadIdx.x & 31;
  const uint64_t len = 1ull << n;
  const uint64_t runs = len >> KW;
  const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) sm[i] = 0.0;
    __syncthreads();
    const typename OT<R>::T2* p = psi + (uint64_t)b * len;
    double s_acc = 0.0, ms_acc[5], qs_acc[10];
#pragma unroll
    for (int k = 0; k < 5; ++k) ms_acc[k] = 0.0;
#pragma unroll
    for (int k = 0; k < 10; ++k) qs_acc[k] = 0.0;
    for (uint64_t run = wid; run < runs; run += nw) {
      const typename OT<R>::T2* pr = p + (run << KW) + lane;
      // a lane's 32 terms summed in the working precision (complex64: FP32,
      // about 1e-7 relative for 32 terms), everything beyond in FP64
      R sr = 0, msr[5] = {0, 0, 0, 0, 0}, qsr[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        const typename OT<R>::T2 u = pr[r * 32];
        const R w = u.x * u.x + u.y * u.y;
        sr += w;
#pragma unroll
        for (int k = 0; k < 5; ++k)
          if ((r >> k) & 1) msr[k] += w;
        int t = 0;
#pragma unroll
        for (int k = 0; k < 5; ++k)
#pragma unroll
          for (int k2 = k + 1; k2 < 5; ++k2, ++t)
            if (((r >> k) & 1) && ((r >> k2) & 1)) qsr[t] += w;
      }
      const double s = (double)sr;
      double ms[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) ms[k] = (double)msr[k];
#pragma unroll
      for (int k = 0; k < 10; ++k) qs_acc[k] += (double)qsr[k];
      s_acc += s;
#pragma unroll
      for (int k = 0; k < 5; ++k) ms_acc[k] += ms[k];
      const uint32_t hm = (uint32_t)((run << KW) & 0xffffffffull);   // the run's set high bits
      if (hm == 0) continue;
      // the run's weight and its ten low-bit moments, on every lane
      double m[KW];
#pragma unroll
      for (int j = 0; j < 5; ++j) m[j] = warp_allsum(((lane >> j) & 1) ? s : 0.0);
#pragma unroll
      for (int k = 0; k < 5; ++k) m[5 + k] = warp_allsum(ms[k]);
      const double S = warp_allsum(s);
      if (S == 0.0) continue;
      const int h = __popc(hm);
      for (int u = lane; u < (KW + 1) * h; u += 32) {   // (j, a) += m_j; (a, a) += S
        const int ia = u / (KW + 1), c = u - ia * (KW + 1);
        const int a = (int)__fns(hm, 0, ia + 1);
        double v = S;
#pragma unroll
        for (int j = 0; j < KW; ++j)
          if (c == j) v = m[j];
        atomicAdd(&sm[(c == KW ? a : c) * n + a], v);
      }
      for (int u = lane; u < h * h; u += 32) {   // (a, b) += S for set high bits a < b
        const int ia = u / h, ib = u - ia * h;
        if (ia < ib) atomicAdd(&sm[(int)__fns(hm, 0, ia + 1) * n + (int)__fns(hm, 0, ib + 1)], S);
      }
    }
    // the low block, reduced once over the warp: bits 0-4 from the lanes,
    // bits 5-9 from the slots
    double lo[KW], q[KW * (KW - 1) / 2];
#pragma unroll
    for (int j = 0; j < 5; ++j) lo[j] = warp_allsum(((lane >> j) & 1) ? s_acc : 0.0);
#pragma unroll
    for (int k = 0; k < 5; ++k) lo[5 + k] = warp_allsum(ms_acc[k]);
    int t = 0, tt = 0;
#pragma unroll
    for (int j = 0; j < KW; ++j)
#pragma unroll
      for (int j2 = j + 1; j2 < KW; ++j2, ++t) {
        double v;
        if (j2 < 5) v = ((lane >> j) & 1) && ((lane >> j2) & 1) ? s_acc : 0.0;   // lane, lane
        else if (j < 5) v = ((lane >> j) & 1) ? ms_acc[j2 - 5] : 0.0;             // lane, slot
        else v = qs_acc[tt++];                                                     // slot, slot
        q[t] = warp_allsum(v);
      }
    if (lane == 0) {
      int t2 = 0;
#pragma unroll
      for (int j = 0; j < KW; ++j) {
        atomicAdd(&sm[j * n + j], lo[j]);
#pragma unroll
        for (int j2 = j + 1; j2 < KW; ++j2, ++t2) atomicAdd(&sm[j * n + j2], q[t2]);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n * n; i += blockDim.x)
      if (sm[i] != 0.0) atomicAdd(&M[(uint64_t)b * n * n + i], sm[i]);
    __syncthreads();
  }
}

// C[b][i][j] = (1/4) (<(n_iu - n_id)(n_ju - n_jd)> - <n_iu - n_id><n_ju - n_jd>)
// from the upper triangle of M.
__global__ void spin_corr_kernel(const double* __restrict__ M, int n, const int32_t* __restrict__ up,
                                 const int32_t* __restrict__ dn, int L, double* __restrict__ C,
                                 int64_t batch) {
  const int64_t total = batch * L * L;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = idx / (L * L);
    const int i = (int)((idx / L) % L), j = (int)(idx % L);
    const double* Mb = M + (uint64_t)b * n * n;
    auto mm = [&](int k, int l) { return k <= l ? Mb[k * n + l] : Mb[l * n + k]; };
    const int ui = up[i], di = dn[i], uj = up[j], dj = dn[j];
    const double corr = mm(ui, uj) - mm(ui, dj) - mm(di, uj) + mm(di, dj);
    const double zi = mm(ui, ui) - mm(di, di), zj = mm(uj, uj) - mm(dj, dj);
    C[idx] = 0.25 * (corr - zi * zj);
  }
}

dim3 vec_grid(uint64_t len, int64_t batch) {
  const uint64_t bx = std::min<uint64_t>((len + 255) / 256, 1216);
  const uint64_t by = std::min<int64_t>(batch, std::max<uint64_t>(1, 65535 / std::max<uint64_t>(bx, 1)));
  return dim3((unsigned)bx, (unsigned)std::min<uint64_t>(by, 65535));
}

}  // namespace

cudaError_t launch_overlap(int dtype, const void* psi, const void* ref, int64_t ref_batch, int n, int64_t batch,
                           double* a, cudaStream_t st) {
  const uint64_t len = 1ull << n;
  const dim3 g = vec_grid(len, batch);
  if (dtype == 0)
    overlap_kernel<float><<<g, 256, 0, st>>>((const float2*)psi, (const float2*)ref, ref_batch, len, batch, a);
  else
    overlap_kernel<double><<<g, 256, 0, st>>>((const double2*)psi, (const double2*)ref, ref_batch, len, batch, a);
  return cudaGetLastError();
}

cudaError_t launch_scale_ref(int dtype, const void* ref, int64_t ref_batch, void* lam, int n, int64_t batch,
                             const double* a, cudaStream_t st) {
  const uint64_t len = 1ull << n;
  const dim3 g = vec_grid(len, batch);
  if (dtype == 0)
    scale_ref_kernel<float><<<g, 256, 0, st>>>((const float2*)ref, ref_batch, (float2*)lam, len, batch, a);
  else
    scale_ref_kernel<double><<<g, 256, 0, st>>>((const double2*)ref, ref_batch, (double2*)lam, len, batch, a);
  return cudaGetLastError();
}

cudaError_t launch_overlap_finalize(const double* acc, int n_slots, int P, const double* a, double* F, double* f,
                                    double* grad, int64_t batch, cudaStream_t st) {
  const int64_t total = batch * (P + 1);
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 1024);
  overlap_finalize_kernel<<<grid, 256, 0, st>>>(acc, n_slots, P, a, F, f, grad, batch);
  return cudaGetLastError();
}

cudaError_t launch_sector_overlap(int dtype, const void* mat, const uint32_t* xrow, const uint32_t* xin, int n_rows,
                                  int row_len, const void* ref, int64_t ref_batch, int n, int64_t batch, double* a,
                                  cudaStream_t st) {
  const dim3 g = vec_grid((uint64_t)n_rows * (uint64_t)row_len, batch);
  if (dtype == 0)
    sector_overlap_kernel<float><<<g, 256, 0, st>>>((const float2*)mat, xrow, xin, n_rows, row_len,
                                                    (const float2*)ref, ref_batch, n, batch, a);
  else
    sector_overlap_kernel<double><<<g, 256, 0, st>>>((const double2*)mat, xrow, xin, n_rows, row_len,
                                                     (const double2*)ref, ref_batch, n, batch, a);
  return cudaGetLastError();
}

cudaError_t launch_sector_scale_ref(int dtype, const void* ref, int64_t ref_batch, const uint32_t* xrow,
                                    const uint32_t* xin, int n_rows, int row_len, int n, int64_t batch,
                                    const double* a, void* lam, cudaStream_t st) {
  const dim3 g = vec_grid((uint64_t)n_rows * (uint64_t)row_len, batch);
  if (dtype == 0)
    sector_scale_ref_kernel<float><<<g, 256, 0, st>>>((const float2*)ref, ref_batch, xrow, xin, n_rows, row_len, n,
                                                      batch, a, (float2*)lam);
  else
    sector_scale_ref_kernel<double><<<g, 256, 0, st>>>((const double2*)ref, ref_batch, xrow, xin, n_rows, row_len,
                                                       n, batch, a, (double2*)lam);
  return cudaGetLastError();
}

cudaError_t launch_occ_corr(int dtype, const void* psi, int n, int64_t batch, double* M, cudaStream_t st) {
  if (n >= KW) {   // one warp per run of 2^KW amplitudes
    const uint64_t runs = 1ull << (n - KW);
    const uint64_t bx = std::min<uint64_t>((runs + 7) / 8, 4 * 152);
    const dim3 g((unsigned)bx, (unsigned)std::min<int64_t>(batch, 65535));
    if (dtype == 0)
      occ_corr_warp_kernel<float><<<g, 256, 0, st>>>((const float2*)psi, n, batch, M);
    else
      occ_corr_warp_kernel<double><<<g, 256, 0, st>>>((const double2*)psi, n, batch, M);
    return cudaGetLastError();
  }
  const int kr = n < KR ? n : KR;
  const uint64_t runs = 1ull << (n - kr);
  const uint64_t bx = std::min<uint64_t>((runs + 127) / 128, 2 * 152);
  const dim3 g((unsigned)bx, (unsigned)std::min<int64_t>(batch, 65535));
  if (dtype == 0)
    occ_corr_kernel<float><<<g, 128, 0, st>>>((const float2*)psi, n, batch, M);
  else
    occ_corr_kernel<double><<<g, 128, 0, st>>>((const double2*)psi, n, batch, M);
  return cudaGetLastError();
}

cudaError_t launch_spin_corr(const double* M, int n, const int32_t* up, const int32_t* dn, int L, double* C,
                             int64_t batch, cudaStream_t st) {
  const int64_t total = batch * L * L;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 1024);
  spin_corr_kernel<<<grid, 256, 0, st>>>(M, n, up, dn, L, C, batch);
  return cudaGetLastError();
}

}  // namespace hubsv
