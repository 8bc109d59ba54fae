// energy_noalloc: the energy call without any device allocation.
//
// Some callers cannot call cudaMalloc while they compute: code that runs
// while another framework owns the device memory pool (its allocator has
// reserved the free memory), or code on a latency-critical path where an
// allocation would synchronise the device.  energy() allocates its
// per-call scratch (coefficient and phase tables, the FP64 accumulators)
// and its static tables on first use; this entry point instead places every
// table and all scratch in one file-scope device array of fixed size, so a
// call allocates nothing.
//
// The array lives in every GPU that loads the library until the process
// exits.  Each device's address of it is looked up once, on the first call
// made with that device current; that first call belongs before any stream
// capture begins.  All calls share the array: each call
// rewrites the tables it uses and clears the accumulators, and two calls
// that overlap on the GPU (different streams, or different threads) race on
// it.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hubsv_host.h"

namespace {

constexpr size_t kScratchBytes = HUB_NOALLOC_SCRATCH_BYTES;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the static array on the current device (looked up once
// per device).
hub_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hubsv::cuda_fail(e, "energy_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return hubsv::fail(HUB_EUNSUPPORTED, "energy_noalloc: device index too large");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return hubsv::cuda_fail(e, "energy_noalloc: cudaGetSymbolAddress");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HUB_OK;
}

// Bump layout of the tables inside the array (256-byte aligned pieces).
struct Layout {
  size_t used = 0;
  size_t take(size_t bytes) {
    const size_t off = used;
    used += (bytes + 255) & ~(size_t)255;
    return off;
  }
};

}  // namespace

extern "C" hub_status energy_noalloc(ans_t a, const double* theta, void* psi, double* E, int32_t dtype,
                                     int64_t batch, uint32_t flags, hub_stream_t stream) {
  using namespace hubsv;
  if (!a) return fail(HUB_EINVAL, "energy_noalloc: NULL ansatz");
  if (dtype != HUB_C64 && dtype != HUB_C128) return fail(HUB_EINVAL, "energy_noalloc: bad dtype");
  if (batch < 1) return fail(HUB_EINVAL, "energy_noalloc: batch must be >= 1");
  if (!psi || !E || (a->P > 0 && !theta)) return fail(HUB_EINVAL, "energy_noalloc: NULL buffer");
  if (((uintptr_t)psi & (dtype == HUB_C64 ? 7u : 15u)) != 0)
    return fail(HUB_EINVAL, "energy_noalloc: psi must be aligned to its element size (8 or 16 bytes)");
  if (flags & ~(uint32_t)(HUB_FLAG_PREP_FUSED | HUB_FLAG_KEEP_STATE))
    return fail(HUB_EINVAL, "energy_noalloc: unknown flags");
  const bool fused = (flags & HUB_FLAG_PREP_FUSED) != 0;
  if (fused && a->prep_kind < 0) return fail(HUB_EINVAL, "energy_noalloc: HUB_FLAG_PREP_FUSED needs a prior state_prepare");
  if (a->n + 63 - __builtin_clzll((unsigned long long)batch) > 62) return fail(HUB_EINVAL, "energy_noalloc: batch too large");
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return cuda_fail(ce, "energy_noalloc: earlier asynchronous error");
  // the plan (host data only; cached in the ansatz)
  const int key = 0 * 16 + dtype * 8 + (int)(flags & 3u);   // the plan cache key of energy()
  Plan* pl = nullptr;
  auto it = a->plans.find(key);
  if (it != a->plans.end()) {
    pl = it->second;
  } else {
    hub_status st = make_plan(a, 0, dtype, flags, pl);
    if (st != HUB_OK) return st;
    a->plans[key] = pl;
  }
  const int n = a->n, n_slots = a->P + 2;
  const size_t r2 = dtype == HUB_C64 ? 8 : 16;
  const uint64_t n_tiles = ((uint64_t)batch) << (n - pl->k);
  if (n_tiles >= (1ull << 31)) return fail(HUB_EUNSUPPORTED, "energy_noalloc: batch too large for one launch");
  const bool sd_needed = fused && a->prep_kind == 0;
  if (sd_needed && a->sd_host.empty()) return fail(HUB_EINVAL, "energy_noalloc: no Slater tables; call state_prepare");
  const std::vector<float> real32(a->real_tabs.begin(), a->real_tabs.end());
  const std::vector<float> sd32(a->sd_host.begin(), a->sd_host.end());
  // layout
  Layout lay;
  const size_t o_gp = lay.take(4 * a->gate_param.size());
  const size_t o_gt = lay.take(8 * a->gate_t.size());
  const size_t o_tp = lay.take(4 * a->tab_param.size());
  const size_t o_tv = lay.take(8 * a->tab_val.size());
  const size_t o_tl = lay.take(4 * a->tab_live.size());
  const size_t o_hc = lay.take(8 * a->hcoef.size());
  const size_t o_rt = lay.take(8 * a->real_tabs.size());
  const size_t o_r32 = lay.take(4 * real32.size());
  const size_t o_dg = lay.take(sizeof(DiagOpDev) * a->diag_ops.size());
  const size_t o_sd = lay.take(sd_needed ? 8 * a->sd_host.size() : 0);
  const size_t o_sd32 = lay.take(sd_needed ? 4 * sd32.size() : 0);
  const size_t o_ops = lay.take(sizeof(OpDev) * std::max<size_t>(1, pl->hops.size()));
  const size_t o_ph = lay.take(sizeof(PhaseDev) * pl->hphases.size());
  const size_t o_sm = lay.take(4 * std::max<size_t>(1, pl->slot_map.size()));
  const size_t o_cf = lay.take(16 * (size_t)batch * a->n_gates);   // Givens (cos, sin): 16 bytes in both dtypes
  const size_t o_pt = lay.take(r2 * (size_t)batch * a->n_tab);
  const size_t o_acc = lay.take(8 * (size_t)batch * n_slots);
  if (lay.used > kScratchBytes)
    return fail(HUB_EINVAL, "energy_noalloc: this problem needs " + std::to_string(lay.used) +
                                " bytes of scratch; the static buffer holds " + std::to_string(kScratchBytes));
  void* base = nullptr;
  hub_status st = scratch_address(&base);
  if (st != HUB_OK) return st;
  unsigned char* S = static_cast<unsigned char*>(base);
  cudaStream_t s = (cudaStream_t)stream;
  auto put = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(S + off, src, bytes, cudaMemcpyHostToDevice, s);
  };
  ce = cudaSuccess;
  if (ce == cudaSuccess) ce = put(o_gp, a->gate_param.data(), 4 * a->gate_param.size());
  if (ce == cudaSuccess) ce = put(o_gt, a->gate_t.data(), 8 * a->gate_t.size());
  if (ce == cudaSuccess) ce = put(o_tp, a->tab_param.data(), 4 * a->tab_param.size());
  if (ce == cudaSuccess) ce = put(o_tv, a->tab_val.data(), 8 * a->tab_val.size());
  if (ce == cudaSuccess) ce = put(o_tl, a->tab_live.data(), 4 * a->tab_live.size());
  if (ce == cudaSuccess) ce = put(o_hc, a->hcoef.data(), 8 * a->hcoef.size());
  if (ce == cudaSuccess) ce = put(o_rt, a->real_tabs.data(), 8 * a->real_tabs.size());
  if (ce == cudaSuccess) ce = put(o_r32, real32.data(), 4 * real32.size());
  if (ce == cudaSuccess) ce = put(o_dg, a->diag_ops.data(), sizeof(DiagOpDev) * a->diag_ops.size());
  if (ce == cudaSuccess && sd_needed) ce = put(o_sd, a->sd_host.data(), 8 * a->sd_host.size());
  if (ce == cudaSuccess && sd_needed) ce = put(o_sd32, sd32.data(), 4 * sd32.size());
  if (ce == cudaSuccess) ce = put(o_ops, pl->hops.data(), sizeof(OpDev) * pl->hops.size());
  if (ce == cudaSuccess) ce = put(o_ph, pl->hphases.data(), sizeof(PhaseDev) * pl->hphases.size());
  if (ce == cudaSuccess) ce = put(o_sm, pl->slot_map.data(), 4 * pl->slot_map.size());
  if (ce != cudaSuccess) return cuda_fail(ce, "energy_noalloc: table copy");
  // the accumulators keep the previous call's sums: clear them
  HUB_CUDA(launch_zero(reinterpret_cast<double*>(S + o_acc), batch * n_slots, s), "energy_noalloc: zero accumulators");
  if (pl->sector)   // sweeps visit only sector tiles: the rest of psi must read as zero
    HUB_CUDA(cudaMemsetAsync(psi, 0, (size_t)batch * ((size_t)1 << n) * r2, s), "energy_noalloc: clear psi");
  HUB_CUDA(launch_coef(dtype, theta, a->P, reinterpret_cast<const int32_t*>(S + o_gp),
                       reinterpret_cast<const double*>(S + o_gt), a->n_gates, S + o_cf,
                       reinterpret_cast<const int32_t*>(S + o_tp), reinterpret_cast<const double*>(S + o_tv),
                       a->n_tab, reinterpret_cast<const int32_t*>(S + o_tl), (int)a->tab_live.size(),
                       S + o_pt, batch, a->n_inst, s),
           "energy_noalloc: coefficient kernel");
  KernelArgs ka;
  std::memset(&ka, 0, sizeof(ka));
  ka.psi = psi;
  ka.ops = reinterpret_cast<const OpDev*>(S + o_ops);
  ka.phases = reinterpret_cast<const PhaseDev*>(S + o_ph);
  ka.diag_ops = reinterpret_cast<const DiagOpDev*>(S + o_dg);
  ka.theta = theta;
  ka.P = a->P;
  ka.coef = S + o_cf;
  ka.n_gates = a->n_gates;
  ka.hcoef = reinterpret_cast<const double*>(S + o_hc);
  ka.n_hterms = a->n_hcol;
  ka.real_tabs = reinterpret_cast<const double*>(S + o_rt);
  ka.real_tabs32 = reinterpret_cast<const float*>(S + o_r32);
  ka.real_stride = a->real_stride;
  ka.phase_tabs = S + o_pt;
  ka.phase_stride = a->n_tab;
  ka.n_inst = a->n_inst;
  ka.n = n;
  ka.s = a->s;
  ka.upmask = a->upmask;
  ka.batch = batch;
  ka.n_tiles = n_tiles;
  ka.acc = reinterpret_cast<double*>(S + o_acc);
  ka.n_slots = n_slots;
  ka.slot_E = a->P;
  ka.slot_N = a->P + 1;
  ka.slot_map = reinterpret_cast<const int32_t*>(S + o_sm);
  ka.prep.kind = a->prep_kind < 0 ? 0 : a->prep_kind;
  ka.prep.L = a->L;
  ka.prep.s = a->s;
  ka.prep.layout = a->layout;
  ka.prep.neel_x0 = a->neel_x0;
  ka.prep.sd = sd_needed ? reinterpret_cast<const double*>(S + o_sd) : nullptr;
  ka.prep.sd32 = sd_needed ? reinterpret_cast<const float*>(S + o_sd32) : nullptr;
  const int sms = device_sm_count();
  if (sms <= 0) return fail(HUB_ECUDA, "energy_noalloc: no CUDA device");
  const int optin = sweep_max_smem_optin();
  for (size_t i = 0; i < pl->sweeps.size(); ++i) {
    const SweepDev& sw = pl->sweeps[i];
    const int nv = pl->nvec[i];
    const int nph = sw.phase_end - sw.phase_begin;
    const size_t smem = sweep_smem_bytes(dtype, nv, sw.k, sw.n_lslot, nph, sw.op_end - sw.op_begin, 32 << sw.w);
    if ((int)smem > optin) return fail(HUB_EUNSUPPORTED, "energy_noalloc: tile does not fit in shared memory");
    HUB_CUDA(sweep_set_smem(dtype, nv, sw.r, 32 << sw.w, (sw.flags & SW_VPOP) != 0, smem), "energy_noalloc: cudaFuncSetAttribute");
    const int threads = 32 << sw.w;
    const int regs = std::max(1, sweep_regs(dtype, nv, sw.r, 32 << sw.w, (sw.flags & SW_VPOP) != 0));
    int per_sm = (int)((size_t)(228 * 1024) / (smem + 1024));
    per_sm = std::min(per_sm, 2048 / threads);
    per_sm = std::min(per_sm, 65536 / (regs * threads));
    per_sm = std::max(per_sm, 1);
    const uint64_t sweep_tiles = sw.sector ? (uint64_t)batch * sw.live : n_tiles;
    const uint64_t grid = std::min<uint64_t>((uint64_t)sms * per_sm, std::max<uint64_t>(1, sweep_tiles));
    HUB_CUDA(launch_sweep(dtype, sw, ka, (int)grid, smem, s), "energy_noalloc: sweep kernel launch");
  }
  HUB_CUDA(launch_finalize(ka.acc, n_slots, a->P, a->P, E, nullptr, batch, s), "energy_noalloc: finalize kernel");
  return HUB_OK;
}
