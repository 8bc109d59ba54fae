// Instantiations of the sweep kernel for float amplitudes that count
// uniform V terms with popcounts (sweeps flagged SW_VPOP), at the default
// register bits; compiled as a unit of its own so the builds run in parallel.
#include "hubsv_sweep.cuh"

namespace hubsv {

const void* sweep_ptr_fv(int nv, int r, int threads) {
  if (r != 4) return nullptr;
  if (nv == 2) return (const void*)sweep_kernel<float, 2, 4, 1, true>;
  if (threads <= 256) return (const void*)sweep_kernel<float, 1, 4, 4, true>;
  return (const void*)sweep_kernel<float, 1, 4, 1, true>;
}

}  // namespace hubsv
