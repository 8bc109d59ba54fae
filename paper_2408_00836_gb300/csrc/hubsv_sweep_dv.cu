// Instantiations of the sweep kernel for double amplitudes that count
// uniform V terms with popcounts (sweeps flagged SW_VPOP), at the default
// register bits; compiled as a unit of its own so the builds run in parallel.
#include "hubsv_sweep.cuh"

namespace hubsv {

const void* sweep_ptr_dv(int nv, int r, int /*threads*/) {
  if (r != 3) return nullptr;
  return nv == 2 ? (const void*)sweep_kernel<double, 2, 3, 1, true>
                 : (const void*)sweep_kernel<double, 1, 3, 1, true>;
}

}  // namespace hubsv
