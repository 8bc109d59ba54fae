// Instantiations of the sweep kernel for double amplitudes, 1 vector(s)
// per tile; compiled as a unit of its own so the builds run in parallel.
#include "hubsv_sweep.cuh"

namespace hubsv {

const void* sweep_ptr_d1(int r) {
  switch (r) {
    case 1: return (const void*)sweep_kernel<double, 1, 1>;
    case 2: return (const void*)sweep_kernel<double, 1, 2>;
    case 3: return (const void*)sweep_kernel<double, 1, 3>;
    default: return nullptr;
  }
}

}  // namespace hubsv
