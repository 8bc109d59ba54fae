// Instantiations of the sweep kernel for float amplitudes, 1 vector(s)
// per tile; compiled as a unit of its own so the builds run in parallel.
#include "hubsv_sweep.cuh"

namespace hubsv {

const void* sweep_ptr_f1(int r) {
  switch (r) {
    case 1: return (const void*)sweep_kernel<float, 1, 1>;
    case 2: return (const void*)sweep_kernel<float, 1, 2>;
    case 3: return (const void*)sweep_kernel<float, 1, 3>;
    case 4: return (const void*)sweep_kernel<float, 1, 4>;
    default: return nullptr;
  }
}

// Four CTAs of at most 256 threads per SM.
const void* sweep_ptr_f1_narrow(int r) {
  switch (r) {
    case 4: return (const void*)sweep_kernel<float, 1, 4, 4>;
    default: return nullptr;
  }
}

}  // namespace hubsv
