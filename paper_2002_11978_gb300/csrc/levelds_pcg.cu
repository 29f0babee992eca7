// levelds_pcg.cu -- mixed level kernels of the grid engine, double-single inner
// solve, PCG on the symmetrised system.
#include "levels.cuh"

namespace tsfde {

const void* leveldsp_kernel(int kp) {
  return kp == 2 ? (const void*)k_level_mixed_ds<2, true> : (const void*)k_level_mixed_ds<4, true>;
}

}  // namespace tsfde
