// level32_pcg.cu -- mixed level kernels of the grid engine, FP32 inner solve,
// PCG on the symmetrised system.
#include "levels.cuh"

namespace tsfde {

const void* level32p_kernel(int kp) {
  return kp == 2 ? (const void*)k_level_mixed<2, true> : (const void*)k_level_mixed<4, true>;
}

}  // namespace tsfde
