// level64_pcg.cu -- FP64 level kernels of the grid engine with PCG on the symmetrised
// system.
#include "levels.cuh"

namespace tsfde {

const void* level64p_kernel(int kp) {
  return kp == 2 ? (const void*)k_level64<2, true> : (const void*)k_level64<4, true>;
}

}  // namespace tsfde
