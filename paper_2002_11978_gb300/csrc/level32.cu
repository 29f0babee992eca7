// level32.cu -- mixed level kernels of the grid engine, FP32 inner solve,
// BiCGSTAB (TSFDE_MIXED).
#include "levels.cuh"

namespace tsfde {

const void* level32p_kernel(int kp);  // level32_pcg.cu

const void* level32_kernel(int kp, int pcg) {
  if (pcg) return level32p_kernel(kp);
  return kp == 2 ? (const void*)k_level_mixed<2, false> : (const void*)k_level_mixed<4, false>;
}

}  // namespace tsfde
