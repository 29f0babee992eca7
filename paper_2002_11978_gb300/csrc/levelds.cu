// levelds.cu -- mixed level kernels of the grid engine, double-single inner
// solve, BiCGSTAB (TSFDE_MIXED_DS; arithmetic in dsf.cuh).
#include "levels.cuh"

namespace tsfde {

const void* leveldsp_kernel(int kp);  // levelds_pcg.cu

const void* levelds_kernel(int kp, int pcg) {
  if (pcg) return leveldsp_kernel(kp);
  return kp == 2 ? (const void*)k_level_mixed_ds<2, false> : (const void*)k_level_mixed_ds<4, false>;
}

const void* precond_ds_kernel(int kp) {
  return kp == 2 ? (const void*)k_precond_ds<2> : (const void*)k_precond_ds<4>;
}

}  // namespace tsfde
