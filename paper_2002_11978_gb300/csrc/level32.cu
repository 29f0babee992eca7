// level32.cu -- mixed level kernel of the grid engine with the FP32 inner
// PBiCGSTAB (TSFDE_MIXED).
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/tsfde.h"
#include "dev.cuh"
#include "grid.cuh"
#include "plan.h"

namespace tsfde {

// Mixed level solve on the grid engine: the refinement loop of mixed_level
// (grid.cuh) with the FP32 PBiCGSTAB spread over the whole cooperative grid.
template <int KP>
__global__ void __launch_bounds__(kThreads, 2) k_level_mixed(LevelArgs A) {
  const DevPlan& P = A.P;
  if (!kp_fits(P, KP)) { write_stat(A.stat, TSFDE_EINVAL, 0, 0, 0.0); return; }
  SmemAll S = smem_setup(P);
  auto conv = [&](int k) {
    if (!A.precond) return;
    P.saG32[k] = (float)P.saG64[k];
    P.sbG32[k] = (float)P.sbG64[k];
  };
  auto inner = [&](double sc, double, SolveRes& ir) -> bool {
    auto binit = [&](int i) -> float { return (float)(A.r64[i] * sc); };
    ir = bicgstab<float, decltype(binit), false, KP>(P, S.f, A.k32, A.kappa32, A.ahat, A.precond != 0,
                                                     A.inner_tol, A.inner_max_it, binit);
    return ir.status != TSFDE_ETIMEOUT;
  };
  mixed_level(A, S, conv, inner, A.k32.x);
}

const void* level32_kernel(int kp) {
  return kp == 2 ? (const void*)k_level_mixed<2> : (const void*)k_level_mixed<4>;
}

}  // namespace tsfde
