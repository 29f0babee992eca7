// levelds.cu -- mixed level kernel of the grid engine with the double-single
// inner PBiCGSTAB (TSFDE_MIXED_DS; arithmetic in dsf.cuh).
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/tsfde.h"
#include "dev.cuh"
#include "grid.cuh"
#include "plan.h"

namespace tsfde {

// Mixed level solve with the inner PBiCGSTAB in double-single arithmetic
// (dsf.cuh): the same refinement loop, every inner vector, product and
// scalar update carried as FP32 pairs.  kappa^m and the preconditioner
// spectrum are rounded from FP64 once per level.  With ~48 bits the inner
// solve resolves the operator, but its true residual cannot go below
// ~u_ds ||M|| ||u|| (u_ds ~ 2^-47), which at the late levels of large
// problems is above tol ||b||.  So the first sweep stops near that floor, at
// kFirstSweep tol ||b|| (never asking for less than a 10x reduction), and
// every later sweep asks for the whole remaining reduction (half the
// target), within max_it iterations and not below 1e-13.  A level takes one
// long sweep and a short one that restarts from the true FP64 residual.
// KP: elements per thread of the inner passes' work items (2 when the
// real-geometry items have <= 512 elements, else 4).
constexpr double kFirstSweep = 100.0;

template <int KP>
__global__ void __launch_bounds__(kThreads, 2) k_level_mixed_ds(LevelArgs A) {
  const DevPlan& P = A.P;
  if (!kp_fits(P, KP)) { write_stat(A.stat, TSFDE_EINVAL, 0, 0, 0.0); return; }
  SmemAll S = smem_setup(P);
  auto conv = [&](int k) {
    if (k < P.n) A.kappads[k] = dsf(A.kappa64[k]);
    if (!A.precond) return;
    P.saGds[k] = dsf(P.saG64[k]);
    P.sbGds[k] = dsf(P.sbG64[k]);
  };
  int sweep = 0;
  auto inner = [&](double sc, double target, SolveRes& ir) -> bool {
    auto binit = [&](int i) -> dsf { return dsf(A.r64[i] * sc); };
    const double tin = sweep++ == 0 ? fmax(fmin(kFirstSweep * target, 0.1), 1e-13)
                                    : fmax(0.5 * target, 1e-13);
    ir = bicgstab<dsf, decltype(binit), false, KP>(P, S.s, A.kds, A.kappads, A.ahat, A.precond != 0,
                                                   tin, A.max_it, binit);
    return ir.status != TSFDE_ETIMEOUT;
  };
  mixed_level(A, S, conv, inner, A.kds.x);
}

const void* levelds_kernel(int kp) {
  return kp == 2 ? (const void*)k_level_mixed_ds<2> : (const void*)k_level_mixed_ds<4>;
}

}  // namespace tsfde
