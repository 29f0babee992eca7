// level64.cu -- FP64 level kernels of the grid engine: the forward level
// solve (Strang-preconditioned PBiCGSTAB, Sec. 4) and the adjoint level
// solve with its gradient epilogue.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/tsfde.h"
#include "dev.cuh"
#include "grid.cuh"
#include "plan.h"

namespace tsfde {

// FP64 level solve: preconditioner build and PBiCGSTAB, all in FP64.
// KP: prefetch depth of the Krylov passes (see kPre).
template <int KP>
__global__ void __launch_bounds__(kThreads, 2) k_level64(LevelArgs A) {
  const DevPlan& P = A.P;
  if (!kp_fits(P, KP)) { write_stat(A.stat, TSFDE_EINVAL, 0, 0, 0.0); return; }
  SmemAll S = smem_setup(P);
  const double kbar = mean_kappa(P, A.kappa64, S.d.red);
  if (kbar < 0.0) { write_stat(A.stat, TSFDE_ETIMEOUT, 0, 0, 0.0); return; }
  if (A.precond && !build_precond<double>(P, S.d, A.ahat, kbar)) {
    write_stat(A.stat, TSFDE_ETIMEOUT, 0, 0, 0.0);
    return;
  }
  if (!A.u_prev) {
    KVecs<double> V = A.k64;
    V.x = A.u;
    auto binit = [&](int i) -> double { return A.b[i]; };
    SolveRes r = bicgstab<double, decltype(binit), false, KP>(P, S.d, V, A.kappa64, A.ahat, A.precond != 0,
                                                               A.tol, A.max_it, binit);
    write_stat(A.stat, r.status, r.iters, 0, r.relres);
    return;
  }
  // warm start: solve M d = b - M u_prev to ||r|| < tol ||b||, u = u_prev + d
  double bb, rr;
  if (!warm_residual(A, S, bb, rr)) { write_stat(A.stat, TSFDE_ETIMEOUT, 0, 0, 0.0); return; }
  if (!isfinite(bb) || !isfinite(rr)) { write_stat(A.stat, TSFDE_ENONFINITE, 0, 0, 0.0); return; }
  if (bb == 0.0 || rr == 0.0) { write_stat(A.stat, TSFDE_OK, 0, 0, 0.0); return; }
  const double scale = sqrt(rr / bb);
  KVecs<double> V = A.k64;  // V.x: the correction d
  auto binit = [&](int i) -> double { return A.r64[i]; };
  SolveRes r = bicgstab<double, decltype(binit), false, KP>(P, S.d, V, A.kappa64, A.ahat, A.precond != 0,
                                                             A.tol / scale, A.max_it, binit);
  if (r.status == TSFDE_OK) {
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = gtid; i < P.n; i += gridDim.x * blockDim.x) A.u[i] += V.x[i];
  }
  write_stat(A.stat, r.status, r.iters, 0, r.relres * scale);
}

// Adjoint level solve: (ahat I + A K) lambda = g in FP64 (transposed
// operator; the Strang preconditioner is symmetric, so the same P serves),
// then y = A u^m with grad_kappa -= lambda .* y and grad_f += lambda in the
// product's epilogue.
__global__ void __launch_bounds__(kThreads, 2) k_level_adj(LevelArgs A, AdjGradArgs Gd) {
  const DevPlan& P = A.P;
  SmemAll S = smem_setup(P);
  const double kbar = mean_kappa(P, A.kappa64, S.d.red);
  if (kbar < 0.0) { write_stat(A.stat, TSFDE_ETIMEOUT, 0, 0, 0.0); return; }
  if (A.precond && !build_precond<double>(P, S.d, A.ahat, kbar)) {
    write_stat(A.stat, TSFDE_ETIMEOUT, 0, 0, 0.0);
    return;
  }
  KVecs<double> V = A.k64;
  V.x = A.u;
  auto binit = [&](int i) -> double { return A.b[i]; };
  SolveRes r = bicgstab<double, decltype(binit), true>(P, S.d, V, A.kappa64, A.ahat, A.precond != 0,
                                                       A.tol, A.max_it, binit);
  if (r.status == TSFDE_OK) {
    auto pro = [&](int i) -> double { return Gd.um[i]; };
    passA_real<double, false>(P, S.d, P.n, pro);
    if (!gsync(P, S.d.red)) { write_stat(A.stat, TSFDE_ETIMEOUT, r.iters, 0, r.relres); return; }
    passB<double, MID_APPLY>(P, S.d, P.saT64, P.sbT64, nullptr, nullptr, nullptr);
    if (!gsync(P, S.d.red)) { write_stat(A.stat, TSFDE_ETIMEOUT, r.iters, 0, r.relres); return; }
    auto epi = [&](int i, double y) -> double {
      const double li = A.u[i];
      Gd.grad_kappa[i] -= li * y;
      Gd.grad_f[i] += li;
      return 0.0;
    };
    passCA_real<double, false>(P, S.d, epi);
  }
  write_stat(A.stat, r.status, r.iters, 0, r.relres);
}

const void* level64_kernel(int kp) {
  return kp == 2 ? (const void*)k_level64<2> : (const void*)k_level64<4>;
}
const void* level_adj_kernel() { return (const void*)k_level_adj; }

}  // namespace tsfde
