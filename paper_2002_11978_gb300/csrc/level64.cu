// level64.cu -- FP64 level kernels of the grid engine with the paper's
// BiCGSTAB, and the adjoint level solve with its gradient epilogue.
#include "levels.cuh"

namespace tsfde {

// Adjoint level solve: (ahat I + A K) lambda = g in FP64 (transposed
// operator; the Strang preconditioner is symmetric, so the same P serves),
// by BiCGSTAB on the transposed operator or (PCG) by CG on the symmetrised
// (ahat K^{-1} + A) mu = g with lambda = K^{-1} mu; then y = A u^m with
// grad_kappa -= lambda .* y and grad_f += lambda in the product's epilogue.
template <bool PCG>
__global__ void __launch_bounds__(kThreads, 2) k_level_adj(LevelArgs A, AdjGradArgs Gd) {
  const DevPlan& P = A.P;
  SmemAll S = smem_setup(P);
  if constexpr (PCG) {
    // 1/kappa for the symmetrised system; ordered by mean_kappa's barrier
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x)
      A.hinv64[i] = 1.0 / A.kappa64[i];
  }
  const double kbar = mean_kappa(P, A.kappa64, S.d.red);
  if (kbar < 0.0) { write_stat(A.stat, TSFDE_ETIMEOUT, 0, 0, 0.0); return; }
  if (A.precond && !build_precond<double>(P, S.d, A.ahat, kbar)) {
    write_stat(A.stat, TSFDE_ETIMEOUT, 0, 0, 0.0);
    return;
  }
  KVecs<double> V = A.k64;
  V.x = A.u;
  auto binit = [&](int i) -> double { return A.b[i]; };
  SolveRes r;
  if constexpr (PCG) {
    r = pcg<double, decltype(binit), kPre, true>(P, S.d, V, A.kappa64, A.hinv64, A.ahat, A.precond != 0,
                                                 A.tol, A.max_it, binit);
    // lambda = K^{-1} mu, ordered before the epilogue by the barriers of
    // the product below
    if (r.status == TSFDE_OK)
      for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x)
        A.u[i] *= A.hinv64[i];
  } else {
    r = bicgstab<double, decltype(binit), true>(P, S.d, V, A.kappa64, A.ahat, A.precond != 0, A.tol,
                                                A.max_it, binit);
  }
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
  if (blockIdx.x == 0 && threadIdx.x == 0 && A.stat) A.stat->method = PCG ? 1 : 0;
}

const void* level64p_kernel(int kp);  // level64_pcg.cu

const void* level64_kernel(int kp, int pcg) {
  if (pcg) return level64p_kernel(kp);
  return kp == 2 ? (const void*)k_level64<2, false> : (const void*)k_level64<4, false>;
}
const void* level_adj_kernel(int pcg) {
  return pcg ? (const void*)k_level_adj<true> : (const void*)k_level_adj<false>;
}

}  // namespace tsfde
