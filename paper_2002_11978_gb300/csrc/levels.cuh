// levels.cuh -- the level kernels of the grid engine, templated on the
// prefetch depth KP of their Krylov passes (see kPre) and on the Krylov
// method: PCG (CG on the symmetrised system, see pcg in grid.cuh) or the
// paper's right-preconditioned BiCGSTAB.  Each (arithmetic, method) pair is
// instantiated in a translation unit of its own (level64.cu,
// level64_pcg.cu, level32.cu, level32_pcg.cu, levelds.cu, levelds_pcg.cu)
// so that they compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/tsfde.h"
#include "dev.cuh"
#include "grid.cuh"
#include "plan.h"

namespace tsfde {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// TSFDE_KRYLOV_AUTO (KrylovAuto, plan.h): true when the kernel of method
// PCG solves level A.m (always true for a fixed method).  Read by every
// thread before any work; the state changes only between kernels.
__device__ __forceinline__ bool auto_mine(const LevelArgs& A, bool pcg) {
  if (!A.kauto) return true;
  return __ldcg(&A.kauto->for_level) == A.m && __ldcg(&A.kauto->choice) == (pcg ? 1 : 0);
}

// End of a level solved by method `pcg`: block 0's thread 0 (which wrote the
// level's status) records the method in the level's stats and, for AUTO,
// hands the level's device time to the choice rule (auto_rule_next,
// plan.h) for the next level's method.
__device__ __forceinline__ void level_done(const LevelArgs& A, bool pcg, unsigned long long t0) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  if (A.stat) A.stat->method = pcg ? 1 : 0;
  KrylovAuto* k = A.kauto;
  if (!k) return;
  const int me = pcg ? 1 : 0;
  double dt = (double)(global_ns() - t0);
  if (A.stat && A.stat->status != TSFDE_OK) dt = INFINITY;
  k->used[me] += 1;
  k->choice = auto_rule_next(k->rule, me, A.m, dt);
  k->for_level = A.m + 1;
}

// FP64 level solve: preconditioner build and the Krylov solve, all in FP64.
template <int KP, bool PCG>
__device__ void level64_run(const LevelArgs& A) {
  const DevPlan& P = A.P;
  if (!kp_fits(P, KP)) { write_stat(A.stat, TSFDE_EINVAL, 0, 0, 0.0); return; }
  SmemAll S = smem_setup(P);
  if constexpr (PCG) {
    // 1/kappa for the symmetrised system; ordered by mean_kappa's barrier
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x)
      A.hinv64[i] = 1.0 / A.kappa64[i];
  }
  const double kbar = mean_kappa(P, A.kappa64, S.d.red);
  if (kbar < 0.0) { write_stat(A.stat, TSFDE_ETIMEOUT, 0, 0, 0.0); return; }
  if (A.precond && !build_precond<double, KP>(P, S.d, A.ahat, kbar)) {
    write_stat(A.stat, TSFDE_ETIMEOUT, 0, 0, 0.0);
    return;
  }
  if (!A.u_prev) {
    KVecs<double> V = A.k64;
    V.x = A.u;
    auto binit = [&](int i) -> double { return A.b[i]; };
    SolveRes r = level_krylov<PCG, KP>(P, S.d, V, A.kappa64, A.hinv64, A.ahat, A.precond != 0,
                                       A.tol, A.max_it, binit);
    write_stat(A.stat, r.status, r.iters, 0, r.relres);
    return;
  }
  // warm start: solve M d = b - M u_prev to ||r|| < tol ||b||, u = u_prev + d
  double bb, rr;
  if (!warm_residual<KP>(A, S, bb, rr)) { write_stat(A.stat, TSFDE_ETIMEOUT, 0, 0, 0.0); return; }
  if (!isfinite(bb) || !isfinite(rr)) { write_stat(A.stat, TSFDE_ENONFINITE, 0, 0, 0.0); return; }
  if (bb == 0.0 || rr == 0.0) { write_stat(A.stat, TSFDE_OK, 0, 0, 0.0); return; }
  const double scale = sqrt(rr / bb);
  KVecs<double> V = A.k64;  // V.x: the correction d
  auto binit = [&](int i) -> double { return A.r64[i]; };
  SolveRes r = level_krylov<PCG, KP>(P, S.d, V, A.kappa64, A.hinv64, A.ahat, A.precond != 0,
                                     A.tol / scale, A.max_it, binit);
  if (r.status == TSFDE_OK) {
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = gtid; i < P.n; i += gridDim.x * blockDim.x) A.u[i] += V.x[i];
  }
  write_stat(A.stat, r.status, r.iters, 0, r.relres * scale);
}

template <int KP, bool PCG>
__global__ void __launch_bounds__(kThreads, 2) k_level64(LevelArgs A) {
  if (!auto_mine(A, PCG)) return;
  const unsigned long long t0 = global_ns();
  level64_run<KP, PCG>(A);
  level_done(A, PCG, t0);
}

// Mixed level solve on the grid engine: the refinement loop of mixed_level
// (grid.cuh) with the FP32 inner solve spread over the whole cooperative grid.
template <int KP, bool PCG>
__device__ void level_mixed_run(const LevelArgs& A) {
  const DevPlan& P = A.P;
  if (!kp_fits(P, KP)) { write_stat(A.stat, TSFDE_EINVAL, 0, 0, 0.0); return; }
  SmemAll S = smem_setup(P);
  auto conv = [&](int k) {
    if (PCG && k < P.n) {
      const double h = 1.0 / A.kappa64[k];
      A.hinv64[k] = h;
      A.hinv32[k] = (float)h;
    }
    if (!A.precond) return;
    P.saG32[k] = (float)P.saG64[k];
    P.sbG32[k] = (float)P.sbG64[k];
  };
  auto inner = [&](double sc, double, SolveRes& ir) -> bool {
    auto binit = [&](int i) -> float { return (float)(A.r64[i] * sc); };
    ir = level_krylov<PCG, KP>(P, S.f, A.k32, A.kappa32, A.hinv32, A.ahat, A.precond != 0,
                               A.inner_tol, A.inner_max_it, binit);
    return ir.status != TSFDE_ETIMEOUT;
  };
  mixed_level<PCG, KP>(A, S, conv, inner, A.k32.x);
}

template <int KP, bool PCG>
__global__ void __launch_bounds__(kThreads, 2) k_level_mixed(LevelArgs A) {
  if (!auto_mine(A, PCG)) return;
  const unsigned long long t0 = global_ns();
  level_mixed_run<KP, PCG>(A);
  level_done(A, PCG, t0);
}

// Mixed level solve with the inner solve in double-single arithmetic
// (dsf.cuh): the same refinement loop, every inner vector, product and
// scalar update carried as FP32 pairs.  kappa^m (and 1/kappa^m for PCG) are
// rounded from FP64 once per level; the preconditioner spectrum comes from
// k_precond_ds, launched just before (mixed_level's PRE form).  With
// ~48 bits the inner solve resolves the operator, but its true residual
// cannot go below ~u_ds ||M|| ||u|| (u_ds ~ 2^-47), which at the late levels
// of large problems is above tol ||b||.  So the first sweep stops near that
// floor, at kFirstSweep tol ||b|| (never asking for less than a 10x
// reduction), and every later sweep asks for the whole remaining reduction
// (half the target), within max_it iterations and not below 1e-13.  A
// level takes one long sweep and a short one that restarts from the true
// FP64 residual.  That floor is relative to the sweep's own right-hand
// side, so when the start is good enough that the whole reduction is at
// most 1/kOneSweep (an extrapolated start), the first sweep asks for all of
// it and the level usually ends after one sweep.
constexpr double kFirstSweep = 100.0;
constexpr double kOneSweep = 1e-6;

template <int KP, bool PCG>
__device__ void level_mixed_ds_run(const LevelArgs& A) {
  const DevPlan& P = A.P;
  if (!kp_fits(P, KP)) { write_stat(A.stat, TSFDE_EINVAL, 0, 0, 0.0); return; }
  SmemAll S = smem_setup(P);
  auto conv = [&](int k) {
    if (k < P.n) {
      A.kappads[k] = dsf(A.kappa64[k]);
      if (PCG) {
        const double h = 1.0 / A.kappa64[k];
        A.hinv64[k] = h;
        A.hinvds[k] = dsf(h);
      }
    }
  };
  int sweep = 0;
  auto inner = [&](double sc, double target, SolveRes& ir) -> bool {
    auto binit = [&](int i) -> dsf { return dsf(A.r64[i] * sc); };
    const double tin = (sweep++ == 0 && target < kOneSweep) ? fmax(fmin(kFirstSweep * target, 0.1), 1e-13)
                                                             : fmax(0.5 * target, 1e-13);
    ir = level_krylov<PCG, KP>(P, S.s, A.kds, A.kappads, A.hinvds, A.ahat, A.precond != 0, tin,
                               A.max_it, binit);
    return ir.status != TSFDE_ETIMEOUT;
  };
  mixed_level<PCG, KP, true>(A, S, conv, inner, A.kds.x);
}

// The preconditioner of a double-single level, built in its own cooperative
// launch before the level kernel(s): kbar = mean(kappa^m), then the
// Bluestein build of P^{-1} (build_precond) in double-single arithmetic,
// whose ~48 bits keep the spectrum to ~1e-14 of its largest entry (FP32
// would bury the smallest eigenvalues, ~1e-8 of the largest at
// n = 2^17 - 1), at a fraction of the FP64 pipe time of an FP64 build; the
// FP64 tables (for an FP64 finish) are rounded from it.  Kept out of the
// level kernel so that the level kernel's registers are not spent on it.
template <int KP>
__global__ void __launch_bounds__(kThreads, 2) k_precond_ds(LevelArgs A) {
  const DevPlan& P = A.P;
  int st = TSFDE_OK;
  if (!kp_fits(P, KP)) {
    st = TSFDE_EINVAL;
  } else {
    SmemAll S = smem_setup(P);
    const double kbar = mean_kappa(P, A.kappa64, S.d.red);
    if (kbar < 0.0 || !build_precond<dsf, KP>(P, S.s, A.ahat, kbar)) {
      st = TSFDE_ETIMEOUT;
    } else {
      const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
      for (int k = gtid; k < P.Nc; k += gridDim.x * blockDim.x) {
        P.saG64[k] = (double)P.saGds[k];
        P.sbG64[k] = (double)P.sbGds[k];
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.pre_status = st;
}

template <int KP, bool PCG>
__global__ void __launch_bounds__(kThreads, 2) k_level_mixed_ds(LevelArgs A) {
  if (!auto_mine(A, PCG)) return;
  const unsigned long long t0 = global_ns();
  level_mixed_ds_run<KP, PCG>(A);
  level_done(A, PCG, t0);
}

}  // namespace tsfde
