// cluster.cu -- cluster engine of the mixed-precision FIDS level solve
// (sm_103a).
//
// One cooperative launch per time level.  The whole grid runs the FP64 parts
// of the mixed solve (the Strang preconditioner build of Sec. 4.1, the FP64
// residual products and the refinement updates; mixed_level in grid.cuh),
// and every FP32 inner PBiCGSTAB runs on the first thread-block cluster
// alone: Q <= 16 CTAs that hold the length-Nc complex FFT of each Toeplitz
// or circulant product in their shared memory and exchange the transposes
// through distributed shared memory.  An inner iteration then costs cluster
// barriers instead of grid barriers and touches global memory only for the
// Krylov vectors (L2-resident) and the spectra; the CTAs outside the first
// cluster wait at the grid barrier meanwhile.
//
// Per product: column pass (length-N1 FFTs of the CTA's own columns, twiddle
// W_Nc^{j2 k1}, push to the row owners), row pass (length-N2 FFTs of the
// CTA's row pairs, the spectral middle step of Sec. 4.1 in its stable form,
// inverse row FFTs, twiddle conj, push back to the column owners), inverse
// column pass (inverse FFTs, epilogue on the owned vector entries, optionally
// the forward column pass of the next product).  Each pass ends with one
// cluster barrier; cluster barriers are hardware barriers whose arrival set
// is every thread of the cluster, and every CTA takes the same branches
// (all decisions use cluster-reduced scalars that are bitwise equal in every
// CTA), so no wait can be left without its partners.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/tsfde.h"
#include "cluster.cuh"
#include "dev.cuh"
#include "grid.cuh"
#include "plan.h"

namespace tsfde {

constexpr int kCT = 512;  // threads per CTA of the cluster engine

// grid slots that carry the inner solve's result to the whole grid
enum { SL_CIT = 10, SL_CST = 11 };

static __host__ __device__ CeLay cluster_layout(const CGeo& g) {
  CeLay y{};
  y.capB = g.cap * (int)sizeof(float2);
  y.nbufB = g.nbuf * (int)sizeof(float2);
  y.T1 = g.T1;
  y.LT = g.LT;
  y.has64 = 0;
  return y;
}

size_t cluster_smem_bytes(const DevPlan& P) {
  return ce_ctx_offset(cluster_layout(P.cl)) + sizeof(CeCtx<float>);
}

// Mixed level solve, cluster engine.  Same refinement loop as the grid
// engine's k_level_mixed (mixed_level, grid.cuh); only the FP32 inner solves
// move to cluster 0, whose CTAs hold each FFT in distributed shared memory
// while the rest of the grid waits at the grid barrier.
__global__ void __launch_bounds__(kCT, 1) k_level_cluster(LevelArgs A) {
  if (A.probe) return;
  const DevPlan& P = A.P;
  const CGeo& cg_ = P.cl;
  SmemAll S = smem_setup(P);
  const int N1 = P.gr.N1, N2 = P.gr.N2, lgN2 = P.gr.lgN2;
  auto conv = [&](int k) {
    if (!A.precond) return;
    const int k1 = k >> lgN2, k2 = k & (N2 - 1);
    int u, b;
    unit_of(k1, N1, u, b);
    const int r = u >> cg_.lgU, slot = 2 * (u & (cg_.U - 1)) + b;
    P.spG_cl[(size_t)r * cg_.nbuf + (k2 << cg_.lgBq) + slot] =
        make_float2((float)P.saG64[k], (float)P.sbG64[k]);
  };
  auto inner = [&](double sc, double, SolveRes& ir) -> bool {
    double its = 0.0, stv = 0.0;
    if ((int)blockIdx.x < cg_.Q) {
      const CeLay lay = cluster_layout(cg_);
      ce_load_tables(lay, cg_.T1, cg_.LT, cg_.lgLT, P.twL64, P.twL32);
      const CeSm<float> cs = ce_sm<float>(lay);
      CeCtx<float>* cx = reinterpret_cast<CeCtx<float>*>(cs.ctx);
      if (threadIdx.x == 0) {
        CeGeo& g = cx->g;
        g.n = P.n; g.L = P.L; g.tws = 2;
        g.N1 = N1; g.N2 = N2; g.lgN1 = P.gr.lgN1; g.lgN2 = lgN2;
        g.Q = cg_.Q; g.cQ = cg_.cQ; g.lgcQ = cg_.lgcQ; g.U = cg_.U; g.lgU = cg_.lgU;
        g.Bq = cg_.Bq; g.lgBq = cg_.lgBq; g.nbuf = cg_.nbuf;
        g.T1 = cg_.T1; g.LT = cg_.LT; g.lgLT = cg_.lgLT; g.q = 0;
        cx->lay = lay;
        cx->spT = P.spT_cl; cx->spG = P.spG_cl;
        cx->V = A.k32; cx->kap = A.kappa32; cx->hinv = nullptr; cx->a = (float)A.ahat;
      }
      __syncthreads();
      const SolveRes r = ce_bicgstab<float>(cx, A.precond != 0, A.inner_tol, A.inner_max_it, A.r64, sc);
      if (blockIdx.x == 0) { its = (double)r.iters; stv = (double)r.status; }
    }
    put_partial(P, SL_CIT, its);
    put_partial(P, SL_CST, stv);
    double o_its, o_st;
    const bool ok = gsync_sum2(P, S.d.red, SL_CIT, SL_CST, 0u, o_its, o_st);
    S = smem_setup(P, false);  // the cluster passes overwrote the grid tables
    ir.iters = (int)o_its;
    ir.status = (int)o_st;
    return ok;
  };
  mixed_level(A, S, conv, inner, A.k32.x);
}

// ------------------------------------------------------------- host side
bool cluster_geometry(DevPlan& P) {
  CGeo& g = P.cl;
  g = CGeo{};
  const int N1 = P.gr.N1, N2 = P.gr.N2;
  if (N1 < N2 || N1 < 2 || N2 < 1) return false;
  int Q = kMaxQ;
  while (Q > 1 && (2 * Q > N1 || Q > N2)) Q >>= 1;
  auto lg = [](int x) { int l = 0; while ((1 << l) < x) ++l; return l; };
  g.Q = Q; g.lgQ = lg(Q);
  g.cQ = N2 / Q; g.lgcQ = lg(g.cQ);
  g.U = N1 / (2 * Q); g.lgU = lg(g.U);
  g.Bq = 2 * g.U; g.lgBq = lg(g.Bq);
  g.nbuf = P.Nc / Q;
  g.cap = g.nbuf + N1;
  g.T1 = N1;
  g.LT = P.L / N1; g.lgLT = lg(g.LT);
  g.G = Q;
  return g.cQ >= 1 && g.U >= 1 && g.cQ * Q == N2 && g.U * 2 * Q == N1;
}

static cudaLaunchConfig_t cluster_config(const DevPlan& P, size_t smem, int grid, cudaStream_t s,
                                         cudaLaunchAttribute* at, bool coop) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = P.cl.Q;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeCooperative;
  at[1].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = coop ? 2 : 1;
  return cfg;
}

// The dynamic shared-memory limit only ever grows, so a context set up earlier
// with a larger plan can still launch.
static size_t g_cl_smem_limit = 0;

int cluster_max_grid(const DevPlan& P, size_t smem) {
  if (smem > g_cl_smem_limit) {
    if (cudaFuncSetAttribute(k_level_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return 0;
    g_cl_smem_limit = smem;
  }
  if (P.cl.Q > 8 &&
      cudaFuncSetAttribute(k_level_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return 0;
  cudaLaunchAttribute at[2];
  cudaLaunchConfig_t cfg = cluster_config(P, smem, P.cl.Q, 0, at, false);
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, k_level_cluster, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return ncl * P.cl.Q;
}

cudaError_t launch_level_cluster(const LevelArgs& a, cudaStream_t s) {
  const size_t smem = std::max(plan_smem_bytes(a.P), cluster_smem_bytes(a.P));
  if (!a.probe) {
    cudaError_t e = cudaMemsetAsync(a.P.bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchAttribute at[2];
  cudaLaunchConfig_t cfg = cluster_config(a.P, smem, a.P.cl.G, s, at, true);
  return cudaLaunchKernelEx(&cfg, k_level_cluster, a);
}

}  // namespace tsfde
