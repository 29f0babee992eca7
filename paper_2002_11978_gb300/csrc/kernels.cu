// kernels.cu -- grid-engine kernels of the FIDS hot path (sm_103a): single
// products, the SOE history / RHS update (forward and adjoint), and the
// launchers of every grid kernel.  The level kernels live in level64.cu,
// level32.cu and levelds.cu (one translation unit each, compiled in
// parallel); the device code they share with the cluster engine is in
// grid.cuh.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "../../include/tsfde.h"
#include "dev.cuh"
#include "grid.cuh"
#include "plan.h"

namespace tsfde {

// Shared memory: [tw64 T][tw32 T][twds T][bufA W][bufB W][red 64]
size_t plan_smem_bytes(const DevPlan& P) {
  return (size_t)tpad_len(P.T) * (2 * sizeof(double2) + sizeof(float2)) +
         2 * (size_t)P.W * sizeof(double2) + 64 * sizeof(double);
}


// Level kernels: level64.cu (FP64, adjoint), level32.cu (FP32 inner),
// levelds.cu (double-single inner).





// Reversed SOE recurrence and adjoint right-hand side (see AdjRhsArgs).
__global__ void __launch_bounds__(kThreads) k_adj_rhs(AdjRhsArgs a) {
  extern __shared__ double sh[];
  double* s_eps = sh;
  double* s_c1 = sh + a.Eact;
  double* s_c2 = sh + 2 * a.Eact;
  for (int j = threadIdx.x; j < a.Eact; j += blockDim.x) {
    s_eps[j] = a.eps1[j];
    s_c1[j] = a.c1[j];
    s_c2[j] = a.c2 ? a.c2[j] : 0.0;
  }
  __syncthreads();
  const int gstr = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gstr) {
    const double lam = a.lam1[i];
    double acc = 0.0;
    double* Yi = a.Y + i;
    const size_t ld = (size_t)a.ld;
    for (int j = 0; j < a.Eact; ++j) {
      const double yo = Yi[j * ld];
      const double yn = s_eps[j] * (lam + yo);
      Yi[j * ld] = yn;
      acc += s_c1[j] * yn - s_c2[j] * yo;
    }
    a.g[i] = a.ahat1 * lam - acc;
  }
}

// ------------------------------------------------------ single products
template <typename R>
__device__ void apply_kernel_body(const ApplyArgs& A, const Smem<R>& sm, const Smem<double>& sd) {
  const DevPlan& P = A.P;
  const int n = P.n;
  if (A.kind == 1) {
    bool ok;
    if constexpr (is_ds<R>) {
      // built in FP64 and rounded, as in the double-single level solve
      ok = build_precond<double>(P, sd, A.a, A.kbar);
      for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.Nc; k += gridDim.x * blockDim.x) {
        P.saGds[k] = dsf(P.saG64[k]);
        P.sbGds[k] = dsf(P.sbG64[k]);
      }
    } else {
      ok = build_precond<R>(P, sm, A.a, A.kbar);
    }
    if (!ok) {
      if (blockIdx.x == 0 && threadIdx.x == 0) *A.status = TSFDE_ETIMEOUT;
      return;
    }
  }
  auto pro = [&](int i) -> R { return (R)A.v[i]; };
  passA_real<R, false>(P, sm, n, pro);
  if (!gsync(P, sm.red)) goto fail;
  if (A.kind == 1)
    passB<R, MID_APPLY>(P, sm, saG<R>(P), sbG<R>(P), nullptr, nullptr, nullptr);
  else
    passB<R, MID_APPLY>(P, sm, saT<R>(P), sbT<R>(P), nullptr, nullptr, nullptr);
  if (!gsync(P, sm.red)) goto fail;
  {
    auto epi = [&](int i, R y) -> R {
      double yi = (double)y;
      if (A.kind == 0) yi = A.a * A.v[i] + (A.kappa ? A.kappa[i] : 1.0) * yi;
      A.y[i] = yi;
      return R(0);
    };
    passCA_real<R, false>(P, sm, epi);
  }
  if (!gsync(P, sm.red)) goto fail;
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.status = TSFDE_OK;
  return;
fail:
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.status = TSFDE_ETIMEOUT;
}

__global__ void __launch_bounds__(kThreads, 2) k_apply64(ApplyArgs A) {
  SmemAll S = smem_setup(A.P);
  apply_kernel_body<double>(A, S.d, S.d);
}
__global__ void __launch_bounds__(kThreads, 2) k_apply32(ApplyArgs A) {
  SmemAll S = smem_setup(A.P);
  apply_kernel_body<float>(A, S.f, S.d);
}
__global__ void __launch_bounds__(kThreads, 2) k_apply_ds(ApplyArgs A) {
  SmemAll S = smem_setup(A.P);
  apply_kernel_body<dsf>(A, S.s, S.d);
}

// ------------------------------------------------- SOE history and RHS
// G_j <- e^{-s_j tau_m} (G_j + c_j d), d = u^{m-1} - u^{m-2}, for the active
// exponentials (G_j = w_j H_j / Gamma(1-gamma), c_j = w_j beta_{j,m-1} /
// Gamma(1-gamma)); b = ahat u^{m-1} - sum_j G_j + f^m (Eq. (3.16gu) with the
// history sum written through the SOE recurrence).  Also materialises
// kappa^m in FP64 and FP32.
constexpr int kRhsU = 8;      // exponentials whose history loads are issued together
constexpr int kRhsPairs = 64; // entry pairs per block
constexpr int kRhsGroups = kThreads / kRhsPairs;  // row groups per pair

// Block = kRhsPairs entry pairs (i, i+1) x kRhsGroups row groups: the warps
// of group g update rows [g c, (g+1) c) of the E x ld history for the
// block's 64 pairs with 16-byte accesses (1 KB contiguous per row), kRhsU
// rows' loads in flight at a time; the groups' partial sums are added in a
// fixed order.
__global__ void __launch_bounds__(kThreads) k_rhs(RhsArgs a) {
  extern __shared__ double sh[];
  double* s_eps = sh;
  double* s_cw = sh + a.Eact;
  double2* s_part = reinterpret_cast<double2*>(sh + 2 * a.Eact);  // 16-byte aligned
  for (int j = threadIdx.x; j < a.Eact; j += blockDim.x) {
    s_eps[j] = a.eps[j];
    s_cw[j] = a.cw[j];
  }
  __syncthreads();
  const int npair = (a.n + 1) >> 1;
  const size_t ld2 = (size_t)a.ld >> 1;  // row stride in pairs (ld is even)
  const int lane = threadIdx.x % kRhsPairs, grp = threadIdx.x / kRhsPairs;
  const int chunk = (a.Eact + kRhsGroups - 1) / kRhsGroups;
  const int j0 = grp * chunk, j1 = min(a.Eact, j0 + chunk);
  for (int base = blockIdx.x * kRhsPairs; base < npair; base += gridDim.x * kRhsPairs) {
    const int pp = base + lane;
    const int i = 2 * pp;
    const bool in = pp < npair;
    const bool two = i + 1 < a.n;
    double sx = 0.0, sy = 0.0;
    if (in && j1 > j0) {
      const double dx = a.u1[i] - a.u2[i];
      const double dy = two ? a.u1[i + 1] - a.u2[i + 1] : 0.0;
      double2* G = reinterpret_cast<double2*>(a.Gm + i);
      for (int j = j0; j < j1; j += kRhsU) {
        double2 g[kRhsU];
#pragma unroll
        for (int u = 0; u < kRhsU; ++u)
          if (j + u < j1) g[u] = G[(j + u) * ld2];
#pragma unroll
        for (int u = 0; u < kRhsU; ++u) {
          if (j + u < j1) {
            const double e = s_eps[j + u], c = s_cw[j + u];
            g[u].x = e * fma(c, dx, g[u].x);
            g[u].y = e * fma(c, dy, g[u].y);
            G[(j + u) * ld2] = g[u];
            sx += g[u].x;
            sy += g[u].y;
          }
        }
      }
    }
    s_part[threadIdx.x] = make_double2(sx, sy);
    __syncthreads();
    if (grp == 0 && in) {
      for (int q = 1; q < kRhsGroups; ++q) {
        const double2 v = s_part[q * kRhsPairs + lane];
        sx += v.x;
        sy += v.y;
      }
      for (int h = 0; h < (two ? 2 : 1); ++h) {
        const int ii = i + h;
        double f;
        if (a.f_m) {
          f = a.f_m[ii];
        } else {
          f = 0.0;
          for (int q = 0; q < a.rank; ++q) f += a.Gr[q] * a.F[(size_t)q * a.n + ii];
        }
        const double bi = a.ahat * a.u1[ii] - (h ? sy : sx) + f;
        a.b[ii] = bi;
        if (a.rhs_copy) a.rhs_copy[ii] = bi;
        double k;
        if (a.kap_m) k = a.kap_m[ii];
        else k = a.kap0[ii] + (a.kap1 ? a.theta * a.kap1[ii] : 0.0);
        a.kappa64[ii] = k;
        a.kappa32[ii] = (float)k;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------ direct history (DIDS) and RHS
// b = sum_{k<m} w_k u^k + f^m (Eq. (4.1): w_0 = a_1/Gamma(1-gamma),
// w_k = (a_{k+1} - a_k)/Gamma(1-gamma)), from every stored level.  Same
// block shape as k_rhs: 64 entry pairs x 4 row groups, 16-byte loads of the
// history rows (streamed: each is read once per level, and the level solve's
// vectors should keep L2), kDirU rows in flight per thread; the weights are
// staged in shared memory kDirChunk at a time; the groups' partial sums are
// added in a fixed order.  One FP64 FMA per 8 bytes read.
constexpr int kDirU = 8;
constexpr int kDirChunk = 2048;

__global__ void __launch_bounds__(kThreads) k_rhs_direct(RhsArgs a) {
  extern __shared__ double sh[];
  double* s_w = sh;
  double2* s_part = reinterpret_cast<double2*>(sh + kDirChunk);  // 16-byte aligned
  const int npair = (a.n + 1) >> 1;
  const size_t ld2 = (size_t)a.ld >> 1;
  const int lane = threadIdx.x % kRhsPairs, grp = threadIdx.x / kRhsPairs;
  for (int base = blockIdx.x * kRhsPairs; base < npair; base += gridDim.x * kRhsPairs) {
    const int pp = base + lane;
    const int i = 2 * pp;
    const bool in = pp < npair;
    const bool two = i + 1 < a.n;
    double sx = 0.0, sy = 0.0;
    for (int k0 = 0; k0 < a.m_hist; k0 += kDirChunk) {
      const int kn = min(kDirChunk, a.m_hist - k0);
      __syncthreads();  // the previous chunk's weights are no longer read
      for (int q = threadIdx.x; q < kn; q += blockDim.x) s_w[q] = a.w_dir[k0 + q];
      __syncthreads();
      const int chunk = (kn + kRhsGroups - 1) / kRhsGroups;
      const int j0 = grp * chunk, j1 = min(kn, j0 + chunk);
      if (!in) continue;
      const double2* Ub = reinterpret_cast<const double2*>(a.U_hist + i) + (size_t)k0 * ld2;
      for (int j = j0; j < j1; j += kDirU) {
        double2 g[kDirU];
#pragma unroll
        for (int u = 0; u < kDirU; ++u)
          if (j + u < j1) g[u] = __ldcs(Ub + (size_t)(j + u) * ld2);
#pragma unroll
        for (int u = 0; u < kDirU; ++u) {
          if (j + u < j1) {
            const double w = s_w[j + u];
            sx = fma(w, g[u].x, sx);
            sy = fma(w, g[u].y, sy);
          }
        }
      }
    }
    s_part[threadIdx.x] = make_double2(sx, sy);
    __syncthreads();
    if (grp == 0 && in) {
      for (int q = 1; q < kRhsGroups; ++q) {
        const double2 v = s_part[q * kRhsPairs + lane];
        sx += v.x;
        sy += v.y;
      }
      for (int h = 0; h < (two ? 2 : 1); ++h) {
        const int ii = i + h;
        double f;
        if (a.f_m) {
          f = a.f_m[ii];
        } else {
          f = 0.0;
          for (int q = 0; q < a.rank; ++q) f += a.Gr[q] * a.F[(size_t)q * a.n + ii];
        }
        const double bi = (h ? sy : sx) + f;
        a.b[ii] = bi;
        if (a.rhs_copy) a.rhs_copy[ii] = bi;
        double k;
        if (a.kap_m) k = a.kap_m[ii];
        else k = a.kap0[ii] + (a.kap1 ? a.theta * a.kap1[ii] : 0.0);
        a.kappa64[ii] = k;
        a.kappa32[ii] = (float)k;
      }
    }
    __syncthreads();
  }
}

__global__ void k_convert(const double* in, double* o64, float* o32, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double v = in[i];
    o64[i] = v;
    o32[i] = (float)v;
  }
}

// ------------------------------------------------------------- launchers
// The dynamic shared-memory limit of the cooperative kernels only ever grows,
// so a context set up earlier with a larger plan can still launch.
static size_t g_smem_limit = 0;

static cudaError_t set_attrs(size_t smem) {
  cudaError_t e = cudaSuccess;
  if (smem <= g_smem_limit) return e;
  const void* ks[] = {level64_kernel(2, 0), level64_kernel(4, 0), level32_kernel(2, 0),
                      level32_kernel(4, 0), levelds_kernel(2, 0), levelds_kernel(4, 0),
                      level64_kernel(2, 1), level64_kernel(4, 1), level32_kernel(2, 1),
                      level32_kernel(4, 1), levelds_kernel(2, 1), levelds_kernel(4, 1),
                      (const void*)k_apply64, (const void*)k_apply32, (const void*)k_apply_ds,
                      level_adj_kernel(0), level_adj_kernel(1), precond_ds_kernel(2), precond_ds_kernel(4)};
  for (const void* k : ks) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  g_smem_limit = smem;
  return e;
}

int coop_blocks_per_sm(size_t smem) {
  if (set_attrs(smem) != cudaSuccess) return 0;
  int best = 1 << 30;
  const void* ks[] = {level64_kernel(2, 0), level64_kernel(4, 0), level32_kernel(2, 0),
                      level32_kernel(4, 0), levelds_kernel(2, 0), levelds_kernel(4, 0),
                      level64_kernel(2, 1), level64_kernel(4, 1), level32_kernel(2, 1),
                      level32_kernel(4, 1), levelds_kernel(2, 1), levelds_kernel(4, 1),
                      (const void*)k_apply64, (const void*)k_apply32, (const void*)k_apply_ds,
                      level_adj_kernel(0), level_adj_kernel(1), precond_ds_kernel(2), precond_ds_kernel(4)};
  for (const void* k : ks) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kThreads, smem) != cudaSuccess) return 0;
    best = nb < best ? nb : best;
  }
  return best;
}

cudaError_t launch_rhs(const RhsArgs& a, cudaStream_t s) {
  const int npair = (a.n + 1) / 2;
  int grid = (npair + kRhsPairs - 1) / kRhsPairs;
  if (grid < 1) grid = 1;
  const size_t smem = (2 * (size_t)(a.Eact > 0 ? a.Eact : 1) + 1) * sizeof(double) +
                      kThreads * sizeof(double2);
  k_rhs<<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rhs_direct(const RhsArgs& a, cudaStream_t s) {
  const int npair = (a.n + 1) / 2;
  int grid = (npair + kRhsPairs - 1) / kRhsPairs;
  if (grid < 1) grid = 1;
  const size_t smem = kDirChunk * sizeof(double) + kThreads * sizeof(double2);
  k_rhs_direct<<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_convert(const double* in, double* o64, float* o32, int n, cudaStream_t s) {
  int grid = (n + kThreads - 1) / kThreads;
  k_convert<<<grid < 1 ? 1 : grid, kThreads, 0, s>>>(in, o64, o32, n);
  return cudaGetLastError();
}

// With TSFDE_KRYLOV_AUTO (a.kauto set) both method kernels are launched;
// the one not chosen for the level returns before any work.  A
// double-single level with a preconditioner first runs k_precond_ds.
cudaError_t launch_level(const LevelArgs& a0, int precision, cudaStream_t s) {
  size_t smem = plan_smem_bytes(a0.P);
  const bool kp2 = kp_fits(a0.P, 2);
  const int kp = kp2 ? 2 : 4;
  LevelArgs a = a0;
  void* args[] = {(void*)&a};
  if (precision == TSFDE_MIXED_DS && a.precond && a.pre_status) {
    a.prebuilt = 1;
    cudaError_t e = cudaMemsetAsync(a.P.bar, 0, sizeof(GridBarrier), s);
    if (e == cudaSuccess)
      e = cudaLaunchCooperativeKernel(precond_ds_kernel(kp), dim3(a.P.G), dim3(kThreads), args, smem, s);
    if (e != cudaSuccess) return e;
  }
  const bool autok = a.krylov == TSFDE_KRYLOV_AUTO && a.kauto;
  for (int pcg = 0; pcg < 2; ++pcg) {
    if (!autok && pcg != (a.krylov == TSFDE_KRYLOV_PCG ? 1 : 0)) continue;
    cudaError_t e = cudaMemsetAsync(a.P.bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    const void* k = precision == TSFDE_MIXED_DS ? levelds_kernel(kp, pcg)
                    : precision == TSFDE_MIXED  ? level32_kernel(kp, pcg)
                                                : level64_kernel(kp, pcg);
    e = cudaLaunchCooperativeKernel(k, dim3(a.P.G), dim3(kThreads), args, smem, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_adj_rhs(const AdjRhsArgs& a, cudaStream_t s) {
  int grid = (a.n + kThreads - 1) / kThreads;
  if (grid < 1) grid = 1;
  const size_t smem = 3 * (size_t)(a.Eact > 0 ? a.Eact : 1) * sizeof(double);
  k_adj_rhs<<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_level_adj(const LevelArgs& a, const AdjGradArgs& g, cudaStream_t s) {
  size_t smem = plan_smem_bytes(a.P);
  cudaError_t e = cudaMemsetAsync(a.P.bar, 0, sizeof(GridBarrier), s);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&a, (void*)&g};
  const int pcg = a.krylov == TSFDE_KRYLOV_PCG ? 1 : 0;
  return cudaLaunchCooperativeKernel(level_adj_kernel(pcg), dim3(a.P.G), dim3(kThreads), args, smem, s);
}

cudaError_t launch_apply(const ApplyArgs& a, int precision, cudaStream_t s) {
  size_t smem = plan_smem_bytes(a.P);
  cudaError_t e = cudaMemsetAsync(a.P.bar, 0, sizeof(GridBarrier), s);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&a};
  const void* k = precision == TSFDE_MIXED_DS ? (const void*)k_apply_ds
                  : precision == TSFDE_MIXED  ? (const void*)k_apply32
                                              : (const void*)k_apply64;
  return cudaLaunchCooperativeKernel(k, dim3(a.P.G), dim3(kThreads), args, smem, s);
}

}  // namespace tsfde

// =====================================================================
// Toeplitz product without any device allocation.
//
// For callers that cannot call cudaMalloc themselves: code running inside
// a pooled-memory framework that forbids raw device allocations, or a host
// thread that must not trigger allocator synchronisation.  Every work
// buffer and table lives in the one fixed-size array below, which each GPU
// that loads this library holds until the process exits.  The kernel builds
// the twiddles, the IFL symbol of Eq. (3.16x) and its circulant-embedding
// spectrum itself, then applies the product; nothing persists between calls
// except the array's contents.
// =====================================================================
namespace tsfde {

constexpr int kStaticMaxN = 16383;   // largest n accepted
constexpr int kStaticMaxL = 32768;   // embedding length for kStaticMaxN
constexpr int kStaticMaxG = 1024;    // largest cooperative grid
// layout (bytes, each block 256-aligned): barrier | partials | status |
// tw64 | tw32 | sym | sig | rho | S1 | S2
constexpr size_t kSA_bar = 0;
constexpr size_t kSA_part = 256;
constexpr size_t kSA_status = kSA_part + sizeof(double) * 2 * kSlots * kStaticMaxG;
constexpr size_t kSA_tw64 = kSA_status + 256;
constexpr size_t kSA_tw32 = kSA_tw64 + sizeof(double2) * kStaticMaxL;
constexpr size_t kSA_sym = kSA_tw32 + sizeof(float2) * kStaticMaxL;
constexpr size_t kSA_sig = kSA_sym + sizeof(double) * (kStaticMaxN + 1);
constexpr size_t kSA_rho = kSA_sig + sizeof(double) * (kStaticMaxL / 2) + 256;
constexpr size_t kSA_S1 = kSA_rho + sizeof(double2) * (kStaticMaxL / 2);
constexpr size_t kSA_S2 = kSA_S1 + sizeof(double2) * (kStaticMaxL / 2);
constexpr size_t kStaticBytes = kSA_S2 + sizeof(double2) * (kStaticMaxL / 2);

static __device__ __align__(256) unsigned char g_toeplitz_scratch[kStaticBytes];

struct StaticApplyArgs {
  DevPlan P;
  double alpha, mu, kappa_mu, C;  // C = c_{1,alpha} / (nu h^alpha)
  double* sym;
  const double* v;
  double* y;
  int* status;
};

__device__ double static_gap_pow(double k, double nu) {
  if (k == 1.0) return pow(2.0, nu);
  return pow(k, nu) * (expm1(nu * log1p(1.0 / k)) - expm1(nu * log1p(-1.0 / k)));
}

__global__ void __launch_bounds__(kThreads, 2) k_apply_static(StaticApplyArgs A) {
  grid_epoch_init();
  const DevPlan& P = A.P;
  const int n = P.n, L = P.L;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gstr = gridDim.x * blockDim.x;
  const double nu = A.mu - A.alpha;
  const int N = n + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* red0 = reinterpret_cast<double*>(smem_raw);
  // twiddles W_L^k and off-diagonal symbol entries; partial sums of the
  // diagonal's long sum (Eq. (3.16x))
  double2* tw64 = const_cast<double2*>(P.twL64);
  float2* tw32 = const_cast<float2*>(P.twL32);
  double acc = 0.0;
  for (int k = gtid; k < L; k += gstr) {
    double s, c;
    sincospi(-2.0 * (double)k / (double)L, &s, &c);
    tw64[k] = make_double2(c, s);
    tw32[k] = make_float2((float)c, (float)s);
  }
  for (int k = gtid; k < n; k += gstr) {
    if (k == 1) A.sym[1] = -0.5 * A.C * (pow(2.0, nu) + A.kappa_mu - 1.0);
    if (k >= 2) A.sym[k] = -0.5 * A.C * static_gap_pow((double)k, nu) * pow((double)k, -A.mu);
  }
  for (int q = 2 + gtid; q <= N - 1; q += gstr) {
    const double Q = (double)q;
    acc += static_gap_pow(Q, nu) * pow(Q, -A.mu);
  }
  put_partial(P, SL_KAP, block_sum(acc, red0));
  double big;
  if (!gsync_sum(P, red0, SL_KAP, big)) { if (blockIdx.x == 0 && threadIdx.x == 0) *A.status = TSFDE_ETIMEOUT; return; }
  if (gtid == 0) {
    const double Nd = (double)N;
    const double lastN = pow(Nd, nu - A.mu) * (-expm1(nu * log1p(-1.0 / Nd)));
    A.sym[0] = A.C * (big + lastN + (pow(2.0, nu) + A.kappa_mu - 1.0) +
                      2.0 * nu / (A.alpha * pow(Nd, A.alpha)));
  }
  if (!gsync(P, red0)) { if (blockIdx.x == 0 && threadIdx.x == 0) *A.status = TSFDE_ETIMEOUT; return; }
  SmemAll S = smem_setup(P, false);  // the barrier epoch runs on from grid_epoch_init
  // spectrum of the even embedding of the symbol -> (sigma, rho) tables
  const double* sym = A.sym;
  auto proE = [&](int i) -> double {
    if (i < n) return sym[i];
    const int k = L - i;
    return (k < n) ? sym[k] : 0.0;
  };
  passA_real<double, true>(P, S.d, L, proE);
  if (!gsync(P, S.d.red)) goto fail;
  passB<double, MID_SPEC>(P, S.d, nullptr, nullptr, const_cast<double*>(P.saT64),
                          const_cast<double*>(P.sbT64), nullptr);
  if (!gsync(P, S.d.red)) goto fail;
  {
    auto pro = [&](int i) -> double { return A.v[i]; };
    passA_real<double, false>(P, S.d, n, pro);
  }
  if (!gsync(P, S.d.red)) goto fail;
  passB<double, MID_APPLY>(P, S.d, P.saT64, P.sbT64, nullptr, nullptr, nullptr);
  if (!gsync(P, S.d.red)) goto fail;
  {
    auto epi = [&](int i, double yv) -> double { A.y[i] = yv; return 0.0; };
    passCA_real<double, false>(P, S.d, epi);
  }
  if (!gsync(P, S.d.red)) goto fail;
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.status = TSFDE_OK;
  return;
fail:
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.status = TSFDE_ETIMEOUT;
}

// Device address of g_toeplitz_scratch, looked up once per device (with that
// device current) on the first call made on it.
static unsigned char* g_scratch_addr[64];
static int g_scratch_ready[64];

static int static_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= 64) return TSFDE_ENOTSUP;
  if (!__atomic_load_n(&g_scratch_ready[dev], __ATOMIC_ACQUIRE)) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_toeplitz_scratch);
    if (e != cudaSuccess) {
      std::fprintf(stderr, "tsfde_toeplitz_apply_static: cudaGetSymbolAddress failed: %s\n",
                   cudaGetErrorString(e));
      return TSFDE_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    __atomic_store_n(&g_scratch_ready[dev], 1, __ATOMIC_RELEASE);
  }
  *out = g_scratch_addr[dev];
  return TSFDE_OK;
}

static Geo static_geo(int Nfft) {
  Geo g{};
  int lg = 0;
  while ((1 << lg) < Nfft) ++lg;
  g.Nfft = Nfft;
  g.lgN1 = (lg + 1) / 2;
  g.N1 = 1 << g.lgN1;
  g.lgN2 = lg - g.lgN1;
  g.N2 = 1 << g.lgN2;
  g.lgct64 = 0;
  g.lgct32 = 0;
  return g;
}

}  // namespace tsfde

extern "C" int tsfde_toeplitz_apply_static(double alpha, double mu, int kappa_mu, double l,
                                           int64_t n, const double* v, double* y, void* stream) {
  using namespace tsfde;
  if (!v || !y) return TSFDE_EINVAL;
  if (!(alpha > 0.0 && alpha < 2.0) || !(l > 0.0) || n < 1) return TSFDE_EINVAL;
  if (mu <= 0.0) mu = 1.0 + 0.5 * alpha;
  if (!(mu > alpha && mu <= 2.0)) return TSFDE_EINVAL;
  if (kappa_mu <= 0) kappa_mu = (mu == 2.0) ? 2 : 1;
  if (n > kStaticMaxN) {
    std::fprintf(stderr,
                 "tsfde_toeplitz_apply_static: n = %lld exceeds the fixed scratch capacity "
                 "n <= %d; use tsfde_toeplitz_apply on a context instead\n",
                 (long long)n, kStaticMaxN);
    return TSFDE_ENOTSUP;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return TSFDE_ECUDA;
  unsigned char* base = nullptr;
  int st = static_scratch(dev, &base);
  if (st != TSFDE_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  DevPlan P{};
  int L = 8;
  while (L < 2 * n - 1) L *= 2;
  P.n = (int)n;
  P.L = L;
  P.Nc = L / 2;
  P.gr = static_geo(P.Nc);
  P.gc = static_geo(P.L);
  P.T = P.gr.N1 > P.gr.N2 ? P.gr.N1 : P.gr.N2;
  P.W = (P.gr.N1 << P.gr.lgct64) > 2 * P.gr.N2 ? (P.gr.N1 << P.gr.lgct64) : 2 * P.gr.N2;
  P.timeout = 2000000000LL;
  P.bar = reinterpret_cast<GridBarrier*>(base + kSA_bar);
  P.part = reinterpret_cast<double*>(base + kSA_part);
  P.twL64 = reinterpret_cast<const double2*>(base + kSA_tw64);
  P.twL32 = reinterpret_cast<const float2*>(base + kSA_tw32);
  P.saT64 = reinterpret_cast<const double*>(base + kSA_sig);
  P.sbT64 = reinterpret_cast<const double*>(base + kSA_rho);
  P.S1 = reinterpret_cast<double2*>(base + kSA_S1);
  P.S2 = reinterpret_cast<double2*>(base + kSA_S2);

  const size_t smem = plan_smem_bytes(P);
  int nsm = 0, bps = 0;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_apply_static, kThreads, smem)) != cudaSuccess)
    return TSFDE_ECUDA;
  if (bps < 1) return TSFDE_ECUDA;
  int items = (P.gr.N2 >> P.gr.lgct64);
  if ((P.gr.N1 >> 1) + 1 > items) items = (P.gr.N1 >> 1) + 1;
  int G = nsm * (bps < 2 ? bps : 2);
  if (G > items) G = items;
  if (G > kStaticMaxG) G = kStaticMaxG;
  if (G < 1) G = 1;
  P.G = G;

  StaticApplyArgs A{};
  A.P = P;
  A.alpha = alpha;
  A.mu = mu;
  A.kappa_mu = (double)kappa_mu;
  const double nu = mu - alpha;
  const double h = 2.0 * l / (double)(n + 1);
  const double pi = 3.14159265358979323846;
  const double c1 = std::pow(2.0, alpha - 1.0) * alpha * std::tgamma(0.5 * (alpha + 1.0)) /
                    (std::sqrt(pi) * std::tgamma(1.0 - 0.5 * alpha));
  A.C = c1 / (nu * std::pow(h, alpha));
  A.sym = reinterpret_cast<double*>(base + kSA_sym);
  A.v = v;
  A.y = y;
  A.status = reinterpret_cast<int*>(base + kSA_status);
  // the barrier counters and the status word must start at zero/unknown
  if ((e = cudaMemsetAsync(P.bar, 0, sizeof(GridBarrier), s)) != cudaSuccess) return TSFDE_ECUDA;
  if ((e = cudaMemsetAsync(A.status, 0xff, sizeof(int), s)) != cudaSuccess) return TSFDE_ECUDA;
  void* args[] = {(void*)&A};
  e = cudaLaunchCooperativeKernel((const void*)k_apply_static, dim3(G), dim3(kThreads), args, smem, s);
  if (e != cudaSuccess) return TSFDE_ECUDA;
  int status = -1;
  if ((e = cudaMemcpyAsync(&status, A.status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return TSFDE_ECUDA;
  return status < 0 ? (int)TSFDE_ECUDA : status;
}
