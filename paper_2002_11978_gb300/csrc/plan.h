// plan.h -- plain-data structures shared by the host launcher code and the
// CUDA kernels (no CUDA-only types beyond vector types).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tsfde {

// Double-single number: the unevaluated sum hi + lo of two FP32 values
// (|lo| <= ulp(hi)/2), about 48 significant bits; device arithmetic in
// dsf.cuh.  Conversions from FP64 round hi to nearest and keep the FP32
// rounding of the remainder.
struct __align__(8) dsf {
  float hi, lo;
  dsf() = default;
  __host__ __device__ constexpr dsf(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dsf(int i) : hi((float)i), lo(0.0f) {}  // |i| < 2^24: exact
  __host__ __device__ explicit dsf(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};
struct __align__(16) dsf2 { dsf x, y; };

// Bounded grid barrier state (cleared by the host before each cooperative
// launch); see grid_sync_red in dev.cuh.
struct GridBarrier {
  unsigned int count;     // arrivals, monotonic within one launch
  int err;                // set once any CTA gave up waiting
  unsigned int pad0[30];
};

// One factorisation Nfft = N1 * N2 of a power-of-two transform, driven by
// three passes: column FFTs of length N1 over tiles of 2^lgct columns,
// row FFTs of length N2 (rows k1 and N1-k1 together), column inverse FFTs.
struct Geo {
  int Nfft, N1, N2, lgN1, lgN2;
  int lgct64, lgct32;  // log2 columns per tile for double / float data
};

// Cluster engine: one thread-block cluster of Q CTAs holds a length-Nc
// complex FFT (geometry gr) in distributed shared memory.  CTA q owns the
// columns j2 in [q cQ, (q+1) cQ) and the vector entries i with
// (i/2) mod N2 in that range; for the row pass it owns the row units
// [q U, (q+1) U), unit 0 = rows {0, N1/2}, unit u > 0 = rows {u, N1-u}, held
// as row slots 2(u - qU) and 2(u - qU) + 1.
struct CGeo {
  int Q, lgQ;    // CTAs of the cluster
  int cQ, lgcQ;  // columns per CTA, N2 / Q
  int U, lgU;    // row units per CTA, N1 / (2Q)
  int Bq, lgBq;  // row slots per CTA, 2U
  int nbuf;      // complex elements per CTA, Nc / Q
  int cap;       // staging capacity, nbuf + N1
  int T1;        // stage twiddle table W_{T1}^k, T1 = N1 >= N2
  int LT, lgLT;  // low twiddle table W_L^l, l < LT = L / T1
  int G;         // CTAs of the cluster-engine launch (a multiple of Q)
};

// One transform geometry on the cluster, held in registers by every pass.
struct CeGeo {
  int n;           // vector entries the epilogues see
  int L;           // base of the twiddle tables W_L
  int tws;         // column-twiddle stride L / Nfft
  int N1, N2, lgN1, lgN2;
  int Q, cQ, lgcQ, U, lgU, Bq, lgBq, nbuf;
  int T1, LT, lgLT;  // tables: hi = W_{T1}^k (k < T1), lo = W_L^l (l < LT = L/T1)
  int q;           // this CTA's rank
};

// Shared-memory layout (bytes): C [capB] | S [capB] | R [nbufB] |
// FP64 tables (if has64) | FP32 tables | part [6 x kMaxQ doubles] | red [64]
// | context.  C and S hold nbuf elements plus the staging padding.
struct CeLay {
  int capB, nbufB;
  int T1, LT;
  int has64;
};

// Result of one Krylov solve.
struct SolveRes {
  int status;
  int iters;
  double relres;
};

// Everything a cooperative kernel needs to run the FIDS level solve.
struct DevPlan {
  int n;       // unknowns
  int L;       // circulant embedding length (power of two, >= 2n-1, >= 8)
  int Nc;      // L/2: complex size of the real-input transforms
  Geo gr;      // real-mode geometry, Nfft = Nc
  Geo gc;      // complex-mode geometry (Bluestein), Nfft = L
  int T;       // shared twiddle table size (>= every sub-FFT length)
  int W;       // work-buffer capacity per buffer, in double2 elements
  int G;       // CTAs of the cooperative grid
  long long timeout;  // barrier wait budget (SM cycles)
  GridBarrier* bar;
  double* part;       // [2][kSlots][G] per-CTA partial sums, by barrier parity
  const double2* twL64;  // W_L^k, k < L
  const float2* twL32;
  // Toeplitz symbol spectrum S (DFT_L of the even embedding), in the (k1,k2)
  // layout of gr and scaled by 1/Nc: sa = S_k / Nc, sb = S_{k'} / Nc with
  // k = k1 + N1 k2 and k' = Nc - k (k' = Nc for k = 0)
  const double* saT64; const double* sbT64;
  const float* saT32;  const float* sbT32;
  const double* lam;       // Strang eigenvalues (n)
  const double2* chirp64;  // e^{+pi i j^2/n}, j < n
  const float2* chirp32;
  const double2* Bh64;     // spectrum of the Bluestein kernel / L, (k1,k2) layout of gc
  const float2* Bh32;
  // per-level preconditioner spectrum, same format (written by the build)
  double* saG64; double* sbG64;
  float* saG32;  float* sbG32;
  double* g64; float* g32;  // first column of the circulant inverse (n)
  // double-single copies (mixed solves with the double-single inner solver;
  // NULL otherwise): twiddles, Toeplitz spectrum, per-level preconditioner
  // spectrum (written by k_precond_ds), and the Bluestein tables and
  // circulant-inverse column that build uses
  const dsf2* twLds;
  const dsf* saTds; const dsf* sbTds;
  dsf* saGds; dsf* sbGds;
  const dsf2* chirpds; const dsf2* Bhds; dsf* gds;
  double2* S1;  // work: Nfft complex (double capacity, reused as float2 / dsf2)
  double2* S2;
  CGeo cl;
  // (sa, sb) pairs in the cluster engine's row-pass order: entry
  // q nbuf + (k2 << lgBq) + slot for the row k1 held in slot `slot` of CTA q
  const float2* spT_cl;  // Toeplitz symbol
  float2* spG_cl;        // per-level preconditioner (written by the build)
};

enum { kSlots = 12 };

struct StepStat {
  int status;
  int iterations;
  int outer;
  int E_active;
  double rel_residual;
  int method;           // Krylov method that solved the level (0 BiCGSTAB, 1 PCG)
  int pad;
};

// Per-level Krylov choice (TSFDE_KRYLOV_AUTO), shared by the grid engine
// (one state per context) and the batched engine (one per instance).  After
// each level, the method that solved it records its device time, and the
// next level runs
//  - the other method if that has no sample yet, if its latest sample was
//    faster, or if this level failed (a failed level counts as infinitely
//    slow);
//  - else the same method, until a trial of the other is due: 8 r^2 levels
//    (8..64) after the other's latest sample, r = how many times slower it
//    was, times 2^k for k (at most 4) trials of it lost in a row.
// A lost trial sends the march back at once; a trial that wins clears its
// method's loss count and the march stays with it.
struct AutoRule {
  double t[2];      // device time (ns) of the latest level of each method
  long long at[2];  // level of that sample (0: none yet)
  int loss[2];      // trials of each method lost in a row
  int trial;        // method run as a trial at the current level, -1 none
  int pad;
};

__host__ __device__ inline void auto_rule_init(AutoRule& k) {
  k.t[0] = k.t[1] = 0.0;
  k.at[0] = k.at[1] = 0;
  k.loss[0] = k.loss[1] = 0;
  k.trial = -1;
  k.pad = 0;
}

// Records level m solved by method `me` (0 BiCGSTAB, 1 PCG) in dt ns
// (anything not below 1e300 for a failed level); returns the method of
// level m + 1.
__host__ __device__ inline int auto_rule_next(AutoRule& k, int me, long long m, double dt) {
  const int ot = 1 - me;
  const bool was_trial = k.trial == me;
  k.trial = -1;
  k.t[me] = dt;
  k.at[me] = m;
  if (k.at[ot] == 0) {
    k.trial = ot;
    return ot;
  }
  if (!(dt < 1e300) || !(k.t[ot] >= dt)) {
    if (was_trial) k.loss[me] += 1;
    return ot;
  }
  if (was_trial) k.loss[me] = 0;
  const double r = k.t[ot] / dt;
  double interval = 8.0 * r * r;
  interval = interval < 8.0 ? 8.0 : (interval > 64.0 ? 64.0 : interval);
  interval *= (double)(1 << (k.loss[ot] < 4 ? k.loss[ot] : 4));
  if ((double)(m + 1 - k.at[ot]) >= interval) {
    k.trial = ot;
    return ot;
  }
  return me;
}

// Per-level choice of the Krylov method (TSFDE_KRYLOV_AUTO).  Every level
// launches the BiCGSTAB and the PCG kernel; the one whose method is `choice`
// for level `for_level` solves it, the other returns at once.  Block 0 of
// the solving kernel then records the level's device time (globaltimer) for
// its method and picks the method of the next level by auto_rule_next.
// Cleared by the host at every reset (choice BiCGSTAB for level 1).
struct KrylovAuto {
  long long for_level;  // level the choice applies to
  int choice;           // 0 BiCGSTAB, 1 PCG
  int pad;
  AutoRule rule;
  long long used[2];    // levels solved by each method since the reset
};

// Krylov workspace of one precision.
template <typename R> struct KVecs {
  R *x, *r, *rh, *p, *v, *s, *t, *ph, *sh;
};

// Highest order of the extrapolated start of a level solve (LevelArgs.up).
constexpr int kMaxStartOrder = 4;

struct LevelArgs {
  DevPlan P;
  double ahat;        // a_m / Gamma(1-gamma)
  const double* b;    // right-hand side (n)
  const double* kappa64;  // kappa^m (n)
  const float* kappa32;
  double* u;          // solution (n)
  int precond;        // 1 = Strang
  double tol;         // FP64: recursive residual tol; mixed: correction tol
  int max_it;
  double inner_tol;
  int max_outer;
  int inner_max_it;
  KVecs<double> k64;
  KVecs<float> k32;
  KVecs<dsf> kds;     // double-single inner solver (TSFDE_MIXED_DS)
  dsf* kappads;       // kappa^m rounded to double-single (written by the level kernel)
  int krylov;         // TSFDE_KRYLOV_BICGSTAB or TSFDE_KRYLOV_PCG
  double* hinv64;     // PCG: 1/kappa^m in FP64 (n), FP32 and double-single (ld),
  float* hinv32;      //   written by the level kernel
  dsf* hinvds;
  double* r64;        // mixed: FP64 residual
  StepStat* stat;
  int probe;          // cluster engine: return at once (launch check)
  // double-single mixed solve: the level's preconditioner was built by
  // k_precond_ds just before (prebuilt = 1; tables in double-single and
  // FP64), which wrote its status to *pre_status
  int prebuilt;
  int* pre_status;
  const double* u_prev;   // warm start from u^{m-1} (NULL: x0 = 0)
  // with u_prev, an extrapolated start of order xorder (0: x0 = u^{m-1}):
  // x0 = sum_{j=0..xorder} xw[j] up[j], the polynomial through up[0..xorder]
  // evaluated at level m (Lagrange weights xw from the host).  up[j] =
  // u^{m-1-j} (up[0] = u_prev); up[xorder] may be the array u itself, each
  // entry read before it is overwritten.
  const double* up[kMaxStartOrder + 1];
  double xw[kMaxStartOrder + 1];
  int xorder;
  const StepStat* prev;   // mixed: the previous level's stats (NULL: none)
  int retry_mixed;        // mixed: refine even after a level finished in FP64
  KrylovAuto* kauto;      // TSFDE_KRYLOV_AUTO: method choice state (NULL: fixed method)
  long long m;            // level index (with kauto)
};

// One instance of the batched solve (device-resident descriptor).  All
// vectors are per-instance slices of pooled device arrays; FP32 / FP64
// Krylov vectors have an even length.
struct BInst {
  int n, E, ld;          // unknowns, SOE size, leading dimension of H (even)
  CeGeo gr, gc;          // real-input (Nfft = L/2) and complex (Nfft = L) geometry
  int tstride;           // twiddle stride: Lmax / L
  double kbar;           // mean of kappa (time independent)
  const double* phi;
  const double* kap64;
  const float* kap32;
  const double* hinv64;  // 1/kappa (PCG)
  const float* hinv32;
  const double* f;
  double* H;             // E x ld scaled SOE history
  double* u[4];          // rotating levels (an extrapolated start reads u^{m-1} .. u^{m-4})
  double* r64;           // FP64 residual (holds b at the start of a level)
  double* w;             // FP64 scratch (M e, preconditioner column g)
  KVecs<float> v32;
  KVecs<double> v64;
  const double* ahat;    // M+1
  const double* eps;     // (M+1) x E
  const double* cw;      // (M+1) x E
  const int* Eact;       // M+1
  const double* lam;     // Strang eigenvalues (n)
  const double2* chirp;  // e^{+pi i j^2/n}, j < n
  const double2* Bh;     // Bluestein kernel spectrum / L, row-pass order of gc
  const double2* spT64;  // Toeplitz spectrum pairs, row-pass order of gr
  const float2* spT32;
  double2* spG64;        // preconditioner spectrum pairs (per level)
  float2* spG32;
  double* u_out;         // caller's u^M (set by each solve)
  StepStat* stat;        // totals: iterations, outer (sum of |outer|),
                         // E_active = FP64-finished levels, worst relres
};

struct BatchArgs {
  BInst* inst;
  int count;
  int M;
  int* next;             // instance counter (zeroed before the launch)
  int precision;         // TSFDE_FP64 or TSFDE_MIXED
  int precond;
  double tol, inner_tol;
  int max_it, max_outer, inner_max_it;
  int warm;              // start each level from u^{m-1}
  int krylov;            // TSFDE_KRYLOV_BICGSTAB or TSFDE_KRYLOV_PCG
  const double2* tw64;   // W_Lmax^k
  const float2* tw32;
  CeLay lay;             // shared-memory layout (sized for the largest instance)
};

struct RhsArgs {
  int n, ld, Eact;
  double ahat;
  double* Gm;              // E x ld scaled history w_j H_j / Gamma(1-gamma)
  const double* eps;       // e^{-s_j tau_m}, Eact entries
  const double* cw;        // w_j beta_{j,m-1} / Gamma(1-gamma)
  const double* u1;        // u^{m-1}
  const double* u2;        // u^{m-2}
  const double* kap_m;     // explicit kappa^m or NULL
  const double* kap0;
  const double* kap1;      // NULL if kappa has no time factor
  double theta;
  const double* f_m;       // explicit f^m or NULL
  const double* F;         // rank x n source factors
  int rank;
  double Gr[4];
  double* b;
  double* rhs_copy;        // NULL or user buffer
  double* kappa64;
  float* kappa32;
  // direct history (DIDS, Eq. (4.1)); used by k_rhs_direct only
  const double* U_hist;    // (m_hist rows) x ld: u^0 .. u^{m-1}
  const double* w_dir;     // m_hist weights: b = sum_k w_k u^k + f^m
  int m_hist;
};

// Adjoint sweep (reverse time): the right-hand side g^m of the transposed
// level system from lambda^{m+1} through the reversed SOE recurrence
//   Y_j <- eps_{j,m+1} (lambda^{m+1} + Y_j),
//   g^m = ahat_{m+1} lambda^{m+1} - sum_j (c_{j,m+1} Y_j^new - c_{j,m+2} Y_j^old)
// (c_{j,k} = w_j beta_{j,k-1} / Gamma(1-gamma), the forward coefficients).
struct AdjRhsArgs {
  int n, ld, Eact;      // Eact = active exponentials at level m+1
  double ahat1;         // ahat_{m+1}
  double* Y;            // E x ld reversed history
  const double* eps1;   // eps_{j,m+1}
  const double* c1;     // c_{j,m+1}
  const double* c2;     // c_{j,m+2}, NULL when m+2 > M
  const double* lam1;   // lambda^{m+1}
  double* g;
};

// Gradient terms of one adjoint level: grad_kappa -= lambda .* (A u^m),
// grad_f += lambda, after the transposed solve of that level.
struct AdjGradArgs {
  const double* um;     // forward solution u^m
  double* grad_kappa;
  double* grad_f;
};

struct ApplyArgs {
  DevPlan P;
  int kind;         // 0: y = a v + kappa .* (A v)  (kappa NULL -> 1)
                    // 1: z = P^{-1} v (builds the preconditioner first)
  double a, kbar;
  const double* kappa;
  const double* v;
  double* y;
  int status_slot;
  int* status;
};

// launchers (kernels.cu)
cudaError_t launch_rhs(const RhsArgs& a, cudaStream_t s);
// DIDS right-hand side from the stored levels (a.U_hist, a.w_dir, a.m_hist)
cudaError_t launch_rhs_direct(const RhsArgs& a, cudaStream_t s);
// precision: TSFDE_FP64, TSFDE_MIXED (FP32 inner) or TSFDE_MIXED_DS
cudaError_t launch_level(const LevelArgs& a, int precision, cudaStream_t s);
// level kernels by prefetch depth kp (2 or 4) and Krylov method (pcg = 1:
// PCG on the symmetrised system, 0: BiCGSTAB): level64*.cu, level32*.cu,
// levelds*.cu
const void* level64_kernel(int kp, int pcg);
const void* level32_kernel(int kp, int pcg);
const void* levelds_kernel(int kp, int pcg);
const void* precond_ds_kernel(int kp);
const void* level_adj_kernel(int pcg);
// cluster engine (cluster.cu): mixed level solve with the FP32 inner solves
// on one thread-block cluster; a.P.G must equal a.P.cl.G.
cudaError_t launch_level_cluster(const LevelArgs& a, cudaStream_t s);
// Fills P.cl for P's real geometry; false if the sizes do not allow it.
bool cluster_geometry(DevPlan& P);
size_t cluster_smem_bytes(const DevPlan& P);
// Largest cluster-engine grid (CTAs) that can be co-resident with `smem`
// dynamic shared bytes per CTA, 0 if the engine cannot be launched.
int cluster_max_grid(const DevPlan& P, size_t smem);
// precision: TSFDE_FP64, TSFDE_MIXED (FP32 product) or TSFDE_MIXED_DS
// (double-single product; a preconditioner is built in FP64 and rounded)
cudaError_t launch_apply(const ApplyArgs& a, int precision, cudaStream_t s);
// batched engine (batch.cu): one persistent launch of clusters of Q CTAs,
// each marching whole instances through all M levels
size_t batch_smem_bytes(const CeLay& lay);
int batch_max_clusters(int Q, size_t smem);
cudaError_t launch_batch(const BatchArgs& a, int Q, int clusters, cudaStream_t s);
// adjoint: reversed SOE right-hand side; FP64 transposed level solve with
// the gradient accumulation fused behind it
cudaError_t launch_adj_rhs(const AdjRhsArgs& a, cudaStream_t s);
cudaError_t launch_level_adj(const LevelArgs& a, const AdjGradArgs& g, cudaStream_t s);
// out64 = in, out32 = (float) in
cudaError_t launch_convert(const double* in, double* out64, float* out32, int n, cudaStream_t s);
// CTAs per SM that every cooperative kernel can co-schedule with `smem`
// dynamic shared bytes; 0 on failure.
int coop_blocks_per_sm(size_t smem);
size_t plan_smem_bytes(const DevPlan& P);

}  // namespace tsfde
