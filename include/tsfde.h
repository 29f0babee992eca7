/*
 * tsfde.h -- C ABI of the GB300 (sm_103a) implementation of the fast implicit
 * difference scheme (FIDS) of Gu, Sun, Zhang and Zhao for the 1-D
 * time-space fractional diffusion equation with the integral fractional
 * Laplacian (arXiv 2002.11978):
 *
 *   C_0D_t^gamma u = -kappa(x,t) (-Delta)^{alpha/2} u + f   on (-l,l) x (0,T]
 *   u = 0 outside (-l,l),  u(x,0) = phi(x)                      (Eq. (1.1))
 *
 * Each time level m solves (Eq. (3.16gu))
 *   (a_m/Gamma(1-gamma) I + diag(kappa^m) A) u^m = b^m,
 * where A is the symmetric Toeplitz IFL matrix of Eq. (3.16x) and b^m is
 * built from the sum-of-exponentials history (Lemma 2.2, Eq. (lem2.3)), by
 * Strang-circulant-preconditioned BiCGSTAB (Sec. 4.1, Eq. (4.3); Sec. 5) or,
 * with tsfde_opts.krylov = TSFDE_KRYLOV_PCG, by preconditioned CG on the
 * equivalent symmetric positive definite system.
 *
 * Conventions for every entry point:
 *  - Return value: a tsfde_status (0 = TSFDE_OK).  No C++ exception crosses
 *    the ABI.  tsfde_strerror() gives a static message.
 *  - "dev" pointers are CUDA device pointers to contiguous IEEE doubles owned
 *    by the caller; they must stay valid until the call's work has completed
 *    on the context's stream.  "host" pointers are read during the call only.
 *  - All device work is enqueued on the stream given in tsfde_opts.stream
 *    (NULL = legacy default stream).  Calls that return per-call statistics
 *    through an info struct synchronise that stream; others are asynchronous.
 *  - A context owns all of its device workspaces; one context per stream.
 *    Nothing is global.  Contexts are not thread-safe.
 *  - n is the number of interior grid points (the paper's N - 1), so the
 *    mesh size is h = 2l/(n+1) and x_i = -l + i h, i = 1..n.
 */
#ifndef TSFDE_H
#define TSFDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tsfde_status {
  TSFDE_OK = 0,
  TSFDE_EINVAL = 1,      /* invalid argument (message names it)            */
  TSFDE_ENOMEM = 2,      /* device or host allocation failed               */
  TSFDE_ECUDA = 3,       /* a CUDA runtime call failed                     */
  TSFDE_ENOCONV = 4,     /* Krylov iteration cap reached                   */
  TSFDE_EBREAKDOWN = 5,  /* Krylov breakdown: BiCGSTAB rho, (r0,v) or (t,t)
                            = 0; PCG (p,Sp) or (r,z) not positive          */
  TSFDE_ETIMEOUT = 6,    /* a device-side grid barrier gave up waiting     */
  TSFDE_ESTATE = 7,      /* call not valid in the context's current state  */
  TSFDE_ENONFINITE = 8,  /* NaN or Inf met in a residual or scalar         */
  TSFDE_ENOTSUP = 9      /* option not supported by this build             */
} tsfde_status;

/* tsfde_opts.precision.  FP64: the Krylov solve (tsfde_opts.krylov) in FP64.
 * MIXED and MIXED_DS: FP64 iterative refinement (FP64 residual b - M u and
 * update) around an inner Krylov solve that runs in FP32 (MIXED) or in
 * double-single arithmetic
 * (MIXED_DS: every value an unevaluated sum of two FP32 numbers, about 48
 * significant bits, computed on the FP32 pipes).  FP32 products cannot
 * resolve a spectral range of ~1e8 (the IFL symbol at n ~ 1e5), so MIXED
 * needs more inner iterations and may finish levels in FP64; MIXED_DS
 * resolves it and converges like FP64 at FP32-pipe cost.  The
 * preconditioner is always built in FP64 and rounded. */
enum { TSFDE_FP64 = 0, TSFDE_MIXED = 1, TSFDE_MIXED_DS = 2 };
enum { TSFDE_STRANG = 0, TSFDE_PRECOND_NONE = 1 }; /* tsfde_opts.precond */
/* tsfde_opts.history: how the Caputo history term of the right-hand side is
 * formed.  SOE: the fast scheme FIDS (Eq. (3.16gu)), a sum-of-exponentials
 * recurrence over E exponentials, O(n E) per level.  DIRECT: the direct
 * scheme DIDS (Eq. (4.1)), the L1 sum over every earlier level, O(n m) per
 * level m; the context then keeps all M+1 levels on the device
 * ((M+1) x n doubles) and a table of the M(M+1)/2 direct weights. */
enum { TSFDE_HISTORY_SOE = 0, TSFDE_HISTORY_DIRECT = 1 };
/* tsfde_opts.krylov: the level solver.  BICGSTAB: the paper's
 * right-preconditioned BiCGSTAB on (a I + K A) x = b (Sec. 4.1, Sec. 5).
 * PCG: conjugate gradients on the equivalent symmetric positive definite
 * system (a K^{-1} + A) x = K^{-1} b (K = diag(kappa); A is SPD by the
 * proposition after Eq. (3.16x)), preconditioned by a/kbar I + s(A), the
 * Strang preconditioner of Eq. (4.3) up to a constant factor.  Sec. 4.2
 * proposes PCG for kappa independent of x; the symmetrisation extends it to
 * any kappa > 0.  One product with A and one with the preconditioner per
 * iteration instead of two of each; the stopping test is the same, on the
 * residual of the original system.  The mixed paths use it for their inner
 * solves and their FP64 finish, and tsfde_adjoint its transposed solves.
 * The batched solve runs it on its clusters (ce_pcg); the single-problem
 * cluster engine runs BiCGSTAB only. */
/* AUTO: each level of tsfde_step / tsfde_solve takes whichever of the two
 * is cheaper there, decided on the device from measured level times: the
 * method of the previous level, unless the other one was faster at its latest
 * sample, or a trial of the other one is due: 8 r^2 levels (8..64; r = how
 * many times slower it was) after its latest sample, doubled for each
 * trial of it lost in a row (at most 16 times).  The first level uses
 * BiCGSTAB, the second PCG.  PCG is weak where a K^{-1}
 * dominates (large a_m, the first levels of a graded mesh: its circulant
 * preconditioner cannot follow the variation of 1/kappa) and strong where A
 * dominates; BiCGSTAB the other way round.  Per-level stats report the
 * method used (tsfde_step_info.krylov).  tsfde_linear_solve takes BiCGSTAB
 * in an AUTO context.  Both methods reach the same stopping test, so the
 * results agree to the tolerance. */
enum { TSFDE_KRYLOV_BICGSTAB = 0, TSFDE_KRYLOV_PCG = 1, TSFDE_KRYLOV_AUTO = 2 };
/* tsfde_opts.engine: how a mixed level solve runs its FP32 inner solves.
 * GRID: spread over the whole cooperative grid (grid barriers between the
 * FFT passes).  CLUSTER: on one thread-block cluster of up to 16 CTAs that
 * keeps each FFT in distributed shared memory (cluster barriers), while the
 * grid runs the FP64 parts.  AUTO takes GRID for a single problem: at the
 * sizes where the cluster engine fits (n <= 2^17 - 1) one cluster of 16 SMs
 * has less FFT throughput than the whole grid loses to grid barriers.
 * FP64 level solves always use the grid. */
enum { TSFDE_ENGINE_AUTO = 0, TSFDE_ENGINE_GRID = 1, TSFDE_ENGINE_CLUSTER = 2 };

typedef struct tsfde_opts {
  double mu;            /* splitting parameter of Eq. (2.11), mu in (alpha,2];
                           <= 0 selects the paper's default 1 + alpha/2     */
  int kappa_mu;         /* 1 for mu < 2, 2 for mu = 2; 0 derives it from mu */
  double krylov_tol;    /* FP64 path: stop when ||r_k||_2/||r_0||_2 < tol
                           (recursive residual, x0 = 0, Sec. 5); mixed paths:
                           stop the FP64 refinement when the true FP64
                           residual satisfies ||b - M u|| <= tol ||b||, or
                           the last correction max|e| <= tol * max|u|, or a
                           sweep no longer halves the FP64 residual (it has
                           reached its rounding floor).  Default 1e-12      */
  int max_it;           /* Krylov iteration cap per solve (default 2000)    */
  int precision;        /* TSFDE_FP64 (default), TSFDE_MIXED or
                           TSFDE_MIXED_DS                                   */
  int precond;          /* TSFDE_STRANG (default) or TSFDE_PRECOND_NONE     */
  double inner_tol;     /* MIXED: FP32 inner relative tolerance (default
                           1e-2).  MIXED_DS ignores it and inner_max_it:
                           its first inner solve of a level stops at
                           100 tol ||b|| (near the double-single residual
                           floor), every later one asks for the whole
                           remaining reduction (to tol ||b|| / 2), each
                           within max_it iterations                         */
  int max_outer;        /* mixed: FP64 refinement cap (default 60)          */
  int inner_max_it;     /* MIXED: inner BiCGSTAB iterations per refinement
                           sweep (default 40).  The inner solve stops there
                           even short of inner_tol: at large n its FP32
                           products cannot resolve every residual, and the
                           FP64 refinement carries the accuracy.            */
  int soe_E;            /* > 0: use the caller's SOE table below instead of
                           building one (exponentials sorted ascending)     */
  const double* soe_s;  /* host, soe_E nodes s_j > 0                        */
  const double* soe_w;  /* host, soe_E weights w_j > 0                      */
  int profile;          /* 1: time every launch with CUDA events on the
                           context's stream (see tsfde_get_timing)          */
  long long barrier_timeout_cycles; /* device barrier wait budget in SM
                           clock cycles; 0 = default (about 2 s).  A tiny
                           value makes every barrier give up and the call
                           return TSFDE_ETIMEOUT: used to test that path.  */
  void* stream;         /* cudaStream_t; NULL = default stream              */
  int engine;           /* TSFDE_ENGINE_* (default AUTO); a MIXED context
                           asking for CLUSTER where it cannot run fails
                           tsfde_setup with TSFDE_ENOTSUP; FP64 and
                           MIXED_DS contexts ignore the field (grid only)   */
  int cluster_size;     /* batched solve: CTAs per thread-block cluster,
                           4, 8 or 16; 0 (default) picks the size that keeps
                           the most CTAs resident                           */
  int warm_start;       /* 1: start every level's solve from u^{m-1} and stop
                           at ||r|| < krylov_tol ||b^m|| (mixed: same
                           refinement rules); 2: the same stopping rule from
                           the cubic extrapolation in the level index,
                           x0 = 4 u^{m-1} - 6 u^{m-2} + 4 u^{m-3} - u^{m-4}
                           (lower orders at levels 1-3; the batched solve
                           too); 0 (default): x0 = 0 and the
                           residual relative to ||r_0|| = ||b^m|| (Sec. 5);
                           other values: TSFDE_EINVAL                       */
  int history;          /* TSFDE_HISTORY_SOE (default, FIDS) or
                           TSFDE_HISTORY_DIRECT (DIDS); the batched solve
                           accepts SOE only                                 */
  int krylov;           /* TSFDE_KRYLOV_BICGSTAB (default), TSFDE_KRYLOV_PCG
                           or TSFDE_KRYLOV_AUTO; in the batched solve AUTO
                           chooses per level within each instance's march */
  int ckpt_stride;      /* adjoint checkpoints: every ckpt_stride-th level of
                           the forward march (level 0 at each reset) keeps
                           u^{k-3} .. u^k and the SOE history, so that
                           tsfde_adjoint can run with u_all = NULL by
                           marching each segment again from its checkpoint.
                           -1: ceil(sqrt(M)); 0 (default): none.  Device
                           memory (M/stride + 1) (E + 4) n + stride n
                           doubles; SOE history only                        */
} tsfde_opts;

typedef struct tsfde_step_info {
  int64_t m;            /* time level just computed (1..M)                  */
  int status;           /* tsfde_status of this level                       */
  int iterations;       /* Krylov iterations (mixed: summed inner ones)     */
  int outer;            /* mixed: FP64 refinement sweeps (0 for FP64 path);
                           negative: the level was finished (or, after such
                           a level, solved directly) by the FP64 Krylov
                           solve                                            */
  int E_active;         /* exponentials still non-zero at this level        */
  double rel_residual;  /* FP64 path: recursive ||r||/||b||; mixed: last
                           computed FP64 ||b - M u||/||b||                  */
  int krylov;           /* method that solved the level: TSFDE_KRYLOV_BICGSTAB
                           or TSFDE_KRYLOV_PCG                              */
} tsfde_step_info;

typedef struct tsfde_solve_info {
  int status;           /* first non-OK level status, else TSFDE_OK          */
  int64_t failed_level; /* level of that status, 0 if none                  */
  int64_t levels;       /* levels computed by this call                     */
  int64_t iterations;   /* total Krylov iterations over those levels        */
  int min_iterations, max_iterations;
  int64_t outer;        /* total refinement sweeps (mixed)                  */
  double max_rel_residual;
  int E;                /* size of the SOE table                            */
  int64_t E_active_sum; /* sum over the levels of the active exponentials   */
  int64_t pcg_levels;   /* levels of this call solved by PCG (the rest by
                           BiCGSTAB)                                        */
} tsfde_solve_info;

typedef struct tsfde_timing {
  int64_t levels;       /* levels timed since the last tsfde_get_timing     */
  double rhs_ms;        /* total device time of the SOE/right-hand-side
                           kernel over those levels (CUDA events)           */
  double level_ms;      /* total device time of the level-solve kernel      */
} tsfde_timing;

typedef struct tsfde_adjoint_info {
  int status;           /* first non-OK level status, else TSFDE_OK          */
  int64_t failed_level; /* level of that status, 0 if none                  */
  int64_t iterations;   /* total Krylov iterations of the transposed solves */
  int max_iterations;
  double max_rel_residual;
  int64_t recomputed_levels; /* forward levels marched again from the
                           checkpoints (u_all = NULL), else 0               */
} tsfde_adjoint_info;

typedef struct tsfde_ctx tsfde_ctx;

/* Defaults documented in tsfde_opts. */
int tsfde_default_opts(tsfde_opts* opts);

/* Build a context: graded mesh t_m = T (m/M)^r (Sec. 3.1), SOE table for
 * t^{-gamma} on [tau_1, T] with relative tolerance soe_tol (Lemma 2.2; see
 * tsfde_get_soe), the Toeplitz symbol of Eq. (3.16x) and its circulant
 * embedding spectrum, the Strang eigenvalues of Sec. 4.1, and all device
 * workspaces.  Validation: 0<alpha<2, 0<gamma<1, l>0, T>0, n>=1, M>=1, r>=1,
 * soe_tol in (0, 1e-2], mu in (alpha, 2]; n <= 2^18 (else TSFDE_ENOTSUP).
 * opts may be NULL (defaults).
 * On error *out is NULL. */
int tsfde_setup(tsfde_ctx** out, double alpha, double gamma, double l, double T,
                int64_t n, int64_t M, double r, double soe_tol,
                const tsfde_opts* opts);

void tsfde_destroy(tsfde_ctx* ctx);
const char* tsfde_strerror(int status);
/* Message of the last failing call on this context ("" if none). */
const char* tsfde_last_error(const tsfde_ctx* ctx);

/* Problem data.  phi: dev n.  Diffusivity kappa(x_i, t_m) = kappa0_i +
 * theta[m] kappa1_i (kappa1 dev n or NULL; theta host M+1 or NULL).  Source
 * f(x_i, t_m) = sum_{q<rank} G[q*(M+1)+m] F[q][i] with rank <= 4, F a host
 * array of rank dev pointers (n each), G host rank x (M+1).  Either part may
 * instead be supplied per level to tsfde_step.  The context copies all of it.
 * Resets the time level to 0. */
int tsfde_set_problem(tsfde_ctx* ctx, const double* phi, const double* kappa0,
                      const double* kappa1, const double* theta, int rank,
                      const double* const* F, const double* G);

/* Back to level 0 with the same problem (history cleared, u^0 = phi). */
int tsfde_reset(tsfde_ctx* ctx);

/* Advance one time level m -> m+1: SOE history update and right-hand side
 * (Eq. (3.16gu) through the recurrence of the history sums), preconditioner
 * for this level (Eq. (4.3)), and the Krylov solve.  kappa_m / f_m (dev n)
 * override the separable data for this level when non-NULL.  u_out (dev n)
 * receives u^{m+1} and rhs_out (dev n) the right-hand side b^{m+1}, when
 * non-NULL.  info (nullable) synchronises.  TSFDE_ESTATE after level M. */
int tsfde_step(tsfde_ctx* ctx, const double* kappa_m, const double* f_m,
               double* u_out, double* rhs_out, tsfde_step_info* info);

/* Run all remaining levels with the separable problem data.  u_final (dev n)
 * receives u^M; u_all (dev (M+1) x n, row m = u^m, nullable) every level.
 * info (nullable) synchronises and summarises. */
int tsfde_solve(tsfde_ctx* ctx, double* u_final, double* u_all,
                tsfde_solve_info* info);

/* Per-level statistics of levels m0..m1 (1 <= m0 <= m1 <= current level)
 * into out[0 .. m1-m0] (host).  Synchronises the stream. */
int tsfde_get_level_stats(tsfde_ctx* ctx, int64_t m0, int64_t m1, tsfde_step_info* out);

/* Copy the current level's solution u^m (m = 0 after set_problem/reset)
 * into u (dev n).  Asynchronous. */
int tsfde_get_solution(tsfde_ctx* ctx, double* u);

/* Copy the SOE table (ascending s_j, Lemma 2.2) to host arrays of capacity
 * *E (either may be NULL); *E returns the table size. */
int tsfde_get_soe(const tsfde_ctx* ctx, int* E, double* s, double* w);

/* Copy the graded mesh t_0..t_M (host, M+1). */
int tsfde_get_times(const tsfde_ctx* ctx, double* t);

/* Copy the first column t_0..t_{n-1} of A (Eq. (3.16x)) to host. */
int tsfde_get_symbol(const tsfde_ctx* ctx, double* t);

/* ---- adjoint sweep (gradients of a scalar J(u^M)) ---------------------
 * The paper solves only the forward problem; this is the discrete adjoint of
 * the FIDS march of Eq. (3.16gu) (with the history written through the SOE
 * recurrence of Sec. 3), for a problem whose kappa is time independent
 * (tsfde_set_problem with kappa1 = NULL) and whose source f^m is the
 * caller's fixed f for every level.
 *
 * Reverse in time, m = M..1, in FP64 with the context's level solver on the
 * transposed operator (BiCGSTAB; or PCG on (ahat_m K^{-1} + A) mu = g^m,
 * lambda^m = K^{-1} mu, whose residual is that of the transposed system;
 * with TSFDE_KRYLOV_AUTO the method that solved forward level m):
 *   (ahat_m I + A K) lambda^m = g^m,   g^M = dJ/du^M,
 *   g^m = ahat_{m+1} lambda^{m+1}
 *         - sum_j (c_{j,m+1} Y_j^{(m+1)} - c_{j,m+2} Y_j^{(m+2)}),  m < M,
 *   Y_j^{(m)} = eps_{j,m} (lambda^m + Y_j^{(m+1)}),  Y^{(M+1)} = 0,
 * with eps_{j,m} = e^{-s_j tau_m} and c_{j,m} = w_j beta_{j,m-1}/Gamma(1-gamma)
 * the forward SOE coefficients.  Gradients:
 *   dJ/dkappa = -sum_m lambda^m .* (A u^m),   dJ/df = sum_m lambda^m.
 *
 * u_all:   dev (M+1) x n, the forward levels u^0..u^M (as tsfde_solve writes
 *          them with this context's problem; row m = u^m); or NULL in a
 *          context set up with ckpt_stride != 0 whose march has reached
 *          level M from level 0 with the separable problem data: the sweep
 *          then takes the segments between checkpoints last to first,
 *          marches each again from its checkpoint (one extra forward march
 *          in all, with the context's own level solver) and sweeps it in
 *          reverse.  With TSFDE_KRYLOV_AUTO a recomputed level may take the
 *          other method than the first march did; both meet krylov_tol.
 * dJ_duM:  dev n.  grad_kappa, grad_f: dev n, overwritten.
 * Uses the context's krylov_tol / max_it / precond (always FP64).  Does not
 * change the forward state (tsfde_step continues where it was).  Device
 * work buffers are allocated on the first call.  Synchronises the stream.
 * Errors: TSFDE_ESTATE without a problem (or, with u_all = NULL, without the
 * checkpoints of a whole march), TSFDE_ENOTSUP if kappa1 was set or
 * the context uses the direct history (the sweep is the adjoint of FIDS),
 * TSFDE_EINVAL for NULL pointers, else the first failing level's status. */
int tsfde_adjoint(tsfde_ctx* ctx, const double* u_all, const double* dJ_duM,
                  double* grad_kappa, double* grad_f, tsfde_adjoint_info* info);

/* ---- batched solve: many independent problems in one launch ----------
 * The paper solves one problem at a time; this runs B independent FIDS
 * problems (each with its own n, alpha, gamma, grading, SOE table and
 * data) over a common number of levels M, as one persistent launch of
 * thread-block clusters: a cluster claims an instance, marches it through
 * all M levels (SOE update, FP64 Strang preconditioner, level solve) with
 * its transforms in distributed shared memory, writes u^M and claims the
 * next.  Instances are taken largest first.  kappa and f are time
 * independent per instance.  Options (tsfde_opts): mu / kappa_mu (common),
 * precision (MIXED: FP32 Krylov sweeps refined in FP64 with the FP64
 * fallback of the single-problem path; FP64: the Krylov solve in FP64),
 * krylov (BICGSTAB, PCG on the symmetrised system, or AUTO: the per-level
 * choice of TSFDE_KRYLOV_AUTO made within each instance's march from the
 * cluster's own level times), krylov_tol, max_it, inner_tol, max_outer,
 * inner_max_it, precond, stream.
 * Each instance needs n >= 31 (its transforms are split over the cluster). */
typedef struct tsfde_instance {
  double alpha, gamma, l, T, r;  /* as tsfde_setup                           */
  int64_t n;                     /* interior nodes, 31 <= n <= 16383         */
  double soe_tol;                /* SOE relative tolerance, (0, 1e-2]        */
  const double* phi;             /* dev n: u^0                               */
  const double* kappa;           /* dev n: diffusivity (> 0), all levels     */
  const double* f;               /* dev n: source, all levels                */
} tsfde_instance;

typedef struct tsfde_batch tsfde_batch;

typedef struct tsfde_batch_info {
  int status;              /* first non-OK instance status, else TSFDE_OK   */
  int failed_instance;     /* index of that instance, -1 if none            */
  int64_t levels;          /* instances x levels solved                     */
  int64_t iterations;      /* all Krylov iterations (inner + FP64)          */
  int64_t outer;           /* refinement sweeps (mixed)                     */
  int64_t fp64_levels;     /* levels finished by the FP64 fallback          */
  double max_rel_residual; /* worst final relative residual of any level    */
} tsfde_batch_info;

/* Copies phi, kappa, f of every instance and builds all tables; the caller's
 * buffers need not outlive the call.  Errors: TSFDE_EINVAL (arguments, as
 * tsfde_setup per instance), TSFDE_ENOTSUP (an instance too small or too
 * large for the cluster transforms), TSFDE_ENOMEM. */
int tsfde_batch_setup(tsfde_batch** out, int B, const tsfde_instance* inst, int64_t M,
                      const tsfde_opts* opts);
/* Solve every instance from u^0 through level `levels` (1..M; 0 = M) of
 * its M-level mesh; u_final: host array of B device pointers (n_i doubles
 * each) that receive u^levels.  Synchronises. */
int tsfde_batch_solve(tsfde_batch* b, int64_t levels, double* const* u_final,
                      tsfde_batch_info* info);
/* Per-instance totals of the last solve (status, iterations, outer = sweeps,
 * E_active = levels finished in FP64, rel_residual = worst level). */
int tsfde_batch_instance_stats(const tsfde_batch* b, int i, tsfde_step_info* out);
/* Thread-block clusters the persistent launch uses and CTAs per cluster
 * (of the first launch; tsfde_batch_get_plan has every launch). */
int tsfde_batch_shape(const tsfde_batch* b, int* clusters, int* cluster_size);

/* Launch plan of a batched solve.  The instances form one persistent launch
 * (classes = 1) or two launched side by side on two streams (classes = 2:
 * instances with n >= split_n in the first).  Every launch has one cluster
 * size (CTAs per cluster, 4, 8 or 16; 0 in a requested plan: the size that
 * keeps the most CTAs resident) and one shared-memory layout sized for its
 * largest transform, because CUDA fixes both per launch.  The cluster size
 * is the tile schedule of the cluster FFTs: CTA q of Q owns N2/Q columns of
 * the column passes and N1/(2Q) row pairs of the row pass; the FFT stages
 * are radix 16 in registers (last stage radix 2^(lg N mod 4)). */
typedef struct tsfde_batch_plan {
  int classes;             /* persistent launches, 1 or 2                   */
  int64_t split_n;         /* classes = 2: n >= split_n go to the first     */
  int cluster_size[2];     /* per launch                                    */
  int clusters[2];         /* clusters resident per launch (filled by setup) */
  double probe_ms;         /* tsfde_batch_tune: the probe solve's time      */
} tsfde_batch_plan;

/* tsfde_batch_setup with an explicit launch plan (NULL: the default plan,
 * two classes split at n = 8193, each with its most-resident cluster size,
 * or opts.cluster_size when set). */
int tsfde_batch_setup_plan(tsfde_batch** out, int B, const tsfde_instance* inst, int64_t M,
                           const tsfde_opts* opts, const tsfde_batch_plan* plan);
/* The plan a batch was set up with (cluster sizes and residency filled in). */
int tsfde_batch_get_plan(const tsfde_batch* b, tsfde_batch_plan* plan);
/* Autotuner of the launch plan (the paper has none: it solves one problem at
 * a time).  Candidates: one launch with cluster size 4, 8 or 16; two launches
 * split at n = 8193 or n = 4097 with cluster sizes (8 or 16, 4 or 8).  Each
 * candidate that fits the device is set up for these instances and times a
 * solve of the first probe_levels levels (1..M) with CUDA events on
 * opts->stream, after one untimed solve; identical plans are timed once.
 * *best receives the fastest (probe_ms set); tried (capacity *ntried, both
 * nullable) every timed plan, *ntried their count.  The caller then passes
 * *best to tsfde_batch_setup_plan.  Allocates and frees its own device
 * buffers; synchronises. */
int tsfde_batch_tune(int B, const tsfde_instance* inst, int64_t M, const tsfde_opts* opts,
                     int64_t probe_levels, tsfde_batch_plan* best, tsfde_batch_plan* tried,
                     int* ntried);
void tsfde_batch_destroy(tsfde_batch* b);

/* Engine the context's mixed level solves use: TSFDE_ENGINE_GRID or
 * TSFDE_ENGINE_CLUSTER (never AUTO); -1 if ctx is NULL. */
int tsfde_get_engine(const tsfde_ctx* ctx);

/* Device time of the kernels launched since the previous call (opts.profile
 * must be 1).  Synchronises the stream and resets the counters. */
int tsfde_get_timing(tsfde_ctx* ctx, tsfde_timing* out);

/* ---- single operations of the hot path (used by tests and tools) ------ */

/* y = A v (Toeplitz product by zero-padded FFT circulant embedding,
 * Sec. 4.1).  v, y: dev n.  precision: TSFDE_FP64, TSFDE_MIXED (FP32
 * transform) or TSFDE_MIXED_DS (double-single transform; only in a context
 * set up with that precision, else TSFDE_EINVAL); FP64 in/out. */
int tsfde_toeplitz_apply(tsfde_ctx* ctx, const double* v, double* y, int precision);

/* y = (a I + diag(kappa) A) v, the matrix-free product of Sec. 4.1.
 * kappa, v, y: dev n. */
int tsfde_operator_apply(tsfde_ctx* ctx, double a, const double* kappa,
                         const double* v, double* y, int precision);

/* z = P^{-1} v with P = a I + kbar s(A), the Strang circulant preconditioner
 * of Eq. (4.3) (kbar = mean of kappa).  Builds the preconditioner (circulant
 * inverse kernel by a Bluestein length-n inverse DFT) and applies it.
 * v, z: dev n. */
int tsfde_precond_apply(tsfde_ctx* ctx, double a, double kbar, const double* v,
                        double* z, int precision);

/* Solve (a I + diag(kappa) A) x = b with the level solver selected by the
 * context options (BiCGSTAB or PCG, FP64 or mixed refinement).  kappa, b,
 * x: dev n. */
int tsfde_linear_solve(tsfde_ctx* ctx, double a, const double* kappa,
                       const double* b, double* x, tsfde_step_info* info);

/* ---- product without any device allocation ---------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc themselves (for example code whose device
 * memory all comes from a framework's pool, or a thread that must not
 * trigger the allocator's implicit synchronisation).
 *
 * y = A v for the IFL Toeplitz matrix of Eq. (3.16x) with n interior points
 * on (-l, l), splitting mu (<= 0: 1 + alpha/2) and kappa_mu (<= 0: derived
 * from mu).  v, y: dev n, owned by the caller.  No context is needed and
 * no memory is allocated: the twiddles, symbol, spectrum and work buffers
 * live in one fixed array of about 1.6 MB inside the library, which every
 * GPU that loads the library keeps until the process exits.
 *  - n must be <= 16383; larger n returns TSFDE_ENOTSUP (with a message on
 *    stderr) without touching the device.
 *  - The first call on a device looks up the array's device address (with
 *    that device current); make that first call before any stream capture.
 *  - All calls on a device share the array and it keeps the last call's
 *    contents; the call clears what must start at zero itself.  Calls whose
 *    work overlaps on the GPU (other streams, other host threads) race on
 *    the array: serialise them.
 *  - Enqueued on `stream` (cudaStream_t, NULL = default); the call waits
 *    for its own completion and returns the kernel's status. */
int tsfde_toeplitz_apply_static(double alpha, double mu, int kappa_mu, double l,
                                int64_t n, const double* v, double* y, void* stream);

/* ---- measurement helper ------------------------------------------------
 * Not part of the method.  Streams 16-byte loads that bypass L1 over the
 * device buffer buf (bytes long, 16-byte aligned, a multiple of 16) `reps`
 * times with every resident thread of the GPU, enqueued on `stream`
 * (cudaStream_t, NULL = default) without waiting.  The caller sizes buf to
 * fit in L2, warms it with one call and times a second one (CUDA events on
 * the same stream): bytes * reps / time is the L2 read bandwidth against
 * which the level kernels, whose vectors stay in L2, are reported.  No
 * allocation; nothing is written.  TSFDE_EINVAL for a NULL, unaligned or
 * short buffer or reps < 1; TSFDE_ECUDA if the launch fails. */
int tsfde_probe_l2_read(const void* buf, size_t bytes, int reps, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TSFDE_H */
