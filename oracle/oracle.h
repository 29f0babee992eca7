/*
 * oracle.h -- CPU reference ("oracle") for the fast and direct implicit
 * difference schemes (FIDS / DIDS) of Gu, Sun, Zhang and Zhao for the 1-D
 * time-space fractional diffusion equation with the integral fractional
 * Laplacian (arXiv 2002.11978).
 *
 * THIS IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline leg may load it.
 * It shares no code with the CUDA path.  Everything is plain, slow and
 * written to be checked against the paper by eye: dense matrices, dense LU
 * with partial pivoting, and the O(M^2 n) direct history sums.
 *
 * Floating point is IEEE double throughout.  Where a printed formula is a
 * difference of nearly equal quantities the oracle evaluates the same
 * quantity through expm1/log1p; each such place says so.
 *
 * Pins (see tests/test_oracle_*.py): closed forms of the fractional
 * Laplacian, Prop. 3.1 structure of A, the L1 weights against a
 * 50-digit decimal evaluation of Eq. (2.8), exactness of the L1 formula for
 * piecewise-linear functions, the SOE bound of Lemma 2.2, dense LU against
 * LAPACK, and the printed Err values of Tables 1-11.
 */
#ifndef TSFDE_ORACLE_H
#define TSFDE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* c_{1,alpha} of Eq. (1.4). */
double or_c1alpha(double alpha);

/* First column t_0..t_{n-1} of the symmetric Toeplitz matrix A of
 * Eq. (3.16x) (equivalently Eq. (2.11)), n = N-1 unknowns, h = 2l/N.
 * Returns 0 on success, -1 on bad arguments. */
int or_ifl_symbol(double alpha, double mu, int kappa_mu, int64_t n, double l,
                  double* t);

/* Graded mesh of Sec. 3.1: t_m = T (m/M)^r, tau_m = t_m - t_{m-1}
 * (tau[0] = 0).  Arrays have M+1 entries. */
int or_graded_mesh(double T, int64_t M, double r, double* t, double* tau);

/* t_m - t_k for 0 <= k <= m on the graded mesh, without cancellation. */
double or_mesh_gap(double T, int64_t M, double r, int64_t m, int64_t k);

/* L1 weight a_k^{(m,gamma)} of Eq. (2.8), 1 <= k <= m. */
double or_l1_weight(double T, int64_t M, double r, double gamma, int64_t m,
                    int64_t k);

/* Sum-of-exponentials table for t^{-gamma} on [delta, T] (Lemma 2.2),
 * built by the trapezoidal rule in x = ln s applied to
 * t^{-gamma} = Gamma(gamma)^{-1} int_R exp(-t e^x + gamma x) dx.
 * The relative error max |t^gamma sum_j w_j e^{-s_j t} - 1| over [delta,T]
 * is verified on a dense log grid and is <= tol on return.
 * Returns E (number of exponentials) or -1 if maxE is too small. */
int or_soe_build(double gamma, double delta, double T, double tol, int maxE,
                 double* s, double* w);

/* max over nsamp log-spaced t in [delta,T] (ends included) of
 * |t^gamma sum_j w_j exp(-s_j t) - 1|. */
double or_soe_rel_err(double gamma, double delta, double T, int E,
                      const double* s, const double* w, int nsamp);

/* FIDS weight b_k^{(m,gamma)} (definition under Eq. (lem2.3)) for a given
 * SOE table; b_m^{(m)} = a_m^{(m)}. */
double or_fids_weight(double T, int64_t M, double r, double gamma, int64_t m,
                      int64_t k, int E, const double* s, const double* w);

/* Dense LU with partial pivoting; A is n x n row-major and is overwritten,
 * b holds the right-hand side on entry and the solution on exit.
 * Returns 0, or -1 if a zero pivot was met. */
/* Row-update threads of or_lu_solve (default 1; results do not depend on it). */
void or_set_threads(int t);
int or_get_threads(void);
/* d = b - (a u + kappa .* (A u)), A the symmetric Toeplitz matrix of first
 * column t, in double-double arithmetic rounded once (threads as or_lu_solve). */
void or_level_defect(int64_t n, const double* t, double a, const double* kappa, const double* u,
                     const double* b, double* d);
int or_lu_solve(int64_t n, double* A, double* b);

/* y = A v for the symmetric Toeplitz matrix with first column t (dense
 * O(n^2) summation). */
void or_toeplitz_matvec(int64_t n, const double* t, const double* v, double* y);

/* Strang circulant of Sec. 4.1: first column c_S and its eigenvalues
 * Lambda = F c_S by the O(n^2) DFT (both length n). */
void or_strang_column(int64_t n, const double* t, double* cS);
void or_strang_eigs(int64_t n, const double* t, double* lam);

/* Time marching of FIDS (Eq. (3.15), matrix form Eq. (3.16gu)) or DIDS
 * (Eq. (3.16), matrix form Eq. (4.1)) with dense LU at every level.
 *   kappa, f: (M+1) x n row-major tables, row m = values at t_m.
 *   U       : (M+1) x n output, row 0 = phi.
 * scheme: 0 = DIDS, 1 = FIDS with the given SOE table.
 * Returns 0 on success. */
typedef struct {
  double alpha, gamma, l, T, r, mu;
  int kappa_mu;
  int64_t n, M;
  const double* phi;
  const double* kappa;
  const double* f;
  int soe_E;
  const double* soe_s;
  const double* soe_w;
  int64_t levels;  /* march levels 1..levels only (0 = all M) */
} or_problem;

int or_march(const or_problem* p, int scheme, double* U);
/* Right-hand side of level m (scheme 0 DIDS, 1 FIDS) from the levels U
 * (rows 0..m-1 of n) and the source fm (n), with the mesh, weights and
 * SOE table of p (p->kappa and p->f are not read).  0 on success. */
int or_level_rhs(const or_problem* p, int scheme, int64_t m, const double* U, const double* fm,
                 double* rhs);

/* Adjoint of the FIDS march for J = 1/2 ||u^M - u_obs||^2 with
 * time-independent kappa (row 0 of p->kappa used for every level) and
 * time-independent source f (row 0 of p->f used for every level):
 * dense transposed solves in reverse time.  Outputs dJ/dkappa and dJ/df
 * (length n each); U is the forward solution from or_march. */
int or_adjoint(const or_problem* p, const double* U, const double* u_obs,
               double* grad_kappa, double* grad_f);

#ifdef __cplusplus
}
#endif
#endif
