/*
 * oracle.c -- plain CPU reference for FIDS/DIDS (arXiv 2002.11978).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Plain C99, IEEE double.
 * Nothing here is blocked, fused or reordered beyond what the formulas in
 * the paper state; each function names the passage it follows.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Eq. (1.4): c_{1,a} = 2^{a-1} a Gamma((a+1)/2) / (sqrt(pi) Gamma(1-a/2)) */
double or_c1alpha(double alpha) {
  const double pi = 3.14159265358979323846;
  return pow(2.0, alpha - 1.0) * alpha * tgamma(0.5 * (alpha + 1.0)) /
         (sqrt(pi) * tgamma(1.0 - 0.5 * alpha));
}

/* (l+1)^nu - (l-1)^nu for l >= 1.  Evaluated as
 * l^nu [ expm1(nu log1p(1/l)) - expm1(nu log1p(-1/l)) ]: the two expm1
 * terms have opposite signs, so no cancellation (the plain difference of
 * powers loses ~log10(l/nu) digits). */
static double diff_pow(double l, double nu) {
  if (l == 1.0) return pow(2.0, nu);  /* (2)^nu - 0^nu, nu > 0 */
  return pow(l, nu) * (expm1(nu * log1p(1.0 / l)) - expm1(nu * log1p(-1.0 / l)));
}

/* Eq. (3.16x), entries of A = C^h_{alpha,mu} [...] with C = c_{1,a}/(nu h^a),
 * nu = mu - alpha, N = n + 1 intervals, h = 2l/N. */
int or_ifl_symbol(double alpha, double mu, int kappa_mu, int64_t n, double l,
                  double* t) {
  if (!(alpha > 0.0 && alpha < 2.0) || !(mu > alpha && mu <= 2.0) || n < 1 ||
      !(l > 0.0) || !t)
    return -1;
  const int64_t N = n + 1;
  const double nu = mu - alpha;
  const double h = 2.0 * l / (double)N;
  const double C = or_c1alpha(alpha) / (nu * pow(h, alpha));
  const double km = (double)kappa_mu;
  /* diagonal: sum_{l=2}^{N-1} ((l+1)^nu-(l-1)^nu)/l^mu + (N^nu-(N-1)^nu)/N^mu
   *           + (2^nu + kappa_mu - 1) + 2 nu / (alpha N^alpha).
   * The sum is accumulated from the smallest term up. */
  double sum = 0.0;
  for (int64_t ell = N - 1; ell >= 2; --ell) {
    double L = (double)ell;
    sum += diff_pow(L, nu) / pow(L, mu);
  }
  double Nd = (double)N;
  /* N^nu - (N-1)^nu = N^nu * (-expm1(nu log1p(-1/N))) */
  double tailN = pow(Nd, nu) * (-expm1(nu * log1p(-1.0 / Nd))) / pow(Nd, mu);
  t[0] = C * (sum + tailN + (pow(2.0, nu) + km - 1.0) +
              2.0 * nu / (alpha * pow(Nd, alpha)));
  if (n > 1) t[1] = -C * (pow(2.0, nu) + km - 1.0) / 2.0;
  for (int64_t k = 2; k < n; ++k) {
    double K = (double)k;
    t[k] = -C * diff_pow(K, nu) / (2.0 * pow(K, mu));
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Graded mesh, Sec. 3.1: t_m = T (m/M)^r. */
static double mesh_t(double T, int64_t M, double r, int64_t m) {
  return T * pow((double)m / (double)M, r);
}

/* t_m - t_k = t_m (1 - (k/m)^r) = -t_m expm1(r log(k/m)) for 0 < k < m. */
double or_mesh_gap(double T, int64_t M, double r, int64_t m, int64_t k) {
  if (k >= m) return 0.0;
  double tm = mesh_t(T, M, r, m);
  if (k == 0) return tm;
  return -tm * expm1(r * log((double)k / (double)m));
}

int or_graded_mesh(double T, int64_t M, double r, double* t, double* tau) {
  if (M < 1 || !(r >= 1.0) || !(T > 0.0)) return -1;
  for (int64_t m = 0; m <= M; ++m) t[m] = mesh_t(T, M, r, m);
  tau[0] = 0.0;
  for (int64_t m = 1; m <= M; ++m) tau[m] = or_mesh_gap(T, M, r, m, m - 1);
  return 0;
}

/* Eq. (2.8): a_k^{(m)} = (1/tau_k) int_{t_{k-1}}^{t_k} (t_m - s)^{-gamma} ds
 *          = [D_{k-1}^{1-g} - D_k^{1-g}] / ((1-g) tau_k),  D_j = t_m - t_j.
 * For k < m the bracket is D_k^{1-g} expm1((1-g) log1p(tau_k/D_k)); for
 * k = m it is tau_m^{1-g}. */
double or_l1_weight(double T, int64_t M, double r, double gamma, int64_t m,
                    int64_t k) {
  double tau = or_mesh_gap(T, M, r, k, k - 1);
  double g1 = 1.0 - gamma;
  if (k == m) return pow(tau, -gamma) / g1;
  double D = or_mesh_gap(T, M, r, m, k);
  return pow(D, g1) * expm1(g1 * log1p(tau / D)) / (g1 * tau);
}

/* ------------------------------------------------------------------ */
/* Lemma 2.2 SOE table, plain trapezoidal rule in x = ln s on
 * t^{-g} = Gamma(g)^{-1} int exp(-t e^x + g x) dx:
 *   s_j = exp(x_j), w_j = h exp(g x_j) / Gamma(g), x_j = x_lo + j h.
 * Range: the left tail is <= e^{g x_lo} t^g / (g Gamma(g)) relative; the
 * right tail is <= (delta s_hi)^{g-1} e^{-delta s_hi} / Gamma(g).  The step
 * h is shrunk until the verified relative error is <= tol. */
double or_soe_rel_err(double gamma, double delta, double T, int E,
                      const double* s, const double* w, int nsamp) {
  double worst = 0.0;
  double la = log(delta), lb = log(T);
  for (int i = 0; i < nsamp; ++i) {
    double tt = (nsamp == 1) ? delta : exp(la + (lb - la) * (double)i / (double)(nsamp - 1));
    if (i == nsamp - 1) tt = T;
    double acc = 0.0;
    for (int j = 0; j < E; ++j) acc += w[j] * exp(-s[j] * tt);
    double e = fabs(pow(tt, gamma) * acc - 1.0);
    if (e > worst) worst = e;
  }
  return worst;
}

int or_soe_build(double gamma, double delta, double T, double tol, int maxE,
                 double* s, double* w) {
  if (!(gamma > 0.0 && gamma < 1.0) || !(delta > 0.0) || !(T >= delta) ||
      !(tol > 0.0))
    return -1;
  double gg = tgamma(gamma);
  double x_lo = (log(0.1 * tol * gamma * gg) - gamma * log(T)) / gamma;
  /* right end: smallest z with z^{g-1} e^{-z} <= 0.1 tol Gamma(g) */
  double z = 1.0;
  for (int it = 0; it < 200; ++it) {
    double zn = log(10.0 / (tol * gg)) + (gamma - 1.0) * log(z);
    if (zn < 1.0) zn = 1.0;
    if (fabs(zn - z) < 1e-12) { z = zn; break; }
    z = zn;
  }
  double x_hi = log((z + 2.0) / delta);
  double h = 0.5;
  for (int attempt = 0; attempt < 40; ++attempt) {
    int E = (int)ceil((x_hi - x_lo) / h) + 1;
    if (E > maxE) return -1;
    for (int j = 0; j < E; ++j) {
      double x = x_lo + h * (double)j;
      s[j] = exp(x);
      w[j] = h * exp(gamma * x) / gg;
    }
    if (or_soe_rel_err(gamma, delta, T, E, s, w, 4001) <= tol) return E;
    h *= 0.9;
  }
  return -1;
}

/* b_k^{(m)} = sum_j w_j (1/tau_k) int_{t_{k-1}}^{t_k} e^{-s_j (t_m - s)} ds
 *           = sum_j w_j e^{-s_j (t_m - t_k)} (1 - e^{-s_j tau_k}) / (s_j tau_k)
 * for k < m (the factor (1 - e^{-x})/x is written -expm1(-x)/x);
 * b_m^{(m)} = a_m^{(m)}. */
double or_fids_weight(double T, int64_t M, double r, double gamma, int64_t m,
                      int64_t k, int E, const double* s, const double* w) {
  if (k == m) return or_l1_weight(T, M, r, gamma, m, m);
  double tau = or_mesh_gap(T, M, r, k, k - 1);
  double D = or_mesh_gap(T, M, r, m, k);
  double acc = 0.0;
  for (int j = 0; j < E; ++j) {
    double x = s[j] * tau;
    double frac = (x == 0.0) ? 1.0 : -expm1(-x) / x;
    acc += w[j] * exp(-s[j] * D) * frac;
  }
  return acc;
}

/* ------------------------------------------------------------------ */
/* Threads of the elimination's row updates (1 unless the caller asks for
 * more: only the timed CPU baseline does).  Each row's update is the same
 * sequence of operations whichever thread runs it, so the result does not
 * depend on the thread count. */
static int or_threads = 1;
void or_set_threads(int t) { or_threads = t > 0 ? t : 1; }
int or_get_threads(void) { return or_threads; }

/* Gaussian elimination with partial pivoting (the paper's direct solver,
 * Sec. 5 "MATLAB's backslash"). */
int or_lu_solve(int64_t n, double* A, double* b) {
  for (int64_t c = 0; c < n; ++c) {
    int64_t piv = c;
    double best = fabs(A[c * n + c]);
    for (int64_t i = c + 1; i < n; ++i) {
      double v = fabs(A[i * n + c]);
      if (v > best) { best = v; piv = i; }
    }
    if (best == 0.0) return -1;
    if (piv != c) {
      for (int64_t j = 0; j < n; ++j) {
        double tmp = A[c * n + j]; A[c * n + j] = A[piv * n + j]; A[piv * n + j] = tmp;
      }
      double tb = b[c]; b[c] = b[piv]; b[piv] = tb;
    }
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_threads > 1 && n - c > 64)
    for (int64_t i = c + 1; i < n; ++i) {
      double f = A[i * n + c] / A[c * n + c];
      A[i * n + c] = f;
      for (int64_t j = c + 1; j < n; ++j) A[i * n + j] -= f * A[c * n + j];
      b[i] -= f * b[c];
    }
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double acc = b[i];
    for (int64_t j = i + 1; j < n; ++j) acc -= A[i * n + j] * b[j];
    b[i] = acc / A[i * n + i];
  }
  return 0;
}

void or_toeplitz_matvec(int64_t n, const double* t, const double* v, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      int64_t d = i > j ? i - j : j - i;
      acc += t[d] * v[j];
    }
    y[i] = acc;
  }
}

/* Sec. 4.1: c_S = [a_11, ..., a_{1,floor((N+1)/2)}, a_{1,floor(N/2)}, ..., a_12]
 * with N - 1 = n entries: entry k (0-based) is t_k for k <= floor(n/2) and
 * t_{n-k} otherwise. */
void or_strang_column(int64_t n, const double* t, double* cS) {
  for (int64_t k = 0; k < n; ++k) cS[k] = (k <= n / 2) ? t[k] : t[n - k];
}

/* Lambda = diag(F c_S): plain O(n^2) DFT; c_S is real and symmetric so the
 * transform is real. */
void or_strang_eigs(int64_t n, const double* t, double* lam) {
  const double pi = 3.14159265358979323846;
  double* cS = (double*)malloc(sizeof(double) * (size_t)n);
  or_strang_column(n, t, cS);
  for (int64_t k = 0; k < n; ++k) {
    double acc = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      int64_t p = (j * k) % n;
      acc += cS[j] * cos(2.0 * pi * (double)p / (double)n);
    }
    lam[k] = acc;
  }
  free(cS);
}

/* ------------------------------------------------------------------ */
/* Weights c_k^{(m)}, k = 1..m, of the scheme: a_k (DIDS, Eq. (4.1)) or
 * b_k (FIDS, Eq. (3.16gu)). */
static void level_weights(const or_problem* p, int scheme, int64_t m,
                          double* c) {
  for (int64_t k = 1; k <= m; ++k) {
    if (scheme == 0)
      c[k] = or_l1_weight(p->T, p->M, p->r, p->gamma, m, k);
    else
      c[k] = or_fids_weight(p->T, p->M, p->r, p->gamma, m, k, p->soe_E,
                            p->soe_s, p->soe_w);
  }
}

/* Right-hand side of level m of Eq. (3.16gu) (FIDS) / Eq. (4.1) (DIDS)
 * from the levels U (rows 0..m-1 of n) and the weights c_k = c_k^{(m)}:
 * Gamma(1-g)^{-1}[ sum_{k=1}^{m-1} (c_{k+1}-c_k) u^k + c_1 u^0 ] + f^m. */
static void level_rhs(const or_problem* p, int64_t m, const double* c, const double* U,
                      const double* fm, double* rhs) {
  const int64_t n = p->n;
  const double Gg = tgamma(1.0 - p->gamma);
  for (int64_t i = 0; i < n; ++i) rhs[i] = c[1] * U[i];
  for (int64_t k = 1; k <= m - 1; ++k) {
    double d = c[k + 1] - c[k];
    const double* uk = U + k * n;
    for (int64_t i = 0; i < n; ++i) rhs[i] += d * uk[i];
  }
  for (int64_t i = 0; i < n; ++i) rhs[i] = rhs[i] / Gg + fm[i];
}

int or_level_rhs(const or_problem* p, int scheme, int64_t m, const double* U, const double* fm,
                 double* rhs) {
  if (m < 1 || m > p->M || (scheme == 1 && p->soe_E < 1)) return -1;
  double* c = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  level_weights(p, scheme, m, c);
  level_rhs(p, m, c, U, fm, rhs);
  free(c);
  return 0;
}

int or_march(const or_problem* p, int scheme, double* U) {
  const int64_t n = p->n, M = p->M;
  double* t = (double*)malloc(sizeof(double) * (size_t)n);
  if (or_ifl_symbol(p->alpha, p->mu, p->kappa_mu, n, p->l, t) != 0) { free(t); return -1; }
  const double Gg = tgamma(1.0 - p->gamma);
  double* c = (double*)malloc(sizeof(double) * (size_t)(M + 1));
  double* Mat = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* rhs = (double*)malloc(sizeof(double) * (size_t)n);
  memcpy(U, p->phi, sizeof(double) * (size_t)n);
  int status = 0;
  const int64_t last = (p->levels > 0 && p->levels < M) ? p->levels : M;
  for (int64_t m = 1; m <= last && status == 0; ++m) {
    level_weights(p, scheme, m, c);
    level_rhs(p, m, c, U, p->f + m * n, rhs);
    /* M^{(m)} = c_m/Gamma(1-g) I + K^{(m)} A */
    const double* km = p->kappa + m * n;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        int64_t d = i > j ? i - j : j - i;
        Mat[i * n + j] = km[i] * t[d] + (i == j ? c[m] / Gg : 0.0);
      }
    if (or_lu_solve(n, Mat, rhs) != 0) status = -2;
    memcpy(U + m * n, rhs, sizeof(double) * (size_t)n);
  }
  free(t); free(c); free(Mat); free(rhs);
  return status;
}

/* Adjoint of the FIDS march (not in the paper).  With
 * R^m = M^{(m)} u^m - Gamma^{-1}[sum_{k<m}(c_{k+1}^{(m)}-c_k^{(m)}) u^k + c_1^{(m)} u^0] - f,
 * stationarity of J - sum_m lambda^m . R^m in u^m gives, for m = M..1,
 *   M^{(m)T} lambda^m = dJ/du^m + Gamma^{-1} sum_{j>m} (c_{m+1}^{(j)} - c_m^{(j)}) lambda^j,
 * M^{(m)T} = c_m^{(m)}/Gamma I + A K, and
 *   dJ/dkappa = -sum_m lambda^m .* (A u^m),   dJ/df = sum_m lambda^m. */
int or_adjoint(const or_problem* p, const double* U, const double* u_obs,
               double* grad_kappa, double* grad_f) {
  const int64_t n = p->n, M = p->M;
  double* t = (double*)malloc(sizeof(double) * (size_t)n);
  if (or_ifl_symbol(p->alpha, p->mu, p->kappa_mu, n, p->l, t) != 0) { free(t); return -1; }
  const double Gg = tgamma(1.0 - p->gamma);
  /* C[j][k] = c_k^{(j)}, k = 1..j, all levels (O(M^2) table) */
  double* C = (double*)calloc((size_t)((M + 1) * (M + 2)), sizeof(double));
  for (int64_t j = 1; j <= M; ++j) level_weights(p, 1, j, C + j * (M + 2));
  double* Lam = (double*)calloc((size_t)((M + 1) * n), sizeof(double));
  double* Mat = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* rhs = (double*)malloc(sizeof(double) * (size_t)n);
  double* Au = (double*)malloc(sizeof(double) * (size_t)n);
  const double* kap = p->kappa;  /* row 0: time-independent */
  for (int64_t i = 0; i < n; ++i) { grad_kappa[i] = 0.0; grad_f[i] = 0.0; }
  int status = 0;
  for (int64_t m = M; m >= 1 && status == 0; --m) {
    for (int64_t i = 0; i < n; ++i)
      rhs[i] = (m == M) ? (U[M * n + i] - u_obs[i]) : 0.0;
    for (int64_t j = m + 1; j <= M; ++j) {
      const double* cj = C + j * (M + 2);
      double d = (cj[m + 1] - cj[m]) / Gg;
      for (int64_t i = 0; i < n; ++i) rhs[i] += d * Lam[j * n + i];
    }
    const double cm = C[m * (M + 2) + m];
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        int64_t d = i > j ? i - j : j - i;
        Mat[i * n + j] = t[d] * kap[j] + (i == j ? cm / Gg : 0.0);
      }
    if (or_lu_solve(n, Mat, rhs) != 0) status = -2;
    memcpy(Lam + m * n, rhs, sizeof(double) * (size_t)n);
    or_toeplitz_matvec(n, t, U + m * n, Au);
    for (int64_t i = 0; i < n; ++i) {
      grad_kappa[i] -= rhs[i] * Au[i];
      grad_f[i] += rhs[i];
    }
  }
  free(t); free(C); free(Lam); free(Mat); free(rhs); free(Au);
  return status;
}

/* ------------------------------------------------------------------ */
/* Defect of a level equation, d = b - (a u + kappa .* (A u)), evaluated in
 * double-double arithmetic and rounded once: every product is split exactly
 * by an FMA (the error-free product), every sum by Knuth's TwoSum, as in
 * the compensated dot product Dot2 of Ogita, Rump and Oishi (SIAM J. Sci.
 * Comput. 26, 2005).  The result carries an error of a few units of
 * 2^-104 times sum_j |terms|, so it stays meaningful where the defect is
 * 1e-12 of b while the terms kappa_i t_{|i-j|} u_j are ~1e8 times larger
 * (a plain FP64 sum would carry errors ~1e-16 of those).  Used to certify
 * GPU levels through the bound of Lemma 3.3 and Theorem 3.1:
 * ||u - u_exact||_inf <= ||d||_inf / a (diagonal dominance of a I + K A). */
static void two_sum(double a, double b, double* s, double* e) {
  const double x = a + b;
  const double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}
static void two_prod(double a, double b, double* p, double* e) {
  const double x = a * b;
  *e = fma(a, b, -x);
  *p = x;
}
/* (hi, lo) += x * y */
static void dd_add_prod(double* hi, double* lo, double x, double y) {
  double p, ep, s, es;
  two_prod(x, y, &p, &ep);
  two_sum(*hi, p, &s, &es);
  *hi = s;
  *lo += es + ep;
}

void or_level_defect(int64_t n, const double* t, double a, const double* kappa, const double* u,
                     const double* b, double* d) {
#pragma omp parallel for schedule(dynamic, 16) num_threads(or_threads) if (or_threads > 1)
  for (int64_t i = 0; i < n; ++i) {
    /* (A u)_i as a double-double */
    double h = 0.0, l = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      const int64_t k = i > j ? i - j : j - i;
      dd_add_prod(&h, &l, t[k], u[j]);
    }
    double ah, al;
    two_sum(h, l, &ah, &al);  /* normalise */
    /* kappa_i (ah + al): exact product of the high part, rounded low part */
    double kh, kl;
    two_prod(kappa[i], ah, &kh, &kl);
    kl += kappa[i] * al;
    /* b_i - a u_i - (kh + kl) */
    double rh = b[i], rl = 0.0;
    dd_add_prod(&rh, &rl, -a, u[i]);
    double s, e;
    two_sum(rh, -kh, &s, &e);
    rh = s;
    rl += e - kl;
    d[i] = rh + rl;
  }
}
