// host_math.cpp -- setup-time host mathematics for the FIDS solver.
#include "host_math.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace tsfde {

static const double kPi = 3.14159265358979323846;

double mesh_t(double T, int64_t M, double r, int64_t m) {
  return T * std::pow((double)m / (double)M, r);
}

double mesh_gap(double T, int64_t M, double r, int64_t m, int64_t k) {
  if (k >= m) return 0.0;
  double tm = mesh_t(T, M, r, m);
  if (k == 0) return tm;
  return -tm * std::expm1(r * std::log((double)k / (double)m));
}

double l1_weight(double T, int64_t M, double r, double gamma, int64_t m, int64_t k) {
  const double tau = mesh_gap(T, M, r, k, k - 1);
  const double g1 = 1.0 - gamma;
  if (k == m) return std::pow(tau, -gamma) / g1;
  // (D_{k-1}^{g1} - D_k^{g1}) / (g1 tau) with D_{k-1} = D_k + tau, written
  // D_k^{g1} ((1 + tau/D_k)^{g1} - 1) so that nothing cancels when tau << D_k
  const double D = mesh_gap(T, M, r, m, k);
  return std::pow(D, g1) * std::expm1(g1 * std::log1p(tau / D)) / (g1 * tau);
}

double c1alpha(double alpha) {
  return std::pow(2.0, alpha - 1.0) * alpha * std::tgamma(0.5 * (alpha + 1.0)) /
         (std::sqrt(kPi) * std::tgamma(1.0 - 0.5 * alpha));
}

// (k+1)^nu - (k-1)^nu without cancellation: the two expm1 terms below have
// opposite signs.
static double gap_pow(double k, double nu) {
  if (k == 1.0) return std::pow(2.0, nu);
  return std::pow(k, nu) * (std::expm1(nu * std::log1p(1.0 / k)) -
                            std::expm1(nu * std::log1p(-1.0 / k)));
}

std::vector<double> ifl_symbol(double alpha, double mu, int kappa_mu, int64_t n,
                               double l) {
  std::vector<double> t(n);
  const int64_t N = n + 1;
  const double nu = mu - alpha;
  const double h = 2.0 * l / (double)N;
  const double C = c1alpha(alpha) / (nu * std::pow(h, alpha));
  const double neighbour = std::pow(2.0, nu) + (double)kappa_mu - 1.0;
  // diagonal bracket; the long sum is accumulated from its smallest term
  double acc = 0.0;
  for (int64_t q = N - 1; q >= 2; --q) {
    double Q = (double)q;
    acc += gap_pow(Q, nu) * std::pow(Q, -mu);
  }
  const double Nd = (double)N;
  const double lastN = std::pow(Nd, nu - mu) * (-std::expm1(nu * std::log1p(-1.0 / Nd)));
  t[0] = C * (acc + lastN + neighbour + 2.0 * nu / (alpha * std::pow(Nd, alpha)));
  if (n > 1) t[1] = -0.5 * C * neighbour;
  for (int64_t k = 2; k < n; ++k) {
    double K = (double)k;
    t[k] = -0.5 * C * gap_pow(K, nu) * std::pow(K, -mu);
  }
  return t;
}

// ---------------------------------------------------------------- SOE
double soe_rel_err(double gamma, double delta, double T, const std::vector<double>& s,
                   const std::vector<double>& w, int nsamp) {
  double worst = 0.0;
  const double la = std::log(delta), lb = std::log(T);
  for (int i = 0; i < nsamp; ++i) {
    double tt = std::exp(la + (lb - la) * (double)i / (double)(nsamp - 1));
    if (i == 0) tt = delta;
    if (i == nsamp - 1) tt = T;
    double acc = 0.0;
    for (size_t j = 0; j < s.size(); ++j) acc += w[j] * std::exp(-s[j] * tt);
    worst = std::max(worst, std::fabs(std::pow(tt, gamma) * acc - 1.0));
  }
  return worst;
}

// Cyclic Jacobi eigen-solver for a small dense symmetric matrix (row-major);
// returns eigenvalues and the first row of the eigenvector matrix.
static void jacobi_eig(int p, std::vector<double> A, std::vector<double>& lam,
                       std::vector<double>& v0) {
  std::vector<double> V(p * p, 0.0);
  for (int i = 0; i < p; ++i) V[i * p + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < p; ++i)
      for (int j = i + 1; j < p; ++j) off += A[i * p + j] * A[i * p + j];
    if (off < 1e-300) break;
    for (int a = 0; a < p; ++a)
      for (int b = a + 1; b < p; ++b) {
        double apq = A[a * p + b];
        if (std::fabs(apq) < 1e-300) continue;
        double theta = (A[b * p + b] - A[a * p + a]) / (2.0 * apq);
        double tq = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(tq * tq + 1.0), sn = tq * c;
        for (int k = 0; k < p; ++k) {  // A <- A J
          double x = A[k * p + a], y = A[k * p + b];
          A[k * p + a] = c * x - sn * y;
          A[k * p + b] = sn * x + c * y;
        }
        for (int k = 0; k < p; ++k) {  // A <- J^T A
          double x = A[a * p + k], y = A[b * p + k];
          A[a * p + k] = c * x - sn * y;
          A[b * p + k] = sn * x + c * y;
        }
        for (int k = 0; k < p; ++k) {  // V <- V J
          double x = V[k * p + a], y = V[k * p + b];
          V[k * p + a] = c * x - sn * y;
          V[k * p + b] = sn * x + c * y;
        }
      }
  }
  lam.resize(p);
  v0.resize(p);
  for (int i = 0; i < p; ++i) {
    lam[i] = A[i * p + i];
    v0[i] = V[0 * p + i];
  }
}

// p-point Gauss rule for the discrete measure sum_j w_j delta(y - y_j),
// y_j in (0,1]: Lanczos with full re-orthogonalisation builds the Jacobi
// matrix of the measure; its eigenvalues are the nodes and mu0 times the
// squared first eigenvector components the weights.
static void discrete_gauss(const std::vector<double>& y, const std::vector<double>& w, int p,
                           std::vector<double>& ny, std::vector<double>& nw) {
  const size_t K = y.size();
  double mu0 = 0.0;
  for (double x : w) mu0 += x;
  p = std::min<int>(p, (int)K);
  std::vector<std::vector<double>> Q;
  std::vector<double> q(K);
  for (size_t j = 0; j < K; ++j) q[j] = std::sqrt(w[j] / mu0);
  std::vector<double> a, b;
  for (int k = 0; k < p; ++k) {
    Q.push_back(q);
    std::vector<double> v(K);
    for (size_t j = 0; j < K; ++j) v[j] = y[j] * q[j];
    double ak = 0.0;
    for (size_t j = 0; j < K; ++j) ak += q[j] * v[j];
    a.push_back(ak);
    for (int pass = 0; pass < 2; ++pass)
      for (auto& qq : Q) {
        double d = 0.0;
        for (size_t j = 0; j < K; ++j) d += qq[j] * v[j];
        for (size_t j = 0; j < K; ++j) v[j] -= d * qq[j];
      }
    double bk = 0.0;
    for (double x : v) bk += x * x;
    bk = std::sqrt(bk);
    if (k + 1 < p) {
      if (bk < 1e-14) { p = k + 1; break; }
      b.push_back(bk);
      for (size_t j = 0; j < K; ++j) q[j] = v[j] / bk;
    }
  }
  p = (int)a.size();
  std::vector<double> J(p * p, 0.0);
  for (int i = 0; i < p; ++i) {
    J[i * p + i] = a[i];
    if (i + 1 < p) J[i * p + i + 1] = J[(i + 1) * p + i] = b[i];
  }
  std::vector<double> lam, v0;
  jacobi_eig(p, J, lam, v0);
  ny = lam;
  nw.resize(p);
  for (int i = 0; i < p; ++i) nw[i] = mu0 * v0[i] * v0[i];
}

bool soe_build(double gamma, double delta, double T, double tol, std::vector<double>& s,
               std::vector<double>& w, std::string* why) {
  const double gg = std::tgamma(gamma);
  // left end: int_{-inf}^{x_lo} e^{g x} dx = e^{g x_lo}/g, relative to
  // Gamma(g) t^{-g} at t = T
  const double x_lo = (std::log(0.02 * tol * gamma * gg) - gamma * std::log(T)) / gamma;
  // right end: (delta s_hi)^{g-1} e^{-delta s_hi} / Gamma(g) <= 0.02 tol
  double z = 1.0;
  for (int it = 0; it < 100; ++it) z = std::max(1.0, std::log(50.0 / (tol * gg)) + (gamma - 1.0) * std::log(z));
  const double x_hi = std::log((z + 1.0) / delta);
  // step: discretisation error ~ 2 (cos d)^{-g} e^{-2 pi d / h}, d = 1.45
  const double d = 1.45;
  // start coarser than the bound (it is pessimistic) and shrink until the
  // verified error meets tol
  double h = 1.3 * 2.0 * kPi * d / std::log(2.0 * std::pow(std::cos(d), -gamma) * 20.0 / tol);
  const double s_c = 8.0 / T;
  for (int attempt = 0; attempt < 60; ++attempt, h *= 0.96) {
    std::vector<double> ys, yw, bs, bw;
    const int J = (int)std::ceil((x_hi - x_lo) / h);
    for (int j = 0; j <= J; ++j) {
      double x = x_lo + h * j;
      double sj = std::exp(x), wj = h * std::exp(gamma * x) / gg;
      if (sj < s_c) { ys.push_back(sj / s_c); yw.push_back(wj); }
      else { bs.push_back(sj); bw.push_back(wj); }
    }
    for (int p : {12, 16, 20}) {
      std::vector<double> gy, gw;
      discrete_gauss(ys, yw, p, gy, gw);
      std::vector<std::pair<double, double>> all;
      for (size_t i = 0; i < gy.size(); ++i)
        if (gw[i] > 0.0 && gy[i] > 0.0) all.push_back({gy[i] * s_c, gw[i]});
      for (size_t i = 0; i < bs.size(); ++i) all.push_back({bs[i], bw[i]});
      std::sort(all.begin(), all.end());
      s.clear(); w.clear();
      for (auto& pr : all) { s.push_back(pr.first); w.push_back(pr.second); }
      if (soe_rel_err(gamma, delta, T, s, w, 20001) <= tol) return true;
    }
  }
  if (why) *why = "SOE construction did not reach the requested tolerance";
  return false;
}

// ---------------------------------------------------------------- FFT
// cos(pi num/den), sin(pi num/den) for integers num >= 0, den > 0, with the
// angle reduced exactly to [0, pi/4] before calling the libm functions.
static void cospi_sinpi(int64_t num, int64_t den, double* c, double* s) {
  num %= 2 * den;
  double sc = 1.0, ss = 1.0;
  if (num >= den) { num -= den; sc = -1.0; ss = -1.0; }  // phi + pi
  if (2 * num > den) { num = den - num; sc = -sc; }        // pi - phi
  double cc, sv;
  if (4 * num > den) {  // pi/2 - phi'
    double a = kPi * (double)(den - 2 * num) / (2.0 * (double)den);
    cc = std::sin(a); sv = std::cos(a);
  } else {
    double a = kPi * (double)num / (double)den;
    cc = std::cos(a); sv = std::sin(a);
  }
  *c = sc * cc;
  *s = ss * sv;
}

std::vector<cd> twiddles(int64_t L) {
  std::vector<cd> tw(L);
  for (int64_t k = 0; k < L; ++k) {
    double c, s;
    cospi_sinpi(2 * k, L, &c, &s);
    tw[k] = cd(c, -s);  // e^{-2 pi i k / L}
  }
  return tw;
}

cd chirp(int64_t m, int64_t n, int sign) {
  // e^{sign pi i m^2 / n}; m^2 reduced mod 2n in integers
  int64_t q = (m % (2 * n)) * (m % (2 * n)) % (2 * n);
  double c, s;
  cospi_sinpi(q, n, &c, &s);
  return cd(c, sign * s);
}

void fft_inplace(std::vector<cd>& a, int sign) {
  const int64_t N = (int64_t)a.size();
  for (int64_t i = 1, j = 0; i < N; ++i) {
    int64_t bit = N >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  std::vector<cd> tw = twiddles(N);
  for (int64_t len = 2; len <= N; len <<= 1) {
    int64_t step = N / len;
    for (int64_t i = 0; i < N; i += len)
      for (int64_t k = 0; k < len / 2; ++k) {
        cd w = tw[k * step];
        if (sign > 0) w = std::conj(w);
        cd u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
  }
}

// ---------------------------------------------------------------------
// Double-double arithmetic for the symbol spectrum.  A value is hi + lo
// with |lo| <= ulp(hi)/2 (Dekker 1971); sums use Knuth's TwoSum, products
// the exact FMA split, and results are renormalised (the "accurate"
// double-double sum of Hida, Li and Bailey).  About 106 significant bits.
namespace {

struct ddv {
  double hi, lo;
};

inline ddv quick_two_sum(double a, double b) {
  const double s = a + b;
  return {s, b - (s - a)};
}
inline ddv two_sum_dd(double a, double b) {
  const double s = a + b;
  const double bv = s - a;
  return {s, (a - (s - bv)) + (b - bv)};
}
inline ddv dd_add(ddv a, ddv b) {
  ddv s = two_sum_dd(a.hi, b.hi);
  const ddv t = two_sum_dd(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
inline ddv dd_neg(ddv a) { return {-a.hi, -a.lo}; }
inline ddv dd_sub(ddv a, ddv b) { return dd_add(a, dd_neg(b)); }
inline ddv dd_mul(ddv a, ddv b) {
  const double p = a.hi * b.hi;
  double e = std::fma(a.hi, b.hi, -p);
  e += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p, e);
}
inline ddv dd_div_d(ddv a, double b) {
  const double q1 = a.hi / b;
  const double p = q1 * b;
  const double pe = std::fma(q1, b, -p);
  const double r = ((a.hi - p) - pe) + a.lo;
  return quick_two_sum(q1, r / b);
}

struct ddc {
  ddv re, im;
};
inline ddc dc_add(ddc a, ddc b) { return {dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
inline ddc dc_sub(ddc a, ddc b) { return {dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; }
inline ddc dc_mul(ddc a, ddc b) {
  return {dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im)), dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))};
}

// cos and sin of x, |x| <= pi/4, by their Taylor series in Horner form, up
// to x^28/28! and x^29/29! (the next terms are below 1e-35).
void dd_sincos_small(ddv x, ddv& c, ddv& s) {
  constexpr int K = 29;
  ddv inv[K + 1];  // 1/k!
  inv[0] = {1.0, 0.0};
  for (int k = 1; k <= K; ++k) inv[k] = dd_div_d(inv[k - 1], (double)k);
  const ddv x2 = dd_mul(x, x);
  ddv sc = {0.0, 0.0}, ss = {0.0, 0.0};
  for (int k = 14; k >= 0; --k) {
    // cos: sum (-1)^k x^{2k} / (2k)!;  sin / x: sum (-1)^k x^{2k} / (2k+1)!
    const ddv ck = (k & 1) ? dd_neg(inv[2 * k]) : inv[2 * k];
    const ddv sk = (k & 1) ? dd_neg(inv[2 * k + 1]) : inv[2 * k + 1];
    sc = dd_add(dd_mul(sc, x2), ck);
    ss = dd_add(dd_mul(ss, x2), sk);
  }
  c = sc;
  s = dd_mul(ss, x);
}

// e^{-2 pi i m / L} in double-double for 0 <= m < L (L a power of two >= 8):
// the angle is reduced to the first octant by exact integer symmetries.
void dd_twiddle_table(int64_t L, std::vector<ddc>& w) {
  const ddv two_pi = {6.283185307179586232, 2.449293598294706414e-16};
  const int64_t L8 = L / 8, L4 = L / 4, L2 = L / 2;
  std::vector<ddv> co(L8 + 1), si(L8 + 1);
  for (int64_t m = 0; m <= L8; ++m) {
    const ddv x = {two_pi.hi * ((double)m / (double)L), two_pi.lo * ((double)m / (double)L)};
    dd_sincos_small(x, co[m], si[m]);
  }
  auto cs = [&](int64_t m, ddv& c, ddv& s) {  // 0 <= m <= L/4
    if (m <= L8) { c = co[m]; s = si[m]; }
    else { c = si[L4 - m]; s = co[L4 - m]; }
  };
  w.resize(L);
  for (int64_t m = 0; m < L; ++m) {
    ddv c, s;
    int64_t q = m;
    bool neg_c = false, neg_s = false, swap = false;
    if (q >= L2) { q -= L2; neg_c = !neg_c; neg_s = !neg_s; }   // theta = pi + psi
    if (q > L4) { q -= L4; swap = true; }                      // theta = pi/2 + phi
    cs(q, c, s);
    if (swap) { const ddv t = c; c = dd_neg(s); s = t; }       // cos = -sin phi, sin = cos phi
    if (neg_c) c = dd_neg(c);
    if (neg_s) s = dd_neg(s);
    w[m] = {c, dd_neg(s)};
  }
}

}  // namespace

// The spectrum of the even embedding is computed in double-double and rounded
// once.  Its low-frequency values (S_0 is the row-sum excess of A, ~0.1 at
// n = 2^17 - 1) are differences of sums of entries up to t_0 ~ 1e8, so a
// double FFT leaves them absolute errors ~1e-16 log L sum|t_k|, i.e. 1e-9
// relative at S_0, an error every product with A would carry into the
// smooth modes of the solution.
std::vector<double> embed_spectrum(const std::vector<double>& t, int64_t L) {
  const int64_t n = (int64_t)t.size();
  std::vector<ddc> e(L, ddc{{0.0, 0.0}, {0.0, 0.0}});
  for (int64_t k = 0; k < n; ++k) e[k].re = {t[k], 0.0};
  for (int64_t k = 1; k < n; ++k) e[L - k].re = {t[k], 0.0};
  for (int64_t i = 1, j = 0; i < L; ++i) {
    int64_t bit = L >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(e[i], e[j]);
  }
  std::vector<ddc> tw;
  dd_twiddle_table(L, tw);
  for (int64_t len = 2; len <= L; len <<= 1) {
    const int64_t step = L / len;
    for (int64_t i = 0; i < L; i += len)
      for (int64_t k = 0; k < len / 2; ++k) {
        const ddc u = e[i + k], v = dc_mul(e[i + k + len / 2], tw[k * step]);
        e[i + k] = dc_add(u, v);
        e[i + k + len / 2] = dc_sub(u, v);
      }
  }
  std::vector<double> S(L);
  for (int64_t k = 0; k < L; ++k) S[k] = e[k].re.hi + e[k].re.lo;
  return S;
}

std::vector<double> strang_eigs(const std::vector<double>& t, int64_t L) {
  const int64_t n = (int64_t)t.size();
  std::vector<double> cS(n);
  for (int64_t k = 0; k < n; ++k) cS[k] = (k <= n / 2) ? t[k] : t[n - k];
  if (n == 1) return cS;
  // lambda_k = sum_j cS_j e^{-2 pi i jk/n}; jk = (j^2 + k^2 - (k-j)^2)/2
  // with chirp c_m = e^{-pi i m^2 / n}: lambda_k = c_k sum_j (cS_j c_j) conj(c_{k-j})
  std::vector<cd> ch(n);
  for (int64_t m = 0; m < n; ++m) ch[m] = chirp(m, n, -1);
  std::vector<cd> a(L, cd(0, 0)), b(L, cd(0, 0));
  for (int64_t j = 0; j < n; ++j) a[j] = cS[j] * ch[j];
  for (int64_t m = 0; m < n; ++m) b[m] = std::conj(ch[m]);
  for (int64_t m = 1; m < n; ++m) b[L - m] = std::conj(ch[m]);
  fft_inplace(a, -1);
  fft_inplace(b, -1);
  for (int64_t k = 0; k < L; ++k) a[k] *= b[k];
  fft_inplace(a, +1);
  std::vector<double> lam(n);
  for (int64_t k = 0; k < n; ++k) lam[k] = (ch[k] * a[k] / (double)L).real();
  return lam;
}

}  // namespace tsfde
