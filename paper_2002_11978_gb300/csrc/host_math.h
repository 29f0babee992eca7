// host_math.h -- setup-time host mathematics (no CUDA): graded mesh,
// sum-of-exponentials table, IFL Toeplitz symbol, a host FFT for the
// one-off spectra, and the per-level scalar tables.
#pragma once
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

namespace tsfde {

using cd = std::complex<double>;

// t_m = T (m/M)^r, m = 0..M (Sec. 3.1).
double mesh_t(double T, int64_t M, double r, int64_t m);
// t_m - t_k, 0 <= k <= m, via -t_m expm1(r log(k/m)) (no cancellation).
double mesh_gap(double T, int64_t M, double r, int64_t m, int64_t k);

// a_k^{(m)} of Eq. (2.8), 1 <= k <= m: the L1 weight of the interval
// [t_{k-1}, t_k] at level m, (1/tau_k) int (t_m - s)^{-gamma} ds.
double l1_weight(double T, int64_t M, double r, double gamma, int64_t m, int64_t k);

// c_{1,alpha} of Eq. (1.4).
double c1alpha(double alpha);

// First column of A, Eq. (3.16x); n = paper N - 1.
std::vector<double> ifl_symbol(double alpha, double mu, int kappa_mu, int64_t n,
                               double l);

// SOE table for t^{-gamma} on [delta, T] with relative error <= tol
// (Lemma 2.2).  Construction: trapezoidal rule in x = ln s for
// t^{-g} = Gamma(g)^{-1} int exp(-t e^x + g x) dx, with every node below
// s_c = c/T replaced by a p-point Gauss rule for the discrete measure those
// nodes define (Lanczos on the nodes, Jacobi eigen-solve of the p x p
// tridiagonal matrix).  The final table is verified on a dense log grid.
// Returns false if no table within the limits met tol.
bool soe_build(double gamma, double delta, double T, double tol,
               std::vector<double>& s, std::vector<double>& w, std::string* why);
double soe_rel_err(double gamma, double delta, double T, const std::vector<double>& s,
                   const std::vector<double>& w, int nsamp);

// In-place iterative radix-2 complex FFT of power-of-two size; sign = -1
// forward (e^{-2 pi i jk/N}), +1 inverse (unnormalised).
void fft_inplace(std::vector<cd>& a, int sign);
// W_L^k = e^{-2 pi i k / L}, k = 0..L-1, with octant symmetry for accuracy.
std::vector<cd> twiddles(int64_t L);
// e^{sign pi i m^2 / n} (Bluestein chirp) with m^2 reduced modulo 2n exactly.
cd chirp(int64_t m, int64_t n, int sign);

// Strang circulant first column (Sec. 4.1) and its eigenvalues F c_S by a
// Bluestein length-n DFT on length-L FFTs (L >= 2n-1, power of two).
std::vector<double> strang_eigs(const std::vector<double>& t, int64_t L);

// Even embedding [t_0..t_{n-1}, 0.., t_{n-1}..t_1] of length L and its
// (real) DFT S_0..S_{L-1}.
std::vector<double> embed_spectrum(const std::vector<double>& t, int64_t L);

}  // namespace tsfde
