// abi.cpp -- C ABI of the FIDS solver: argument validation, setup tables,
// device workspaces and the per-level launch sequence.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/tsfde.h"
#include "host_math.h"
#include "plan.h"

using namespace tsfde;

// Order of the extrapolated start (warm_start = 2): the level solve starts
// from the polynomial in the level index through the last kStartOrder + 1
// levels.  The SOE-history context rotates kRoll = kStartOrder + 1 level
// buffers (at least 3: the right-hand side reads u^{m-1} and u^{m-2} while
// u^m is written).
constexpr int kStartOrder = 3;
constexpr int kRoll = kStartOrder + 1 > 3 ? kStartOrder + 1 : 3;
static_assert(kStartOrder <= kMaxStartOrder, "LevelArgs.up holds kMaxStartOrder + 1 levels");

struct tsfde_ctx {
  double alpha = 0, gamma = 0, l = 0, T = 0, r = 0, soe_tol = 0, mu = 0;
  int kappa_mu = 1;
  int64_t n = 0, M = 0;
  tsfde_opts opts{};
  cudaStream_t stream = nullptr;
  int64_t m = 0;
  bool have_problem = false;
  std::string err;
  // host tables
  std::vector<double> tmesh, ahat, soe_s, soe_w, symbol, theta, Gsrc, eps_h, cw_h;
  std::vector<int> Eact;
  int E = 0, rank = 0, ld = 0;
  bool kap1 = false;
  // device
  DevPlan P{};
  std::vector<void*> allocs;
  double *G = nullptr, *eps = nullptr, *cw = nullptr;
  double* u[kRoll] = {};  // rotating levels u^m, u^{m-1}, ... (SOE history)
  double *b = nullptr, *kappa64 = nullptr, *phi = nullptr, *kap0 = nullptr, *kap1d = nullptr;
  double* F = nullptr;
  float* kappa32 = nullptr;
  KVecs<double> k64{};
  KVecs<float> k32{};
  KVecs<dsf> kds{};        // TSFDE_MIXED_DS inner vectors
  dsf* kappads = nullptr;
  double* hinv64 = nullptr;  // PCG: 1/kappa^m
  float* hinv32 = nullptr;
  dsf* hinvds = nullptr;
  double* r64 = nullptr;
  // direct history (DIDS): every level u^0..u^M (rows of ld doubles) and the
  // packed weights, row m (m entries) at offset m(m-1)/2
  double* Uh = nullptr;
  double* wdir = nullptr;
  StepStat* stats = nullptr;
  int* status = nullptr;
  KrylovAuto* kauto = nullptr;  // TSFDE_KRYLOV_AUTO: per-level method choice
  int* pre_status = nullptr;     // double-single: status of the separate preconditioner build
  KrylovAuto kauto_init{};       // host source of the reset copy (outlives it)
  int engine = TSFDE_ENGINE_GRID;  // engine of the mixed level solves
  // checkpoints of the forward march for the adjoint sweep (ckpt_stride):
  // slot j = level k = j * ck_stride holds [u^{k-1} | u^k | G^k] (rows of
  // ld doubles; G^k = the E x ld history after level k's right-hand side),
  // everything needed to march on from level k
  int64_t ck_stride = 0, ck_slots = 0;
  size_t ck_slot = 0;               // doubles per slot, (kRoll + E) ld
  double* ck = nullptr;
  double* ck_seg = nullptr;         // ck_stride recomputed levels, rows of n
  double* ck_save = nullptr;        // forward state kept across a sweep: u[kRoll], G
  KrylovAuto* ck_kauto = nullptr;   // ... and the method-choice state
  std::vector<char> ck_ok;          // slot recorded in the current march
  bool ck_override = false;         // a level took per-level kappa_m / f_m
  bool ck_recomputing = false;
  std::vector<int> ck_kry;          // Krylov method of each level, replayed when recomputing
  // adjoint work buffers (allocated by the first tsfde_adjoint)
  double* adjY = nullptr;       // E x ld reversed SOE history
  double* adjLam[2] = {nullptr, nullptr};
  double* adjG = nullptr;
  StepStat* adjStats = nullptr;
  // profiling: three events per level (before rhs, after rhs, after level)
  std::vector<cudaEvent_t> ev_free, ev_used;
};

namespace {

const double kTimeoutDefault = 2.0e9;

int fail(tsfde_ctx* c, int st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

int cuda_fail(tsfde_ctx* c, cudaError_t e, const char* where) {
  return fail(c, TSFDE_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Every workspace starts zeroed: a buffer read before its first write (a
// Krylov direction at beta = 0, the padding of an FP32 or double-single
// vector) must never see what an earlier user of the memory left there, since
// 0 * NaN is NaN.
template <typename T> bool dalloc(tsfde_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) return false;
  c->allocs.push_back(q);
  if (cudaMemset(q, 0, count * sizeof(T)) != cudaSuccess) return false;
  *p = static_cast<T*>(q);
  return true;
}

template <typename T> cudaError_t upload(T* dst, const std::vector<T>& src) {
  return cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Device vector of level m: a row of the stored levels with the direct
// history, else one of kRoll rotating buffers.
double* ulev(tsfde_ctx* c, int64_t m) {
  return c->Uh ? c->Uh + (size_t)m * c->ld : c->u[m % kRoll];
}

// Checkpoint of level k (a multiple of ck_stride): u^{k-kStartOrder} .. u^k
// (the levels an extrapolated start of level k + 1 reads) and the SOE
// history after level k's right-hand side, copied on the context's stream.
cudaError_t record_ckpt(tsfde_ctx* c, int64_t k) {
  const int64_t j = k / c->ck_stride;
  double* slot = c->ck + c->ck_slot * (size_t)j;
  const size_t nb = sizeof(double) * (size_t)c->n;
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < kRoll && e == cudaSuccess; ++q)  // u^{k-kRoll+1} .. u^k (those that exist)
    if (k - kRoll + 1 + q >= 0)
      e = cudaMemcpyAsync(slot + q * (size_t)c->ld, ulev(c, k - kRoll + 1 + q), nb, cudaMemcpyDeviceToDevice,
                          c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(slot + kRoll * (size_t)c->ld, c->G, sizeof(double) * (size_t)std::max(c->E, 1) * c->ld,
                        cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) c->ck_ok[j] = 1;
  return e;
}

// Make checkpoint k the current state of the march (c->m = k).
cudaError_t restore_ckpt(tsfde_ctx* c, int64_t k) {
  const double* slot = c->ck + c->ck_slot * (size_t)(k / c->ck_stride);
  const size_t nb = sizeof(double) * (size_t)c->n;
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < kRoll && e == cudaSuccess; ++q)
    if (k - kRoll + 1 + q >= 0)
      e = cudaMemcpyAsync(ulev(c, k - kRoll + 1 + q), slot + q * (size_t)c->ld, nb, cudaMemcpyDeviceToDevice,
                          c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->G, slot + kRoll * (size_t)c->ld, sizeof(double) * (size_t)std::max(c->E, 1) * c->ld,
                        cudaMemcpyDeviceToDevice, c->stream);
  c->m = k;
  return e;
}

// Keep (save = true) or bring back the forward state: the rotating levels,
// the SOE history and the method-choice state.
cudaError_t keep_forward_state(tsfde_ctx* c, bool save) {
  const size_t nb = sizeof(double) * (size_t)c->n;
  const size_t gb = sizeof(double) * (size_t)std::max(c->E, 1) * c->ld;
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < kRoll && e == cudaSuccess; ++q) {
    double* keep = c->ck_save + (size_t)q * c->ld;
    e = save ? cudaMemcpyAsync(keep, c->u[q], nb, cudaMemcpyDeviceToDevice, c->stream)
             : cudaMemcpyAsync(c->u[q], keep, nb, cudaMemcpyDeviceToDevice, c->stream);
  }
  double* gkeep = c->ck_save + kRoll * (size_t)c->ld;
  if (e == cudaSuccess)
    e = save ? cudaMemcpyAsync(gkeep, c->G, gb, cudaMemcpyDeviceToDevice, c->stream)
             : cudaMemcpyAsync(c->G, gkeep, gb, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess && c->kauto)
    e = save ? cudaMemcpyAsync(c->ck_kauto, c->kauto, sizeof(KrylovAuto), cudaMemcpyDeviceToDevice, c->stream)
             : cudaMemcpyAsync(c->kauto, c->ck_kauto, sizeof(KrylovAuto), cudaMemcpyDeviceToDevice, c->stream);
  return e;
}


int ilog2(int64_t x) {
  int k = 0;
  while ((int64_t(1) << k) < x) ++k;
  return k;
}

// Column tiles are sized so that their count matches the N1/2 + 1 row pairs
// (one work item per CTA in every pass): one column per tile when
// N1 = 2 N2, two when N1 = N2.  The real-input geometry keeps one column
// (its passes run at prefetch depth 2, which covers N1 elements per item up
// to n = 2^17 - 1); the complex geometry of the preconditioner build (depth
// 4) takes two when N1 = N2.
Geo make_geo(int Nfft, bool pair_columns) {
  Geo g{};
  const int lg = ilog2(Nfft);
  g.Nfft = Nfft;
  g.lgN1 = (lg + 1) / 2;
  g.N1 = 1 << g.lgN1;
  g.lgN2 = lg - g.lgN1;
  g.N2 = 1 << g.lgN2;
  const int lc = (pair_columns && g.N1 == g.N2 && g.N2 >= 2) ? 1 : 0;
  g.lgct64 = lc;
  g.lgct32 = lc;
  return g;
}

int items(const Geo& g) {
  return std::max((g.N2 >> std::min(g.lgct64, g.lgct32)), (g.N1 >> 1) + 1);
}

}  // namespace

extern "C" {

int tsfde_default_opts(tsfde_opts* o) {
  if (!o) return TSFDE_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->mu = 0.0;
  o->kappa_mu = 0;
  o->krylov_tol = 1e-12;
  o->max_it = 2000;
  o->precision = TSFDE_FP64;
  o->precond = TSFDE_STRANG;
  o->inner_tol = 1e-2;
  o->max_outer = 60;
  o->inner_max_it = 40;
  o->soe_E = 0;
  o->soe_s = nullptr;
  o->soe_w = nullptr;
  o->profile = 0;
  o->barrier_timeout_cycles = 0;
  o->stream = nullptr;
  o->engine = TSFDE_ENGINE_AUTO;
  o->cluster_size = 0;
  o->warm_start = 0;
  o->history = TSFDE_HISTORY_SOE;
  o->krylov = TSFDE_KRYLOV_BICGSTAB;
  o->ckpt_stride = 0;
  return TSFDE_OK;
}

const char* tsfde_strerror(int s) {
  switch (s) {
    case TSFDE_OK: return "ok";
    case TSFDE_EINVAL: return "invalid argument";
    case TSFDE_ENOMEM: return "out of memory";
    case TSFDE_ECUDA: return "CUDA runtime error";
    case TSFDE_ENOCONV: return "Krylov iteration cap reached";
    case TSFDE_EBREAKDOWN: return "BiCGSTAB breakdown";
    case TSFDE_ETIMEOUT: return "device barrier timed out";
    case TSFDE_ESTATE: return "call not valid in the current state";
    case TSFDE_ENONFINITE: return "non-finite value in the solver";
    case TSFDE_ENOTSUP: return "unsupported option";
    default: return "unknown status";
  }
}

const char* tsfde_last_error(const tsfde_ctx* c) { return c ? c->err.c_str() : ""; }

void tsfde_destroy(tsfde_ctx* c) {
  if (!c) return;
  for (cudaEvent_t e : c->ev_used) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
  for (void* p : c->allocs) cudaFree(p);
  delete c;
}

static int setup_impl(tsfde_ctx* c, double alpha, double gamma, double l, double T, int64_t n,
                      int64_t M, double r, double soe_tol, const tsfde_opts* opts) {
  if (opts) c->opts = *opts; else tsfde_default_opts(&c->opts);
  tsfde_opts& o = c->opts;
  if (!(alpha > 0.0 && alpha < 2.0)) return fail(c, TSFDE_EINVAL, "alpha must be in (0,2)");
  if (!(gamma > 0.0 && gamma < 1.0)) return fail(c, TSFDE_EINVAL, "gamma must be in (0,1)");
  if (!(l > 0.0) || !std::isfinite(l)) return fail(c, TSFDE_EINVAL, "l must be positive");
  if (!(T > 0.0) || !std::isfinite(T)) return fail(c, TSFDE_EINVAL, "T must be positive");
  if (n < 1) return fail(c, TSFDE_EINVAL, "n must be >= 1");
  if (n > (int64_t(1) << 18)) return fail(c, TSFDE_ENOTSUP, "n > 2^18 is not supported");
  if (M < 1) return fail(c, TSFDE_EINVAL, "M must be >= 1");
  if (!(r >= 1.0) || !std::isfinite(r)) return fail(c, TSFDE_EINVAL, "grading r must be >= 1");
  if (!(soe_tol > 0.0 && soe_tol <= 1e-2)) return fail(c, TSFDE_EINVAL, "soe_tol must be in (0,1e-2]");
  double mu = o.mu > 0.0 ? o.mu : 1.0 + 0.5 * alpha;
  if (!(mu > alpha && mu <= 2.0)) return fail(c, TSFDE_EINVAL, "mu must be in (alpha,2]");
  int kmu = o.kappa_mu > 0 ? o.kappa_mu : (mu == 2.0 ? 2 : 1);
  if (kmu != 1 && kmu != 2) return fail(c, TSFDE_EINVAL, "kappa_mu must be 1 or 2");
  if (!(o.krylov_tol > 0.0)) return fail(c, TSFDE_EINVAL, "krylov_tol must be positive");
  if (o.max_it < 1) return fail(c, TSFDE_EINVAL, "max_it must be >= 1");
  if (o.precision != TSFDE_FP64 && o.precision != TSFDE_MIXED && o.precision != TSFDE_MIXED_DS)
    return fail(c, TSFDE_EINVAL, "precision must be TSFDE_FP64, TSFDE_MIXED or TSFDE_MIXED_DS");
  if (o.precond != TSFDE_STRANG && o.precond != TSFDE_PRECOND_NONE)
    return fail(c, TSFDE_EINVAL, "precond must be TSFDE_STRANG or TSFDE_PRECOND_NONE");
  if (o.precision != TSFDE_FP64 &&
      (!(o.inner_tol > 0.0 && o.inner_tol < 1.0) || o.max_outer < 1 || o.inner_max_it < 1))
    return fail(c, TSFDE_EINVAL, "mixed needs inner_tol in (0,1), max_outer >= 1, inner_max_it >= 1");
  if (o.barrier_timeout_cycles < 0) return fail(c, TSFDE_EINVAL, "barrier_timeout_cycles < 0");
  if (o.engine != TSFDE_ENGINE_AUTO && o.engine != TSFDE_ENGINE_GRID && o.engine != TSFDE_ENGINE_CLUSTER)
    return fail(c, TSFDE_EINVAL, "engine must be TSFDE_ENGINE_AUTO, _GRID or _CLUSTER");
  if (o.history != TSFDE_HISTORY_SOE && o.history != TSFDE_HISTORY_DIRECT)
    return fail(c, TSFDE_EINVAL, "history must be TSFDE_HISTORY_SOE or TSFDE_HISTORY_DIRECT");
  if (o.krylov != TSFDE_KRYLOV_BICGSTAB && o.krylov != TSFDE_KRYLOV_PCG && o.krylov != TSFDE_KRYLOV_AUTO)
    return fail(c, TSFDE_EINVAL, "krylov must be TSFDE_KRYLOV_BICGSTAB, _PCG or _AUTO");
  if (o.warm_start < 0 || o.warm_start > 2) return fail(c, TSFDE_EINVAL, "warm_start must be 0, 1 or 2");
  if (o.ckpt_stride < -1) return fail(c, TSFDE_EINVAL, "ckpt_stride must be -1 (sqrt M), 0 (off) or positive");
  if (o.ckpt_stride != 0 && o.history != TSFDE_HISTORY_SOE)
    return fail(c, TSFDE_EINVAL, "checkpoints serve the FIDS adjoint (history = SOE)");
  if (o.krylov != TSFDE_KRYLOV_BICGSTAB && o.precision == TSFDE_MIXED && o.engine == TSFDE_ENGINE_CLUSTER)
    return fail(c, TSFDE_ENOTSUP, "the cluster engine runs BiCGSTAB only");
  c->alpha = alpha; c->gamma = gamma; c->l = l; c->T = T; c->n = n; c->M = M; c->r = r;
  c->soe_tol = soe_tol; c->mu = mu; c->kappa_mu = kmu;
  c->stream = static_cast<cudaStream_t>(o.stream);

  // ---- mesh and per-level scalars (Sec. 3.1, Eq. (2.8))
  c->tmesh.resize(M + 1);
  for (int64_t m = 0; m <= M; ++m) c->tmesh[m] = mesh_t(T, M, r, m);
  std::vector<double> tau(M + 1, 0.0);
  for (int64_t m = 1; m <= M; ++m) tau[m] = mesh_gap(T, M, r, m, m - 1);
  const double G2 = std::tgamma(2.0 - gamma), G1 = std::tgamma(1.0 - gamma);
  c->ahat.assign(M + 1, 0.0);
  for (int64_t m = 1; m <= M; ++m) c->ahat[m] = std::pow(tau[m], -gamma) / G2;

  // ---- SOE table (Lemma 2.2)
  if (o.soe_E > 0) {
    if (!o.soe_s || !o.soe_w) return fail(c, TSFDE_EINVAL, "soe_E > 0 needs soe_s and soe_w");
    c->soe_s.assign(o.soe_s, o.soe_s + o.soe_E);
    c->soe_w.assign(o.soe_w, o.soe_w + o.soe_E);
    for (int j = 0; j < o.soe_E; ++j) {
      if (!(c->soe_s[j] > 0.0) || !(c->soe_w[j] > 0.0)) return fail(c, TSFDE_EINVAL, "SOE nodes/weights must be positive");
      if (j > 0 && c->soe_s[j] < c->soe_s[j - 1]) return fail(c, TSFDE_EINVAL, "SOE nodes must be ascending");
    }
  } else {
    std::string why;
    if (!soe_build(gamma, tau[1], T, soe_tol, c->soe_s, c->soe_w, &why)) return fail(c, TSFDE_EINVAL, why);
  }
  const int E = c->E = (int)c->soe_s.size();
  c->eps_h.assign((size_t)(M + 1) * E, 0.0);
  c->cw_h.assign((size_t)(M + 1) * E, 0.0);
  c->Eact.assign(M + 1, 0);
  for (int64_t m = 2; m <= M; ++m) {
    int act = 0;
    for (int j = 0; j < E; ++j) {
      const double sj = c->soe_s[j];
      const double e = std::exp(-sj * tau[m]);
      const double x = sj * tau[m - 1];
      const double beta = (x == 0.0) ? 1.0 : -std::expm1(-x) / x;
      c->eps_h[m * E + j] = e;
      c->cw_h[m * E + j] = c->soe_w[j] * beta / G1;
      if (e > 0.0) act = j + 1;
    }
    c->Eact[m] = act;
  }
  c->Eact[1] = 0;

  // ---- IFL symbol (Eq. (3.16x)), spectra and Strang eigenvalues (Sec. 4.1)
  c->symbol = ifl_symbol(alpha, mu, kmu, n, l);
  int64_t L = 8;
  while (L < 2 * n - 1) L *= 2;
  DevPlan& P = c->P;
  P.n = (int)n;
  P.L = (int)L;
  P.Nc = (int)(L / 2);
  P.gr = make_geo(P.Nc, false);
  P.gc = make_geo(P.L, true);
  P.T = std::max(std::max(P.gr.N1, P.gr.N2), std::max(P.gc.N1, P.gc.N2));
  P.W = std::max(std::max(P.gr.N1 << P.gr.lgct64, 2 * P.gr.N2),
                 std::max(P.gc.N1 << P.gc.lgct64, 2 * P.gc.N2));
  P.timeout = o.barrier_timeout_cycles > 0 ? o.barrier_timeout_cycles : (long long)kTimeoutDefault;

  std::vector<double> S = embed_spectrum(c->symbol, L);
  std::vector<cd> tw = twiddles(L);
  std::vector<double> lam = strang_eigs(c->symbol, L);
  for (double x : lam)
    if (!(x > 0.0)) return fail(c, TSFDE_EINVAL, "Strang eigenvalue not positive (Lemma 4.1 violated)");
  const int Nc = P.Nc, N1 = P.gr.N1, N2 = P.gr.N2;
  std::vector<double> sa(Nc), sb(Nc);
  for (int k1 = 0; k1 < N1; ++k1)
    for (int k2 = 0; k2 < N2; ++k2) {
      const int k = k1 + N1 * k2;
      const int kp = (k == 0) ? Nc : Nc - k;
      sa[k1 * N2 + k2] = S[k] / Nc;
      sb[k1 * N2 + k2] = S[kp] / Nc;
    }
  std::vector<double2> ch64(n), tw64(L);
  std::vector<float2> ch32(n), tw32(L);
  for (int64_t j = 0; j < n; ++j) {
    cd v = chirp(j, n, +1);
    ch64[j] = make_double2(v.real(), v.imag());
    ch32[j] = make_float2((float)v.real(), (float)v.imag());
  }
  for (int64_t k = 0; k < L; ++k) {
    tw64[k] = make_double2(tw[k].real(), tw[k].imag());
    tw32[k] = make_float2((float)tw[k].real(), (float)tw[k].imag());
  }
  std::vector<cd> bk(L, cd(0, 0));
  for (int64_t m = 0; m < n; ++m) bk[m] = std::conj(chirp(m, n, +1));
  for (int64_t m = 1; m < n; ++m) bk[L - m] = std::conj(chirp(m, n, +1));
  fft_inplace(bk, -1);
  std::vector<double2> Bh64(L);
  std::vector<float2> Bh32(L);
  {
    const int M1 = P.gc.N1, M2 = P.gc.N2;
    for (int k1 = 0; k1 < M1; ++k1)
      for (int k2 = 0; k2 < M2; ++k2) {
        cd v = bk[k1 + (int64_t)M1 * k2] / (double)L;
        Bh64[k1 * M2 + k2] = make_double2(v.real(), v.imag());
        Bh32[k1 * M2 + k2] = make_float2((float)v.real(), (float)v.imag());
      }
  }
  std::vector<float> sa32(Nc), sb32(Nc);
  for (int i = 0; i < Nc; ++i) {
    sa32[i] = (float)sa[i];
    sb32[i] = (float)sb[i];
  }

  // ---- grid size
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaDeviceGetAttribute");
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return fail(c, TSFDE_ENOTSUP, "device lacks cooperative launch");
  const size_t smem = plan_smem_bytes(P);
  const int bps = coop_blocks_per_sm(smem);
  if (bps < 1) return fail(c, TSFDE_ECUDA, "cooperative kernels do not fit on an SM");
  const int maxG = nsm * std::min(bps, 2);
  P.G = std::max(1, std::min(maxG, std::max(items(P.gr), items(P.gc))));

  // ---- cluster engine (mixed level solves only): one cooperative launch of
  // whole clusters; cluster 0 runs the FP32 inner solves
  bool use_cluster = false;
  if (o.precision == TSFDE_MIXED && o.krylov == TSFDE_KRYLOV_BICGSTAB &&
      o.engine == TSFDE_ENGINE_CLUSTER && cluster_geometry(P)) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t csmem = std::max(plan_smem_bytes(P), cluster_smem_bytes(P));
    const int gmax = (csmem <= (size_t)optin) ? cluster_max_grid(P, csmem) : 0;
    if (gmax >= P.cl.Q) {
      P.cl.G = gmax;
      use_cluster = true;
    }
  }
  if (o.precision == TSFDE_MIXED && o.engine == TSFDE_ENGINE_CLUSTER && !use_cluster)
    return fail(c, TSFDE_ENOTSUP, "cluster engine unavailable for this size or device");

  // ---- device allocations
  const int64_t ld = ((n + 31) / 32) * 32;
  c->ld = (int)ld;
  bool ok = true;
  double2 *dtw64, *dch64, *dBh64, *dS1, *dS2;
  float2 *dtw32, *dch32, *dBh32;
  double *dsa64, *dsb64, *dlam, *dsaG64, *dsbG64, *dg64, *dpart;
  float *dsa32, *dsb32, *dsaG32, *dsbG32, *dg32;
  GridBarrier* dbar;
  ok &= dalloc(c, &dtw64, L) && dalloc(c, &dtw32, L);
  ok &= dalloc(c, &dsa64, Nc) && dalloc(c, &dsb64, Nc) && dalloc(c, &dsa32, Nc) && dalloc(c, &dsb32, Nc);
  ok &= dalloc(c, &dlam, n) && dalloc(c, &dch64, n) && dalloc(c, &dch32, n);
  ok &= dalloc(c, &dBh64, L) && dalloc(c, &dBh32, L);
  ok &= dalloc(c, &dsaG64, Nc) && dalloc(c, &dsbG64, Nc) && dalloc(c, &dsaG32, Nc) && dalloc(c, &dsbG32, Nc);
  ok &= dalloc(c, &dg64, n) && dalloc(c, &dg32, n);
  ok &= dalloc(c, &dS1, L) && dalloc(c, &dS2, L);
  ok &= dalloc(c, &dpart, (size_t)2 * kSlots * std::max(P.G, P.cl.G)) && dalloc(c, &dbar, 1);
  float2* dspT = nullptr;
  float2* dspG = nullptr;
  if (use_cluster) ok &= dalloc(c, &dspT, Nc) && dalloc(c, &dspG, Nc);
  ok &= dalloc(c, &c->G, (size_t)std::max(E, 1) * ld);
  ok &= dalloc(c, &c->eps, c->eps_h.size()) && dalloc(c, &c->cw, c->cw_h.size());
  for (int q = 0; q < kRoll; ++q) ok &= dalloc(c, &c->u[q], n);
  // FP32 vectors: length ld (even, zero-padded) -- the cluster engine moves
  // entries in aligned pairs
  ok &= dalloc(c, &c->b, n) && dalloc(c, &c->kappa64, n) && dalloc(c, &c->kappa32, ld);
  ok &= dalloc(c, &c->phi, n) && dalloc(c, &c->kap0, n) && dalloc(c, &c->kap1d, n);
  ok &= dalloc(c, &c->F, 4 * n) && dalloc(c, &c->r64, n);
  // Krylov vectors of every arithmetic: length ld (even, zero padded), so
  // that entries can be moved in aligned pairs
  double** v64[] = {&c->k64.r, &c->k64.rh, &c->k64.p, &c->k64.v, &c->k64.s, &c->k64.t, &c->k64.ph, &c->k64.sh};
  for (double** p : v64) ok &= dalloc(c, p, ld);
  float** v32[] = {&c->k32.x, &c->k32.r, &c->k32.rh, &c->k32.p, &c->k32.v, &c->k32.s, &c->k32.t, &c->k32.ph, &c->k32.sh};
  for (float** p : v32) ok &= dalloc(c, p, ld);
  ok &= dalloc(c, &c->stats, M + 1) && dalloc(c, &c->status, 1);
  ok &= dalloc(c, &c->k64.x, n);  // FP64 correction of the mixed fallback
  // double-single tables and inner vectors
  const bool ds = o.precision == TSFDE_MIXED_DS;
  dsf2* dtwds = nullptr;
  dsf *dsads = nullptr, *dsbds = nullptr, *dsaGds = nullptr, *dsbGds = nullptr, *dgds = nullptr;
  dsf2 *dchds = nullptr, *dBhds = nullptr;
  if (ds) {
    ok &= dalloc(c, &dtwds, L) && dalloc(c, &dsads, Nc) && dalloc(c, &dsbds, Nc) &&
          dalloc(c, &dsaGds, Nc) && dalloc(c, &dsbGds, Nc) && dalloc(c, &c->kappads, ld);
    ok &= dalloc(c, &dchds, n) && dalloc(c, &dBhds, L) && dalloc(c, &dgds, n);
    dsf** vds[] = {&c->kds.x, &c->kds.r, &c->kds.rh, &c->kds.p, &c->kds.v, &c->kds.s, &c->kds.t,
                   &c->kds.ph, &c->kds.sh};
    for (dsf** p : vds) ok &= dalloc(c, p, ld);
  }
  if (o.krylov != TSFDE_KRYLOV_BICGSTAB) {
    ok &= dalloc(c, &c->hinv64, n) && dalloc(c, &c->hinv32, ld);
    if (ds) ok &= dalloc(c, &c->hinvds, ld);
  }
  if (o.krylov == TSFDE_KRYLOV_AUTO) ok &= dalloc(c, &c->kauto, 1);
  if (ds) ok &= dalloc(c, &c->pre_status, 1);
  if (o.ckpt_stride != 0) {
    int64_t S = o.ckpt_stride;
    if (S < 0) S = std::max<int64_t>(1, (int64_t)std::ceil(std::sqrt((double)M)));
    S = std::min<int64_t>(S, M);
    c->ck_stride = S;
    c->ck_slots = M / S + 1;
    c->ck_slot = (size_t)(kRoll + std::max(E, 1)) * ld;
    c->ck_ok.assign(c->ck_slots, 0);
    ok &= dalloc(c, &c->ck, c->ck_slot * c->ck_slots) && dalloc(c, &c->ck_seg, (size_t)S * n) &&
          dalloc(c, &c->ck_save, (size_t)(kRoll + std::max(E, 1)) * ld);
    if (c->kauto) ok &= dalloc(c, &c->ck_kauto, 1);
  }
  // direct history: all levels and the weights of Eq. (4.1),
  // w_0 = a_1/Gamma(1-g), w_k = (a_{k+1} - a_k)/Gamma(1-g) (k = 1..m-1)
  std::vector<double> wdir_h;
  if (o.history == TSFDE_HISTORY_DIRECT) {
    ok &= dalloc(c, &c->Uh, (size_t)(M + 1) * ld) && dalloc(c, &c->wdir, (size_t)M * (M + 1) / 2);
    wdir_h.assign((size_t)M * (M + 1) / 2, 0.0);
    const double G1h = std::tgamma(1.0 - gamma);
    std::vector<double> a(M + 2);
    for (int64_t m = 1; m <= M; ++m) {
      for (int64_t k = 1; k <= m; ++k) a[k] = l1_weight(T, M, r, gamma, m, k);
      double* w = wdir_h.data() + (size_t)m * (m - 1) / 2;
      w[0] = a[1] / G1h;
      for (int64_t k = 1; k < m; ++k) w[k] = (a[k + 1] - a[k]) / G1h;
    }
  }
  if (!ok) return fail(c, TSFDE_ENOMEM, "cudaMalloc failed");
  if (c->Uh) {
    if ((e = upload(c->wdir, wdir_h)) != cudaSuccess) return cuda_fail(c, e, "upload");
    if ((e = cudaMemset(c->Uh, 0, sizeof(double) * (size_t)(M + 1) * ld)) != cudaSuccess)
      return cuda_fail(c, e, "cudaMemset");
  }
  if (ds) {
    std::vector<dsf2> twds(L);
    for (int64_t k = 0; k < L; ++k) {
      twds[k].x = dsf(tw[k].real());
      twds[k].y = dsf(tw[k].imag());
    }
    std::vector<dsf> sads(Nc), sbds(Nc);
    for (int i = 0; i < Nc; ++i) {
      sads[i] = dsf(sa[i]);
      sbds[i] = dsf(sb[i]);
    }
    std::vector<dsf2> chds(n), Bhds(L);
    for (int64_t j = 0; j < n; ++j) {
      chds[j].x = dsf(ch64[j].x);
      chds[j].y = dsf(ch64[j].y);
    }
    for (int64_t k = 0; k < L; ++k) {
      Bhds[k].x = dsf(Bh64[k].x);
      Bhds[k].y = dsf(Bh64[k].y);
    }
    if ((e = upload(dtwds, twds)) != cudaSuccess || (e = upload(dsads, sads)) != cudaSuccess ||
        (e = upload(dsbds, sbds)) != cudaSuccess || (e = upload(dchds, chds)) != cudaSuccess ||
        (e = upload(dBhds, Bhds)) != cudaSuccess)
      return cuda_fail(c, e, "upload");
    P.twLds = dtwds;
    P.saTds = dsads; P.sbTds = dsbds;
    P.saGds = dsaGds; P.sbGds = dsbGds;
    P.chirpds = dchds; P.Bhds = dBhds; P.gds = dgds;
  }

  if ((e = upload(dtw64, tw64)) != cudaSuccess || (e = upload(dtw32, tw32)) != cudaSuccess ||
      (e = upload(dsa64, sa)) != cudaSuccess || (e = upload(dsb64, sb)) != cudaSuccess ||
      (e = upload(dsa32, sa32)) != cudaSuccess || (e = upload(dsb32, sb32)) != cudaSuccess ||
      (e = upload(dlam, lam)) != cudaSuccess || (e = upload(dch64, ch64)) != cudaSuccess ||
      (e = upload(dch32, ch32)) != cudaSuccess || (e = upload(dBh64, Bh64)) != cudaSuccess ||
      (e = upload(dBh32, Bh32)) != cudaSuccess || (e = upload(c->eps, c->eps_h)) != cudaSuccess ||
      (e = upload(c->cw, c->cw_h)) != cudaSuccess)
    return cuda_fail(c, e, "upload");
  if ((e = cudaMemset(c->G, 0, sizeof(double) * (size_t)std::max(E, 1) * ld)) != cudaSuccess)
    return cuda_fail(c, e, "cudaMemset");
  if ((e = cudaMemset(c->stats, 0, sizeof(StepStat) * (M + 1))) != cudaSuccess) return cuda_fail(c, e, "cudaMemset");
  for (float* p : {c->kappa32, c->k32.x, c->k32.r, c->k32.rh, c->k32.p, c->k32.v, c->k32.s, c->k32.t,
                   c->k32.ph, c->k32.sh})
    if ((e = cudaMemset(p, 0, sizeof(float) * ld)) != cudaSuccess) return cuda_fail(c, e, "cudaMemset");
  P.bar = dbar; P.part = dpart;
  P.twL64 = dtw64; P.twL32 = dtw32;
  P.saT64 = dsa64; P.sbT64 = dsb64; P.saT32 = dsa32; P.sbT32 = dsb32;
  P.lam = dlam; P.chirp64 = dch64; P.chirp32 = dch32; P.Bh64 = dBh64; P.Bh32 = dBh32;
  P.saG64 = dsaG64; P.sbG64 = dsbG64; P.saG32 = dsaG32; P.sbG32 = dsbG32;
  P.g64 = dg64; P.g32 = dg32; P.S1 = dS1; P.S2 = dS2;
  if (use_cluster) {
    // Toeplitz spectrum in the cluster engine's row-pass order
    const CGeo& g = P.cl;
    std::vector<float2> spT(Nc);
    for (int k1 = 0; k1 < N1; ++k1) {
      const int h = N1 / 2;
      const int u = (k1 == 0 || k1 == h) ? 0 : (k1 < h ? k1 : N1 - k1);
      const int b = (k1 == 0) ? 0 : (k1 == h ? 1 : (k1 < h ? 0 : 1));
      const int q = u / g.U, slot = 2 * (u % g.U) + b;
      for (int k2 = 0; k2 < N2; ++k2)
        spT[(size_t)q * g.nbuf + (size_t)k2 * g.Bq + slot] =
            make_float2(sa32[k1 * N2 + k2], sb32[k1 * N2 + k2]);
    }
    if ((e = upload(dspT, spT)) != cudaSuccess) return cuda_fail(c, e, "upload");
    P.spT_cl = dspT;
    P.spG_cl = dspG;
    // the launch itself must be accepted (cooperative launch of clusters)
    LevelArgs probe{};
    probe.P = P;
    probe.P.G = P.cl.G;
    probe.probe = 1;
    e = launch_level_cluster(probe, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (o.engine == TSFDE_ENGINE_CLUSTER)
        return fail(c, TSFDE_ENOTSUP, std::string("cluster engine launch refused: ") + cudaGetErrorString(e));
      use_cluster = false;
    }
  }
  c->engine = use_cluster ? TSFDE_ENGINE_CLUSTER : TSFDE_ENGINE_GRID;
  return TSFDE_OK;
}

int tsfde_setup(tsfde_ctx** out, double alpha, double gamma, double l, double T, int64_t n,
                int64_t M, double r, double soe_tol, const tsfde_opts* opts) {
  if (!out) return TSFDE_EINVAL;
  *out = nullptr;
  tsfde_ctx* c = nullptr;
  try {
    c = new tsfde_ctx();
    int st = setup_impl(c, alpha, gamma, l, T, n, M, r, soe_tol, opts);
    if (st != TSFDE_OK) {
      std::fprintf(stderr, "tsfde_setup: %s\n", c->err.c_str());
      tsfde_destroy(c);
      return st;
    }
  } catch (const std::bad_alloc&) {
    tsfde_destroy(c);
    return TSFDE_ENOMEM;
  } catch (...) {
    tsfde_destroy(c);
    return TSFDE_EINVAL;
  }
  *out = c;
  return TSFDE_OK;
}

int tsfde_set_problem(tsfde_ctx* c, const double* phi, const double* kappa0, const double* kappa1,
                      const double* theta, int rank, const double* const* F, const double* G) {
  if (!c) return TSFDE_EINVAL;
  if (!phi || !kappa0) return fail(c, TSFDE_EINVAL, "phi and kappa0 are required");
  if (kappa1 && !theta) return fail(c, TSFDE_EINVAL, "kappa1 needs theta");
  if (rank < 0 || rank > 4) return fail(c, TSFDE_EINVAL, "source rank must be 0..4");
  if (rank > 0 && (!F || !G)) return fail(c, TSFDE_EINVAL, "rank > 0 needs F and G");
  const size_t nb = sizeof(double) * (size_t)c->n;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->phi, phi, nb, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->kap0, kappa0, nb, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "set_problem copy");
  c->kap1 = kappa1 != nullptr;
  if (kappa1 && (e = cudaMemcpyAsync(c->kap1d, kappa1, nb, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "set_problem copy");
  c->theta.assign(c->M + 1, 0.0);
  if (theta) c->theta.assign(theta, theta + c->M + 1);
  c->rank = rank;
  c->Gsrc.assign(4 * (c->M + 1), 0.0);
  for (int q = 0; q < rank; ++q) {
    if (!F[q]) return fail(c, TSFDE_EINVAL, "F[q] is NULL");
    if ((e = cudaMemcpyAsync(c->F + (size_t)q * c->n, F[q], nb, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "set_problem copy");
    for (int64_t m = 0; m <= c->M; ++m) c->Gsrc[q * (c->M + 1) + m] = G[q * (c->M + 1) + m];
  }
  c->have_problem = true;
  return tsfde_reset(c);
}

int tsfde_reset(tsfde_ctx* c) {
  if (!c) return TSFDE_EINVAL;
  if (!c->have_problem) return fail(c, TSFDE_ESTATE, "no problem set");
  cudaError_t e;
  if ((e = cudaMemcpyAsync(ulev(c, 0), c->phi, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "reset copy");
  if ((e = cudaMemsetAsync(c->G, 0, sizeof(double) * (size_t)std::max(c->E, 1) * c->ld, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "reset memset");
  if (c->kauto) {
    KrylovAuto k0{};
    k0.for_level = 1;
    k0.choice = 0;
    auto_rule_init(k0.rule);
    c->kauto_init = k0;
    if ((e = cudaMemcpyAsync(c->kauto, &c->kauto_init, sizeof(KrylovAuto), cudaMemcpyHostToDevice, c->stream)) !=
        cudaSuccess)
      return cuda_fail(c, e, "reset copy");
  }
  c->m = 0;
  if (c->ck) {
    std::fill(c->ck_ok.begin(), c->ck_ok.end(), 0);
    c->ck_override = false;
    if ((e = record_ckpt(c, 0)) != cudaSuccess) return cuda_fail(c, e, "checkpoint copy");
  }
  return TSFDE_OK;
}

static LevelArgs level_args(tsfde_ctx* c, double ahat, const double* b, double* u, StepStat* st) {
  LevelArgs A{};
  A.P = c->P;
  A.ahat = ahat;
  A.b = b;
  A.kappa64 = c->kappa64;
  A.kappa32 = c->kappa32;
  A.u = u;
  A.precond = c->opts.precond == TSFDE_STRANG ? 1 : 0;
  A.tol = c->opts.krylov_tol;
  A.max_it = c->opts.max_it;
  A.inner_tol = c->opts.inner_tol;
  A.max_outer = c->opts.max_outer;
  A.inner_max_it = c->opts.inner_max_it;
  A.k64 = c->k64;
  A.k32 = c->k32;
  A.kds = c->kds;
  A.pre_status = c->pre_status;
  A.kappads = c->kappads;
  A.krylov = c->opts.krylov;
  A.hinv64 = c->hinv64;
  A.hinv32 = c->hinv32;
  A.hinvds = c->hinvds;
  A.r64 = c->r64;
  A.stat = st;
  return A;
}

static cudaError_t record(tsfde_ctx* c) {
  if (!c->opts.profile) return cudaSuccess;
  cudaEvent_t e;
  if (c->ev_free.empty()) {
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
  } else {
    e = c->ev_free.back();
    c->ev_free.pop_back();
  }
  c->ev_used.push_back(e);
  return cudaEventRecord(e, c->stream);
}

static cudaError_t launch_level_ctx(tsfde_ctx* c, LevelArgs& A) {
  if (c->opts.precision == TSFDE_MIXED && c->engine == TSFDE_ENGINE_CLUSTER) {
    A.P.G = A.P.cl.G;
    return launch_level_cluster(A, c->stream);
  }
  return launch_level(A, c->opts.precision, c->stream);
}

// Enqueue level m = c->m + 1.
static int enqueue_level(tsfde_ctx* c, const double* kappa_m, const double* f_m, double* rhs_out) {
  const int64_t m = c->m + 1;
  RhsArgs R{};
  R.n = (int)c->n;
  R.ld = c->ld;
  R.Eact = (m >= 2) ? c->Eact[m] : 0;
  R.ahat = c->ahat[m];
  R.Gm = c->G;
  R.eps = c->eps + m * c->E;
  R.cw = c->cw + m * c->E;
  R.u1 = ulev(c, m - 1);
  R.u2 = (m >= 2) ? ulev(c, m - 2) : ulev(c, m - 1);
  R.kap_m = kappa_m;
  R.kap0 = c->kap0;
  R.kap1 = c->kap1 ? c->kap1d : nullptr;
  R.theta = c->theta[m];
  R.f_m = f_m;
  R.F = c->F;
  R.rank = c->rank;
  for (int q = 0; q < 4; ++q) R.Gr[q] = (q < c->rank) ? c->Gsrc[q * (c->M + 1) + m] : 0.0;
  R.b = c->b;
  R.rhs_copy = rhs_out;
  R.kappa64 = c->kappa64;
  R.kappa32 = c->kappa32;
  if (c->Uh) {
    R.U_hist = c->Uh;
    R.w_dir = c->wdir + (size_t)m * (m - 1) / 2;
    R.m_hist = (int)m;
    R.Eact = 0;
  }
  cudaError_t e = record(c);
  if (e == cudaSuccess) e = c->Uh ? launch_rhs_direct(R, c->stream) : launch_rhs(R, c->stream);
  if (e == cudaSuccess) e = record(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "rhs kernel");
  LevelArgs A = level_args(c, c->ahat[m], c->b, ulev(c, m), c->stats + m);
  A.u_prev = c->opts.warm_start ? ulev(c, m - 1) : nullptr;
  if (c->opts.warm_start == 2) {
    // polynomial extrapolation in the level index through the last
    // kStartOrder + 1 levels (fewer at the first levels); with the SOE
    // history the oldest of them shares its buffer with u^m
    A.xorder = (int)std::min<int64_t>(kStartOrder, m - 1);
    for (int j = 0; j <= A.xorder; ++j) A.up[j] = ulev(c, m - 1 - j);
    // Lagrange weights of the nodes m-1-j at m: (-1)^j C(q+1, j+1)
    // (4, -6, 4, -1 for q = 3), exact in FP64
    for (int j = 0; j <= A.xorder; ++j) {
      double w = 1.0;
      for (int k = 0; k <= A.xorder; ++k)
        if (k != j) w *= (double)(1 + k) / (double)(k - j);
      A.xw[j] = w;
    }
  }
  A.prev = (m >= 2) ? c->stats + (m - 1) : nullptr;
  A.retry_mixed = (m % 64 == 0) ? 1 : 0;
  A.kauto = c->kauto;
  A.m = m;
  if (c->ck_recomputing && c->kauto) {
    // a recomputed level takes the method the forward march took there
    A.kauto = nullptr;
    A.krylov = c->ck_kry[m];
  }
  e = launch_level_ctx(c, A);
  if (e == cudaSuccess) e = record(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "level kernel");
  c->m = m;
  if (c->ck && !c->ck_recomputing) {
    if (kappa_m || f_m) c->ck_override = true;
    if (m % c->ck_stride == 0 && (e = record_ckpt(c, m)) != cudaSuccess) return cuda_fail(c, e, "checkpoint copy");
  }
  return TSFDE_OK;
}

int tsfde_step(tsfde_ctx* c, const double* kappa_m, const double* f_m, double* u_out, double* rhs_out,
               tsfde_step_info* info) {
  if (!c) return TSFDE_EINVAL;
  if (!c->have_problem) return fail(c, TSFDE_ESTATE, "no problem set");
  if (c->m >= c->M) return fail(c, TSFDE_ESTATE, "all levels already computed");
  int st = enqueue_level(c, kappa_m, f_m, rhs_out);
  if (st != TSFDE_OK) return st;
  const int64_t m = c->m;
  cudaError_t e;
  if (u_out && (e = cudaMemcpyAsync(u_out, ulev(c, m), sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "u copy");
  if (info) {
    StepStat s{};
    if ((e = cudaMemcpyAsync(&s, c->stats + m, sizeof(s), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "step sync");
    info->m = m;
    info->status = s.status;
    info->iterations = s.iterations;
    info->outer = s.outer;
    info->E_active = c->Eact[m];
    info->rel_residual = s.rel_residual;
    info->krylov = s.method;
    if (s.status != TSFDE_OK) return fail(c, s.status, std::string("level ") + std::to_string(m) + ": " + tsfde_strerror(s.status));
  }
  return TSFDE_OK;
}

int tsfde_solve(tsfde_ctx* c, double* u_final, double* u_all, tsfde_solve_info* info) {
  if (!c) return TSFDE_EINVAL;
  if (!c->have_problem) return fail(c, TSFDE_ESTATE, "no problem set");
  const int64_t m0 = c->m;
  const size_t nb = sizeof(double) * c->n;
  cudaError_t e;
  if (u_all && m0 == 0 && (e = cudaMemcpyAsync(u_all, ulev(c, 0), nb, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "u copy");
  while (c->m < c->M) {
    int st = enqueue_level(c, nullptr, nullptr, nullptr);
    if (st != TSFDE_OK) return st;
    if (u_all && (e = cudaMemcpyAsync(u_all + c->m * c->n, ulev(c, c->m), nb, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "u copy");
  }
  if (u_final && (e = cudaMemcpyAsync(u_final, ulev(c, c->m), nb, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "u copy");
  if (info) {
    std::vector<StepStat> s(c->M + 1);
    if ((e = cudaMemcpyAsync(s.data(), c->stats, sizeof(StepStat) * (c->M + 1), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "solve sync");
    std::memset(info, 0, sizeof(*info));
    info->E = c->E;
    info->min_iterations = 1 << 30;
    for (int64_t m = m0 + 1; m <= c->M; ++m) {
      if (s[m].status != TSFDE_OK && info->status == TSFDE_OK) {
        info->status = s[m].status;
        info->failed_level = m;
      }
      info->iterations += s[m].iterations;
      info->outer += s[m].outer;
      info->min_iterations = std::min(info->min_iterations, s[m].iterations);
      info->max_iterations = std::max(info->max_iterations, s[m].iterations);
      info->max_rel_residual = std::max(info->max_rel_residual, s[m].rel_residual);
      info->E_active_sum += c->Eact[m];
      info->pcg_levels += s[m].method == 1 ? 1 : 0;
    }
    info->levels = c->M - m0;
    if (info->levels == 0) info->min_iterations = 0;
    if (info->status != TSFDE_OK)
      return fail(c, info->status, std::string("level ") + std::to_string(info->failed_level) + ": " + tsfde_strerror(info->status));
  }
  return TSFDE_OK;
}

int tsfde_get_level_stats(tsfde_ctx* c, int64_t m0, int64_t m1, tsfde_step_info* out) {
  if (!c || !out) return TSFDE_EINVAL;
  if (m0 < 1 || m1 < m0 || m1 > c->m) return fail(c, TSFDE_EINVAL, "level range outside 1..current level");
  std::vector<StepStat> s(m1 - m0 + 1);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(s.data(), c->stats + m0, sizeof(StepStat) * s.size(), cudaMemcpyDeviceToHost,
                           c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "level stats");
  for (size_t q = 0; q < s.size(); ++q) {
    out[q].m = m0 + (int64_t)q;
    out[q].status = s[q].status;
    out[q].iterations = s[q].iterations;
    out[q].outer = s[q].outer;
    out[q].E_active = c->Eact[m0 + q];
    out[q].rel_residual = s[q].rel_residual;
    out[q].krylov = s[q].method;
  }
  return TSFDE_OK;
}

int tsfde_get_solution(tsfde_ctx* c, double* u) {
  if (!c || !u) return TSFDE_EINVAL;
  if (!c->have_problem) return fail(c, TSFDE_ESTATE, "no problem set");
  cudaError_t e = cudaMemcpyAsync(u, ulev(c, c->m), sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "solution copy");
  return TSFDE_OK;
}

int tsfde_get_timing(tsfde_ctx* c, tsfde_timing* out) {
  if (!c || !out) return TSFDE_EINVAL;
  if (!c->opts.profile) return fail(c, TSFDE_ESTATE, "profiling is off (opts.profile = 0)");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "timing sync");
  std::memset(out, 0, sizeof(*out));
  for (size_t q = 0; q + 2 < c->ev_used.size(); q += 3) {
    float a = 0.f, b = 0.f;
    if ((e = cudaEventElapsedTime(&a, c->ev_used[q], c->ev_used[q + 1])) != cudaSuccess ||
        (e = cudaEventElapsedTime(&b, c->ev_used[q + 1], c->ev_used[q + 2])) != cudaSuccess)
      return cuda_fail(c, e, "cudaEventElapsedTime");
    out->rhs_ms += a;
    out->level_ms += b;
    out->levels += 1;
  }
  for (cudaEvent_t ev : c->ev_used) c->ev_free.push_back(ev);
  c->ev_used.clear();
  return TSFDE_OK;
}

int tsfde_get_soe(const tsfde_ctx* c, int* E, double* s, double* w) {
  if (!c || !E) return TSFDE_EINVAL;
  const int cap = *E;
  *E = c->E;
  if ((s || w) && cap < c->E) return TSFDE_EINVAL;
  if (s) std::memcpy(s, c->soe_s.data(), sizeof(double) * c->E);
  if (w) std::memcpy(w, c->soe_w.data(), sizeof(double) * c->E);
  return TSFDE_OK;
}

int tsfde_get_times(const tsfde_ctx* c, double* t) {
  if (!c || !t) return TSFDE_EINVAL;
  std::memcpy(t, c->tmesh.data(), sizeof(double) * (c->M + 1));
  return TSFDE_OK;
}

int tsfde_get_symbol(const tsfde_ctx* c, double* t) {
  if (!c || !t) return TSFDE_EINVAL;
  std::memcpy(t, c->symbol.data(), sizeof(double) * c->n);
  return TSFDE_OK;
}

static int run_apply(tsfde_ctx* c, int kind, double a, double kbar, const double* kappa, const double* v,
                     double* y, int precision) {
  if (!c || !v || !y) return TSFDE_EINVAL;
  if (precision != TSFDE_FP64 && precision != TSFDE_MIXED && precision != TSFDE_MIXED_DS)
    return fail(c, TSFDE_EINVAL, "bad precision");
  if (precision == TSFDE_MIXED_DS && !c->P.twLds)
    return fail(c, TSFDE_EINVAL, "double-single products need a context set up with TSFDE_MIXED_DS");
  ApplyArgs A{};
  A.P = c->P;
  A.kind = kind;
  A.a = a;
  A.kbar = kbar;
  A.kappa = kappa;
  A.v = v;
  A.y = y;
  A.status = c->status;
  cudaError_t e = launch_apply(A, precision, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "apply kernel");
  int st = 0;
  if ((e = cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "apply sync");
  if (st != TSFDE_OK) return fail(c, st, tsfde_strerror(st));
  return TSFDE_OK;
}

int tsfde_toeplitz_apply(tsfde_ctx* c, const double* v, double* y, int precision) {
  return run_apply(c, 0, 0.0, 0.0, nullptr, v, y, precision);
}

int tsfde_operator_apply(tsfde_ctx* c, double a, const double* kappa, const double* v, double* y, int precision) {
  if (!kappa) return fail(c, TSFDE_EINVAL, "kappa is required");
  return run_apply(c, 0, a, 0.0, kappa, v, y, precision);
}

int tsfde_precond_apply(tsfde_ctx* c, double a, double kbar, const double* v, double* z, int precision) {
  if (!(a > 0.0) || !(kbar > 0.0)) return fail(c, TSFDE_EINVAL, "a and kbar must be positive");
  return run_apply(c, 1, a, kbar, nullptr, v, z, precision);
}

int tsfde_get_engine(const tsfde_ctx* c) { return c ? c->engine : -1; }

// One reverse level m of the adjoint sweep: g^m (from lambda^{m+1} through
// the reversed SOE recurrence, or dJ/du^M at m = M), the transposed level
// solve into lambda^m and the gradient terms with u^m (dev n).
static int adjoint_level(tsfde_ctx* c, int64_t m, const double* um, const double* dJ, double* grad_kappa,
                         double* grad_f, int krylov) {
  const int64_t n = c->n, M = c->M;
  cudaStream_t s = c->stream;
  cudaError_t e;
  double* lam = c->adjLam[m & 1];
  const double* lam1 = c->adjLam[(m + 1) & 1];
  if (m == M) {
    if ((e = cudaMemcpyAsync(c->adjG, dJ, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return cuda_fail(c, e, "adjoint copy");
  } else {
    AdjRhsArgs R{};
    R.n = (int)n;
    R.ld = c->ld;
    R.Eact = c->Eact[m + 1];
    R.ahat1 = c->ahat[m + 1];
    R.Y = c->adjY;
    R.eps1 = c->eps + (m + 1) * c->E;
    R.c1 = c->cw + (m + 1) * c->E;
    R.c2 = (m + 2 <= M) ? c->cw + (m + 2) * c->E : nullptr;
    R.lam1 = lam1;
    R.g = c->adjG;
    if ((e = launch_adj_rhs(R, s)) != cudaSuccess) return cuda_fail(c, e, "adjoint rhs kernel");
  }
  LevelArgs A{};
  A.P = c->P;
  A.ahat = c->ahat[m];
  A.b = c->adjG;
  A.kappa64 = c->kappa64;
  A.kappa32 = c->kappa32;
  A.u = lam;
  A.precond = c->opts.precond == TSFDE_STRANG ? 1 : 0;
  A.tol = c->opts.krylov_tol;
  A.max_it = c->opts.max_it;
  A.k64 = c->k64;
  A.k32 = c->k32;
  A.r64 = c->r64;
  A.stat = c->adjStats + m;
  A.krylov = krylov;
  A.hinv64 = c->hinv64;
  AdjGradArgs Gd{um, grad_kappa, grad_f};
  if ((e = launch_level_adj(A, Gd, s)) != cudaSuccess) return cuda_fail(c, e, "adjoint level kernel");
  return TSFDE_OK;
}

int tsfde_adjoint(tsfde_ctx* c, const double* u_all, const double* dJ, double* grad_kappa,
                  double* grad_f, tsfde_adjoint_info* info) {
  if (!c || !dJ || !grad_kappa || !grad_f) return TSFDE_EINVAL;
  if (!c->have_problem) return fail(c, TSFDE_ESTATE, "no problem set");
  if (c->kap1) return fail(c, TSFDE_ENOTSUP, "adjoint needs a time-independent kappa (kappa1 = NULL)");
  if (c->Uh) return fail(c, TSFDE_ENOTSUP, "the adjoint sweep is that of FIDS (history = SOE)");
  const int64_t n = c->n, M = c->M;
  if (!u_all) {
    if (!c->ck) return fail(c, TSFDE_ESTATE, "u_all is NULL and the context keeps no checkpoints (ckpt_stride = 0)");
    if (c->m != M) return fail(c, TSFDE_ESTATE, "checkpointed adjoint: march to level M first");
    if (c->ck_override) return fail(c, TSFDE_ESTATE, "checkpointed adjoint: a level used per-level kappa_m / f_m");
    for (int64_t j = 0; j * c->ck_stride < M; ++j)
      if (!c->ck_ok[j]) return fail(c, TSFDE_ESTATE, "checkpointed adjoint: the march was not run from level 0");
  }
  const int E = std::max(c->E, 1);
  if (!c->adjY) {
    bool ok = dalloc(c, &c->adjY, (size_t)E * c->ld) && dalloc(c, &c->adjLam[0], n) &&
              dalloc(c, &c->adjLam[1], n) && dalloc(c, &c->adjG, n) && dalloc(c, &c->adjStats, M + 1);
    if (!ok) {
      c->adjY = nullptr;
      return fail(c, TSFDE_ENOMEM, "cudaMalloc failed (adjoint buffers)");
    }
  }
  cudaStream_t s = c->stream;
  cudaError_t e;
  const size_t nb = sizeof(double) * (size_t)n;
  if ((e = cudaMemsetAsync(c->adjY, 0, sizeof(double) * (size_t)E * c->ld, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(grad_kappa, 0, nb, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(grad_f, 0, nb, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->adjStats, 0, sizeof(StepStat) * (M + 1), s)) != cudaSuccess)
    return cuda_fail(c, e, "adjoint memset");
  // kappa of every level is kappa0
  if ((e = launch_convert(c->kap0, c->kappa64, c->kappa32, (int)n, s)) != cudaSuccess)
    return cuda_fail(c, e, "convert kernel");
  // Krylov method of each reverse level: the context's; with AUTO, the one
  // that solved the same forward level (the transposed system has the same
  // balance of ahat K^{-1} against A)
  std::vector<int> kry(M + 1, c->opts.krylov == TSFDE_KRYLOV_PCG ? TSFDE_KRYLOV_PCG : TSFDE_KRYLOV_BICGSTAB);
  if (c->opts.krylov == TSFDE_KRYLOV_AUTO && c->m == M) {
    std::vector<StepStat> fw(M + 1);
    if ((e = cudaMemcpyAsync(fw.data(), c->stats, sizeof(StepStat) * (M + 1), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(c, e, "adjoint sync");
    for (int64_t m = 1; m <= M; ++m) kry[m] = fw[m].method == 1 ? TSFDE_KRYLOV_PCG : TSFDE_KRYLOV_BICGSTAB;
  }
  int st0 = TSFDE_OK;
  if (u_all) {
    for (int64_t m = M; m >= 1 && st0 == TSFDE_OK; --m)
      st0 = adjoint_level(c, m, u_all + (size_t)m * n, dJ, grad_kappa, grad_f, kry[m]);
  } else {
    // Checkpointed sweep: segments (k0, k1] of ck_stride levels, last first;
    // each is marched again from its checkpoint k0 into ck_seg, then swept
    // in reverse.  The forward state is kept aside and brought back.
    const int64_t S = c->ck_stride;
    if ((e = keep_forward_state(c, true)) != cudaSuccess) return cuda_fail(c, e, "checkpoint copy");
    c->ck_kry = kry;
    c->ck_recomputing = true;
    for (int64_t k0 = ((M - 1) / S) * S; k0 >= 0 && st0 == TSFDE_OK; k0 -= S) {
      const int64_t k1 = std::min(k0 + S, M);
      if ((e = restore_ckpt(c, k0)) != cudaSuccess) { st0 = cuda_fail(c, e, "checkpoint copy"); break; }
      for (int64_t m = k0 + 1; m <= k1 && st0 == TSFDE_OK; ++m) {
        st0 = enqueue_level(c, nullptr, nullptr, nullptr);
        if (st0 == TSFDE_OK &&
            (e = cudaMemcpyAsync(c->ck_seg + (size_t)(m - k0 - 1) * n, ulev(c, m), nb, cudaMemcpyDeviceToDevice,
                                 s)) != cudaSuccess)
          st0 = cuda_fail(c, e, "checkpoint copy");
      }
      // the recomputed forward levels wrote kappa^m = kappa0 again: unchanged
      for (int64_t m = k1; m > k0 && st0 == TSFDE_OK; --m)
        st0 = adjoint_level(c, m, c->ck_seg + (size_t)(m - k0 - 1) * n, dJ, grad_kappa, grad_f, kry[m]);
    }
    c->ck_recomputing = false;
    c->m = M;
    if ((e = keep_forward_state(c, false)) != cudaSuccess && st0 == TSFDE_OK) st0 = cuda_fail(c, e, "checkpoint copy");
  }
  if (st0 != TSFDE_OK) return st0;
  std::vector<StepStat> st(M + 1);
  if ((e = cudaMemcpyAsync(st.data(), c->adjStats, sizeof(StepStat) * (M + 1), cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(c, e, "adjoint sync");
  tsfde_adjoint_info inf{};
  for (int64_t m = M; m >= 1; --m) {
    inf.iterations += st[m].iterations;
    inf.max_iterations = std::max(inf.max_iterations, st[m].iterations);
    inf.max_rel_residual = std::max(inf.max_rel_residual, st[m].rel_residual);
    if (st[m].status != TSFDE_OK && inf.status == TSFDE_OK) {
      inf.status = st[m].status;
      inf.failed_level = m;
    }
  }
  if (!u_all) {
    // the recomputed forward levels must have converged as well
    std::vector<StepStat> fw(M + 1);
    if ((e = cudaMemcpy(fw.data(), c->stats, sizeof(StepStat) * (M + 1), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(c, e, "adjoint sync");
    for (int64_t m = 1; m <= M; ++m)
      if (fw[m].status != TSFDE_OK && inf.status == TSFDE_OK) {
        inf.status = fw[m].status;
        inf.failed_level = m;
      }
    inf.recomputed_levels = M;
  }
  if (info) *info = inf;
  if (inf.status != TSFDE_OK) return fail(c, inf.status, tsfde_strerror(inf.status));
  return TSFDE_OK;
}

int tsfde_linear_solve(tsfde_ctx* c, double a, const double* kappa, const double* b, double* x,
                       tsfde_step_info* info) {
  if (!c || !kappa || !b || !x) return TSFDE_EINVAL;
  if (!(a > 0.0)) return fail(c, TSFDE_EINVAL, "a must be positive");
  cudaError_t e = launch_convert(kappa, c->kappa64, c->kappa32, (int)c->n, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "convert kernel");
  LevelArgs A = level_args(c, a, b, x, c->stats);
  A.kappa64 = c->kappa64;
  if (A.krylov == TSFDE_KRYLOV_AUTO) A.krylov = TSFDE_KRYLOV_BICGSTAB;  // no level history here
  e = launch_level_ctx(c, A);
  if (e != cudaSuccess) return cuda_fail(c, e, "level kernel");
  StepStat s{};
  if ((e = cudaMemcpyAsync(&s, c->stats, sizeof(s), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "solve sync");
  if (info) {
    info->m = 0;
    info->status = s.status;
    info->iterations = s.iterations;
    info->outer = s.outer;
    info->E_active = 0;
    info->rel_residual = s.rel_residual;
    info->krylov = s.method;
  }
  if (s.status != TSFDE_OK) return fail(c, s.status, tsfde_strerror(s.status));
  return TSFDE_OK;
}

}  // extern "C"
