// batch_host.cpp -- C ABI of the batched solve (tsfde_batch_*): per-instance
// setup tables (built on host threads), pooled device memory, and the
// persistent cluster launch of batch.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tsfde.h"
#include "host_math.h"
#include "plan.h"

using namespace tsfde;

namespace {

int ilg(int64_t x) {
  int k = 0;
  while ((int64_t(1) << k) < x) ++k;
  return k;
}

// Cluster geometry of a length-Nfft transform with L the twiddle base.
bool make_ce_geo(int n, int L, int Nfft, int Q, int T1, CeGeo& g) {
  g = CeGeo{};
  const int lg = ilg(Nfft);
  g.n = n;
  g.L = L;
  g.tws = L / Nfft;
  g.lgN1 = (lg + 1) / 2;
  g.N1 = 1 << g.lgN1;
  g.lgN2 = lg - g.lgN1;
  g.N2 = 1 << g.lgN2;
  if (2 * Q > g.N1 || Q > g.N2) return false;
  g.Q = Q;
  g.cQ = g.N2 / Q;
  g.lgcQ = ilg(g.cQ);
  g.U = g.N1 / (2 * Q);
  g.lgU = ilg(g.U);
  g.Bq = 2 * g.U;
  g.lgBq = ilg(g.Bq);
  g.nbuf = Nfft / Q;
  g.T1 = T1;
  g.LT = L / T1;
  g.lgLT = ilg(g.LT);
  g.q = 0;
  return true;
}

void unit_slot(int k1, int N1, int U, int& q, int& slot) {
  const int h = N1 / 2;
  int u, b;
  if (k1 == 0) { u = 0; b = 0; }
  else if (k1 == h) { u = 0; b = 1; }
  else if (k1 < h) { u = k1; b = 0; }
  else { u = N1 - k1; b = 1; }
  q = u / U;
  slot = 2 * (u % U) + b;
}

// Host tables of one instance.
struct HostInst {
  int n = 0, L = 0, Nc = 0, E = 0, ld = 0;
  CeGeo gr{}, gc{};
  std::vector<double> ahat, eps, cw, lam;
  std::vector<int> Eact;
  std::vector<double2> chirp, Bh, spT64;
  std::vector<float2> spT32;
  std::string err;
};

bool build_instance(const tsfde_instance& in, int64_t M, double mu_opt, int kmu_opt, int Q,
                    HostInst& h) {
  const double alpha = in.alpha, gamma = in.gamma, T = in.T, r = in.r, l = in.l;
  const int64_t n = in.n;
  const double mu = mu_opt > 0.0 ? mu_opt : 1.0 + 0.5 * alpha;
  if (!(mu > alpha && mu <= 2.0)) { h.err = "mu must be in (alpha,2]"; return false; }
  const int kmu = kmu_opt > 0 ? kmu_opt : (mu == 2.0 ? 2 : 1);
  h.n = (int)n;
  int L = 8;
  while (L < 2 * n - 1) L *= 2;
  h.L = L;
  h.Nc = L / 2;
  h.ld = (int)((n + 1) / 2 * 2);
  // geometry: tables sized for the complex transform (the larger N1)
  const int lgL = ilg(L);
  const int T1 = 1 << ((lgL + 1) / 2);
  if (!make_ce_geo((int)n, L, h.Nc, Q, T1, h.gr) || !make_ce_geo((int)n, L, L, Q, T1, h.gc)) {
    h.err = "instance too small for the cluster size";
    return false;
  }
  // mesh and per-level scalars (Sec. 3.1, Eq. (2.8))
  std::vector<double> tau(M + 1, 0.0);
  for (int64_t m = 1; m <= M; ++m) tau[m] = mesh_gap(T, M, r, m, m - 1);
  const double G2 = std::tgamma(2.0 - gamma), G1 = std::tgamma(1.0 - gamma);
  h.ahat.assign(M + 1, 0.0);
  for (int64_t m = 1; m <= M; ++m) h.ahat[m] = std::pow(tau[m], -gamma) / G2;
  // SOE table (Lemma 2.2) and its per-level factors
  std::vector<double> s, w;
  std::string why;
  if (!soe_build(gamma, tau[1], T, in.soe_tol, s, w, &why)) { h.err = why; return false; }
  const int E = h.E = (int)s.size();
  h.eps.assign((size_t)(M + 1) * std::max(E, 1), 0.0);
  h.cw.assign((size_t)(M + 1) * std::max(E, 1), 0.0);
  h.Eact.assign(M + 1, 0);
  for (int64_t m = 2; m <= M; ++m) {
    int act = 0;
    for (int j = 0; j < E; ++j) {
      const double e = std::exp(-s[j] * tau[m]);
      const double x = s[j] * tau[m - 1];
      const double beta = (x == 0.0) ? 1.0 : -std::expm1(-x) / x;
      h.eps[m * E + j] = e;
      h.cw[m * E + j] = w[j] * beta / G1;
      if (e > 0.0) act = j + 1;
    }
    h.Eact[m] = act;
  }
  // symbol, spectrum pairs in row-pass order, Strang eigenvalues
  std::vector<double> sym = ifl_symbol(alpha, mu, kmu, n, l);
  std::vector<double> S = embed_spectrum(sym, L);
  h.lam = strang_eigs(sym, L);
  for (double x : h.lam)
    if (!(x > 0.0)) { h.err = "Strang eigenvalue not positive"; return false; }
  const int Nc = h.Nc;
  h.spT64.assign(Nc, make_double2(0, 0));
  h.spT32.assign(Nc, make_float2(0, 0));
  {
    const CeGeo& g = h.gr;
    for (int k1 = 0; k1 < g.N1; ++k1) {
      int q, slot;
      unit_slot(k1, g.N1, g.U, q, slot);
      for (int k2 = 0; k2 < g.N2; ++k2) {
        const int k = k1 + g.N1 * k2;
        const int kp = (k == 0) ? Nc : Nc - k;
        const size_t at = (size_t)q * g.nbuf + (size_t)k2 * g.Bq + slot;
        h.spT64[at] = make_double2(S[k] / Nc, S[kp] / Nc);
        h.spT32[at] = make_float2((float)(S[k] / Nc), (float)(S[kp] / Nc));
      }
    }
  }
  // Bluestein chirp and kernel spectrum / L in the complex geometry's order
  h.chirp.resize(n);
  for (int64_t j = 0; j < n; ++j) {
    const cd v = chirp(j, n, +1);
    h.chirp[j] = make_double2(v.real(), v.imag());
  }
  std::vector<cd> bk(L, cd(0, 0));
  for (int64_t m = 0; m < n; ++m) bk[m] = std::conj(chirp(m, n, +1));
  for (int64_t m = 1; m < n; ++m) bk[L - m] = std::conj(chirp(m, n, +1));
  fft_inplace(bk, -1);
  h.Bh.assign(L, make_double2(0, 0));
  {
    const CeGeo& g = h.gc;
    for (int k1 = 0; k1 < g.N1; ++k1) {
      int q, slot;
      unit_slot(k1, g.N1, g.U, q, slot);
      for (int k2 = 0; k2 < g.N2; ++k2) {
        const cd v = bk[k1 + (size_t)g.N1 * k2] / (double)L;
        h.Bh[(size_t)q * g.nbuf + (size_t)k2 * g.Bq + slot] = make_double2(v.real(), v.imag());
      }
    }
  }
  return true;
}

}  // namespace

// Instances of one size class share a cluster size, a shared-memory layout and
// a persistent launch; the classes' launches run side by side on two streams.
struct BClass {
  std::vector<int> members;  // caller indices in launch order (largest first)
  int Q = 0, clusters = 0;
  CeLay lay{};
  BInst* dinst = nullptr;
  int* dnext = nullptr;
  StepStat* dstats = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
};

struct tsfde_batch {
  int B = 0;
  int64_t M = 0;
  tsfde_opts opts{};
  tsfde_batch_plan plan{};
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<BClass> cls;
  std::vector<BInst> inst;     // host copies (device pointers inside)
  std::vector<StepStat> stats; // per caller index, last solve
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

template <typename T> bool balloc(tsfde_batch* b, T** p, size_t count) {
  void* q = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) return false;
  b->allocs.push_back(q);
  // zeroed, so that no buffer read before its first write sees stale NaNs
  if (cudaMemset(q, 0, count * sizeof(T)) != cudaSuccess) return false;
  *p = static_cast<T*>(q);
  return true;
}

template <typename T> cudaError_t up(T* dst, const std::vector<T>& src) {
  return cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

int bfail(tsfde_batch* b, int st, const std::string& msg) {
  if (b) b->err = msg;
  std::fprintf(stderr, "tsfde_batch_setup: %s\n", msg.c_str());
  return st;
}

// Cluster size for instances with nmin <= n <= nmax: among 4, 8, 16 (or the
// caller's), those every instance can split and whose shared-memory layout
// fits; the one keeping the most CTAs resident (ties: the smaller cluster).
int pick_q(int64_t nmin, int64_t nmax, int want) {
  int Lmin = 8, Lmax0 = 8;
  while (Lmin < 2 * nmin - 1) Lmin *= 2;
  while (Lmax0 < 2 * nmax - 1) Lmax0 *= 2;
  const int lgs = ilg(Lmin / 2);
  const int N1s = 1 << ((lgs + 1) / 2), N2s = (Lmin / 2) / N1s;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int best = 0, Q = 0;
  for (int q : {4, 8, 16}) {
    if (want > 0 && q != want) continue;
    if (2 * q > N1s || q > N2s) continue;
    const int lgL = ilg(Lmax0);
    const int N1c = 1 << ((lgL + 1) / 2);
    CeLay y{};
    y.has64 = 1;
    y.capB = std::max((Lmax0 / q + N1c) * (int)sizeof(double2), 2 * 4096 * (int)sizeof(double));
    y.nbufB = (Lmax0 / q) * (int)sizeof(double2);
    y.T1 = N1c;
    y.LT = Lmax0 / N1c;
    const size_t sm = batch_smem_bytes(y);
    if (sm > (size_t)optin) continue;
    const int res = batch_max_clusters(q, sm) * q;
    if (res > best) { best = res; Q = q; }
  }
  return Q;
}

}  // namespace

extern "C" {

int tsfde_batch_setup_plan(tsfde_batch** out, int B, const tsfde_instance* inst, int64_t M,
                           const tsfde_opts* opts, const tsfde_batch_plan* plan) {
  if (!out) return TSFDE_EINVAL;
  *out = nullptr;
  if (plan && (plan->classes < 1 || plan->classes > 2)) return TSFDE_EINVAL;
  for (int k = 0; plan && k < plan->classes; ++k)
    if (plan->cluster_size[k] != 0 && plan->cluster_size[k] != 4 && plan->cluster_size[k] != 8 &&
        plan->cluster_size[k] != 16)
      return TSFDE_EINVAL;
  if (B < 1 || !inst || M < 1) return TSFDE_EINVAL;
  tsfde_opts o;
  if (opts) o = *opts; else tsfde_default_opts(&o);
  if (o.precision != TSFDE_FP64 && o.precision != TSFDE_MIXED) return TSFDE_EINVAL;
  if (o.history == TSFDE_HISTORY_DIRECT) return TSFDE_ENOTSUP;  // FIDS only
  if (o.krylov != TSFDE_KRYLOV_BICGSTAB && o.krylov != TSFDE_KRYLOV_PCG && o.krylov != TSFDE_KRYLOV_AUTO)
    return TSFDE_EINVAL;
  if (o.warm_start < 0 || o.warm_start > 2) return TSFDE_EINVAL;
  if (o.history != TSFDE_HISTORY_SOE) return TSFDE_EINVAL;
  if (o.precond != TSFDE_STRANG && o.precond != TSFDE_PRECOND_NONE) return TSFDE_EINVAL;
  if (!(o.krylov_tol > 0.0) || o.max_it < 1) return TSFDE_EINVAL;
  if (o.precision == TSFDE_MIXED &&
      (!(o.inner_tol > 0.0 && o.inner_tol < 1.0) || o.max_outer < 1 || o.inner_max_it < 1))
    return TSFDE_EINVAL;
  int64_t nmin = INT64_MAX, nmax = 0;
  for (int i = 0; i < B; ++i) {
    const tsfde_instance& x = inst[i];
    if (!(x.alpha > 0.0 && x.alpha < 2.0) || !(x.gamma > 0.0 && x.gamma < 1.0) || !(x.l > 0.0) ||
        !(x.T > 0.0) || !(x.r >= 1.0) || !(x.soe_tol > 0.0 && x.soe_tol <= 1e-2) || !x.phi ||
        !x.kappa || !x.f || x.n < 1)
      return TSFDE_EINVAL;
    nmin = std::min(nmin, x.n);
    nmax = std::max(nmax, x.n);
  }
  if (nmin < 31 || nmax > 16383) return TSFDE_ENOTSUP;
  if (o.cluster_size != 0 && o.cluster_size != 4 && o.cluster_size != 8 && o.cluster_size != 16)
    return TSFDE_EINVAL;
  tsfde_batch* b = new tsfde_batch();
  b->B = B;
  b->M = M;
  b->opts = o;
  b->stream = static_cast<cudaStream_t>(o.stream);
  // Size classes.  Default plan: transforms of length L >= 16384 (n >= 8193:
  // one CTA per SM with their shared-memory layout) and the rest (several
  // CTAs per SM), each with the cluster size that keeps the most CTAs
  // resident.  A plan (tsfde_batch_tune) may instead put every instance in
  // one persistent launch, move the split, and fix each class's cluster size.
  tsfde_batch_plan pl{};
  if (plan) {
    pl = *plan;
  } else {
    pl.classes = 2;
    pl.split_n = 8193;
    pl.cluster_size[0] = pl.cluster_size[1] = o.cluster_size;
  }
  std::vector<int> order(B);
  for (int i = 0; i < B; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return inst[a].n > inst[c].n; });
  std::vector<int> want_q;
  {
    BClass big, small;
    for (int i : order) (pl.classes == 1 || inst[i].n >= pl.split_n ? big : small).members.push_back(i);
    if (!big.members.empty()) {
      b->cls.push_back(big);
      want_q.push_back(pl.cluster_size[0]);
    }
    if (!small.members.empty()) {
      b->cls.push_back(small);
      want_q.push_back(pl.cluster_size[pl.classes == 2 ? 1 : 0]);
    }
  }
  std::vector<int> cls_of(B, 0);
  for (size_t k = 0; k < b->cls.size(); ++k) {
    BClass& C = b->cls[k];
    int64_t lo = INT64_MAX, hi = 0;
    for (int i : C.members) {
      cls_of[i] = (int)k;
      lo = std::min(lo, inst[i].n);
      hi = std::max(hi, inst[i].n);
    }
    C.Q = pick_q(lo, hi, want_q[k]);
    if (C.Q == 0) {
      const int st = bfail(b, TSFDE_ENOTSUP, "no cluster size fits these instances on this device");
      tsfde_batch_destroy(b);
      return st;
    }
  }
  // host tables, in parallel
  std::vector<HostInst> H(B);
  {
    std::atomic<int> next(0);
    std::atomic<int> bad(-1);
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
      th.emplace_back([&]() {
        for (;;) {
          const int i = next.fetch_add(1);
          if (i >= B) break;
          if (!build_instance(inst[i], M, o.mu, o.kappa_mu, b->cls[cls_of[i]].Q, H[i])) {
            int exp = -1;
            bad.compare_exchange_strong(exp, i);
          }
        }
      });
    for (auto& t : th) t.join();
    if (bad.load() >= 0) {
      const int i = bad.load();
      const int st = bfail(b, TSFDE_EINVAL, "instance " + std::to_string(i) + ": " + H[i].err);
      tsfde_batch_destroy(b);
      return st;
    }
  }
  // shared-memory layout of each class (its largest transform)
  int Lmax = 8;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  for (size_t k = 0; k < b->cls.size(); ++k) {
    BClass& C = b->cls[k];
    CeLay lay{};
    lay.has64 = 1;
    for (int i : C.members) {
      const HostInst& h = H[i];
      Lmax = std::max(Lmax, h.L);
      lay.capB = std::max(lay.capB, (h.gc.nbuf + h.gc.N1) * (int)sizeof(double2));
      lay.nbufB = std::max(lay.nbufB, h.gc.nbuf * (int)sizeof(double2));
      lay.T1 = std::max(lay.T1, h.gc.T1);
      lay.LT = std::max(lay.LT, h.gc.LT);
      // the right-hand side stages the level's SOE factors in S
      lay.capB = std::max(lay.capB, 2 * std::max(h.E, 1) * (int)sizeof(double));
      if (h.E > 4096) {
        const int st = bfail(b, TSFDE_ENOTSUP, "SOE table longer than 4096 exponentials");
        tsfde_batch_destroy(b);
        return st;
      }
    }
    C.lay = lay;
    const size_t smem = batch_smem_bytes(lay);
    C.clusters = (smem <= (size_t)optin) ? batch_max_clusters(C.Q, smem) : 0;
    if (C.clusters < 1) {
      const int st = bfail(b, TSFDE_ENOTSUP, "cluster launch not possible on this device");
      tsfde_batch_destroy(b);
      return st;
    }
    if (k == 0) {
      C.stream = b->stream;
    } else if (cudaStreamCreateWithFlags(&C.stream, cudaStreamNonBlocking) == cudaSuccess) {
      C.own_stream = true;
    } else {
      const int st = bfail(b, TSFDE_ECUDA, "cudaStreamCreate failed");
      tsfde_batch_destroy(b);
      return st;
    }
  }
  if (cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    const int st = bfail(b, TSFDE_ECUDA, "cudaEventCreate failed");
    tsfde_batch_destroy(b);
    return st;
  }
  // device memory
  bool ok = balloc(b, &b->tw64, Lmax) && balloc(b, &b->tw32, Lmax);
  for (BClass& C : b->cls)
    ok = ok && balloc(b, &C.dinst, C.members.size()) && balloc(b, &C.dnext, 1) &&
         balloc(b, &C.dstats, C.members.size());
  b->inst.resize(B);
  std::vector<double> kmean(B, 0.0);
  for (int i = 0; i < B && ok; ++i) {
    const HostInst& h = H[i];
    BInst& I = b->inst[i];
    I = BInst{};
    const int n = h.n, ld = h.ld, E = std::max(h.E, 1);
    I.n = n; I.E = h.E; I.ld = ld;
    I.gr = h.gr; I.gc = h.gc;
    I.tstride = Lmax / h.L;
    double *phi, *k64, *f, *Hh, *u0, *u1, *u2, *u3, *r64, *w, *ah, *eps, *cw, *lam, *h64;
    float *k32, *h32;
    int* ea;
    double2 *ch, *bh, *t64, *g64;
    float2 *t32, *g32;
    ok = ok && balloc(b, &phi, ld) && balloc(b, &k64, ld) && balloc(b, &f, ld) &&
         balloc(b, &Hh, (size_t)E * ld) && balloc(b, &u0, ld) && balloc(b, &u1, ld) &&
         balloc(b, &u2, ld) && balloc(b, &u3, ld) && balloc(b, &r64, ld) && balloc(b, &w, ld) && balloc(b, &k32, ld) &&
         balloc(b, &h64, ld) && balloc(b, &h32, ld) &&
         balloc(b, &ah, M + 1) && balloc(b, &eps, h.eps.size()) && balloc(b, &cw, h.cw.size()) &&
         balloc(b, &ea, M + 1) && balloc(b, &lam, n) && balloc(b, &ch, n) && balloc(b, &bh, h.L) &&
         balloc(b, &t64, h.Nc) && balloc(b, &t32, h.Nc) && balloc(b, &g64, h.Nc) && balloc(b, &g32, h.Nc);
    double* v64[9];
    float* v32[9];
    for (int q = 0; q < 9 && ok; ++q) ok = balloc(b, &v64[q], ld) && balloc(b, &v32[q], ld);
    if (!ok) break;
    I.phi = phi; I.kap64 = k64; I.kap32 = k32; I.hinv64 = h64; I.hinv32 = h32; I.f = f; I.H = Hh;
    I.u[0] = u0; I.u[1] = u1; I.u[2] = u2; I.u[3] = u3; I.r64 = r64; I.w = w;
    I.v64 = KVecs<double>{v64[0], v64[1], v64[2], v64[3], v64[4], v64[5], v64[6], v64[7], v64[8]};
    I.v32 = KVecs<float>{v32[0], v32[1], v32[2], v32[3], v32[4], v32[5], v32[6], v32[7], v32[8]};
    I.ahat = ah; I.eps = eps; I.cw = cw; I.Eact = ea; I.lam = lam; I.chirp = ch; I.Bh = bh;
    I.spT64 = t64; I.spT32 = t32; I.spG64 = g64; I.spG32 = g32;
    cudaError_t e = cudaSuccess;
    const size_t nb = sizeof(double) * n;
    // zero-padded copies of the caller's data
    for (double* p : {phi, k64, f, u0, u1, u2, r64, w})
      if (e == cudaSuccess) e = cudaMemset(p, 0, sizeof(double) * ld);
    if (e == cudaSuccess) e = cudaMemset(k32, 0, sizeof(float) * ld);
    for (int q = 0; q < 9 && e == cudaSuccess; ++q) {
      e = cudaMemset(v64[q], 0, sizeof(double) * ld);
      if (e == cudaSuccess) e = cudaMemset(v32[q], 0, sizeof(float) * ld);
    }
    if (e == cudaSuccess) e = cudaMemcpy(phi, inst[i].phi, nb, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(k64, inst[i].kappa, nb, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f, inst[i].f, nb, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) {
      std::vector<double> kh(n);
      e = cudaMemcpy(kh.data(), k64, nb, cudaMemcpyDeviceToHost);
      std::vector<float> k32h(n), h32h(n);
      std::vector<double> h64h(n);
      double sum = 0.0;
      for (int j = 0; j < n; ++j) {
        if (!(kh[j] > 0.0) || !std::isfinite(kh[j])) ok = false;
        sum += kh[j];
        k32h[j] = (float)kh[j];
        h64h[j] = 1.0 / kh[j];
        h32h[j] = (float)h64h[j];
      }
      kmean[i] = sum / n;
      if (e == cudaSuccess) e = up(k32, k32h);
      if (e == cudaSuccess) e = up(h64, h64h);
      if (e == cudaSuccess) e = up(h32, h32h);
    }
    if (e == cudaSuccess) e = up(ah, h.ahat);
    if (e == cudaSuccess) e = up(eps, h.eps);
    if (e == cudaSuccess) e = up(cw, h.cw);
    if (e == cudaSuccess) e = up(ea, h.Eact);
    if (e == cudaSuccess) e = up(lam, h.lam);
    if (e == cudaSuccess) e = up(ch, h.chirp);
    if (e == cudaSuccess) e = up(bh, h.Bh);
    if (e == cudaSuccess) e = up(t64, h.spT64);
    if (e == cudaSuccess) e = up(t32, h.spT32);
    if (e != cudaSuccess) {
      const int st = bfail(b, TSFDE_ECUDA, std::string("upload: ") + cudaGetErrorString(e));
      tsfde_batch_destroy(b);
      return st;
    }
    if (!ok) {
      const int st = bfail(b, TSFDE_EINVAL, "instance " + std::to_string(i) + ": kappa must be positive");
      tsfde_batch_destroy(b);
      return st;
    }
    I.kbar = kmean[i];
    I.stat = nullptr;  // set per launch slot by each solve
  }
  if (!ok) {
    const int st = bfail(b, TSFDE_ENOMEM, "cudaMalloc failed");
    tsfde_batch_destroy(b);
    return st;
  }
  {
    std::vector<cd> tw = twiddles(Lmax);
    std::vector<double2> t64(Lmax);
    std::vector<float2> t32(Lmax);
    for (int k = 0; k < Lmax; ++k) {
      t64[k] = make_double2(tw[k].real(), tw[k].imag());
      t32[k] = make_float2((float)tw[k].real(), (float)tw[k].imag());
    }
    if (up(b->tw64, t64) != cudaSuccess || up(b->tw32, t32) != cudaSuccess) {
      const int st = bfail(b, TSFDE_ECUDA, "upload twiddles");
      tsfde_batch_destroy(b);
      return st;
    }
  }
  b->stats.assign(B, StepStat{});
  b->plan = pl;
  b->plan.classes = (int)b->cls.size();
  for (int k = 0; k < 2; ++k) {
    b->plan.cluster_size[k] = k < (int)b->cls.size() ? b->cls[k].Q : 0;
    b->plan.clusters[k] = k < (int)b->cls.size() ? b->cls[k].clusters : 0;
  }
  if (b->cls.size() == 1) b->plan.split_n = 0;
  *out = b;
  return TSFDE_OK;
}

int tsfde_batch_setup(tsfde_batch** out, int B, const tsfde_instance* inst, int64_t M,
                      const tsfde_opts* opts) {
  return tsfde_batch_setup_plan(out, B, inst, M, opts, nullptr);
}

int tsfde_batch_get_plan(const tsfde_batch* b, tsfde_batch_plan* plan) {
  if (!b || !plan) return TSFDE_EINVAL;
  *plan = b->plan;
  return TSFDE_OK;
}

// Launch-plan search: every candidate is set up for the real batch and
// times a solve of its first probe_levels levels (CUDA events on the
// options' stream, after one untimed solve); the fastest is returned.
int tsfde_batch_tune(int B, const tsfde_instance* inst, int64_t M, const tsfde_opts* opts,
                     int64_t probe_levels, tsfde_batch_plan* best, tsfde_batch_plan* tried, int* ntried) {
  if (!best || B < 1 || !inst || M < 1) return TSFDE_EINVAL;
  if (probe_levels < 1 || probe_levels > M) return TSFDE_EINVAL;
  const int cap = (ntried && tried) ? *ntried : 0;
  if (ntried) *ntried = 0;
  std::vector<tsfde_batch_plan> cand;
  auto add = [&](int classes, int64_t split, int q0, int q1) {
    tsfde_batch_plan p{};
    p.classes = classes;
    p.split_n = split;
    p.cluster_size[0] = q0;
    p.cluster_size[1] = q1;
    cand.push_back(p);
  };
  for (int q : {4, 8, 16}) add(1, 0, q, 0);
  for (int64_t split : {(int64_t)8193, (int64_t)4097})
    for (int qb : {8, 16})
      for (int qs : {4, 8}) add(2, split, qb, qs);
  int64_t ntot = 0;
  for (int i = 0; i < B; ++i) ntot += std::max<int64_t>(inst[i].n, 1);
  void* out_buf = nullptr;
  if (cudaMalloc(&out_buf, sizeof(double) * (size_t)ntot) != cudaSuccess) return TSFDE_ENOMEM;
  std::vector<double*> outs(B);
  {
    double* q = static_cast<double*>(out_buf);
    for (int i = 0; i < B; ++i) {
      outs[i] = q;
      q += std::max<int64_t>(inst[i].n, 1);
    }
  }
  cudaStream_t s = opts ? static_cast<cudaStream_t>(opts->stream) : nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = TSFDE_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = TSFDE_ECUDA;
  double best_ms = 0.0;
  bool found = false;
  std::vector<tsfde_batch_plan> done;
  for (size_t c = 0; c < cand.size() && st == TSFDE_OK; ++c) {
    tsfde_batch* b = nullptr;
    const int rc = tsfde_batch_setup_plan(&b, B, inst, M, opts, &cand[c]);
    if (rc == TSFDE_ENOTSUP || rc == TSFDE_ENOMEM) continue;  // this plan does not fit
    if (rc != TSFDE_OK) { st = rc; break; }
    // plans that end up identical to one already timed are skipped
    bool dup = false;
    for (const tsfde_batch_plan& d : done)
      if (d.classes == b->plan.classes && d.split_n == b->plan.split_n &&
          d.cluster_size[0] == b->plan.cluster_size[0] && d.cluster_size[1] == b->plan.cluster_size[1])
        dup = true;
    float ms = 0.f;
    int r1 = TSFDE_OK;
    if (!dup) {
      r1 = tsfde_batch_solve(b, probe_levels, outs.data(), nullptr);
      if (r1 == TSFDE_OK && cudaEventRecord(e0, s) == cudaSuccess) {
        r1 = tsfde_batch_solve(b, probe_levels, outs.data(), nullptr);
        if (r1 == TSFDE_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                               cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
          r1 = TSFDE_ECUDA;
      }
    }
    tsfde_batch_plan got = b->plan;
    tsfde_batch_destroy(b);
    if (dup) continue;
    if (r1 != TSFDE_OK) { st = r1; break; }
    got.probe_ms = ms;
    done.push_back(got);
    if (ntried && *ntried < cap) tried[(*ntried)++] = got;
    if (!found || ms < best_ms) {
      best_ms = ms;
      *best = got;
      found = true;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out_buf);
  if (st == TSFDE_OK && !found) st = TSFDE_ENOTSUP;
  return st;
}

int tsfde_batch_solve(tsfde_batch* b, int64_t levels, double* const* u_final,
                      tsfde_batch_info* info) {
  if (!b || !u_final || levels < 0 || levels > b->M) return TSFDE_EINVAL;
  if (levels == 0) levels = b->M;
  for (int i = 0; i < b->B; ++i)
    if (!u_final[i]) return TSFDE_EINVAL;
  BatchArgs A0{};
  A0.M = (int)levels;
  A0.precision = b->opts.precision;
  A0.precond = b->opts.precond == TSFDE_STRANG ? 1 : 0;
  A0.tol = b->opts.krylov_tol;
  A0.inner_tol = b->opts.inner_tol;
  A0.max_it = b->opts.max_it;
  A0.max_outer = b->opts.max_outer;
  A0.inner_max_it = b->opts.inner_max_it;
  A0.warm = b->opts.warm_start;
  A0.krylov = b->opts.krylov;
  A0.tw64 = b->tw64;
  A0.tw32 = b->tw32;
  // the classes' streams start after the caller's stream reaches this point
  // and the caller's stream continues after all of them
  cudaError_t e = cudaEventRecord(b->ev_in, b->stream);
  const size_t nc = b->cls.size();
  std::vector<std::vector<BInst>> d(nc);
  std::vector<std::vector<StepStat>> st(nc);
  for (size_t k = 0; k < nc && e == cudaSuccess; ++k) {
    BClass& C = b->cls[k];
    const int cnt = (int)C.members.size();
    d[k].resize(cnt);
    st[k].resize(cnt);
    for (int j = 0; j < cnt; ++j) {
      const int i = C.members[j];
      d[k][j] = b->inst[i];
      d[k][j].u_out = u_final[i];
      d[k][j].stat = C.dstats + j;
    }
    if (C.stream != b->stream) e = cudaStreamWaitEvent(C.stream, b->ev_in, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(C.dinst, d[k].data(), sizeof(BInst) * cnt, cudaMemcpyHostToDevice, C.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(C.dstats, 0, sizeof(StepStat) * cnt, C.stream);
    BatchArgs A = A0;
    A.inst = C.dinst;
    A.count = cnt;
    A.next = C.dnext;
    A.lay = C.lay;
    if (e == cudaSuccess) e = launch_batch(A, C.Q, C.clusters, C.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(st[k].data(), C.dstats, sizeof(StepStat) * cnt, cudaMemcpyDeviceToHost, C.stream);
    if (e == cudaSuccess && C.stream != b->stream) {
      e = cudaEventRecord(b->ev_out, C.stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_out, 0);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    b->err = std::string("batch launch: ") + cudaGetErrorString(e);
    return TSFDE_ECUDA;
  }
  tsfde_batch_info inf{};
  inf.failed_instance = -1;
  inf.levels = (int64_t)b->B * levels;
  for (size_t k = 0; k < nc; ++k)
    for (size_t j = 0; j < b->cls[k].members.size(); ++j) {
      const int i = b->cls[k].members[j];
      const StepStat& x = st[k][j];
      b->stats[i] = x;
      inf.iterations += x.iterations;
      inf.outer += x.outer;
      inf.fp64_levels += x.E_active;
      inf.max_rel_residual = std::max(inf.max_rel_residual, x.rel_residual);
      if (x.status != TSFDE_OK && (inf.status == TSFDE_OK || i < inf.failed_instance)) {
        inf.status = x.status;
        inf.failed_instance = i;
      }
    }
  if (info) *info = inf;
  return inf.status;
}

int tsfde_batch_instance_stats(const tsfde_batch* b, int i, tsfde_step_info* out) {
  if (!b || !out || i < 0 || i >= b->B) return TSFDE_EINVAL;
  const StepStat& s = b->stats[i];
  out->m = b->M;
  out->status = s.status;
  out->iterations = s.iterations;
  out->outer = s.outer;
  out->E_active = s.E_active;
  out->rel_residual = s.rel_residual;
  return TSFDE_OK;
}

int tsfde_batch_shape(const tsfde_batch* b, int* clusters, int* cluster_size) {
  if (!b) return TSFDE_EINVAL;
  if (clusters) *clusters = b->cls.empty() ? 0 : b->cls[0].clusters;
  if (cluster_size) *cluster_size = b->cls.empty() ? 0 : b->cls[0].Q;
  return TSFDE_OK;
}

void tsfde_batch_destroy(tsfde_batch* b) {
  if (!b) return;
  for (BClass& C : b->cls)
    if (C.own_stream) cudaStreamDestroy(C.stream);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  for (void* p : b->allocs) cudaFree(p);
  delete b;
}

}  // extern "C"
