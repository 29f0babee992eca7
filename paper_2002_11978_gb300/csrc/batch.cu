// batch.cu -- batched FIDS solve (many independent problems) on sm_103a.
//
// One persistent launch of thread-block clusters.  A cluster claims an
// instance from a global counter (largest first: the host sorts them), marches
// it through all M levels, writes u^M, and claims the next.  Everything of a
// level runs inside the cluster, with the transforms in distributed shared
// memory (cluster.cuh):
//   SOE history update and right-hand side of Eq. (3.16gu) (one HBM pass over
//     the E x n history),
//   the Strang preconditioner of Sec. 4.1 built in FP64 (Bluestein length-n
//     inverse DFT of 1/(ahat + kbar lambda) on length-L complex transforms,
//     then the spectrum of its even embedding),
//   the level solve: FP32 Krylov sweeps (PBiCGSTAB, or PCG on the
//     symmetrised system) refined by FP64 residual products and finished in
//     FP64 when the refinement stalls (the rules of mixed_level in grid.cuh),
//     or the plain FP64 Krylov solve.
// Instances never wait on one another, so there is no grid-wide barrier: the
// only waits are cluster barriers, whose partners are co-scheduled by the
// hardware and take the same branches (every decision uses cluster-reduced
// scalars that are bitwise equal in all CTAs).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/tsfde.h"
#include "cluster.cuh"
#include "dev.cuh"
#include "plan.h"

namespace tsfde {

constexpr int kBT = 256;  // threads per CTA

// cluster partial-sum slots of the level loop, apart from ce_bicgstab's 0..5
// (a CTA may start pushing into those while another still reads these)
enum { BS_RW = 6, BS_WW = 7, BS_RES = 8, BS_EMAX = 9, BS_XMAX = 10, BS_BB = 11, BS_R0 = 12 };

// Per-cluster context at CeSm::ctx.
struct BatchCtx {
  CeCtx<float> c32;
  CeCtx<double> c64;
  BInst I;
  int inst;
  int method;  // Krylov method of the current level (TSFDE_KRYLOV_BICGSTAB / _PCG)
};

// rotating level buffers per instance
constexpr int kBRoll = 4;

size_t batch_smem_bytes(const CeLay& lay) { return ce_ctx_offset(lay) + sizeof(BatchCtx); }

__device__ __forceinline__ CeGeo geo_q(const CeGeo& g0) {
  CeGeo g = g0;
  g.q = (int)cg::this_cluster().block_rank();
  return g;
}

// ------------------------------------------------------------ level pieces
// u^0 = phi, H = 0 (owned pairs of gr).
__device__ __noinline__ void bt_init(const BatchCtx* bx) {
  const BInst& I = bx->I;
  const CeGeo g = geo_q(I.gr);
  const int n = g.n, npair = (g.N1 >> 1) << g.lgcQ;
  double** const u = const_cast<double**>(I.u);
  for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) {
    const int i0 = pair_i0(g, pp);
    if (i0 >= n) continue;
    st2(u[0], i0, n, ld2(I.phi, i0));
    for (int j = 0; j < I.E; ++j) st2(I.H + (size_t)j * I.ld, i0, n, make_double2(0.0, 0.0));
  }
}

// History update and right-hand side of level m into r64; u^m = 0, or
// u^{m-1} with warm = 1, or (warm = 2) the polynomial in the level index
// through u^{m-1} .. u^{m-4} evaluated at m (x0 = 4 u^{m-1} - 6 u^{m-2} +
// 4 u^{m-3} - u^{m-4}; lower orders at the first levels; u^{m-4} shares its
// buffer with u^m and is read first); pushes the cluster partial of b.b
// into slot BS_BB.
__device__ __noinline__ void bt_rhs(const BatchCtx* bx, int m, int warm) {
  const BInst& I = bx->I;
  const CeGeo g = geo_q(I.gr);
  const CeSm<double> s = ce_sm<double>(bx->c64.lay);
  const int n = g.n, npair = (g.N1 >> 1) << g.lgcQ;
  const int Eact = (m >= 2) ? I.Eact[m] : 0;
  double* s_eps = reinterpret_cast<double*>(s.S);  // S is free between products
  double* s_cw = s_eps + Eact;
  for (int j = threadIdx.x; j < Eact; j += blockDim.x) {
    s_eps[j] = I.eps[(size_t)m * I.E + j];
    s_cw[j] = I.cw[(size_t)m * I.E + j];
  }
  __syncthreads();
  const double* u1 = I.u[(m - 1) % kBRoll];
  const double* u2 = I.u[(m >= 2 ? m - 2 : m - 1) % kBRoll];
  double* um = I.u[m % kBRoll];
  const double ah = I.ahat[m];
  // extrapolated start: order q and the Lagrange weights (-1)^j C(q+1, j+1)
  const int q = (warm == 2 && m >= 2) ? (m - 1 < 3 ? m - 1 : 3) : 0;
  const double w0 = q + 1, w1 = -0.5 * (q + 1) * q, w2 = (q + 1) * q * (q - 1) / 6.0,
               w3 = -(q + 1) * q * (q - 1) * (q - 2) / 24.0;
  const double* u3 = q >= 2 ? I.u[(m - 3) % kBRoll] : nullptr;
  const double* u4 = q >= 3 ? I.u[(m - 4) % kBRoll] : nullptr;
  double bb = 0.0;
  for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) {
    const int i0 = pair_i0(g, pp);
    if (i0 >= n) continue;
    const double2 a1 = ld2(u1, i0), a2 = ld2(u2, i0);
    const double dx = a1.x - a2.x, dy = a1.y - a2.y;
    double sx = 0.0, sy = 0.0;
    double* Hp = I.H + i0;
    for (int j = 0; j < Eact; ++j) {
      double2* h = reinterpret_cast<double2*>(Hp + (size_t)j * I.ld);
      double2 v = *h;
      v.x = s_eps[j] * fma(s_cw[j], dx, v.x);
      v.y = s_eps[j] * fma(s_cw[j], dy, v.y);
      *h = v;
      sx += v.x;
      sy += v.y;
    }
    const double2 fv = ld2(I.f, i0);
    double2 b = make_double2(ah * a1.x - sx + fv.x, ah * a1.y - sy + fv.y);
    if (i0 + 1 >= n) b.y = 0.0;
    st2(I.r64, i0, n, b);
    double2 x0 = warm ? a1 : make_double2(0.0, 0.0);
    if (q > 0) {
      x0 = make_double2(w0 * a1.x + w1 * a2.x, w0 * a1.y + w1 * a2.y);
      if (q >= 2) {
        const double2 a3 = ld2(u3, i0);
        x0 = make_double2(fma(w2, a3.x, x0.x), fma(w2, a3.y, x0.y));
      }
      if (q >= 3) {
        const double2 a4 = ld2(u4, i0);
        x0 = make_double2(fma(w3, a4.x, x0.x), fma(w3, a4.y, x0.y));
      }
    }
    st2(um, i0, n, x0);
    bb += b.x * b.x + b.y * b.y;
  }
  ce_put(s.part, g.Q, BS_BB, block_sum(bb, s.red));
}

// Preconditioner of level m (FP64): spectrum pairs of the even embedding of
// g = IDFT_n(1/(ahat + kbar lambda)) into spG64 / spG32 (row-pass order).
// Contains its own cluster barriers and ends with one.
__device__ __noinline__ void bt_precond(const BatchCtx* bx, int m) {
  typedef double2 Z;
  cg::cluster_group cl = cg::this_cluster();
  const BInst& I = bx->I;
  const CeSm<double> s = ce_sm<double>(bx->c64.lay);
  const double ah = I.ahat[m], kbar = I.kbar;
  const int n = I.n;
  // (a) Bluestein input a_j = chirp_j / d_j on the complex geometry
  {
    const CeGeo g = geo_q(I.gc);
    Z* X = ce_io(g, s);
    const int nel = (g.N1 >> 1) << g.lgcQ;
    for (int pp = threadIdx.x; pp < nel; pp += blockDim.x) {
      const int j = ((pp >> g.lgcQ) << g.lgN2) + (g.q << g.lgcQ) + (pp & (g.cQ - 1));
      Z v = make_double2(0.0, 0.0);
      if (j < n) {
        const double q = 1.0 / (ah + kbar * I.lam[j]);
        v = cscale(I.chirp[j], q);
      }
      X[pp] = v;
    }
    __syncthreads();
    ce_colfwd_buf(g, s, g.N1 >> 1);
    cl.sync();
    ce_rows<double, CE_CONV>(g, s, I.Bh, nullptr, nullptr);
    cl.sync();
    // (b) inverse transform, g_j = Re(chirp_j z_j) / n into w
    Z* Y = ce_io(g, s);
    const int lgcQ = g.lgcQ;
    auto st = [=](int j1, int c, Z z) {
      if (j1 < (g.N1 >> 1)) Y[(j1 << lgcQ) + c] = z;
    };
    ce_colinv(g, s, st);
    const double invn = 1.0 / (double)n;
    for (int pp = threadIdx.x; pp < nel; pp += blockDim.x) {
      const int j = ((pp >> g.lgcQ) << g.lgN2) + (g.q << g.lgcQ) + (pp & (g.cQ - 1));
      if (j < n) {
        const Z c = I.chirp[j], z = Y[pp];
        I.w[j] = (c.x * z.x - c.y * z.y) * invn;
      }
    }
  }
  cl.sync();  // g complete in global memory for every CTA
  // (c) spectrum of the even embedding e_i = g_i (i < n), g_{L-i} (i > L-n)
  {
    const CeGeo g = geo_q(I.gr);
    const int L = g.L;
    Z* X = ce_io(g, s);
    const int nel = g.N1 << g.lgcQ;  // all rows: the input has length L
    for (int pp = threadIdx.x; pp < nel; pp += blockDim.x) {
      const int j = ((pp >> g.lgcQ) << g.lgN2) + (g.q << g.lgcQ) + (pp & (g.cQ - 1));
      const int i0 = 2 * j, i1 = 2 * j + 1;
      const double x0 = (i0 < n) ? I.w[i0] : ((L - i0 < n && i0 > 0) ? I.w[L - i0] : 0.0);
      const double x1 = (i1 < n) ? I.w[i1] : ((L - i1 < n) ? I.w[L - i1] : 0.0);
      X[pp] = make_double2(x0, x1);
    }
    __syncthreads();
    ce_colfwd_buf(g, s, g.N1);
    cl.sync();
    ce_rows<double, CE_SPEC>(g, s, nullptr, I.spG64, I.spG32);
  }
  cl.sync();
}

// w = M (nr e) in FP64 with e = v32.x; pushes (r64, w) and (w, w).  Ends
// before the barrier of the reduction.
__device__ __noinline__ void bt_resid_product(const BatchCtx* bx, double nr, double ah) {
  typedef double2 Z;
  cg::cluster_group cl = cg::this_cluster();
  const BInst& I = bx->I;
  const CeGeo g = geo_q(I.gr);
  const CeSm<double> s = ce_sm<double>(bx->c64.lay);
  const int n = g.n, npair = (g.N1 >> 1) << g.lgcQ;
  const float* e = I.v32.x;
  Z* X = ce_io(g, s);
  for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) {
    const int i0 = pair_i0(g, pp);
    Z x = make_double2(0.0, 0.0);
    if (i0 < n) {
      const float2 ev = ld2(e, i0);
      x = make_double2(nr * (double)ev.x, i0 + 1 < n ? nr * (double)ev.y : 0.0);
    }
    X[pp] = x;
  }
  __syncthreads();
  ce_colfwd_buf(g, s, g.N1 >> 1);
  cl.sync();
  ce_rows<double, CE_APPLY>(g, s, I.spT64, nullptr, nullptr);
  cl.sync();
  Z* Y = ce_io(g, s);
  {
    const int lgcQ = g.lgcQ, N1 = g.N1;
    auto st = [=](int j1, int c, Z z) {
      if (j1 < (N1 >> 1)) Y[(j1 << lgcQ) + c] = z;
    };
    ce_colinv(g, s, st);
  }
  double rw = 0.0, ww = 0.0;
  for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) {
    const int i0 = pair_i0(g, pp);
    if (i0 >= n) continue;
    const float2 ev = ld2(e, i0);
    const Z y = Y[pp], kv = ld2(I.kap64, i0), rv = ld2((const double*)I.r64, i0);
    Z wv = make_double2(ah * nr * (double)ev.x + kv.x * y.x, ah * nr * (double)ev.y + kv.y * y.y);
    if (i0 + 1 >= n) wv.y = 0.0;
    st2(I.w, i0, n, wv);
    rw += rv.x * wv.x + rv.y * wv.y;
    ww += wv.x * wv.x + wv.y * wv.y;
  }
  const double rwb = block_sum(rw, s.red);
  const double wwb = block_sum(ww, s.red);
  ce_put(s.part, g.Q, BS_RW, rwb);
  ce_put(s.part, g.Q, BS_WW, wwb);
}

// Warm start: r64 = b - M u^m (r64 holds b, u^m = u^{m-1}); pushes r.r into
// BS_R0.  Ends before the barrier of the reduction.
__device__ __noinline__ void bt_warm_residual(const BatchCtx* bx, int m) {
  typedef double2 Z;
  cg::cluster_group cl = cg::this_cluster();
  const BInst& I = bx->I;
  const CeGeo g = geo_q(I.gr);
  const CeSm<double> s = ce_sm<double>(bx->c64.lay);
  const int n = g.n, npair = (g.N1 >> 1) << g.lgcQ;
  const double* um = I.u[m % kBRoll];
  const double ah = I.ahat[m];
  Z* X = ce_io(g, s);
  for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) {
    const int i0 = pair_i0(g, pp);
    Z x = make_double2(0.0, 0.0);
    if (i0 < n) {
      x = ld2(um, i0);
      if (i0 + 1 >= n) x.y = 0.0;
    }
    X[pp] = x;
  }
  __syncthreads();
  ce_colfwd_buf(g, s, g.N1 >> 1);
  cl.sync();
  ce_rows<double, CE_APPLY>(g, s, I.spT64, nullptr, nullptr);
  cl.sync();
  Z* Y = ce_io(g, s);
  {
    const int lgcQ = g.lgcQ, N1 = g.N1;
    auto st = [=](int j1, int c, Z z) {
      if (j1 < (N1 >> 1)) Y[(j1 << lgcQ) + c] = z;
    };
    ce_colinv(g, s, st);
  }
  double rr = 0.0;
  for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) {
    const int i0 = pair_i0(g, pp);
    if (i0 >= n) continue;
    const Z y = Y[pp], kv = ld2(I.kap64, i0), uv = ld2(um, i0), bv = ld2((const double*)I.r64, i0);
    Z r = make_double2(bv.x - (ah * uv.x + kv.x * y.x), bv.y - (ah * uv.y + kv.y * y.y));
    if (i0 + 1 >= n) r.y = 0.0;
    st2(I.r64, i0, n, r);
    rr += r.x * r.x + r.y * r.y;
  }
  ce_put(s.part, g.Q, BS_R0, block_sum(rr, s.red));
}

// u += step e, r64 -= theta w; pushes ||r||^2, max|step e|, max|u|.
__device__ __noinline__ void bt_update(const BatchCtx* bx, int m, double step, double theta) {
  const BInst& I = bx->I;
  const CeGeo g = geo_q(I.gr);
  const CeSm<double> s = ce_sm<double>(bx->c64.lay);
  const int n = g.n, npair = (g.N1 >> 1) << g.lgcQ;
  double* um = I.u[m % kBRoll];
  double rr = 0.0, emax = 0.0, xmax = 0.0;
  for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) {
    const int i0 = pair_i0(g, pp);
    if (i0 >= n) continue;
    const float2 ev = ld2(I.v32.x, i0);
    const double2 uv = ld2((const double*)um, i0), rv = ld2((const double*)I.r64, i0),
                  wv = ld2((const double*)I.w, i0);
    double2 d = make_double2(step * (double)ev.x, step * (double)ev.y);
    double2 x = make_double2(uv.x + d.x, uv.y + d.y);
    double2 r = make_double2(rv.x - theta * wv.x, rv.y - theta * wv.y);
    if (i0 + 1 >= n) { d.y = 0.0; x.y = 0.0; r.y = 0.0; }
    st2(um, i0, n, x);
    st2(I.r64, i0, n, r);
    rr += r.x * r.x + r.y * r.y;
    emax = fmax(emax, fmax(fabs(d.x), fabs(d.y)));
    xmax = fmax(xmax, fmax(fabs(x.x), fabs(x.y)));
  }
  const double a = block_sum(rr, s.red);
  const double b = block_max(emax, s.red);
  const double c = block_max(xmax, s.red);
  ce_put(s.part, g.Q, BS_RES, a);
  ce_put(s.part, g.Q, BS_EMAX, b);
  ce_put(s.part, g.Q, BS_XMAX, c);
}

// u^m += v64.x (the FP64 correction of a level finished in FP64).
__device__ __noinline__ void bt_add_fp64(const BatchCtx* bx, int m) {
  const BInst& I = bx->I;
  const CeGeo g = geo_q(I.gr);
  const int n = g.n, npair = (g.N1 >> 1) << g.lgcQ;
  double* um = I.u[m % kBRoll];
  for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) {
    const int i0 = pair_i0(g, pp);
    if (i0 >= n) continue;
    const double2 uv = ld2((const double*)um, i0), dv = ld2((const double*)I.v64.x, i0);
    st2(um, i0, n, make_double2(uv.x + dv.x, uv.y + dv.y));
  }
}

__device__ __noinline__ void bt_copy_out(const BatchCtx* bx, int m) {
  const BInst& I = bx->I;
  const CeGeo g = geo_q(I.gr);
  const int n = g.n, npair = (g.N1 >> 1) << g.lgcQ;
  const double* um = I.u[m % kBRoll];
  for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) {
    const int i0 = pair_i0(g, pp);
    if (i0 < n) I.u_out[i0] = um[i0];
    if (i0 + 1 < n) I.u_out[i0 + 1] = um[i0 + 1];
  }
}

// The level's Krylov solve on the cluster: BiCGSTAB or PCG on the
// symmetrised system.
template <typename R>
__device__ __forceinline__ SolveRes bt_krylov(const CeCtx<R>* cx, int method, bool prec, double tol,
                                              int max_it, const double* r64, double sc) {
  if (method == TSFDE_KRYLOV_PCG) return ce_pcg<R>(cx, prec, tol, max_it, r64, sc);
  return ce_bicgstab<R>(cx, prec, tol, max_it, r64, sc);
}

struct LevelOut {
  int status, iters, outer;
  bool fp64;
  double relres;
};

// One level: right-hand side, preconditioner, solve.
// prev_fp64: the previous level was finished in FP64 (adaptive precision:
// go to FP64 directly unless m is a retry level).
__device__ LevelOut bt_level(BatchCtx* bx, const BatchArgs& A, int m, bool prev_fp64) {
  cg::cluster_group cl = cg::this_cluster();
  const CeSm<double> s = ce_sm<double>(A.lay);
  const BInst& I = bx->I;
  const int Q = I.gr.Q;
  const bool warm = A.warm != 0;
  LevelOut o{TSFDE_OK, 0, 0, false, 0.0};
  bt_rhs(bx, m, A.warm);
  if (A.precond) bt_precond(bx, m);  // ends with a barrier
  else cl.sync();
  const double bb = ce_total(s.part, Q, BS_BB);
  if (!isfinite(bb)) { o.status = TSFDE_ENONFINITE; return o; }
  if (bb == 0.0) return o;
  double rr0 = bb;
  if (warm) {
    bt_warm_residual(bx, m);
    cl.sync();
    rr0 = ce_total(s.part, Q, BS_R0);
    if (!isfinite(rr0)) { o.status = TSFDE_ENONFINITE; return o; }
    if (rr0 == 0.0) return o;
  }
  const double nb = sqrt(bb);
  const bool prec = A.precond != 0;
  if (threadIdx.x == 0) {
    bx->c32.a = (float)I.ahat[m];
    bx->c64.a = I.ahat[m];
    bx->c64.V.x = (A.precision == TSFDE_FP64 && !warm) ? I.u[m % kBRoll] : I.v64.x;
  }
  __syncthreads();
  if (A.precision == TSFDE_FP64) {
    const double scale = sqrt(rr0 / bb);
    const SolveRes r = bt_krylov<double>(&bx->c64, bx->method, prec, A.tol / scale, A.max_it, I.r64, 1.0);
    cl.sync();
    if (warm && r.status == TSFDE_OK) bt_add_fp64(bx, m);
    o.status = r.status;
    o.iters = r.iters;
    o.relres = r.relres * scale;
    cl.sync();
    return o;
  }
  double nr = sqrt(rr0), relres = nr / nb;
  int stalls = 0;
  bool fallback = prev_fp64 && (m % 64) != 0;
  if (!fallback && relres <= A.tol) { o.relres = relres; cl.sync(); return o; }
  const double ah = I.ahat[m];
  while (!fallback) {
    if (o.outer >= A.max_outer) { fallback = true; break; }
    const SolveRes ir = bt_krylov<float>(&bx->c32, bx->method, prec, A.inner_tol, A.inner_max_it, I.r64, 1.0 / nr);
    o.iters += ir.iters;
    ++o.outer;
    cl.sync();
    // no usable correction (non-finite, or no iteration run): FP64 finish
    if (ir.status == TSFDE_ENONFINITE ||
        (ir.status != TSFDE_OK && ir.status != TSFDE_ENOCONV && ir.iters == 0)) {
      fallback = true;
      break;
    }
    bt_resid_product(bx, nr, ah);
    cl.sync();
    const double rw = ce_total(s.part, Q, BS_RW), ww = ce_total(s.part, Q, BS_WW);
    double theta = 1.0;
    if (ww - 2.0 * rw > 0.0) theta = (ww > 0.0) ? rw / ww : 0.0;
    if (!isfinite(theta) || !(theta > 0.0)) { fallback = true; break; }
    bt_update(bx, m, theta * nr, theta);
    cl.sync();
    const double rr = ce_total(s.part, Q, BS_RES);
    const double emax = ce_maxall(s.part, Q, BS_EMAX), xmax = ce_maxall(s.part, Q, BS_XMAX);
    const double nr_prev = nr;
    nr = sqrt(rr);
    if (!isfinite(nr) || !isfinite(xmax)) { o.status = TSFDE_ENONFINITE; break; }
    relres = nr / nb;
    if (nr == 0.0 || relres <= A.tol) break;
    // a zero correction cannot make progress: never read it as converged
    if (!(emax > 0.0)) { fallback = true; break; }
    if (o.outer >= 2 && emax <= A.tol * xmax) break;  // as in mixed_level (grid.cuh)
    if (o.outer >= 2 && nr > 0.5 * nr_prev) {
      // the FP64 residual is at its rounding floor and u no longer moves at
      // the accuracy asked for
      if (relres <= 1e-9 && emax <= 100.0 * A.tol * xmax) break;
      if (++stalls >= 3) { fallback = true; break; }
    } else {
      stalls = 0;
    }
  }
  if (fallback && o.status == TSFDE_OK) {
    const double tol_d = fmax(A.tol * nb / nr, 1e-14);
    const SolveRes fr = bt_krylov<double>(&bx->c64, bx->method, prec, tol_d, A.max_it, I.r64, 1.0);
    cl.sync();
    if (fr.status == TSFDE_OK) {
      bt_add_fp64(bx, m);
      relres = fr.relres * nr / nb;
    }
    o.status = fr.status;
    o.iters += fr.iters;
    o.fp64 = true;
  }
  o.relres = relres;
  cl.sync();
  return o;
}

__global__ void __launch_bounds__(kBT, 2) k_batch(BatchArgs A) {
  cg::cluster_group cl = cg::this_cluster();
  const CeSm<double> s = ce_sm<double>(A.lay);
  BatchCtx* bx = reinterpret_cast<BatchCtx*>(s.ctx);
  const int Q = (int)cl.num_blocks();
  for (;;) {
    if (cl.block_rank() == 0 && threadIdx.x == 0) {
      const int k = atomicAdd(A.next, 1);
      for (int r = 0; r < Q; ++r) cl.map_shared_rank(&bx->inst, r)[0] = k;
    }
    cl.sync();
    const int k = bx->inst;
    if (k >= A.count) break;
    if (threadIdx.x == 0) {
      bx->I = A.inst[k];
      const BInst& I = bx->I;
      CeCtx<float>& c32 = bx->c32;
      c32.g = I.gr; c32.lay = A.lay; c32.spT = I.spT32; c32.spG = I.spG32;
      c32.V = I.v32; c32.kap = I.kap32; c32.hinv = I.hinv32; c32.a = 0.f;
      CeCtx<double>& c64 = bx->c64;
      c64.g = I.gr; c64.lay = A.lay; c64.spT = I.spT64; c64.spG = I.spG64;
      c64.V = I.v64; c64.kap = I.kap64; c64.hinv = I.hinv64; c64.a = 0.0;
    }
    __syncthreads();
    {
      const BInst& I = bx->I;
      ce_load_tables(A.lay, I.gr.T1, I.gr.LT, I.gr.lgLT, A.tw64, A.tw32, I.tstride);
    }
    bt_init(bx);
    cl.sync();
    long long its = 0, outer = 0;
    int nfp64 = 0, status = TSFDE_OK;
    double worst = 0.0;
    bool prev_fp64 = false;
    // Krylov method: fixed, or chosen per level by auto_rule_next (plan.h)
    // from CTA 0's level times
    AutoRule ka;
    auto_rule_init(ka);
    if (threadIdx.x == 0) bx->method = (A.krylov == TSFDE_KRYLOV_PCG) ? TSFDE_KRYLOV_PCG : TSFDE_KRYLOV_BICGSTAB;
    __syncthreads();
    for (int m = 1; m <= A.M; ++m) {
      unsigned long long t0 = 0;
      if (A.krylov == TSFDE_KRYLOV_AUTO && cl.block_rank() == 0 && threadIdx.x == 0)
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      const LevelOut o = bt_level(bx, A, m, prev_fp64);
      if (A.krylov == TSFDE_KRYLOV_AUTO) {
        // CTA 0 picks the next level's method and hands it to every CTA
        if (cl.block_rank() == 0 && threadIdx.x == 0) {
          unsigned long long t1;
          asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
          const int me = bx->method == TSFDE_KRYLOV_PCG ? 1 : 0;
          const double dt = o.status == TSFDE_OK ? (double)(t1 - t0) : INFINITY;
          const int next = auto_rule_next(ka, me, m, dt) ? TSFDE_KRYLOV_PCG : TSFDE_KRYLOV_BICGSTAB;
          for (int r = 0; r < Q; ++r) cl.map_shared_rank(&bx->method, r)[0] = next;
        }
        cl.sync();
      }
      prev_fp64 = o.fp64;
      its += o.iters;
      outer += o.outer;
      nfp64 += o.fp64 ? 1 : 0;
      worst = fmax(worst, o.relres);
      if (o.status != TSFDE_OK && status == TSFDE_OK) status = o.status;
    }
    bt_copy_out(bx, A.M);
    if (cl.block_rank() == 0 && threadIdx.x == 0) {
      StepStat* st = bx->I.stat;
      st->status = status;
      st->iterations = (int)its;
      st->outer = (int)outer;
      st->E_active = nfp64;
      st->rel_residual = worst;
    }
    cl.sync();
  }
}

// ------------------------------------------------------------- host side
static size_t g_batch_smem_limit = 0;

int batch_max_clusters(int Q, size_t smem) {
  if (smem > g_batch_smem_limit) {
    if (cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return 0;
    g_batch_smem_limit = smem;
  }
  if (Q > 8 && cudaFuncSetAttribute(k_batch, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(Q);
  cfg.blockDim = dim3(kBT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = Q;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, k_batch, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return ncl;
}

cudaError_t launch_batch(const BatchArgs& a, int Q, int clusters, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.next, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(Q * clusters);
  cfg.blockDim = dim3(kBT);
  cfg.dynamicSmemBytes = batch_smem_bytes(a.lay);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = Q;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch, a);
}

}  // namespace tsfde
