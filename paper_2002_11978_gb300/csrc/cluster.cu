// cluster.cu -- cluster engine of the mixed-precision FIDS level solve
// (sm_103a).
//
// One cooperative launch per time level.  The whole grid runs the FP64 parts
// of the mixed solve (the Strang preconditioner build of Sec. 4.1, the FP64
// residual products and the refinement updates; mixed_level in grid.cuh),
// and every FP32 inner PBiCGSTAB runs on the first thread-block cluster
// alone: Q <= 16 CTAs that hold the length-Nc complex FFT of each Toeplitz
// or circulant product in their shared memory and exchange the transposes
// through distributed shared memory.  An inner iteration then costs cluster
// barriers instead of grid barriers and touches global memory only for the
// Krylov vectors (L2-resident) and the spectra; the CTAs outside the first
// cluster wait at the grid barrier meanwhile.
//
// Per product: column pass (length-N1 FFTs of the CTA's own columns, twiddle
// W_Nc^{j2 k1}, push to the row owners), row pass (length-N2 FFTs of the
// CTA's row pairs, the spectral middle step of Sec. 4.1 in its stable form,
// inverse row FFTs, twiddle conj, push back to the column owners), inverse
// column pass (inverse FFTs, epilogue on the owned vector entries, optionally
// the forward column pass of the next product).  Each pass ends with one
// cluster barrier; cluster barriers are hardware barriers whose arrival set
// is every thread of the cluster, and every CTA takes the same branches
// (all decisions use cluster-reduced scalars that are bitwise equal in every
// CTA), so no wait can be left without its partners.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/tsfde.h"
#include "dev.cuh"
#include "grid.cuh"
#include "plan.h"

namespace cg = cooperative_groups;

namespace tsfde {

constexpr int kCT = 512;     // threads per CTA of the cluster engine
constexpr int kMaxQ = 16;    // largest cluster (non-portable size)

// cluster partial-sum slots (per CTA: [slot][16])
enum { CS_BB = 0, CS_RV = 1, CS_TS = 2, CS_TT = 3, CS_RR0 = 4, CS_RR = 5, kCSlots = 6 };
// grid slots that carry the inner solve's result to the whole grid
enum { SL_CIT = 10, SL_CST = 11 };

// Geometry of the cluster passes, held in registers by every pass.
struct CeLoc {
  int n, L, N1, N2, lgN1, lgN2;
  int Q, cQ, lgcQ, U, lgU, Bq, lgBq, nbuf, cap, T1, LT, lgLT;
  int q;  // this CTA's rank in the cluster
};

// What the inner solve reads, kept in shared memory behind the work buffers
// (each pass copies what it needs into registers on entry).
struct CeCtx {
  CeLoc loc;
  const float2* spT;  // Toeplitz spectrum, row-pass order
  const float2* spG;  // preconditioner spectrum, row-pass order
  KVecs<float> V;
  const float* kap;
  float a;            // ahat
};
static_assert(sizeof(CeCtx) <= 512, "CeCtx must fit its shared-memory slot");

// Shared-memory carve of the cluster phase.  Every pointer is formed from the
// extern __shared__ base inside the pass that uses it, so the compiler emits
// shared-memory instructions and keeps the addresses in registers.
struct CSm {
  float2* C;     // column-pass data (receives the row pass's pushes), cap
  float2* S;     // scratch and staging, cap
  float2* R;     // row-pass data (receives the column pass's pushes), nbuf
  float2* hi;    // W_{T1}^k, k < T1 (also the FFT stage table)
  float2* lo;    // W_L^l, l < LT
  double* part;  // [kCSlots][kMaxQ] partial sums pushed by every CTA
  double* red;   // 64 doubles of block-reduction scratch
  CeCtx* cx;
};

size_t cluster_smem_bytes(const DevPlan& P) {
  const CGeo& g = P.cl;
  return sizeof(float2) * (2 * (size_t)g.cap + g.nbuf + g.T1 + g.LT) +
         sizeof(double) * (kCSlots * kMaxQ + 64) + 512;
}

__device__ __forceinline__ CSm ce_ptrs(int cap, int nbuf, int T1, int LT) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CSm s;
  s.C = reinterpret_cast<float2*>(smem_raw);
  s.S = s.C + cap;
  s.R = s.S + cap;
  s.hi = s.R + nbuf;
  s.lo = s.hi + T1;
  s.part = reinterpret_cast<double*>(s.lo + LT);
  s.red = s.part + kCSlots * kMaxQ;
  s.cx = reinterpret_cast<CeCtx*>(s.red + 64);
  return s;
}
__device__ __forceinline__ CSm ce_ptrs(const CeLoc& l) { return ce_ptrs(l.cap, l.nbuf, l.T1, l.LT); }

// Entry of every pass: geometry into registers (then the pointers follow
// from the base with ce_ptrs).
__device__ __forceinline__ CeLoc ce_enter(const CeCtx* cx) {
  CeLoc l = cx->loc;
  l.q = (int)cg::this_cluster().block_rank();
  return l;
}

// W_L^m for 0 <= m < L, as hi * lo.
__device__ __forceinline__ float2 tw_hl(const float2* hi, const float2* lo, int lgLT, int LT, int m) {
  return cmul(hi[m >> lgLT], lo[m & (LT - 1)]);
}

// Row unit and slot parity of frequency row k1.
__device__ __forceinline__ void unit_of(int k1, int N1, int& u, int& b) {
  const int h = N1 >> 1;
  if (k1 == 0) { u = 0; b = 0; }
  else if (k1 == h) { u = 0; b = 1; }
  else if (k1 < h) { u = k1; b = 0; }
  else { u = N1 - k1; b = 1; }
}
// Frequency row held in row slot `slot` of CTA q.
__device__ __forceinline__ int k1_of(int lgU, int N1, int q, int slot) {
  const int u = (q << lgU) + (slot >> 1), b = slot & 1;
  if (u == 0) return b ? (N1 >> 1) : 0;
  return b ? N1 - u : u;
}

// epilogue / prologue modes of the column passes
enum { PRO_P = 0, PRO_S = 1 };                          // forward of p or s
enum { EPI_PH = 0, EPI_SH = 1, EPI_V = 2, EPI_T = 3 };  // inverse into ...

// Forward column pass: FFT over j1 of the CTA's columns (input through ld),
// twiddle W_Nc^{j2 k1}, staging in C as [row owner][column][row slot] (rows
// padded by one element against bank conflicts), push into the row owners' R.
template <class Ld>
__device__ __forceinline__ void ce_colfwd(const CeLoc& l, const CSm& s, Ld& ld, float2* first,
                                          float2* second) {
  cg::cluster_group cl = cg::this_cluster();
  const int q = l.q, N1 = l.N1, Lm = l.L - 1, ldS = l.Bq + 1;
  const int lgcQ = l.lgcQ, lgU = l.lgU, Um = l.U - 1, lgLT = l.lgLT, LT = l.LT;
  float2* const C = s.C;
  const float2* const hi = s.hi;
  const float2* const lo = s.lo;
  auto st = [=](int k1, int c, float2 z) {
    const int j2 = (q << lgcQ) + c;
    z = cmul(z, tw_hl(hi, lo, lgLT, LT, (2 * j2 * k1) & Lm));
    int u, b;
    unit_of(k1, N1, u, b);
    const int r = u >> lgU, slot = 2 * (u & Um) + b;
    C[((r << lgcQ) + c) * ldS + slot] = z;
  };
  fft_pipe<float, false>(l.lgN1, lgcQ, ld, st, first, second, hi, l.T1);
  const int Bm = l.Bq - 1, lgBq = l.lgBq, cm = l.cQ - 1;
  for (int t = threadIdx.x; t < l.nbuf; t += blockDim.x) {
    const int slot = t & Bm;
    const int c = (t >> lgBq) & cm;
    const int r = t >> (lgBq + lgcQ);
    float2* dst = cl.map_shared_rank(s.R, r);
    dst[(((q << lgcQ) + c) << lgBq) + slot] = C[((r << lgcQ) + c) * ldS + slot];
  }
}

// Row pass with the spectral product Y = S X ((sa, sb) pairs in row-pass
// order: the preconditioner's with precG, else the Toeplitz symbol's),
// pushed back into the column owners' C.
__device__ __noinline__ void ce_rows(const CeCtx* cxp, bool precG) {
  cg::cluster_group cl = cg::this_cluster();
  const CeLoc l = ce_enter(cxp);
  const CSm s = ce_ptrs(l);
  const int q = l.q, N1 = l.N1, N2 = l.N2, lgN2 = l.lgN2, Lm = l.L - 1;
  const int lgBq = l.lgBq, Bm = l.Bq - 1, lgU = l.lgU, lgcQ = l.lgcQ, cm = l.cQ - 1;
  const int lgLT = l.lgLT, LT = l.LT;
  const float2* __restrict__ sp = (precG ? cxp->spG : cxp->spT) + (size_t)q * l.nbuf;
  const float2* const hi = s.hi;
  const float2* const lo = s.lo;
  const int ns = pipe_stages(lgN2);
  float2* F = (ns & 1) ? s.S : s.R;   // forward result
  float2* Gm = (ns & 1) ? s.R : s.S;  // after the middle step
  {
    BufIn<float> ld{s.R, lgBq};
    BufOut<float> st{F, lgBq};
    fft_pipe<float, false>(lgN2, lgBq, ld, st, s.S, s.R, hi, l.T1);
  }
  // middle step, Y = S X on the real-input spectrum (see passB in grid.cuh)
  for (int e = threadIdx.x; e < l.nbuf; e += blockDim.x) {
    const int slot = e & Bm, k2 = e >> lgBq;
    const int k1 = k1_of(lgU, N1, q, slot);
    int ps, pk2;
    if (q == 0 && slot == 0) { ps = 0; pk2 = (N2 - k2) & (N2 - 1); }
    else if (q == 0 && slot == 1) { ps = 1; pk2 = N2 - 1 - k2; }
    else { ps = slot ^ 1; pk2 = N2 - 1 - k2; }
    const float2 sab = sp[e];
    const float2 Zk = F[e];
    const float2 Zq = F[(pk2 << lgBq) + ps];
    const float2 E = make_float2(0.5f * (Zk.x + Zq.x), 0.5f * (Zk.y - Zq.y));
    const float2 O = make_float2(0.5f * (Zk.y + Zq.y), -0.5f * (Zk.x - Zq.x));
    const float2 Wk = tw_hl(hi, lo, lgLT, LT, k1 + N1 * k2);
    const float2 WO = cmul(Wk, O);
    const float2 X = cadd(E, WO);
    const float2 Xc = csub(E, WO);
    const float2 Ya = cscale(X, sab.x);
    const float2 Yb = cscale(Xc, sab.y);
    const float2 Ep = cscale(cadd(Ya, Yb), 0.5f);
    const float2 Op = cscale(cmulc(csub(Ya, Yb), Wk), 0.5f);
    Gm[e] = make_float2(Ep.x - Op.y, Ep.y + Op.x);
  }
  __syncthreads();
  const int ldS = l.cQ + 1;
  float2* const Sst = s.S;
  {
    BufIn<float> ld{Gm, lgBq};
    auto st = [=](int j2, int slot, float2 z) {
      const int k1 = k1_of(lgU, N1, q, slot);
      z = cmulc(z, tw_hl(hi, lo, lgLT, LT, (2 * j2 * k1) & Lm));
      Sst[(((j2 >> lgcQ) << lgBq) + slot) * ldS + (j2 & cm)] = z;
    };
    float2* first = (Gm == s.R) ? s.S : s.R;
    fft_pipe<float, true>(lgN2, lgBq, ld, st, first, Gm, hi, l.T1);
  }
  for (int t = threadIdx.x; t < l.nbuf; t += blockDim.x) {
    const int c = t & cm;
    const int slot = (t >> lgcQ) & Bm;
    const int r = t >> (lgcQ + lgBq);
    float2* dst = cl.map_shared_rank(s.C, r);
    dst[(k1_of(lgU, N1, q, slot) << lgcQ) + c] = Sst[((r << lgBq) + slot) * ldS + c];
  }
}

// Owned entry pairs: pair pp = (j1 << lgcQ) + c (j1 < N1/2, c < cQ) holds
// the vector entries i0 = 2 (N2 j1 + q cQ + c) and i0 + 1 -- the real and
// imaginary parts of packed element (j1, c) of the CTA's columns.  The FP32
// vectors are allocated with an even length, so a pair is one aligned float2.
__device__ __forceinline__ int pair_i0(const CeLoc& l, int pp) {
  return 2 * (((pp >> l.lgcQ) << l.lgN2) + (l.q << l.lgcQ) + (pp & (l.cQ - 1)));
}
__device__ __forceinline__ float2 ld2(const float* v, int i0) {
  return reinterpret_cast<const float2*>(v)[i0 >> 1];
}
// store the entries of a pair that lie below n
__device__ __forceinline__ void st2(float* v, int i0, int n, float2 x) {
  if (i0 + 1 < n) reinterpret_cast<float2*>(v)[i0 >> 1] = x;
  else if (i0 < n) v[i0] = x.x;
}

constexpr int kVB = 4;  // pairs per thread whose loads are issued together
constexpr int kXR = 2;  // the same for the six-vector update of x and r

// Inverse column pass: y_{2j}, y_{2j+1} = Re, Im of the inverse FFT for the
// CTA's columns, written into the pair buffer Bn (zero at entries >= n) by
// the last FFT stage and then consumed per mode:
//   EPI_PH / EPI_SH: ph = y (sh = y), then the forward column pass of that
//     vector straight from Bn (the next product's input);
//   EPI_V: v = a ph + kappa y, acc.x = (rh, v);  EPI_T: t = a sh + kappa y,
//     acc.x = (t, s), acc.y = (t, t).
// xin is the vector the operator was applied to (ph or p; sh or s).
__device__ __noinline__ float2 ce_colinv(const CeCtx* cxp, int mode, const float* __restrict__ xin) {
  const CeLoc l = ce_enter(cxp);
  const CSm s = ce_ptrs(l);
  const int q = l.q, N1 = l.N1, lgN2 = l.lgN2, n = l.n, lgcQ = l.lgcQ;
  const bool fused = (mode == EPI_PH || mode == EPI_SH);
  const int ns = pipe_stages(l.lgN1);
  float2* const Bn = (ns & 1) ? s.S : s.C;
  {
    auto st = [=](int j1, int c, float2 z) {
      if (j1 < (N1 >> 1)) {
        const int i0 = 2 * ((j1 << lgN2) + (q << lgcQ) + c);
        Bn[(j1 << lgcQ) + c] = make_float2(i0 < n ? z.x : 0.f, i0 + 1 < n ? z.y : 0.f);
      }
    };
    BufIn<float> ld{s.C, lgcQ};
    fft_pipe<float, true>(l.lgN1, lgcQ, ld, st, s.S, s.C, s.hi, l.T1);
  }
  const int npair = (N1 >> 1) << lgcQ;
  float acc0 = 0.f, acc1 = 0.f;
  if (fused) {
    float* dst = (mode == EPI_PH) ? cxp->V.ph : cxp->V.sh;
    for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) st2(dst, pair_i0(l, pp), n, Bn[pp]);
    auto ldb = [=](int j1, int c) -> float2 {
      return (j1 < (N1 >> 1)) ? Bn[(j1 << lgcQ) + c] : make_float2(0.f, 0.f);
    };
    float2* other = (Bn == s.C) ? s.S : s.C;
    ce_colfwd(l, s, ldb, other, Bn);
  } else {
    float* const dst = (mode == EPI_V) ? cxp->V.v : cxp->V.t;
    const float* const dotv = (mode == EPI_V) ? cxp->V.rh : cxp->V.s;
    const float* const kap = cxp->kap;
    const float a = cxp->a;
    for (int p0 = threadIdx.x; p0 < npair; p0 += kVB * blockDim.x) {
      float2 xv[kVB], kv[kVB], dv[kVB];
#pragma unroll
      for (int u = 0; u < kVB; ++u) {
        const int pp = p0 + u * blockDim.x;
        if (pp < npair) {
          const int i0 = pair_i0(l, pp);
          xv[u] = ld2(xin, i0);
          kv[u] = ld2(kap, i0);
          dv[u] = ld2(dotv, i0);
        }
      }
#pragma unroll
      for (int u = 0; u < kVB; ++u) {
        const int pp = p0 + u * blockDim.x;
        if (pp < npair) {
          const int i0 = pair_i0(l, pp);
          const float2 y = Bn[pp];
          float2 w = make_float2(a * xv[u].x + kv[u].x * y.x, a * xv[u].y + kv[u].y * y.y);
          if (i0 + 1 >= n) w.y = 0.f;
          if (i0 >= n) w.x = 0.f;
          st2(dst, i0, n, w);
          acc0 += dv[u].x * w.x + dv[u].y * w.y;
          acc1 += w.x * w.x + w.y * w.y;
        }
      }
    }
  }
  return make_float2(acc0, acc1);
}

// Forward column pass of p = r + beta (p - omega v) (PRO_P) or of
// s = r - alpha v (PRO_S), storing the new vector.  The new entries are
// formed in a pair buffer first (loads issued together), then transformed.
__device__ __noinline__ void ce_colfwd_vec(const CeCtx* cxp, int mode, float c0, float c1) {
  const CeLoc l = ce_enter(cxp);
  const CSm s = ce_ptrs(l);
  const int N1 = l.N1, n = l.n, lgcQ = l.lgcQ;
  const float* const r_ = cxp->V.r;
  const float* const v_ = cxp->V.v;
  float* const dst = (mode == PRO_P) ? cxp->V.p : cxp->V.s;
  const int ns = pipe_stages(l.lgN1);
  float2* first = ((ns - 1) & 1) ? s.S : s.C;
  float2* second = ((ns - 1) & 1) ? s.C : s.S;
  float2* const X = (first == s.C) ? s.S : s.C;
  const int npair = (N1 >> 1) << lgcQ;
  for (int p0 = threadIdx.x; p0 < npair; p0 += kVB * blockDim.x) {
    float2 rv[kVB], pv[kVB], vv[kVB];
#pragma unroll
    for (int u = 0; u < kVB; ++u) {
      const int pp = p0 + u * blockDim.x;
      if (pp < npair) {
        const int i0 = pair_i0(l, pp);
        rv[u] = ld2(r_, i0);
        vv[u] = ld2(v_, i0);
        pv[u] = (mode == PRO_P) ? ld2(dst, i0) : make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < kVB; ++u) {
      const int pp = p0 + u * blockDim.x;
      if (pp < npair) {
        const int i0 = pair_i0(l, pp);
        float2 x;
        if (mode == PRO_P) {
          x.x = rv[u].x + c0 * (pv[u].x - c1 * vv[u].x);
          x.y = rv[u].y + c0 * (pv[u].y - c1 * vv[u].y);
        } else {
          x.x = rv[u].x - c0 * vv[u].x;
          x.y = rv[u].y - c0 * vv[u].y;
        }
        if (i0 + 1 >= n) x.y = 0.f;
        if (i0 >= n) x.x = 0.f;
        st2(dst, i0, n, x);
        X[pp] = x;
      }
    }
  }
  __syncthreads();
  auto ld = [=](int j1, int c) -> float2 {
    return (j1 < (N1 >> 1)) ? X[(j1 << lgcQ) + c] : make_float2(0.f, 0.f);
  };
  ce_colfwd(l, s, ld, first, second);
}

// Push the block-reduced value v (valid in every thread) into slot `slot` of
// every CTA of the cluster; read back with ce_total after a cluster barrier.
__device__ __forceinline__ void ce_put(const CSm& s, int Q, int slot, double v) {
  cg::cluster_group cl = cg::this_cluster();
  if ((int)threadIdx.x < Q) {
    double* dst = cl.map_shared_rank(s.part, (int)threadIdx.x);
    dst[slot * kMaxQ + (int)cl.block_rank()] = v;
  }
}
__device__ __forceinline__ double ce_total(const CSm& s, int Q, int slot) {
  double t = 0.0;
  for (int r = 0; r < Q; ++r) t += s.part[slot * kMaxQ + r];
  return t;
}

// FP32 right-preconditioned BiCGSTAB (van der Vorst) for
// (ahat I + K A) x = b with b_i = (float)(sc r64_i), x0 = 0, on the cluster;
// the same recurrences and stopping rule as bicgstab in grid.cuh.  Must be
// called by every CTA of the cluster.
__device__ __noinline__ SolveRes ce_bicgstab(const CeCtx* cxp, bool prec, double tol, int max_it,
                                             const double* __restrict__ r64, double sc) {
  cg::cluster_group cl = cg::this_cluster();
  const CeLoc l = ce_enter(cxp);
  const CSm s = ce_ptrs(l);
  const int Q = l.Q, n = l.n;
  const int npair = (l.N1 >> 1) << l.lgcQ;
  SolveRes out{TSFDE_OK, 0, 0.0};
  {
    const KVecs<float> V = cxp->V;
    float acc = 0.f;
    for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) {
      const int i0 = pair_i0(l, pp);
      float2 b2 = make_float2(0.f, 0.f);
      if (i0 + 1 < n) {
        const double2 r2 = reinterpret_cast<const double2*>(r64)[i0 >> 1];
        b2 = make_float2((float)(r2.x * sc), (float)(r2.y * sc));
      } else if (i0 < n) {
        b2.x = (float)(r64[i0] * sc);
      }
      const float2 z = make_float2(0.f, 0.f);
      st2(V.x, i0, n, z); st2(V.r, i0, n, b2); st2(V.rh, i0, n, b2);
      st2(V.p, i0, n, z); st2(V.v, i0, n, z);
      acc += b2.x * b2.x + b2.y * b2.y;
    }
    ce_put(s, Q, CS_BB, block_sum((double)acc, s.red));
  }
  cl.sync();
  const double bb = ce_total(s, Q, CS_BB);
  if (!isfinite(bb)) { out.status = TSFDE_ENONFINITE; return out; }
  if (bb == 0.0) return out;
  const double nb = sqrt(bb);
  double rho = 1.0, alpha = 1.0, omega = 1.0, rho_new = bb, rr = bb;
  int it = 0;
  for (;;) {
    const double relres = sqrt(rr) / nb;
    out.relres = relres;
    out.iters = it;
    if (!isfinite(relres) || !isfinite(rho_new)) { out.status = TSFDE_ENONFINITE; return out; }
    if (relres < tol) return out;
    if (it >= max_it) { out.status = TSFDE_ENOCONV; return out; }
    if (rho_new == 0.0 || omega == 0.0) { out.status = TSFDE_EBREAKDOWN; return out; }
    const double beta = (rho_new / rho) * (alpha / omega);
    rho = rho_new;
    ++it;
    // p = r + beta (p - omega v); v = M P^{-1} p
    ce_colfwd_vec(cxp, PRO_P, (float)beta, (float)omega);
    cl.sync();
    if (prec) {
      ce_rows(cxp, true);
      cl.sync();
      ce_colinv(cxp, EPI_PH, nullptr);
      cl.sync();
    }
    ce_rows(cxp, false);
    cl.sync();
    {
      const float2 acc = ce_colinv(cxp, EPI_V, prec ? cxp->V.ph : cxp->V.p);
      ce_put(s, Q, CS_RV, block_sum((double)acc.x, s.red));
    }
    cl.sync();
    const double rv = ce_total(s, Q, CS_RV);
    if (!isfinite(rv)) { out.status = TSFDE_ENONFINITE; return out; }
    if (rv == 0.0) { out.status = TSFDE_EBREAKDOWN; return out; }
    alpha = rho / rv;
    // s = r - alpha v; t = M P^{-1} s
    ce_colfwd_vec(cxp, PRO_S, (float)alpha, 0.f);
    cl.sync();
    if (prec) {
      ce_rows(cxp, true);
      cl.sync();
      ce_colinv(cxp, EPI_SH, nullptr);
      cl.sync();
    }
    ce_rows(cxp, false);
    cl.sync();
    {
      const float2 acc = ce_colinv(cxp, EPI_T, prec ? cxp->V.sh : cxp->V.s);
      const double ts_b = block_sum((double)acc.x, s.red);
      const double tt_b = block_sum((double)acc.y, s.red);
      ce_put(s, Q, CS_TS, ts_b);
      ce_put(s, Q, CS_TT, tt_b);
    }
    cl.sync();
    const double ts = ce_total(s, Q, CS_TS), tt = ce_total(s, Q, CS_TT);
    omega = (tt > 0.0) ? ts / tt : 0.0;
    if (!isfinite(omega)) { out.status = TSFDE_ENONFINITE; return out; }
    // x += alpha p^ + omega s^, r = s - omega t
    {
      const KVecs<float> V = cxp->V;
      const float* const ph = prec ? V.ph : V.p;
      const float* const sh = prec ? V.sh : V.s;
      const float aR = (float)alpha, oR = (float)omega;
      float arr = 0.f, ar2 = 0.f;
      for (int p0 = threadIdx.x; p0 < npair; p0 += kXR * blockDim.x) {
        float2 xv[kXR], pv[kXR], sv[kXR], ss[kXR], tv[kXR], hv[kXR];
#pragma unroll
        for (int u = 0; u < kXR; ++u) {
          const int pp = p0 + u * blockDim.x;
          if (pp < npair) {
            const int i0 = pair_i0(l, pp);
            xv[u] = ld2(V.x, i0); pv[u] = ld2(ph, i0); sv[u] = ld2(sh, i0);
            ss[u] = ld2(V.s, i0); tv[u] = ld2(V.t, i0); hv[u] = ld2(V.rh, i0);
          }
        }
#pragma unroll
        for (int u = 0; u < kXR; ++u) {
          const int pp = p0 + u * blockDim.x;
          if (pp < npair) {
            const int i0 = pair_i0(l, pp);
            const float2 x = make_float2(xv[u].x + aR * pv[u].x + oR * sv[u].x,
                                         xv[u].y + aR * pv[u].y + oR * sv[u].y);
            float2 r = make_float2(ss[u].x - oR * tv[u].x, ss[u].y - oR * tv[u].y);
            if (i0 + 1 >= n) r.y = 0.f;
            if (i0 >= n) r.x = 0.f;
            st2(V.x, i0, n, x);
            st2(V.r, i0, n, r);
            arr += hv[u].x * r.x + hv[u].y * r.y;
            ar2 += r.x * r.x + r.y * r.y;
          }
        }
      }
      const double rr0_b = block_sum((double)arr, s.red);
      const double rr_b = block_sum((double)ar2, s.red);
      ce_put(s, Q, CS_RR0, rr0_b);
      ce_put(s, Q, CS_RR, rr_b);
    }
    cl.sync();
    rho_new = ce_total(s, Q, CS_RR0);
    rr = ce_total(s, Q, CS_RR);
  }
}

// Mixed level solve, cluster engine.  Same refinement loop as the grid
// engine's k_level_mixed; only the FP32 inner solves move to cluster 0.
__global__ void __launch_bounds__(kCT, 1) k_level_cluster(LevelArgs A) {
  if (A.probe) return;
  const DevPlan& P = A.P;
  const CGeo& g = P.cl;
  SmemAll S = smem_setup(P);
  const int N1 = P.gr.N1, N2 = P.gr.N2, lgN2 = P.gr.lgN2;
  auto conv = [&](int k) {
    const int k1 = k >> lgN2, k2 = k & (N2 - 1);
    int u, b;
    unit_of(k1, N1, u, b);
    const int r = u >> g.lgU, slot = 2 * (u & (g.U - 1)) + b;
    P.spG_cl[(size_t)r * g.nbuf + (k2 << g.lgBq) + slot] =
        make_float2((float)P.saG64[k], (float)P.sbG64[k]);
  };
  auto inner = [&](double sc, SolveRes& ir) -> bool {
    double its = 0.0, stv = 0.0;
    if ((int)blockIdx.x < g.Q) {
      const CSm cs = ce_ptrs(g.cap, g.nbuf, g.T1, g.LT);
      for (int k = threadIdx.x; k < g.T1; k += blockDim.x) cs.hi[k] = P.twL32[k << g.lgLT];
      for (int k = threadIdx.x; k < g.LT; k += blockDim.x) cs.lo[k] = P.twL32[k];
      if (threadIdx.x == 0) {
        CeLoc& l = cs.cx->loc;
        l.n = P.n; l.L = P.L; l.N1 = N1; l.N2 = N2; l.lgN1 = P.gr.lgN1; l.lgN2 = lgN2;
        l.Q = g.Q; l.cQ = g.cQ; l.lgcQ = g.lgcQ; l.U = g.U; l.lgU = g.lgU; l.Bq = g.Bq;
        l.lgBq = g.lgBq; l.nbuf = g.nbuf; l.cap = g.cap; l.T1 = g.T1; l.LT = g.LT; l.lgLT = g.lgLT;
        l.q = 0;
        cs.cx->spT = P.spT_cl; cs.cx->spG = P.spG_cl;
        cs.cx->V = A.k32; cs.cx->kap = A.kappa32; cs.cx->a = (float)A.ahat;
      }
      __syncthreads();
      const SolveRes r = ce_bicgstab(cs.cx, A.precond != 0, A.inner_tol, A.inner_max_it, A.r64, sc);
      if (blockIdx.x == 0) { its = (double)r.iters; stv = (double)r.status; }
    }
    put_partial(P, SL_CIT, its);
    put_partial(P, SL_CST, stv);
    double o_its, o_st;
    const bool ok = gsync_sum2(P, S.d.red, SL_CIT, SL_CST, 0u, o_its, o_st);
    S = smem_setup(P);  // the cluster passes overwrote the grid tables
    ir.iters = (int)o_its;
    ir.status = (int)o_st;
    return ok;
  };
  mixed_level(A, S, conv, inner);
}

// ------------------------------------------------------------- host side
bool cluster_geometry(DevPlan& P) {
  CGeo& g = P.cl;
  g = CGeo{};
  const int N1 = P.gr.N1, N2 = P.gr.N2;
  if (N1 < N2 || N1 < 2 || N2 < 1) return false;
  int Q = kMaxQ;
  while (Q > 1 && (2 * Q > N1 || Q > N2)) Q >>= 1;
  auto lg = [](int x) { int l = 0; while ((1 << l) < x) ++l; return l; };
  g.Q = Q; g.lgQ = lg(Q);
  g.cQ = N2 / Q; g.lgcQ = lg(g.cQ);
  g.U = N1 / (2 * Q); g.lgU = lg(g.U);
  g.Bq = 2 * g.U; g.lgBq = lg(g.Bq);
  g.nbuf = P.Nc / Q;
  g.cap = g.nbuf + N1;
  g.T1 = N1;
  g.LT = P.L / N1; g.lgLT = lg(g.LT);
  g.G = Q;
  return g.cQ >= 1 && g.U >= 1 && g.cQ * Q == N2 && g.U * 2 * Q == N1;
}

static cudaLaunchConfig_t cluster_config(const DevPlan& P, size_t smem, int grid, cudaStream_t s,
                                         cudaLaunchAttribute* at, bool coop) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = P.cl.Q;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeCooperative;
  at[1].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = coop ? 2 : 1;
  return cfg;
}

// The dynamic shared-memory limit only ever grows, so a context set up earlier
// with a larger plan can still launch.
static size_t g_cl_smem_limit = 0;

int cluster_max_grid(const DevPlan& P, size_t smem) {
  if (smem > g_cl_smem_limit) {
    if (cudaFuncSetAttribute(k_level_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return 0;
    g_cl_smem_limit = smem;
  }
  if (P.cl.Q > 8 &&
      cudaFuncSetAttribute(k_level_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return 0;
  cudaLaunchAttribute at[2];
  cudaLaunchConfig_t cfg = cluster_config(P, smem, P.cl.Q, 0, at, false);
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, k_level_cluster, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return ncl * P.cl.Q;
}

cudaError_t launch_level_cluster(const LevelArgs& a, cudaStream_t s) {
  const size_t smem = std::max(plan_smem_bytes(a.P), cluster_smem_bytes(a.P));
  if (!a.probe) {
    cudaError_t e = cudaMemsetAsync(a.P.bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchAttribute at[2];
  cudaLaunchConfig_t cfg = cluster_config(a.P, smem, a.P.cl.G, s, at, true);
  return cudaLaunchKernelEx(&cfg, k_level_cluster, a);
}

}  // namespace tsfde
