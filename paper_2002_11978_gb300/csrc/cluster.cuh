// cluster.cuh -- zero-padded FFT products of Sec. 4.1 on one thread-block
// cluster, with the transform held in the CTAs' shared memory and the
// transposes exchanged through distributed shared memory (sm_90+ clusters).
//
// A length-Nfft complex transform, Nfft = N1 N2 (N1 >= N2, powers of two), is
// split over the Q CTAs of a cluster.  CTA q owns the columns j2 in
// [q cQ, (q+1) cQ) (cQ = N2/Q) for the column passes, and the row units
// [q U, (q+1) U) (U = N1/(2Q)) for the row pass: unit 0 = rows {0, N1/2},
// unit u > 0 = rows {u, N1-u}, held in row slots 2(u - qU) and 2(u - qU)+1,
// so the partner k' = Nfft - k of every frequency k of the real-input
// unpacking lies in the same CTA.  Per product:
//   column pass   FFTs over j1 of the CTA's columns, twiddle W_Nfft^{j2 k1},
//                 staging [row owner][column][slot], push to the row owners;
//   row pass      FFTs over j2, the middle step, inverse FFTs, conjugate
//                 twiddle, staging [column owner][slot][column], push back;
//   inverse col   inverse FFTs over k1, epilogue.
// Each pass ends with one cluster barrier, placed by the caller.  Two uses:
// the real-input products (Nfft = Nc = L/2, packed z_j = x_2j + i x_2j+1,
// column-twiddle stride 2 on the W_L tables) and the complex Bluestein
// transform of the preconditioner build (Nfft = L, stride 1).
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "../../include/tsfde.h"
#include "dev.cuh"
#include "plan.h"

namespace tsfde {

namespace cg = cooperative_groups;

constexpr int kMaxQ = 16;  // largest cluster (non-portable size)

constexpr int kCeSlots = 13;  // cluster partial-sum slots (ce_bicgstab: 0..5)

__host__ __device__ inline size_t ce_tables_bytes(const CeLay& y) {
  return (size_t)(y.T1 + y.LT) * (sizeof(float2) + (y.has64 ? sizeof(double2) : 0));
}
__host__ __device__ inline size_t ce_ctx_offset(const CeLay& y) {
  return 2 * (size_t)y.capB + y.nbufB + ce_tables_bytes(y) + sizeof(double) * (kCeSlots * kMaxQ + 64);
}

template <typename R> struct CeSm {
  cplx<R>* C;
  cplx<R>* S;
  cplx<R>* R_;
  const cplx<R>* hi;
  const cplx<R>* lo;
  double* part;
  double* red;
  unsigned char* ctx;
};

// Pointers of the layout, formed from the extern __shared__ base inside the
// caller so that the compiler knows they address shared memory.
template <typename R> __device__ __forceinline__ CeSm<R> ce_sm(const CeLay& y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CeSm<R> s;
  s.C = reinterpret_cast<cplx<R>*>(smem_raw);
  s.S = reinterpret_cast<cplx<R>*>(smem_raw + y.capB);
  s.R_ = reinterpret_cast<cplx<R>*>(smem_raw + 2 * (size_t)y.capB);
  unsigned char* t = smem_raw + 2 * (size_t)y.capB + y.nbufB;
  unsigned char* t32 = t + (y.has64 ? (size_t)(y.T1 + y.LT) * sizeof(double2) : 0);
  if constexpr (sizeof(R) == 8) {
    s.hi = reinterpret_cast<const cplx<R>*>(t);
  } else {
    s.hi = reinterpret_cast<const cplx<R>*>(t32);
  }
  s.lo = s.hi + y.T1;
  s.part = reinterpret_cast<double*>(t + ce_tables_bytes(y));
  s.red = s.part + kCeSlots * kMaxQ;
  s.ctx = smem_raw + ce_ctx_offset(y);
  return s;
}

// Fill the twiddle tables hi = W_{T1}^k (k < T1) and lo = W_L^l (l < LT) from
// global W_Lg tables with Lg = L * stride (all threads; ends with
// __syncthreads).  T1, LT may be below the layout's capacities.
__device__ __forceinline__ void ce_load_tables(const CeLay& y, int T1, int LT, int lgLT,
                                               const double2* twL64, const float2* twL32,
                                               int stride = 1) {
  CeSm<float> s32 = ce_sm<float>(y);
  float2* hi32 = const_cast<float2*>(s32.hi);
  float2* lo32 = const_cast<float2*>(s32.lo);
  for (int k = threadIdx.x; k < T1; k += blockDim.x) hi32[k] = twL32[(size_t)(k << lgLT) * stride];
  for (int k = threadIdx.x; k < LT; k += blockDim.x) lo32[k] = twL32[(size_t)k * stride];
  if (y.has64) {
    CeSm<double> s64 = ce_sm<double>(y);
    double2* hi64 = const_cast<double2*>(s64.hi);
    double2* lo64 = const_cast<double2*>(s64.lo);
    for (int k = threadIdx.x; k < T1; k += blockDim.x) hi64[k] = twL64[(size_t)(k << lgLT) * stride];
    for (int k = threadIdx.x; k < LT; k += blockDim.x) lo64[k] = twL64[(size_t)k * stride];
  }
  __syncthreads();
}

// W_L^m for 0 <= m < L, as hi * lo.
template <typename Z>
__device__ __forceinline__ Z ce_tw(const Z* hi, const Z* lo, int lgLT, int LT, int m) {
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

// Forward column pass: FFT over j1 of the CTA's columns (input ld(j1, c)),
// twiddle W_Nfft^{j2 k1}, staging in C as [row owner][column][row slot] (rows
// padded by one element against bank conflicts), push into the row owners'
// R.  ld must not read `first`; st writes C, so the buffer the last stage
// reads must not be C (see fft_pipe).
template <typename R, class Ld>
__device__ __forceinline__ void ce_colfwd(const CeGeo& g, const CeSm<R>& s, Ld& ld, cplx<R>* first,
                                          cplx<R>* second) {
  typedef cplx<R> Z;
  cg::cluster_group cl = cg::this_cluster();
  const int q = g.q, N1 = g.N1, Lm = g.L - 1, ldS = g.Bq + 1, tws = g.tws;
  const int lgcQ = g.lgcQ, lgU = g.lgU, Um = g.U - 1, lgLT = g.lgLT, LT = g.LT;
  Z* const C = s.C;
  const Z* const hi = s.hi;
  const Z* const lo = s.lo;
  auto st = [=](int k1, int c, Z z) {
    const int j2 = (q << lgcQ) + c;
    z = cmul(z, ce_tw(hi, lo, lgLT, LT, (tws * j2 * k1) & Lm));
    int u, b;
    unit_of(k1, N1, u, b);
    const int r = u >> lgU, slot = 2 * (u & Um) + b;
    C[((r << lgcQ) + c) * ldS + slot] = z;
  };
  fft_pipe<R, false>(g.lgN1, lgcQ, ld, st, first, second, hi, g.T1);
  const int Bm = g.Bq - 1, lgBq = g.lgBq, cm = g.cQ - 1;
  for (int t = threadIdx.x; t < g.nbuf; t += blockDim.x) {
    const int slot = t & Bm;
    const int c = (t >> lgBq) & cm;
    const int r = t >> (lgBq + lgcQ);
    Z* dst = cl.map_shared_rank(s.R_, r);
    dst[(((q << lgcQ) + c) << lgBq) + slot] = C[((r << lgcQ) + c) * ldS + slot];
  }
}

enum { CE_APPLY = 0, CE_SPEC = 1, CE_CONV = 2 };

// Row pass.  sp holds per-element coefficients in row-pass order (entry
// q nbuf + (k2 << lgBq) + slot):
//   CE_APPLY  (sa, sb) = (S_k, S_k') / Nfft of a real even spectrum S; the
//             real-input product Y = S X, stable form (see passB, grid.cuh);
//   CE_CONV   a complex multiplier c_k: Z'_k = c_k Z_k (complex transforms);
//   CE_SPEC   forward only: writes (Re X_k, Re conj X_k') / Nfft of the
//             real input into out64 (and out32 if non-NULL), no push.
// Otherwise the result goes through the inverse row FFTs back to the column
// owners' C.
template <typename R, int MID>
__device__ __forceinline__ void ce_rows(const CeGeo& g, const CeSm<R>& s, const cplx<R>* __restrict__ sp,
                                        double2* out64, float2* out32) {
  typedef cplx<R> Z;
  cg::cluster_group cl = cg::this_cluster();
  const int q = g.q, N1 = g.N1, N2 = g.N2, lgN2 = g.lgN2, Lm = g.L - 1, tws = g.tws;
  const int lgBq = g.lgBq, Bm = g.Bq - 1, lgU = g.lgU, lgcQ = g.lgcQ, cm = g.cQ - 1;
  const int lgLT = g.lgLT, LT = g.LT;
  const Z* const hi = s.hi;
  const Z* const lo = s.lo;
  const int ns = pipe_stages(lgN2);
  Z* F = (ns & 1) ? s.S : s.R_;   // forward result
  Z* Gm = (ns & 1) ? s.R_ : s.S;  // after the middle step
  {
    BufIn<R> ld{s.R_, lgBq};
    BufOut<R> st{F, lgBq};
    fft_pipe<R, false>(lgN2, lgBq, ld, st, s.S, s.R_, hi, g.T1);
  }
  const size_t base = (size_t)q * g.nbuf;
  const R invN = R(1) / R(N1 * N2);
  for (int e = threadIdx.x; e < g.nbuf; e += blockDim.x) {
    const Z Zk = F[e];
    if constexpr (MID == CE_CONV) {
      Gm[e] = cmul(Zk, sp[base + e]);
    } else {
      const int slot = e & Bm, k2 = e >> lgBq;
      const int k1 = k1_of(lgU, N1, q, slot);
      int ps, pk2;
      if (q == 0 && slot == 0) { ps = 0; pk2 = (N2 - k2) & (N2 - 1); }
      else if (q == 0 && slot == 1) { ps = 1; pk2 = N2 - 1 - k2; }
      else { ps = slot ^ 1; pk2 = N2 - 1 - k2; }
      const Z Zq = F[(pk2 << lgBq) + ps];
      const Z E = mkc<R>(R(0.5) * (Zk.x + Zq.x), R(0.5) * (Zk.y - Zq.y));
      const Z O = mkc<R>(R(0.5) * (Zk.y + Zq.y), R(-0.5) * (Zk.x - Zq.x));
      // W_L^k of the real transform of length L = 2 Nfft
      const Z Wk = ce_tw(hi, lo, lgLT, LT, k1 + N1 * k2);
      const Z WO = cmul(Wk, O);
      const Z X = cadd(E, WO);
      const Z Xc = csub(E, WO);
      if constexpr (MID == CE_SPEC) {
        out64[base + e] = make_double2((double)X.x * (double)invN, (double)Xc.x * (double)invN);
        if (out32) out32[base + e] = make_float2((float)(X.x * invN), (float)(Xc.x * invN));
      } else {
        const Z sab = sp[base + e];
        const Z Ya = cscale(X, sab.x);
        const Z Yb = cscale(Xc, sab.y);
        const Z Ep = cscale(cadd(Ya, Yb), R(0.5));
        const Z Op = cscale(cmulc(csub(Ya, Yb), Wk), R(0.5));
        Gm[e] = mkc<R>(Ep.x - Op.y, Ep.y + Op.x);
      }
    }
  }
  if constexpr (MID == CE_SPEC) return;
  __syncthreads();
  const int ldS = g.cQ + 1;
  Z* const Sst = s.S;
  {
    BufIn<R> ld{Gm, lgBq};
    auto st = [=](int j2, int slot, Z z) {
      const int k1 = k1_of(lgU, N1, q, slot);
      z = cmulc(z, ce_tw(hi, lo, lgLT, LT, (tws * j2 * k1) & Lm));
      Sst[(((j2 >> lgcQ) << lgBq) + slot) * ldS + (j2 & cm)] = z;
    };
    Z* first = (Gm == s.R_) ? s.S : s.R_;
    fft_pipe<R, true>(lgN2, lgBq, ld, st, first, Gm, hi, g.T1);
  }
  for (int t = threadIdx.x; t < g.nbuf; t += blockDim.x) {
    const int c = t & cm;
    const int slot = (t >> lgcQ) & Bm;
    const int r = t >> (lgcQ + lgBq);
    Z* dst = cl.map_shared_rank(s.C, r);
    dst[(k1_of(lgU, N1, q, slot) << lgcQ) + c] = Sst[((r << lgBq) + slot) * ldS + c];
  }
}

// The one buffer (S when the column FFT has an odd number of stages, else C)
// that both the inverse column pass may write (it is not what its last stage
// reads) and the forward column pass may read its input from (it is neither
// the first intermediate nor what the last stage reads, and the last stage
// stages into C).  An inverse pass can therefore leave the next product's
// input there.
template <typename R> __device__ __forceinline__ cplx<R>* ce_io(const CeGeo& g, const CeSm<R>& s) {
  return (pipe_stages(g.lgN1) & 1) ? s.S : s.C;
}

// Inverse column pass over the received C: st(j1, c, z) gets element
// (j1, c) of the CTA's columns and may write ce_io(g, s).
template <typename R, class St>
__device__ __forceinline__ void ce_colinv(const CeGeo& g, const CeSm<R>& s, St& st) {
  BufIn<R> ld{s.C, g.lgcQ};
  fft_pipe<R, true>(g.lgN1, g.lgcQ, ld, st, s.S, s.C, s.hi, g.T1);
}

// Forward column pass of data laid out in X = ce_io(g, s) as
// X[(j1 << lgcQ) + c] for j1 < rows (zero beyond): rows = N1/2 for the
// products (input of length <= Nfft), N1 for a full-length real input.
template <typename R>
__device__ __forceinline__ void ce_colfwd_buf(const CeGeo& g, const CeSm<R>& s, int rows) {
  typedef cplx<R> Z;
  const int lgcQ = g.lgcQ;
  Z* const X = ce_io(g, s);
  auto ld = [=](int j1, int c) -> Z { return (j1 < rows) ? X[(j1 << lgcQ) + c] : mkc<R>(R(0), R(0)); };
  Z* const other = (X == s.C) ? s.S : s.C;
  ce_colfwd(g, s, ld, other, X);
}

// Cluster reductions: push a block-reduced value (valid in every thread) into
// slot `slot` of every CTA; read back with ce_total after a cluster barrier.
__device__ __forceinline__ void ce_put(double* part, int Q, int slot, double v) {
  cg::cluster_group cl = cg::this_cluster();
  if ((int)threadIdx.x < Q) {
    double* dst = cl.map_shared_rank(part, (int)threadIdx.x);
    dst[slot * kMaxQ + (int)cl.block_rank()] = v;
  }
}
__device__ __forceinline__ double ce_total(const double* part, int Q, int slot) {
  double t = 0.0;
  for (int r = 0; r < Q; ++r) t += part[slot * kMaxQ + r];
  return t;
}
__device__ __forceinline__ double ce_maxall(const double* part, int Q, int slot) {
  double t = 0.0;
  for (int r = 0; r < Q; ++r) t = fmax(t, part[slot * kMaxQ + r]);
  return t;
}

// ------------------------------------------------- Krylov solve on a cluster
// Owned entry pairs of the real-input geometry: pair pp = (j1 << lgcQ) + c
// (j1 < N1/2, c < cQ) holds the vector entries i0 = 2 (N2 j1 + q cQ + c) and
// i0 + 1, the real and imaginary parts of packed element (j1, c) of the CTA's
// columns -- the same index as the element in ce_io.  Vectors are allocated
// with an even length, so a pair is one aligned two-element vector load.
__device__ __forceinline__ int pair_i0(const CeGeo& g, int pp) {
  return 2 * (((pp >> g.lgcQ) << g.lgN2) + (g.q << g.lgcQ) + (pp & (g.cQ - 1)));
}
template <typename R> __device__ __forceinline__ cplx<R> ld2(const R* v, int i0) {
  return reinterpret_cast<const cplx<R>*>(v)[i0 >> 1];
}
// store the entries of a pair that lie below n
template <typename R> __device__ __forceinline__ void st2(R* v, int i0, int n, cplx<R> x) {
  if (i0 + 1 < n) reinterpret_cast<cplx<R>*>(v)[i0 >> 1] = x;
  else if (i0 < n) v[i0] = x.x;
}

constexpr int kVB = 4;  // pairs per thread whose loads are issued together
constexpr int kXR = 2;  // the same for the six-vector update of x and r

// What a Krylov solve on the cluster reads, kept at CeSm::ctx (each pass
// copies what it needs into registers on entry).
template <typename R> struct CeCtx {
  CeGeo g;            // real-input geometry (q filled per CTA)
  CeLay lay;
  const cplx<R>* spT;  // Toeplitz spectrum, row-pass order
  const cplx<R>* spG;  // preconditioner spectrum, row-pass order
  KVecs<R> V;
  const R* kap;
  const R* hinv;       // 1/kappa (PCG on the symmetrised system; NULL otherwise)
  R a;                 // ahat
};

template <typename R> __device__ __forceinline__ CeGeo ce_enter(const CeCtx<R>* cx) {
  CeGeo g = cx->g;
  g.q = (int)cg::this_cluster().block_rank();
  return g;
}

// epilogue / prologue modes of the column passes
enum { PRO_P = 0, PRO_S = 1, PRO_R = 2, PRO_PZ = 3 };  // forward of p, s, r, or z + c0 p
enum { EPI_PH = 0, EPI_SH = 1, EPI_V = 2, EPI_T = 3, EPI_Z = 4, EPI_Q = 5 };  // inverse into ...

// Inverse column pass of a product inside the solve; the last FFT stage
// writes y (zero at entries >= n) into ce_io, then per mode:
//   EPI_PH / EPI_SH: ph = y (sh = y), and the forward column pass of that
//     vector straight from ce_io (the next product's input);
//   EPI_V: v = a ph + kappa y, acc.x = (rh, v);  EPI_T: t = a sh + kappa y,
//     acc.x = (t, s), acc.y = (t, t).   xin is ph or p (sh or s).
//   PCG (ce_pcg): EPI_Z: z = y (into V.s), acc.x = (r, z);  EPI_Q:
//     q = a hinv p + y (into V.v), acc.x = (p, q), xin = p.
// TR (transposed operator a I + A K): kappa scales the forwarded input
// instead of the product's output.
template <typename R>
__device__ __noinline__ cplx<R> ce_colinv_op(const CeCtx<R>* cxp, int mode, const R* __restrict__ xin) {
  typedef cplx<R> Z;
  const CeGeo g = ce_enter(cxp);
  const CeSm<R> s = ce_sm<R>(cxp->lay);
  const int q = g.q, N1 = g.N1, lgN2 = g.lgN2, n = g.n, lgcQ = g.lgcQ;
  const bool fused = (mode == EPI_PH || mode == EPI_SH);
  Z* const Bn = ce_io(g, s);
  {
    auto st = [=](int j1, int c, Z z) {
      if (j1 < (N1 >> 1)) {
        const int i0 = 2 * ((j1 << lgN2) + (q << lgcQ) + c);
        Bn[(j1 << lgcQ) + c] = mkc<R>(i0 < n ? z.x : R(0), i0 + 1 < n ? z.y : R(0));
      }
    };
    ce_colinv(g, s, st);
  }
  const int npair = (N1 >> 1) << lgcQ;
  R acc0 = R(0), acc1 = R(0);
  if (fused) {
    R* dst = (mode == EPI_PH) ? cxp->V.ph : cxp->V.sh;
    for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) st2(dst, pair_i0(g, pp), n, Bn[pp]);
    __syncthreads();
    ce_colfwd_buf(g, s, N1 >> 1);
  } else {
    const bool pz = (mode == EPI_Z || mode == EPI_Q);
    R* const dst = (mode == EPI_V || mode == EPI_Q) ? cxp->V.v : (mode == EPI_Z ? cxp->V.s : cxp->V.t);
    const R* const dotv = (mode == EPI_V) ? cxp->V.rh : (mode == EPI_Z ? cxp->V.r : (mode == EPI_Q ? xin : cxp->V.s));
    const R* const kap = (mode == EPI_Q) ? cxp->hinv : cxp->kap;
    const R a = cxp->a;
    for (int p0 = threadIdx.x; p0 < npair; p0 += kVB * blockDim.x) {
      Z xv[kVB], kv[kVB], dv[kVB];
#pragma unroll
      for (int u = 0; u < kVB; ++u) {
        const int pp = p0 + u * blockDim.x;
        const int i0 = pair_i0(g, pp);
        xv[u] = kv[u] = dv[u] = mkc<R>(R(0), R(0));
        if (pp < npair && i0 < n) {
          if (mode != EPI_Z) {
            xv[u] = ld2(xin, i0);
            kv[u] = ld2(kap, i0);
          }
          dv[u] = ld2(dotv, i0);
        }
      }
#pragma unroll
      for (int u = 0; u < kVB; ++u) {
        const int pp = p0 + u * blockDim.x;
        if (pp < npair) {
          const int i0 = pair_i0(g, pp);
          const Z y = Bn[pp];
          Z w;
          if (mode == EPI_Z) w = y;
          else if (mode == EPI_Q) w = mkc<R>(a * kv[u].x * xv[u].x + y.x, a * kv[u].y * xv[u].y + y.y);
          else w = mkc<R>(a * xv[u].x + kv[u].x * y.x, a * xv[u].y + kv[u].y * y.y);
          if (i0 + 1 >= n) w.y = R(0);
          if (i0 >= n) w.x = R(0);
          st2(dst, i0, n, w);
          acc0 += dv[u].x * w.x + dv[u].y * w.y;
          acc1 += w.x * w.x + w.y * w.y;
        }
      }
    }
    (void)pz;
  }
  return mkc<R>(acc0, acc1);
}

// Forward column pass of p = r + beta (p - omega v) (PRO_P), of
// s = r - alpha v (PRO_S), of r itself (PRO_R), or (PCG) of p = z + c0 p with
// z = zsrc (PRO_PZ), storing the new vector (not for PRO_R); the entries are
// formed in ce_io first (loads issued together), then transformed.
template <typename R>
__device__ __noinline__ void ce_colfwd_vec(const CeCtx<R>* cxp, int mode, R c0, R c1,
                                           const R* zsrc = nullptr) {
  typedef cplx<R> Z;
  const CeGeo g = ce_enter(cxp);
  const CeSm<R> s = ce_sm<R>(cxp->lay);
  const int N1 = g.N1, n = g.n, lgcQ = g.lgcQ;
  const R* const r_ = (mode == PRO_PZ) ? zsrc : cxp->V.r;
  const R* const v_ = cxp->V.v;
  R* const dst = (mode == PRO_P || mode == PRO_PZ) ? cxp->V.p : cxp->V.s;
  Z* const X = ce_io(g, s);
  const int npair = (N1 >> 1) << lgcQ;
  for (int p0 = threadIdx.x; p0 < npair; p0 += kVB * blockDim.x) {
    Z rv[kVB], pv[kVB], vv[kVB];
#pragma unroll
    for (int u = 0; u < kVB; ++u) {
      const int pp = p0 + u * blockDim.x;
      const int i0 = pair_i0(g, pp);
      rv[u] = vv[u] = pv[u] = mkc<R>(R(0), R(0));
      if (pp < npair && i0 < n) {
        rv[u] = ld2(r_, i0);
        if (mode == PRO_P || mode == PRO_S) vv[u] = ld2(v_, i0);
        if (mode == PRO_P || mode == PRO_PZ) pv[u] = ld2((const R*)dst, i0);
      }
    }
#pragma unroll
    for (int u = 0; u < kVB; ++u) {
      const int pp = p0 + u * blockDim.x;
      if (pp < npair) {
        const int i0 = pair_i0(g, pp);
        Z x;
        if (mode == PRO_P) {
          x.x = rv[u].x + c0 * (pv[u].x - c1 * vv[u].x);
          x.y = rv[u].y + c0 * (pv[u].y - c1 * vv[u].y);
        } else if (mode == PRO_S) {
          x.x = rv[u].x - c0 * vv[u].x;
          x.y = rv[u].y - c0 * vv[u].y;
        } else if (mode == PRO_PZ) {
          x.x = rv[u].x + c0 * pv[u].x;
          x.y = rv[u].y + c0 * pv[u].y;
        } else {
          x = rv[u];
        }
        if (i0 + 1 >= n) x.y = R(0);
        if (i0 >= n) x.x = R(0);
        if (mode != PRO_R) st2(dst, i0, n, x);
        X[pp] = x;
      }
    }
  }
  __syncthreads();
  ce_colfwd_buf(g, s, N1 >> 1);
}

template <typename R> __device__ __noinline__ void ce_rows_apply(const CeCtx<R>* cxp, bool precG) {
  const CeGeo g = ce_enter(cxp);
  const CeSm<R> s = ce_sm<R>(cxp->lay);
  ce_rows<R, CE_APPLY>(g, s, precG ? cxp->spG : cxp->spT, nullptr, nullptr);
}

// Right-preconditioned BiCGSTAB (van der Vorst) for (ahat I + K A) x = b with
// b_i = (R)(sc r64_i), x0 = 0, on the cluster in precision R; the same
// recurrences and stopping rule as bicgstab in grid.cuh.  Every CTA of the
// cluster calls it with the context at CeSm::ctx filled in.
enum { CS_BB = 0, CS_RV = 1, CS_TS = 2, CS_TT = 3, CS_RR0 = 4, CS_RR = 5 };

template <typename R>
__device__ __noinline__ SolveRes ce_bicgstab(const CeCtx<R>* cxp, bool prec, double tol, int max_it,
                                             const double* __restrict__ r64, double sc) {
  typedef cplx<R> Z;
  cg::cluster_group cl = cg::this_cluster();
  const CeGeo g = ce_enter(cxp);
  const CeSm<R> s = ce_sm<R>(cxp->lay);
  const int Q = g.Q, n = g.n;
  const int npair = (g.N1 >> 1) << g.lgcQ;
  SolveRes out{TSFDE_OK, 0, 0.0};
  {
    const KVecs<R> V = cxp->V;
    R acc = R(0);
    for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) {
      const int i0 = pair_i0(g, pp);
      Z b2 = mkc<R>(R(0), R(0));
      if (i0 + 1 < n) {
        const double2 r2 = reinterpret_cast<const double2*>(r64)[i0 >> 1];
        b2 = mkc<R>((R)(r2.x * sc), (R)(r2.y * sc));
      } else if (i0 < n) {
        b2.x = (R)(r64[i0] * sc);
      }
      const Z z = mkc<R>(R(0), R(0));
      st2(V.x, i0, n, z); st2(V.r, i0, n, b2); st2(V.rh, i0, n, b2);
      st2(V.p, i0, n, z); st2(V.v, i0, n, z);
      acc += b2.x * b2.x + b2.y * b2.y;
    }
    ce_put(s.part, Q, CS_BB, block_sum((double)acc, s.red));
  }
  cl.sync();
  const double bb = ce_total(s.part, Q, CS_BB);
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
    ce_colfwd_vec<R>(cxp, PRO_P, (R)beta, (R)omega);
    cl.sync();
    if (prec) {
      ce_rows_apply<R>(cxp, true);
      cl.sync();
      ce_colinv_op<R>(cxp, EPI_PH, nullptr);
      cl.sync();
    }
    ce_rows_apply<R>(cxp, false);
    cl.sync();
    {
      const Z acc = ce_colinv_op<R>(cxp, EPI_V, prec ? cxp->V.ph : cxp->V.p);
      ce_put(s.part, Q, CS_RV, block_sum((double)acc.x, s.red));
    }
    cl.sync();
    const double rv = ce_total(s.part, Q, CS_RV);
    if (!isfinite(rv)) { out.status = TSFDE_ENONFINITE; return out; }
    if (rv == 0.0) { out.status = TSFDE_EBREAKDOWN; return out; }
    alpha = rho / rv;
    // s = r - alpha v; t = M P^{-1} s
    ce_colfwd_vec<R>(cxp, PRO_S, (R)alpha, R(0));
    cl.sync();
    if (prec) {
      ce_rows_apply<R>(cxp, true);
      cl.sync();
      ce_colinv_op<R>(cxp, EPI_SH, nullptr);
      cl.sync();
    }
    ce_rows_apply<R>(cxp, false);
    cl.sync();
    {
      const Z acc = ce_colinv_op<R>(cxp, EPI_T, prec ? cxp->V.sh : cxp->V.s);
      const double ts_b = block_sum((double)acc.x, s.red);
      const double tt_b = block_sum((double)acc.y, s.red);
      ce_put(s.part, Q, CS_TS, ts_b);
      ce_put(s.part, Q, CS_TT, tt_b);
    }
    cl.sync();
    const double ts = ce_total(s.part, Q, CS_TS), tt = ce_total(s.part, Q, CS_TT);
    omega = (tt > 0.0) ? ts / tt : 0.0;
    if (!isfinite(omega)) { out.status = TSFDE_ENONFINITE; return out; }
    // x += alpha p^ + omega s^, r = s - omega t
    {
      const KVecs<R> V = cxp->V;
      const R* const ph = prec ? V.ph : V.p;
      const R* const sh = prec ? V.sh : V.s;
      const R aR = (R)alpha, oR = (R)omega;
      R arr = R(0), ar2 = R(0);
      for (int p0 = threadIdx.x; p0 < npair; p0 += kXR * blockDim.x) {
        Z xv[kXR], pv[kXR], sv[kXR], ss[kXR], tv[kXR], hv[kXR];
#pragma unroll
        for (int u = 0; u < kXR; ++u) {
          const int pp = p0 + u * blockDim.x;
          const int i0 = pair_i0(g, pp);
          xv[u] = pv[u] = sv[u] = ss[u] = tv[u] = hv[u] = mkc<R>(R(0), R(0));
          if (pp < npair && i0 < n) {
            xv[u] = ld2(V.x, i0); pv[u] = ld2(ph, i0); sv[u] = ld2(sh, i0);
            ss[u] = ld2(V.s, i0); tv[u] = ld2(V.t, i0); hv[u] = ld2(V.rh, i0);
          }
        }
#pragma unroll
        for (int u = 0; u < kXR; ++u) {
          const int pp = p0 + u * blockDim.x;
          if (pp < npair) {
            const int i0 = pair_i0(g, pp);
            const Z x = mkc<R>(xv[u].x + aR * pv[u].x + oR * sv[u].x,
                               xv[u].y + aR * pv[u].y + oR * sv[u].y);
            Z r = mkc<R>(ss[u].x - oR * tv[u].x, ss[u].y - oR * tv[u].y);
            if (i0 + 1 >= n) r.y = R(0);
            if (i0 >= n) r.x = R(0);
            st2(V.x, i0, n, x);
            st2(V.r, i0, n, r);
            arr += hv[u].x * r.x + hv[u].y * r.y;
            ar2 += r.x * r.x + r.y * r.y;
          }
        }
      }
      const double rr0_b = block_sum((double)arr, s.red);
      const double rr_b = block_sum((double)ar2, s.red);
      ce_put(s.part, Q, CS_RR0, rr0_b);
      ce_put(s.part, Q, CS_RR, rr_b);
    }
    cl.sync();
    rho_new = ce_total(s.part, Q, CS_RR0);
    rr = ce_total(s.part, Q, CS_RR);
  }
}

// Preconditioned CG on the symmetrised level system (ahat K^{-1} + A) x =
// K^{-1} b, b_i = (R)(sc r64_i), x0 = 0, with the Strang circulant of
// Eq. (4.3) up to a constant factor (the same spectrum tables), on the
// cluster in precision R: the recurrences and the stopping rule of pcg in
// grid.cuh (||K r|| < tol ||b||, the residual of the original system).
// Needs cxp->hinv = 1/kappa.  Per iteration: forward pass of p = z + beta p,
// row pass (A), q = S p with (p, q), the update of x and r with ||K r||, and
// (with the preconditioner) the forward pass of r, row pass (P^{-1}) and
// z = P^{-1} r with (r, z).
template <typename R>
__device__ __noinline__ SolveRes ce_pcg(const CeCtx<R>* cxp, bool prec, double tol, int max_it,
                                        const double* __restrict__ r64, double sc) {
  typedef cplx<R> Z;
  cg::cluster_group cl = cg::this_cluster();
  const CeGeo g = ce_enter(cxp);
  const CeSm<R> s = ce_sm<R>(cxp->lay);
  const int Q = g.Q, n = g.n;
  const int npair = (g.N1 >> 1) << g.lgcQ;
  SolveRes out{TSFDE_OK, 0, 0.0};
  const KVecs<R> V = cxp->V;
  // x = 0, p = 0, r = K^{-1} b, ||b||^2 and (r, r)
  {
    R acc = R(0), arr = R(0);
    for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) {
      const int i0 = pair_i0(g, pp);
      Z b2 = mkc<R>(R(0), R(0));
      if (i0 + 1 < n) {
        const double2 r2 = reinterpret_cast<const double2*>(r64)[i0 >> 1];
        b2 = mkc<R>((R)(r2.x * sc), (R)(r2.y * sc));
      } else if (i0 < n) {
        b2.x = (R)(r64[i0] * sc);
      }
      const Z h = (i0 < n) ? ld2(cxp->hinv, i0) : mkc<R>(R(0), R(0));
      Z rk = mkc<R>(b2.x * h.x, b2.y * h.y);
      if (i0 + 1 >= n) rk.y = R(0);
      const Z z = mkc<R>(R(0), R(0));
      st2(V.x, i0, n, z); st2(V.p, i0, n, z); st2(V.r, i0, n, rk);
      acc += b2.x * b2.x + b2.y * b2.y;
      arr += rk.x * rk.x + rk.y * rk.y;
    }
    ce_put(s.part, Q, CS_BB, block_sum((double)acc, s.red));
    ce_put(s.part, Q, CS_RR0, block_sum((double)arr, s.red));
  }
  cl.sync();
  const double bb = ce_total(s.part, Q, CS_BB);
  double rho = ce_total(s.part, Q, CS_RR0);
  if (!isfinite(bb)) { out.status = TSFDE_ENONFINITE; return out; }
  if (bb == 0.0) return out;
  const double nb = sqrt(bb);
  // z = P^{-1} r (into V.s), (r, z)
  auto precond = [&](double& rho_out) {
    ce_colfwd_vec<R>(cxp, PRO_R, R(0), R(0));
    cl.sync();
    ce_rows_apply<R>(cxp, true);
    cl.sync();
    const Z acc = ce_colinv_op<R>(cxp, EPI_Z, nullptr);
    ce_put(s.part, Q, CS_RV, block_sum((double)acc.x, s.red));
    cl.sync();
    rho_out = ce_total(s.part, Q, CS_RV);
  };
  if (prec) precond(rho);
  const R* const zv = prec ? V.s : V.r;
  double rr = bb, beta = 0.0;
  int it = 0;
  for (;;) {
    const double relres = sqrt(rr) / nb;
    out.relres = relres;
    out.iters = it;
    if (!isfinite(relres) || !isfinite(rho)) { out.status = TSFDE_ENONFINITE; return out; }
    if (relres < tol) return out;
    if (it >= max_it) { out.status = TSFDE_ENOCONV; return out; }
    if (!(rho > 0.0)) { out.status = TSFDE_EBREAKDOWN; return out; }
    out.iters = ++it;
    // p = z + beta p and its forward pass; q = S p, (p, q)
    ce_colfwd_vec<R>(cxp, PRO_PZ, (R)beta, R(0), zv);
    cl.sync();
    ce_rows_apply<R>(cxp, false);
    cl.sync();
    {
      const Z acc = ce_colinv_op<R>(cxp, EPI_Q, V.p);
      ce_put(s.part, Q, CS_TS, block_sum((double)acc.x, s.red));
    }
    cl.sync();
    const double pq = ce_total(s.part, Q, CS_TS);
    if (!isfinite(pq)) { out.status = TSFDE_ENONFINITE; return out; }
    if (!(pq > 0.0)) { out.status = TSFDE_EBREAKDOWN; return out; }
    const double alpha = rho / pq;
    // x += alpha p, r -= alpha q, ||K r||^2 and (r, r)
    {
      const R aR = (R)alpha;
      R akr = R(0), arr = R(0);
      for (int pp = threadIdx.x; pp < npair; pp += blockDim.x) {
        const int i0 = pair_i0(g, pp);
        if (i0 >= n) continue;
        const Z xv = ld2(V.x, i0), pv = ld2(V.p, i0), rv = ld2(V.r, i0), qv = ld2(V.v, i0);
        const Z kv = ld2(cxp->kap, i0);
        const Z x = mkc<R>(xv.x + aR * pv.x, xv.y + aR * pv.y);
        Z r = mkc<R>(rv.x - aR * qv.x, rv.y - aR * qv.y);
        if (i0 + 1 >= n) r.y = R(0);
        st2(V.x, i0, n, x);
        st2(V.r, i0, n, r);
        const R k0 = kv.x * r.x, k1 = kv.y * r.y;
        akr += k0 * k0 + k1 * k1;
        arr += r.x * r.x + r.y * r.y;
      }
      ce_put(s.part, Q, CS_RR, block_sum((double)akr, s.red));
      ce_put(s.part, Q, CS_RR0, block_sum((double)arr, s.red));
    }
    cl.sync();
    rr = ce_total(s.part, Q, CS_RR);
    double rho_new = ce_total(s.part, Q, CS_RR0);
    if (sqrt(rr) / nb < tol) {
      out.relres = sqrt(rr) / nb;
      if (!isfinite(out.relres)) out.status = TSFDE_ENONFINITE;
      return out;
    }
    if (prec) precond(rho_new);
    beta = rho_new / rho;
    rho = rho_new;
  }
}

}  // namespace tsfde
