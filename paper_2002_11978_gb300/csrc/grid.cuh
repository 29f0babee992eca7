// grid.cuh -- device code of the grid-wide (cooperative) FIDS solver, shared
// by the grid engine and the cluster engine: the three-pass zero-padded FFT
// products (Sec. 4.1), the Strang preconditioner build, PBiCGSTAB on the
// whole grid, and the mixed-precision refinement loop around an inner solver.
//
// Toeplitz and circulant products use a zero-padded real FFT of length L
// computed as a complex FFT of length Nc = L/2 in three passes (column FFTs,
// paired row FFTs with the spectral product in the middle, inverse column
// FFTs).  The inverse column pass of one product and the forward column pass
// of the next product share a CTA tile, so a product that feeds another costs
// two grid barriers.  Grid barriers are bounded (dev.cuh); every kernel
// returns a status instead of hanging or trapping.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "../../include/tsfde.h"
#include "dev.cuh"
#include "plan.h"

namespace tsfde {

constexpr int kThreads = 256;

// partial-sum slots
enum {
  SL_BB = 0, SL_RV = 1, SL_TS = 2, SL_TT = 3, SL_RR0 = 4, SL_RR = 5,
  SL_EMAX = 6, SL_XMAX = 7, SL_RES = 8, SL_KAP = 9
};

template <typename R> struct Smem {
  cplx<R>* tw;  // W_T^k, k < T
  cplx<R>* bA;  // work buffers (W complex each)
  cplx<R>* bB;
  double* red;  // 33 doubles
};

// Tables of each arithmetic type.
template <typename R> constexpr bool is_f64 = std::is_same_v<R, double>;
template <typename R> constexpr bool is_ds = std::is_same_v<R, dsf>;

template <typename R> __device__ __forceinline__ const cplx<R>* twL(const DevPlan& P) {
  if constexpr (is_f64<R>) return P.twL64;
  else if constexpr (is_ds<R>) return P.twLds;
  else return P.twL32;
}
template <typename R> __device__ __forceinline__ int lgct(const Geo& g) {
  if constexpr (sizeof(cplx<R>) == 16) return g.lgct64; else return g.lgct32;
}
template <typename R> __device__ __forceinline__ const R* saT(const DevPlan& P) {
  if constexpr (is_f64<R>) return P.saT64;
  else if constexpr (is_ds<R>) return P.saTds;
  else return P.saT32;
}
template <typename R> __device__ __forceinline__ const R* sbT(const DevPlan& P) {
  if constexpr (is_f64<R>) return P.sbT64;
  else if constexpr (is_ds<R>) return P.sbTds;
  else return P.sbT32;
}
template <typename R> __device__ __forceinline__ R* saG(const DevPlan& P) {
  if constexpr (is_f64<R>) return P.saG64;
  else if constexpr (is_ds<R>) return P.saGds;
  else return P.saG32;
}
template <typename R> __device__ __forceinline__ R* sbG(const DevPlan& P) {
  if constexpr (is_f64<R>) return P.sbG64;
  else if constexpr (is_ds<R>) return P.sbGds;
  else return P.sbG32;
}
template <typename R> __device__ __forceinline__ const cplx<R>* chirp(const DevPlan& P) {
  if constexpr (is_f64<R>) return P.chirp64;
  else if constexpr (is_ds<R>) return P.chirpds;
  else return P.chirp32;
}
template <typename R> __device__ __forceinline__ const cplx<R>* Bh(const DevPlan& P) {
  if constexpr (is_f64<R>) return P.Bh64;
  else if constexpr (is_ds<R>) return P.Bhds;
  else return P.Bh32;
}
template <typename R> __device__ __forceinline__ R* gcol(const DevPlan& P) {
  if constexpr (is_f64<R>) return P.g64;
  else if constexpr (is_ds<R>) return P.gds;
  else return P.g32;
}

struct SmemAll {
  Smem<double> d;
  Smem<float> f;
  Smem<dsf> s;  // tw is NULL unless the plan has double-single tables
};

// Shared memory: [tw64 Tp][tw32 Tp][twds Tp][bufA W][bufB W][red 64], the
// twiddle tables padded (Tp = tpad_len(T), entry k at tpad(k); see dev.cuh)
// init_epoch: also clear the CTA's grid-barrier epoch (at the start of a
// kernel; not when the tables are reloaded in mid-kernel).
__device__ __forceinline__ SmemAll smem_setup(const DevPlan& P, bool init_epoch = true) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (init_epoch && threadIdx.x == 0) s_grid_epoch = 0u;
  char* base = reinterpret_cast<char*>(smem_raw);
  const size_t Tp = (size_t)tpad_len(P.T);
  double2* tw64 = reinterpret_cast<double2*>(base);
  float2* tw32 = reinterpret_cast<float2*>(base + Tp * sizeof(double2));
  dsf2* twds = reinterpret_cast<dsf2*>(base + Tp * (sizeof(double2) + sizeof(float2)));
  char* wbase = base + Tp * (2 * sizeof(double2) + sizeof(float2));
  double2* bA = reinterpret_cast<double2*>(wbase);
  double2* bB = bA + P.W;
  double* red = reinterpret_cast<double*>(bB + P.W);
  const int stride = P.L / P.T;
  const bool ds = P.twLds != nullptr;
  for (int k = threadIdx.x; k < P.T; k += blockDim.x) {
    const int kp = tpad(k);
    tw64[kp] = P.twL64[k * stride];
    tw32[kp] = P.twL32[k * stride];
    if (ds) twds[kp] = P.twLds[k * stride];
  }
  __syncthreads();
  SmemAll s;
  s.d.tw = tw64; s.d.bA = bA; s.d.bB = bB; s.d.red = red;
  s.f.tw = tw32; s.f.bA = reinterpret_cast<float2*>(bA); s.f.bB = reinterpret_cast<float2*>(bB);
  s.f.red = red;
  s.s.tw = ds ? twds : nullptr; s.s.bA = reinterpret_cast<dsf2*>(bA); s.s.bB = reinterpret_cast<dsf2*>(bB);
  s.s.red = red;
  return s;
}

__device__ __forceinline__ void put_partial(const DevPlan& P, int slot, double v) {
  if (threadIdx.x == 0) grid_partials_next(P.part, P.G)[slot * P.G + blockIdx.x] = v;
}
// Grid barrier; the _sum variants also return the grid-wide reduction of
// the partial slots written before the barrier (bit-identical in all CTAs).
__device__ __forceinline__ bool gsync(const DevPlan& P, double* red) {
  return grid_sync_red(P.bar, P.timeout, P.part, P.G, 0, nullptr, 0u, nullptr, red);
}
__device__ __forceinline__ bool gsync_sum(const DevPlan& P, double* red, int s0, double& o0) {
  const int sl[1] = {s0};
  double o[1];
  const bool ok = grid_sync_red(P.bar, P.timeout, P.part, P.G, 1, sl, 0u, o, red);
  o0 = o[0];
  return ok;
}
__device__ __forceinline__ bool gsync_sum2(const DevPlan& P, double* red, int s0, int s1,
                                           unsigned maxmask, double& o0, double& o1) {
  const int sl[2] = {s0, s1};
  double o[2];
  const bool ok = grid_sync_red(P.bar, P.timeout, P.part, P.G, 2, sl, maxmask, o, red);
  o0 = o[0];
  o1 = o[1];
  return ok;
}

__device__ __forceinline__ bool gsync_sum3(const DevPlan& P, double* red, int s0, int s1, int s2,
                                           unsigned maxmask, double& o0, double& o1, double& o2) {
  const int sl[3] = {s0, s1, s2};
  double o[3];
  const bool ok = grid_sync_red(P.bar, P.timeout, P.part, P.G, 3, sl, maxmask, o, red);
  o0 = o[0];
  o1 = o[1];
  o2 = o[2];
  return ok;
}

// True when the real-geometry work items (column tiles, row pairs) have at
// most KP * kThreads elements, so that solvers instantiated with that
// prefetch depth cover them.
__host__ __device__ inline bool kp_fits(const DevPlan& P, int KP) {
  return (P.gr.N1 << P.gr.lgct64) <= KP * kThreads && 2 * P.gr.N2 <= KP * kThreads;
}

// ------------------------------------------------------------------ passes
// Each thread handles at most KP elements of a work item (tile or row
// pair); their store twiddles and spectral coefficients are loaded into
// registers before the shared-memory FFT so the L2 latency overlaps it.
// kPre = 4 covers every size (with 256 threads: work items of <= 1024
// elements, n <= 2^18); solvers whose items are <= 512 elements can be
// instantiated with KP = 2, which frees registers.
constexpr int kPre = 4;

// Pass A, real input: x (length nin, zero beyond) -> z_j = x_{2j} + i x_{2j+1},
// column FFTs over j1 (j = N2 j1 + j2), twiddle W_Nc^{j2 k1}, store
// S1[k1*N2 + j2].  Without FULL only rows j1 < N1/2 can be non-zero
// (nin <= L/2).
// A prologue of passA_real may take the entries in pairs: invocable as
// pro(PairTag{}, i0) for even i0 < nin, returning entries i0 and i0 + 1 (the
// latter is dropped when i0 + 1 >= nin), so that its loads and stores can be
// 16-byte pair accesses issued together.  Otherwise pro(i) gives entry i.
struct PairTag {};
template <typename R> __device__ __forceinline__ cplx<R> ld_pair(const R* v, int i0) {
  return reinterpret_cast<const cplx<R>*>(v)[i0 >> 1];
}
template <typename R> __device__ __forceinline__ void st_pair(R* v, int i0, cplx<R> z) {
  reinterpret_cast<cplx<R>*>(v)[i0 >> 1] = z;
}

// out: where the column transforms go (NULL: S1).
template <typename R, bool FULL, int KP = kPre, class Pro>
__device__ void passA_real(const DevPlan& P, const Smem<R>& sm, int nin, Pro& pro,
                           cplx<R>* out = nullptr) {
  typedef cplx<R> Z;
  const Geo& g = P.gr;
  const int lc = lgct<R>(g), ct = 1 << lc;
  const int N1 = g.N1, N2 = g.N2;
  const int ntiles = N2 >> lc;
  const int total = N1 << lc;
  const int rows = FULL ? N1 : (N1 >> 1);
  const int tstride = P.L / g.Nfft;
  Z* S1 = out ? out : reinterpret_cast<Z*>(P.S1);
  const Z* tw = twL<R>(P);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int c0 = tile << lc;
    Z wp[KP];
#pragma unroll
    for (int q = 0; q < KP; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < total) {
        const int k1 = e >> lc, j2 = c0 + (e & (ct - 1));
        wp[q] = tw[((j2 * k1) & (g.Nfft - 1)) * tstride];
      }
    }
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int j1 = e >> lc, c = e & (ct - 1);
      Z v = mkc<R>(R(0), R(0));
      if (j1 < rows) {
        const int i0 = 2 * (N2 * j1 + c0 + c);
        if constexpr (std::is_invocable_v<Pro&, PairTag, int>) {
          if (i0 < nin) {
            v = pro(PairTag{}, i0);
            if (i0 + 1 >= nin) v.y = R(0);
          }
        } else {
          const R x0 = (i0 < nin) ? pro(i0) : R(0);
          const R x1 = (i0 + 1 < nin) ? pro(i0 + 1) : R(0);
          v = mkc<R>(x0, x1);
        }
      }
      sm.bA[e] = v;
    }
    __syncthreads();
    const Z* res = fft_batch<R, false>(sm.bA, sm.bB, N1, lc, sm.tw, P.T);
#pragma unroll
    for (int q = 0; q < KP; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < total) S1[(e >> lc) * N2 + c0 + (e & (ct - 1))] = cmul(res[e], wp[q]);
    }
    __syncthreads();
  }
}

// Pass A, complex input a_j (j < n, n <= L/2), geometry gc (Nfft = L).
template <typename R, class Pro>
__device__ void passA_cplx(const DevPlan& P, const Smem<R>& sm, Pro& pro) {
  typedef cplx<R> Z;
  const Geo& g = P.gc;
  const int lc = lgct<R>(g), ct = 1 << lc;
  const int N1 = g.N1, N2 = g.N2;
  const int ntiles = N2 >> lc;
  const int total = N1 << lc;
  const int tstride = P.L / g.Nfft;
  Z* S1 = reinterpret_cast<Z*>(P.S1);
  const Z* tw = twL<R>(P);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int c0 = tile << lc;
    Z wp[kPre];
#pragma unroll
    for (int q = 0; q < kPre; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < total) {
        const int k1 = e >> lc, j2 = c0 + (e & (ct - 1));
        wp[q] = tw[((j2 * k1) & (g.Nfft - 1)) * tstride];
      }
    }
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int j1 = e >> lc, c = e & (ct - 1);
      const int j = N2 * j1 + c0 + c;
      sm.bA[e] = (j1 < (N1 >> 1) && j < P.n) ? pro(j) : mkc<R>(R(0), R(0));
    }
    __syncthreads();
    const Z* res = fft_batch<R, false>(sm.bA, sm.bB, N1, lc, sm.tw, P.T);
#pragma unroll
    for (int q = 0; q < kPre; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < total) S1[(e >> lc) * N2 + c0 + (e & (ct - 1))] = cmul(res[e], wp[q]);
    }
    __syncthreads();
  }
}

enum { MID_APPLY = 0, MID_SPEC = 1, MID_CONV = 2 };

// Pass B: row FFTs (rows k1 and N1-k1 together), the spectral middle step,
// inverse row FFTs, twiddle W^{-j2 k1}, store S2.  With Z the complex FFT of
// the packed real input and k' = Nc - k, E = (Z_k + conj Z_k')/2 and
// O = -i (Z_k - conj Z_k')/2 give the real-input spectrum
// X_k = E + W_L^k O and conj(X_k') = E - W_L^k O.
//  MID_APPLY: Y = S X for a real even spectrum S (tables sa = S_k/Nc,
//    sb = S_k'/Nc), repacked as Z'_k = E' + i O' with
//    E' = (sa X_k + sb conj X_k')/2, O' = conj(W_L^k) (sa X_k - sb conj X_k')/2.
//    Each multiplier meets only its own frequency: the split into E and O
//    is never weighted by the partner's S, which for the IFL symbol can be
//    ~1e8 times larger (low against high frequencies) and would swamp the
//    low-frequency result in rounding.
//  MID_SPEC: forward only; stores sa = Re X_k / Nc, sb = Re conj X_k' / Nc
//    (the spectrum of an even real sequence is real).
//  MID_CONV: complex product Z'_k = Z_k * conv_k (geometry gc).
// Row input of a pass B: the combination a + cb b + cc c of up to three
// column transforms (b, c NULL when absent), optionally kept in `keep`.
// The column transforms are linear, so a combination of transforms is the
// transform of the combination: the Krylov loops use this to form the
// transform of a new search direction without a column pass of its own.
template <typename R> struct RowIn {
  const cplx<R>* a;
  const cplx<R>* b;
  R cb;
  const cplx<R>* c;
  R cc;
  cplx<R>* keep;
};

template <typename R, int MID, int KP = kPre, bool COMB = false>
__device__ void passB(const DevPlan& P, const Smem<R>& sm, const R* __restrict__ sa,
                      const R* __restrict__ sb, R* sa_out, R* sb_out,
                      const cplx<R>* __restrict__ conv, const RowIn<R>* in = nullptr) {
  typedef cplx<R> Z;
  const Geo& g = (MID == MID_CONV) ? P.gc : P.gr;
  const int N1 = g.N1, N2 = g.N2;
  const int npairs = (N1 >> 1) + 1;
  const int tstride = P.L / g.Nfft;
  const Z* S1 = reinterpret_cast<const Z*>(P.S1);
  Z* S2 = reinterpret_cast<Z*>(P.S2);
  const Z* tw = twL<R>(P);
  const R invNc = R(1.0 / (double)P.Nc);  // Nc is a power of two: exact
  for (int it = blockIdx.x; it < npairs; it += gridDim.x) {
    const int ka = it;
    const int kb = (it == 0 || it == (N1 >> 1)) ? -1 : N1 - it;
    const int lgB = (kb < 0) ? 0 : 1;
    const int B = 1 << lgB;
    const int total = N2 << lgB;
    // per-element coefficients and store twiddles, fetched early
    Z wp[KP], cf[KP];
    R s1[KP], s2[KP];
#pragma unroll
    for (int q = 0; q < KP; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < total) {
        const int b = e & (B - 1), k2 = e >> lgB;
        const int k1 = b ? kb : ka;
        if constexpr (MID == MID_CONV) {
          cf[q] = conv[k1 * N2 + k2];
        } else {
          cf[q] = tw[k1 + N1 * k2];  // W_L^k, k = k1 + N1 k2
          if constexpr (MID == MID_APPLY) {
            s1[q] = sa[k1 * N2 + k2];
            s2[q] = sb[k1 * N2 + k2];
          }
        }
        if constexpr (MID != MID_SPEC) wp[q] = tw[((k2 * k1) & (g.Nfft - 1)) * tstride];
      }
    }
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int b = e & (B - 1), k2 = e >> lgB;
      const int row = b ? kb : ka;
      if constexpr (COMB) {
        const int at = row * N2 + k2;
        Z v = ldcg(in->a + at);
        if (in->b) {
          const Z w = ldcg(in->b + at);
          v = mkc<R>(v.x + in->cb * w.x, v.y + in->cb * w.y);
        }
        if (in->c) {
          const Z w = ldcg(in->c + at);
          v = mkc<R>(v.x + in->cc * w.x, v.y + in->cc * w.y);
        }
        if (in->keep) in->keep[at] = v;
        sm.bA[e] = v;
      } else {
        sm.bA[e] = ldcg(S1 + row * N2 + k2);
      }
    }
    __syncthreads();
    Z* res = fft_batch<R, false>(sm.bA, sm.bB, N2, lgB, sm.tw, P.T);
    Z* oth = (res == sm.bA) ? sm.bB : sm.bA;
#pragma unroll
    for (int q = 0; q < KP; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e >= total) continue;
      const int b = e & (B - 1), k2 = e >> lgB;
      const int k1 = b ? kb : ka;
      const Z Zk = res[e];
      if constexpr (MID == MID_CONV) {
        oth[e] = cmul(Zk, cf[q]);
      } else {
        const int q2 = (k1 == 0) ? ((N2 - k2) & (N2 - 1)) : (N2 - 1 - k2);
        const int qb = (B == 1) ? 0 : 1 - b;
        const Z Zq = res[(q2 << lgB) + qb];
        const Z E = mkc<R>(R(0.5) * (Zk.x + Zq.x), R(0.5) * (Zk.y - Zq.y));
        const Z O = mkc<R>(R(0.5) * (Zk.y + Zq.y), R(-0.5) * (Zk.x - Zq.x));
        const Z Wk = cf[q];
        const Z WO = cmul(Wk, O);
        const Z X = cadd(E, WO);   // X_k
        const Z Xc = csub(E, WO);  // conj(X_k')
        if constexpr (MID == MID_APPLY) {
          const Z Ya = cscale(X, s1[q]);
          const Z Yb = cscale(Xc, s2[q]);
          const Z Ep = cscale(cadd(Ya, Yb), R(0.5));
          const Z Op = cscale(cmulc(csub(Ya, Yb), Wk), R(0.5));
          oth[e] = mkc<R>(Ep.x - Op.y, Ep.y + Op.x);
        } else {
          sa_out[k1 * N2 + k2] = X.x * invNc;
          sb_out[k1 * N2 + k2] = Xc.x * invNc;
        }
      }
    }
    __syncthreads();
    if constexpr (MID == MID_SPEC) continue;
    const Z* res2 = fft_batch<R, true>(oth, res, N2, lgB, sm.tw, P.T);
#pragma unroll
    for (int q = 0; q < KP; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e < total) {
        const int b = e & (B - 1), j2 = e >> lgB;
        const int k1 = b ? kb : ka;
        S2[k1 * N2 + j2] = cmulc(res2[e], wp[q]);
      }
    }
    __syncthreads();
  }
}

// Pass C (+ optional fused pass A): inverse column FFTs, y_{2j} = Re z_j,
// y_{2j+1} = Im z_j for j1 < N1/2.  epi(i, y_i) consumes each output and
// returns the next product's input x_i (used only with DO_A).
template <typename R, bool DO_A, int KP = kPre, class Epi>
__device__ void passCA_real(const DevPlan& P, const Smem<R>& sm, Epi& epi, cplx<R>* out = nullptr) {
  typedef cplx<R> Z;
  const Geo& g = P.gr;
  const int lc = lgct<R>(g), ct = 1 << lc;
  const int N1 = g.N1, N2 = g.N2, n = P.n;
  const int ntiles = N2 >> lc;
  const int total = N1 << lc;
  const int tstride = P.L / g.Nfft;
  const Z* S2 = reinterpret_cast<const Z*>(P.S2);
  Z* S1 = out ? out : reinterpret_cast<Z*>(P.S1);
  const Z* tw = twL<R>(P);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int c0 = tile << lc;
    Z wp[KP];
    if constexpr (DO_A) {
#pragma unroll
      for (int q = 0; q < KP; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < total) {
          const int k1 = e >> lc, j2 = c0 + (e & (ct - 1));
          wp[q] = tw[((j2 * k1) & (g.Nfft - 1)) * tstride];
        }
      }
    }
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int k1 = e >> lc, c = e & (ct - 1);
      sm.bA[e] = ldcg(S2 + k1 * N2 + c0 + c);
    }
    __syncthreads();
    Z* res = fft_batch<R, true>(sm.bA, sm.bB, N1, lc, sm.tw, P.T);
    Z* oth = (res == sm.bA) ? sm.bB : sm.bA;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int j1 = e >> lc, c = e & (ct - 1);
      if (j1 < (N1 >> 1)) {
        const int i0 = 2 * (N2 * j1 + c0 + c);
        const Z v = res[e];
        R x0 = R(0), x1 = R(0);
        if (i0 < n) x0 = epi(i0, v.x);
        if (i0 + 1 < n) x1 = epi(i0 + 1, v.y);
        if (DO_A) oth[e] = mkc<R>(x0, x1);
      } else if (DO_A) {
        oth[e] = mkc<R>(R(0), R(0));
      }
    }
    __syncthreads();
    if constexpr (DO_A) {
      const Z* res2 = fft_batch<R, false>(oth, res, N1, lc, sm.tw, P.T);
#pragma unroll
      for (int q = 0; q < KP; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < total) S1[(e >> lc) * N2 + c0 + (e & (ct - 1))] = cmul(res2[e], wp[q]);
      }
      __syncthreads();
    }
  }
}

// Pass C, complex output z_j for j < n (geometry gc).
template <typename R, class Epi>
__device__ void passC_cplx(const DevPlan& P, const Smem<R>& sm, Epi& epi) {
  typedef cplx<R> Z;
  const Geo& g = P.gc;
  const int lc = lgct<R>(g), ct = 1 << lc;
  const int N1 = g.N1, N2 = g.N2;
  const int ntiles = N2 >> lc;
  const Z* S2 = reinterpret_cast<const Z*>(P.S2);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int c0 = tile << lc;
    for (int e = threadIdx.x; e < (N1 << lc); e += blockDim.x) {
      const int k1 = e >> lc, c = e & (ct - 1);
      sm.bA[e] = ldcg(S2 + k1 * N2 + c0 + c);
    }
    __syncthreads();
    const Z* res = fft_batch<R, true>(sm.bA, sm.bB, N1, lc, sm.tw, P.T);
    for (int e = threadIdx.x; e < (N1 << lc); e += blockDim.x) {
      const int j1 = e >> lc, c = e & (ct - 1);
      const int j = N2 * j1 + c0 + c;
      if (j1 < (N1 >> 1) && j < P.n) epi(j, res[e]);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------- preconditioner
// P = ahat I + kbar s(A) (Eq. (4.3)) is circulant of size n with eigenvalues
// d_k = ahat + kbar lambda_k.  Its inverse is the symmetric circulant with
// first column g = IDFT_n(1/d), computed by a Bluestein chirp-z transform
// on length-L FFTs; P^{-1} v is then the symmetric Toeplitz product with
// first column g, i.e. the same zero-padded product as A with the spectrum
// of the even embedding of g (built here as (sigma, rho) tables).
template <typename R, int KP = kPre>
__device__ bool build_precond(const DevPlan& P, const Smem<R>& sm, double ahat, double kbar) {
  typedef cplx<R> Z;
  const double* lam = P.lam;
  const Z* ch = chirp<R>(P);
  auto pro = [&](int j) -> Z {
    const R q = (R)(1.0 / (ahat + kbar * lam[j]));
    return cscale(ch[j], q);
  };
  passA_cplx<R>(P, sm, pro);
  if (!gsync(P, sm.red)) return false;
  passB<R, MID_CONV>(P, sm, nullptr, nullptr, nullptr, nullptr, Bh<R>(P));
  if (!gsync(P, sm.red)) return false;
  R* gv = gcol<R>(P);
  const R invn = R(1.0 / (double)P.n);
  auto epi = [&](int j, Z z) { gv[j] = (ch[j].x * z.x - ch[j].y * z.y) * invn; };
  passC_cplx<R>(P, sm, epi);
  if (!gsync(P, sm.red)) return false;
  const int n = P.n, L = P.L;
  auto proE = [&](int i) -> R {
    if (i < n) return gv[i];
    const int k = L - i;
    return (k < n) ? gv[k] : R(0);
  };
  passA_real<R, true, KP>(P, sm, L, proE);
  if (!gsync(P, sm.red)) return false;
  passB<R, MID_SPEC, KP>(P, sm, nullptr, nullptr, saG<R>(P), sbG<R>(P), nullptr);
  return gsync(P, sm.red);
}

// ------------------------------------------------------------- PBiCGSTAB
// Right-preconditioned BiCGSTAB (van der Vorst) for (ahat I + K A) x = b,
// x0 = 0, stop when ||r_k||_2 / ||b||_2 < tol (Sec. 5).  binit(i) gives b_i.
// Per iteration: P^{-1}p, A p^, P^{-1}s, A s^ as zero-padded FFT products.
// TR selects the transposed operator ahat I + A K (the adjoint level solve):
// kappa then scales the input of the Toeplitz product instead of its output.
template <typename R, class BInit, bool TR = false, int KP = kPre>
__device__ SolveRes bicgstab(const DevPlan& P, const Smem<R>& sm, const KVecs<R>& V,
                             const R* __restrict__ kap, double ahat, bool prec, double tol,
                             int max_it, BInit& binit) {
  const int n = P.n;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gstr = gridDim.x * blockDim.x;
  const R a = (R)ahat;
  SolveRes out{TSFDE_OK, 0, 0.0};
  {
    R acc = 0;
    for (int i = gtid; i < n; i += gstr) {
      const R bi = binit(i);
      V.x[i] = R(0); V.r[i] = bi; V.rh[i] = bi; V.p[i] = R(0); V.v[i] = R(0);
      acc += bi * bi;
    }
    put_partial(P, SL_BB, block_sum((double)acc, sm.red));
  }
  double bb;
  if (!gsync_sum(P, sm.red, SL_BB, bb)) { out.status = TSFDE_ETIMEOUT; return out; }
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
    out.iters = ++it;
    // p = r + beta (p - omega v), in pairs (the Krylov vectors are padded)
    {
      const R bR = (R)beta, oR = (R)omega;
      auto pro = [&](PairTag, int i0) -> cplx<R> {
        const cplx<R> r2 = ld_pair(V.r, i0), p2 = ld_pair(V.p, i0), v2 = ld_pair(V.v, i0);
        const cplx<R> q = mkc<R>(r2.x + bR * (p2.x - oR * v2.x), r2.y + bR * (p2.y - oR * v2.y));
        st_pair(V.p, i0, q);
        if (TR && !prec) {
          const cplx<R> k2 = mkc<R>(kap[i0], i0 + 1 < n ? kap[i0 + 1] : R(0));
          return mkc<R>(k2.x * q.x, k2.y * q.y);
        }
        return q;
      };
      passA_real<R, false, KP>(P, sm, n, pro);
    }
    if (!gsync(P, sm.red)) { out.status = TSFDE_ETIMEOUT; return out; }
    if (prec) {
      passB<R, MID_APPLY, KP>(P, sm, saG<R>(P), sbG<R>(P), nullptr, nullptr, nullptr);
      if (!gsync(P, sm.red)) { out.status = TSFDE_ETIMEOUT; return out; }
      auto epi = [&](int i, R y) -> R { V.ph[i] = y; return TR ? kap[i] * y : y; };
      passCA_real<R, true, KP>(P, sm, epi);
      if (!gsync(P, sm.red)) { out.status = TSFDE_ETIMEOUT; return out; }
    }
    passB<R, MID_APPLY, KP>(P, sm, saT<R>(P), sbT<R>(P), nullptr, nullptr, nullptr);
    if (!gsync(P, sm.red)) { out.status = TSFDE_ETIMEOUT; return out; }
    const R* ph = prec ? V.ph : V.p;
    {
      R acc = 0;
      auto epi = [&](int i, R y) -> R {
        const R vi = a * ph[i] + (TR ? y : kap[i] * y);
        V.v[i] = vi;
        acc += V.rh[i] * vi;
        return R(0);
      };
      passCA_real<R, false, KP>(P, sm, epi);
      put_partial(P, SL_RV, block_sum((double)acc, sm.red));
    }
    double rv;
    if (!gsync_sum(P, sm.red, SL_RV, rv)) { out.status = TSFDE_ETIMEOUT; return out; }
    if (!isfinite(rv)) { out.status = TSFDE_ENONFINITE; return out; }
    if (rv == 0.0) { out.status = TSFDE_EBREAKDOWN; return out; }
    alpha = rho / rv;
    // s = r - alpha v, in pairs
    {
      const R aR = (R)alpha;
      auto pro = [&](PairTag, int i0) -> cplx<R> {
        const cplx<R> r2 = ld_pair(V.r, i0), v2 = ld_pair(V.v, i0);
        const cplx<R> q = mkc<R>(r2.x - aR * v2.x, r2.y - aR * v2.y);
        st_pair(V.s, i0, q);
        if (TR && !prec) {
          const cplx<R> k2 = mkc<R>(kap[i0], i0 + 1 < n ? kap[i0 + 1] : R(0));
          return mkc<R>(k2.x * q.x, k2.y * q.y);
        }
        return q;
      };
      passA_real<R, false, KP>(P, sm, n, pro);
    }
    if (!gsync(P, sm.red)) { out.status = TSFDE_ETIMEOUT; return out; }
    if (prec) {
      passB<R, MID_APPLY, KP>(P, sm, saG<R>(P), sbG<R>(P), nullptr, nullptr, nullptr);
      if (!gsync(P, sm.red)) { out.status = TSFDE_ETIMEOUT; return out; }
      auto epi = [&](int i, R y) -> R { V.sh[i] = y; return TR ? kap[i] * y : y; };
      passCA_real<R, true, KP>(P, sm, epi);
      if (!gsync(P, sm.red)) { out.status = TSFDE_ETIMEOUT; return out; }
    }
    passB<R, MID_APPLY, KP>(P, sm, saT<R>(P), sbT<R>(P), nullptr, nullptr, nullptr);
    if (!gsync(P, sm.red)) { out.status = TSFDE_ETIMEOUT; return out; }
    const R* sh = prec ? V.sh : V.s;
    {
      R ats = 0, att = 0;
      auto epi = [&](int i, R y) -> R {
        const R ti = a * sh[i] + (TR ? y : kap[i] * y);
        V.t[i] = ti;
        ats += ti * V.s[i];
        att += ti * ti;
        return R(0);
      };
      passCA_real<R, false, KP>(P, sm, epi);
      put_partial(P, SL_TS, block_sum((double)ats, sm.red));
      put_partial(P, SL_TT, block_sum((double)att, sm.red));
    }
    double ts, tt;
    if (!gsync_sum2(P, sm.red, SL_TS, SL_TT, 0u, ts, tt)) { out.status = TSFDE_ETIMEOUT; return out; }
    omega = (tt > 0.0) ? ts / tt : 0.0;
    if (!isfinite(omega)) { out.status = TSFDE_ENONFINITE; return out; }
    // x += alpha p^ + omega s^, r = s - omega t
    {
      const R aR = (R)alpha, oR = (R)omega;
      R arr = 0, ar2 = 0;
      for (int i = gtid; i < n; i += gstr) {
        V.x[i] = V.x[i] + aR * ph[i] + oR * sh[i];
        const R ri = V.s[i] - oR * V.t[i];
        V.r[i] = ri;
        arr += V.rh[i] * ri;
        ar2 += ri * ri;
      }
      put_partial(P, SL_RR0, block_sum((double)arr, sm.red));
      put_partial(P, SL_RR, block_sum((double)ar2, sm.red));
    }
    if (!gsync_sum2(P, sm.red, SL_RR0, SL_RR, 0u, rho_new, rr)) { out.status = TSFDE_ETIMEOUT; return out; }
  }
}

// ------------------------------------------------------------------ PCG
// Preconditioned conjugate gradients on the symmetrised level system.
// Sec. 4.2 proposes PCG for kappa(x, t) = kappa(t), where the level matrix
// itself is SPD.  For a general kappa, with K = diag(kappa) > 0,
// (ahat I + K A) x = b is equivalent to S x = K^{-1} b with
// S = ahat K^{-1} + A, which is symmetric positive definite (A is, by the
// proposition after Eq. (3.16x); ahat K^{-1} is a positive diagonal), so CG
// applies with the SPD circulant preconditioner
// ahat/kbar I + s(A) = (ahat I + kbar s(A))/kbar: the Strang preconditioner
// of Eq. (4.3) up to a constant factor, which leaves the CG iterates
// unchanged, so its spectrum tables serve as they are.  One product with A
// and one with P^{-1} per iteration (BiCGSTAB needs two of each).  The
// residual r of S relates to the original one by b - (ahat I + K A) x =
// K r, and the stopping test is on that: ||K r|| < tol ||b||, the same
// criterion as bicgstab's.  hinv = 1/kappa.
// Per iteration five grid phases.  The column transforms are linear, so the
// transform of p = z + beta p_old is F(z) + beta F(p_old): F(z) comes out of
// the pass that produces z (its inverse column FFTs fused with the forward
// ones), F(p_old) is kept in the spare half of S1, and the row pass of the
// product with A loads their combination; the spatial p is formed in that
// product's epilogue.  Phases: row pass (A) on F(z) + beta F(p) | q = S p,
// (p, q) | x += alpha p, r -= alpha q, ||K r||, forward column FFTs of r |
// row pass (P^{-1}) | z = P^{-1} r, (r, z), forward column FFTs of z.
// Without a preconditioner z = r and the last two phases drop out.
// TR selects the transposed level system (ahat I + A K) lambda = g of the
// adjoint sweep: with mu = K lambda it reads (ahat K^{-1} + A) mu = g, the
// same S with the right-hand side g itself, and its residual g - S mu is
// that of the transposed system, so r starts at g and the test is on ||r||.
// The caller recovers lambda = K^{-1} mu.
template <typename R, class BInit, int KP = kPre, bool TR = false>
__device__ SolveRes pcg(const DevPlan& P, const Smem<R>& sm, const KVecs<R>& V,
                        const R* __restrict__ kap, const R* __restrict__ hinv, double ahat,
                        bool prec, double tol, int max_it, BInit& binit) {
  const int n = P.n;
  const R a = (R)ahat;
  SolveRes out{TSFDE_OK, 0, 0.0};
  // x = 0, p = 0, r = K^{-1} b and its forward column FFTs, ||b|| (and,
  // without a preconditioner, rho = (r, r)).  p must hold no stale
  // non-finite value: 0 * NaN is NaN.
  {
    R acc = 0, arr = 0;
    auto pro = [&](int i) -> R {
      const R bi = binit(i);
      const R ri = TR ? bi : bi * hinv[i];
      V.x[i] = R(0);
      V.p[i] = R(0);
      V.r[i] = ri;
      acc += bi * bi;
      arr += ri * ri;
      return ri;
    };
    passA_real<R, false, KP>(P, sm, n, pro);
    put_partial(P, SL_BB, block_sum((double)acc, sm.red));
    put_partial(P, SL_RR0, block_sum((double)arr, sm.red));
  }
  double bb, rho;
  if (!gsync_sum2(P, sm.red, SL_BB, SL_RR0, 0u, bb, rho)) { out.status = TSFDE_ETIMEOUT; return out; }
  if (!isfinite(bb)) { out.status = TSFDE_ENONFINITE; return out; }
  if (bb == 0.0) return out;
  const double nb = sqrt(bb);
  const R* z = prec ? V.s : V.r;
  // z = P^{-1} r from the forward column FFTs of r in S1, rho = (r, z); the
  // same tile pass computes the forward column FFTs of z into S1
  auto precond = [&](double& rho_out) -> bool {
    passB<R, MID_APPLY, KP>(P, sm, saG<R>(P), sbG<R>(P), nullptr, nullptr, nullptr);
    if (!gsync(P, sm.red)) return false;
    R acc = 0;
    auto epi = [&](int i, R y) -> R {
      V.s[i] = y;
      acc += V.r[i] * y;
      return y;
    };
    passCA_real<R, true, KP>(P, sm, epi);
    put_partial(P, SL_RR0, block_sum((double)acc, sm.red));
    return gsync_sum(P, sm.red, SL_RR0, rho_out);
  };
  if (prec && !precond(rho)) { out.status = TSFDE_ETIMEOUT; return out; }
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
    const bool first = it == 0;
    out.iters = ++it;
    // row pass of A on F(p) = F(z) + beta F(p_old)
    {
      cplx<R>* Fp = reinterpret_cast<cplx<R>*>(P.S1) + P.Nc;  // F(p), kept between iterations
      const RowIn<R> in{reinterpret_cast<const cplx<R>*>(P.S1), first ? nullptr : Fp, (R)beta, nullptr, R(0), Fp};
      passB<R, MID_APPLY, KP, true>(P, sm, saT<R>(P), sbT<R>(P), nullptr, nullptr, nullptr, &in);
    }
    if (!gsync(P, sm.red)) { out.status = TSFDE_ETIMEOUT; return out; }
    // p = z + beta p, q = S p = ahat K^{-1} p + A p, (p, q)
    {
      const R bR = (R)beta;
      R acc = 0;
      auto epi = [&](int i, R y) -> R {
        const R pi = first ? z[i] : z[i] + bR * V.p[i];
        V.p[i] = pi;
        const R qi = a * hinv[i] * pi + y;
        V.v[i] = qi;
        acc += pi * qi;
        return R(0);
      };
      passCA_real<R, false, KP>(P, sm, epi);
      put_partial(P, SL_RV, block_sum((double)acc, sm.red));
    }
    double pq;
    if (!gsync_sum(P, sm.red, SL_RV, pq)) { out.status = TSFDE_ETIMEOUT; return out; }
    if (!isfinite(pq)) { out.status = TSFDE_ENONFINITE; return out; }
    if (!(pq > 0.0)) { out.status = TSFDE_EBREAKDOWN; return out; }
    const double alpha = rho / pq;
    // x += alpha p, r -= alpha q, ||K r||^2 (and (r, r) without a
    // preconditioner), forward column FFTs of r
    {
      const R aR = (R)alpha;
      R acc = 0, arr = 0;
      auto pro = [&](int i) -> R {
        V.x[i] = V.x[i] + aR * V.p[i];
        const R ri = V.r[i] - aR * V.v[i];
        V.r[i] = ri;
        const R kr = TR ? ri : kap[i] * ri;
        acc += kr * kr;
        arr += ri * ri;
        return ri;
      };
      passA_real<R, false, KP>(P, sm, n, pro);
      put_partial(P, SL_RR, block_sum((double)acc, sm.red));
      put_partial(P, SL_RR0, block_sum((double)arr, sm.red));
    }
    double rho_np;
    if (!gsync_sum2(P, sm.red, SL_RR, SL_RR0, 0u, rr, rho_np)) { out.status = TSFDE_ETIMEOUT; return out; }
    if (sqrt(rr) / nb < tol) {
      out.relres = sqrt(rr) / nb;
      out.iters = it;
      if (!isfinite(out.relres)) out.status = TSFDE_ENONFINITE;
      return out;
    }
    double rho_new = rho_np;
    if (prec && !precond(rho_new)) { out.status = TSFDE_ETIMEOUT; return out; }
    beta = rho_new / rho;
    rho = rho_new;
  }
}

// The Krylov solve of a level, (ahat I + K A) x = b in arithmetic R: PCG on
// the symmetrised system, or the paper's BiCGSTAB (hinv unused).
template <bool PCG, int KP, typename R, class BInit>
__device__ SolveRes level_krylov(const DevPlan& P, const Smem<R>& sm, const KVecs<R>& V,
                                 const R* __restrict__ kap, const R* __restrict__ hinv, double ahat,
                                 bool prec, double tol, int max_it, BInit& binit) {
  if constexpr (PCG)
    return pcg<R, BInit, KP>(P, sm, V, kap, hinv, ahat, prec, tol, max_it, binit);
  else
    return bicgstab<R, BInit, false, KP>(P, sm, V, kap, ahat, prec, tol, max_it, binit);
}

static __device__ double mean_kappa(const DevPlan& P, const double* kap, double* red) {
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gstr = gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int i = gtid; i < P.n; i += gstr) acc += kap[i];
  put_partial(P, SL_KAP, block_sum(acc, red));
  double tot;
  if (!gsync_sum(P, red, SL_KAP, tot)) return -1.0;
  return tot / (double)P.n;
}

static __device__ void write_stat(StepStat* st, int status, int iters, int outer, double relres) {
  if (st && blockIdx.x == 0 && threadIdx.x == 0) {
    st->status = status;
    st->iterations = iters;
    st->outer = outer;
    st->rel_residual = relres;
  }
}


// Warm start of a level solve: u = x0 and r64 = b - (ahat I + K A) x0, with
// x0 = u_prev, or the extrapolation of order A.xorder from the earlier
// levels A.up (one FP64 product); returns b.b and r.r (grid-wide, in every
// CTA).
template <int KP = kPre>
__device__ bool warm_residual(const LevelArgs& A, SmemAll& S, double& bb, double& rr) {
  const DevPlan& P = A.P;
  const int q = A.xorder;
  auto pro = [&](int i) -> double {
    double x = A.u_prev[i];
    if (q > 0) {
      double v[kMaxStartOrder + 1];
#pragma unroll
      for (int j = 1; j <= kMaxStartOrder; ++j)
        if (j <= q) v[j] = A.up[j][i];
      x *= A.xw[0];
#pragma unroll
      for (int j = 1; j <= kMaxStartOrder; ++j)
        if (j <= q) x = fma(A.xw[j], v[j], x);
    }
    A.u[i] = x;
    return x;
  };
  passA_real<double, false, KP>(P, S.d, P.n, pro);
  if (!gsync(P, S.d.red)) return false;
  passB<double, MID_APPLY, KP>(P, S.d, P.saT64, P.sbT64, nullptr, nullptr, nullptr);
  if (!gsync(P, S.d.red)) return false;
  double bacc = 0.0, racc = 0.0;
  auto epi = [&](int i, double y) -> double {
    const double bi = A.b[i];
    const double ri = bi - (A.ahat * A.u[i] + A.kappa64[i] * y);
    A.r64[i] = ri;
    bacc += bi * bi;
    racc += ri * ri;
    return 0.0;
  };
  passCA_real<double, false, KP>(P, S.d, epi);
  put_partial(P, SL_BB, block_sum(bacc, S.d.red));
  put_partial(P, SL_RES, block_sum(racc, S.d.red));
  return gsync_sum2(P, S.d.red, SL_BB, SL_RES, 0u, bb, rr);
}

// Mixed level solve (shared by both engines and both inner arithmetics).
// conv(k), called for every k < Nc after the preconditioner build, rounds
// entry k of the FP64 preconditioner spectrum into the inner solver's
// tables (and whatever else the inner solver needs rounded);
// inner(sc, target, res) solves (ahat I + K A) e = sc r64 in the inner
// arithmetic into e (false on a barrier timeout); target = tol ||b|| / ||r||
// is the relative reduction that would meet the FP64 path's criterion.
// FP64 refinement around a lower-precision PBiCGSTAB: each sweep
// solves (ahat I + K A) e = r / ||r|| (at most inner_max_it
// iterations), forms w = M e in FP64 and updates u += theta e,
// r -= theta w with theta = 1, or the minimal-residual
// theta = (r, w)/(w, w) when the full step would raise ||r||, so the FP64
// residual never grows.  Stops when a step after the first satisfies
// max|theta e| <= tol max|u|, or ||r|| <= tol ||b|| (the FP64 path's
// criterion, on the true residual), or when a sweep no longer halves ||r|| with
// ||r||/||b|| <= 1e-9 (its rounding floor at large n) and the step is below
// 100 tol max|u|.  After three sweeps
// without progress above that, or at max_outer, the level is finished by
// FP64 PBiCGSTAB on the remaining residual, so a level never returns an
// unconverged answer.  PCG selects the Krylov method of that FP64 finish
// (the inner solves choose their own).
// PRE: the caller's preconditioner is always built by a separate launch
// (A.prebuilt; the in-kernel FP64 build is then not compiled in).
template <bool PCG = false, int KP = kPre, bool PRE = false, typename RI, class Conv, class Inner>
__device__ void mixed_level(const LevelArgs& A, SmemAll& S, Conv& conv, Inner& inner, const RI* e) {
  const DevPlan& P = A.P;
  const int n = P.n;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gstr = gridDim.x * blockDim.x;
  if (PRE || A.prebuilt) {
    // built by k_precond_ds before this launch
    const int st = A.precond ? __ldcg(A.pre_status) : TSFDE_OK;
    if (st != TSFDE_OK) { write_stat(A.stat, st, 0, 0, 0.0); return; }
  } else if constexpr (!PRE) {
    const double kbar = mean_kappa(P, A.kappa64, S.d.red);
    if (kbar < 0.0) { write_stat(A.stat, TSFDE_ETIMEOUT, 0, 0, 0.0); return; }
    // The preconditioner is built in FP64 and rounded to FP32; building it in
    // FP32 would bury its smallest eigenvalues (1/(ahat + kbar lambda_max),
    // ~1e-8 of the largest at n = 2^17-1) under rounding.
    if (A.precond && !build_precond<double, KP>(P, S.d, A.ahat, kbar)) {
      write_stat(A.stat, TSFDE_ETIMEOUT, 0, 0, 0.0);
      return;
    }
  }
  double bb, rr0;
  {
    for (int k = gtid; k < P.Nc; k += gstr) conv(k);
    if (A.u_prev) {
      if (!warm_residual<KP>(A, S, bb, rr0)) { write_stat(A.stat, TSFDE_ETIMEOUT, 0, 0, 0.0); return; }
    } else {
      double acc = 0.0;
      for (int i = gtid; i < n; i += gstr) {
        const double bi = A.b[i];
        A.u[i] = 0.0;
        A.r64[i] = bi;
        acc += bi * bi;
      }
      put_partial(P, SL_RES, block_sum(acc, S.d.red));
      if (!gsync_sum(P, S.d.red, SL_RES, bb)) { write_stat(A.stat, TSFDE_ETIMEOUT, 0, 0, 0.0); return; }
      rr0 = bb;
    }
  }
  if (!isfinite(bb) || !isfinite(rr0)) { write_stat(A.stat, TSFDE_ENONFINITE, 0, 0, 0.0); return; }
  if (bb == 0.0 || rr0 == 0.0) { write_stat(A.stat, TSFDE_OK, 0, 0, 0.0); return; }
  const double nb = sqrt(bb);
  double nr = sqrt(rr0), relres = nr / nb;
  int inner_total = 0, outer = 0, status = TSFDE_OK, stalls = 0;
  // After a level that needed the FP64 finish, go to it directly (the
  // levels grow harder along the graded mesh), retrying the refinement on
  // the levels the host marks.
  bool fallback = A.prev && !A.retry_mixed && __ldcg(&A.prev->outer) < 0;
  if (!fallback && relres <= A.tol) { write_stat(A.stat, TSFDE_OK, 0, 0, relres); return; }
  double* w = A.k64.v;  // FP64 scratch for M e
  while (!fallback) {
    if (outer >= A.max_outer) { fallback = true; break; }
    SolveRes ir{TSFDE_OK, 0, 0.0};
    if (!inner(1.0 / nr, A.tol * nb / nr, ir)) { status = TSFDE_ETIMEOUT; break; }
    inner_total += ir.iters;
    ++outer;
    // An inner solve that hit its iteration cap (or broke down after some
    // iterations) still leaves a usable correction: the FP64 step below
    // accepts it only if it lowers the FP64 residual.  One that produced a
    // non-finite value, or stopped before its first iteration, leaves none:
    // the level goes to the FP64 finish.
    if (ir.status == TSFDE_ENONFINITE ||
        (ir.status != TSFDE_OK && ir.status != TSFDE_ENOCONV && ir.iters == 0)) {
      fallback = true;
      break;
    }
    // w = M (nr e) in FP64
    const double ah = A.ahat;
    auto pro = [&](int i) -> double { return nr * (double)e[i]; };
    passA_real<double, false, KP>(P, S.d, n, pro);
    if (!gsync(P, S.d.red)) { status = TSFDE_ETIMEOUT; break; }
    passB<double, MID_APPLY, KP>(P, S.d, P.saT64, P.sbT64, nullptr, nullptr, nullptr);
    if (!gsync(P, S.d.red)) { status = TSFDE_ETIMEOUT; break; }
    {
      double rw = 0.0, ww = 0.0;
      auto epi = [&](int i, double y) -> double {
        const double wi = ah * nr * (double)e[i] + A.kappa64[i] * y;
        w[i] = wi;
        rw += A.r64[i] * wi;
        ww += wi * wi;
        return 0.0;
      };
      passCA_real<double, false, KP>(P, S.d, epi);
      put_partial(P, SL_RV, block_sum(rw, S.d.red));
      put_partial(P, SL_TT, block_sum(ww, S.d.red));
    }
    double rw, ww;
    if (!gsync_sum2(P, S.d.red, SL_RV, SL_TT, 0u, rw, ww)) { status = TSFDE_ETIMEOUT; break; }
    // full step unless it would raise ||r||: ||r - w||^2 = ||r||^2 - 2 (r,w) + (w,w)
    double theta = 1.0;
    if (ww - 2.0 * rw > 0.0) theta = (ww > 0.0) ? rw / ww : 0.0;
    if (!isfinite(theta) || !(theta > 0.0)) { fallback = true; break; }
    {
      double rr = 0.0, emax = 0.0, xmax = 0.0;
      const double step = theta * nr;
      for (int i = gtid; i < n; i += gstr) {
        const double di = step * (double)e[i];
        const double xi = A.u[i] + di;
        A.u[i] = xi;
        const double ri = A.r64[i] - theta * w[i];
        A.r64[i] = ri;
        rr += ri * ri;
        emax = fmax(emax, fabs(di));
        xmax = fmax(xmax, fabs(xi));
      }
      put_partial(P, SL_RES, block_sum(rr, S.d.red));
      put_partial(P, SL_EMAX, block_max(emax, S.d.red));
      put_partial(P, SL_XMAX, block_max(xmax, S.d.red));
    }
    double rr, emax, xmax;
    if (!gsync_sum3(P, S.d.red, SL_RES, SL_EMAX, SL_XMAX, 6u, rr, emax, xmax)) {
      status = TSFDE_ETIMEOUT;
      break;
    }
    const double nr_prev = nr;
    nr = sqrt(rr);
    if (!isfinite(nr) || !isfinite(xmax)) { status = TSFDE_ENONFINITE; break; }
    relres = nr / nb;
    if (nr == 0.0 || relres <= A.tol) break;
    // a zero correction cannot make progress: never read it as converged
    if (!(emax > 0.0)) { fallback = true; break; }
    // a small step ends the refinement from the second sweep on; the first
    // sweep's step only measures how good the starting point was (a warm or
    // extrapolated start leaves it small while ||r|| is still above tol)
    if (outer >= 2 && emax <= A.tol * xmax) break;
    if (outer >= 2 && nr > 0.5 * nr_prev) {
      // the FP64 residual is at its rounding floor and u no longer moves at
      // the accuracy asked for
      if (relres <= 1e-9 && emax <= 100.0 * A.tol * xmax) break;
      if (++stalls >= 3) { fallback = true; break; }
    } else {
      stalls = 0;
    }
  }
  if (fallback && status == TSFDE_OK) {
    // finish in FP64: solve M d = r to the requested overall tolerance
    KVecs<double> V = A.k64;
    auto binit = [&](int i) -> double { return A.r64[i]; };
    const double tol_d = fmax(A.tol * nb / nr, 1e-14);
    SolveRes fr = level_krylov<PCG, KP>(P, S.d, V, A.kappa64, A.hinv64, A.ahat, A.precond != 0,
                                        tol_d, A.max_it, binit);
    if (fr.status == TSFDE_OK) {
      for (int i = gtid; i < n; i += gstr) A.u[i] += V.x[i];
      relres = fr.relres * nr / nb;
      if (!gsync(P, S.d.red)) fr.status = TSFDE_ETIMEOUT;
    }
    status = fr.status;
    inner_total += fr.iters;
    outer = -(outer > 0 ? outer : 1);  // negative: the level was finished in FP64
  }
  write_stat(A.stat, status, inner_total, outer, relres);
}

}  // namespace tsfde
