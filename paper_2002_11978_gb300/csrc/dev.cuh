// dev.cuh -- device primitives for the FIDS hot path on sm_103a:
// complex arithmetic, a bounded grid barrier, a shared-memory Stockham
// radix-4/2 FFT over a batch of short sequences, and deterministic
// block/grid reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dsf.cuh"
#include "plan.h"

namespace tsfde {

// ----------------------------------------------------------------- complex
template <typename R> struct CT;
template <> struct CT<double> { using T = double2; };
template <> struct CT<float> { using T = float2; };
template <> struct CT<dsf> { using T = dsf2; };
template <typename R> using cplx = typename CT<R>::T;

template <typename R> __device__ __forceinline__ cplx<R> mkc(R x, R y) {
  cplx<R> c; c.x = x; c.y = y; return c;
}
template <typename Z> __device__ __forceinline__ Z cadd(Z a, Z b) { a.x += b.x; a.y += b.y; return a; }
template <typename Z> __device__ __forceinline__ Z csub(Z a, Z b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename Z> __device__ __forceinline__ Z cconj(Z a) { a.y = -a.y; return a; }
template <typename Z> __device__ __forceinline__ Z cmul(Z a, Z b) {
  Z c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
// a * conj(b)
template <typename Z> __device__ __forceinline__ Z cmulc(Z a, Z b) {
  Z c; c.x = a.x * b.x + a.y * b.y; c.y = a.y * b.x - a.x * b.y; return c;
}
template <typename Z, typename R> __device__ __forceinline__ Z cscale(Z a, R s) { a.x *= s; a.y *= s; return a; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename Z> __device__ __forceinline__ Z mul_mi(Z a) {
  Z c;
  if (INV) { c.x = -a.y; c.y = a.x; } else { c.x = a.y; c.y = -a.x; }
  return c;
}

// ----------------------------------------------------------- grid barrier
// count/gen/err (GridBarrier, plan.h) live in device memory and are cleared
// by the host before every cooperative launch.  A CTA that waits longer than
// `timeout` SM cycles sets err and stops waiting; every later barrier then
// returns false at once, so the kernel unwinds instead of hanging.

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// --------------------------------------------------- shared-memory FFT
// The shared twiddle table W_T^i is stored with one spare entry after every
// eight (entry i at tpad(i)): the radix-4 stages read it with strides
// T/(4 Ns), multiples of 8 entries (128 bytes for 16-byte entries) in the
// middle stages, which would put up to 16 lanes of a warp on the same banks.
__host__ __device__ __forceinline__ int tpad(int i) { return i + (i >> 3); }
// Entries of the padded table for a table of T, rounded up to even so that
// the following tables stay 16-byte aligned.
__host__ __device__ __forceinline__ int tpad_len(int T) { return (T + (T >> 3) + 1) & ~1; }

// Stockham autosort FFT (radix 4, one radix-2 stage when log2 N is odd) of
// B independent length-N sequences held in shared memory with layout
// [k][b] (element k of sequence b at k*B + b).  `a` holds the input, `b`
// is scratch of the same size; the function returns whichever buffer holds
// the result.  tw[tpad(k)] = e^{-2 pi i k / T} for k < T, T >= N a power of
// two.
// INV selects e^{+...}; neither direction normalises.
template <typename R, bool INV>
__device__ __forceinline__ cplx<R>* fft_batch(cplx<R>* a, cplx<R>* b, int N, int lgB,
                                              const cplx<R>* __restrict__ tw, int T) {
  typedef cplx<R> Z;
  Z* in = a;
  Z* out = b;
  const int B = 1 << lgB;
  int Ns = 1;
#pragma unroll 1
  while (Ns < N) {
    if (N / Ns >= 4) {
      const int Q = N >> 2;
      const int total = Q << lgB;
      const int st = T / (Ns << 2);
#pragma unroll 1
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int bb = t & (B - 1);
        const int j = t >> lgB;
        const int k = j & (Ns - 1);
        Z v0 = in[(j << lgB) + bb];
        Z v1 = in[((j + Q) << lgB) + bb];
        Z v2 = in[((j + 2 * Q) << lgB) + bb];
        Z v3 = in[((j + 3 * Q) << lgB) + bb];
        if (Ns > 1) {
          Z w1 = tw[tpad(k * st)], w2 = tw[tpad(2 * k * st)], w3 = tw[tpad(3 * k * st)];
          if (INV) { w1 = cconj(w1); w2 = cconj(w2); w3 = cconj(w3); }
          v1 = cmul(v1, w1); v2 = cmul(v2, w2); v3 = cmul(v3, w3);
        }
        Z a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3);
        Z a3 = mul_mi<INV>(csub(v1, v3));
        const int base = ((j - k) << 2) + k;
        out[(base << lgB) + bb] = cadd(a0, a2);
        out[((base + Ns) << lgB) + bb] = cadd(a1, a3);
        out[((base + 2 * Ns) << lgB) + bb] = csub(a0, a2);
        out[((base + 3 * Ns) << lgB) + bb] = csub(a1, a3);
      }
      Ns <<= 2;
    } else {
      const int H = N >> 1;
      const int total = H << lgB;
      const int st = T / (Ns << 1);
#pragma unroll 1
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int bb = t & (B - 1);
        const int j = t >> lgB;
        const int k = j & (Ns - 1);
        Z v0 = in[(j << lgB) + bb];
        Z v1 = in[((j + H) << lgB) + bb];
        if (Ns > 1) {
          Z w = tw[tpad(k * st)];
          if (INV) w = cconj(w);
          v1 = cmul(v1, w);
        }
        const int base = ((j - k) << 1) + k;
        out[(base << lgB) + bb] = cadd(v0, v1);
        out[((base + Ns) << lgB) + bb] = csub(v0, v1);
      }
      Ns <<= 1;
    }
    __syncthreads();
    Z* tmp = in; in = out; out = tmp;
  }
  return in;
}

// ------------------------------------------- register-blocked FFT stages
// W_16^m = e^{-2 pi i m/16}; m is a compile-time constant after unrolling,
// so the switch folds to literals (cos/sin of multiples of pi/8).
template <typename R> __device__ __forceinline__ cplx<R> w16(int m) {
  const R c1 = R(0.92387953251128674), s1 = R(0.38268343236508977), c2 = R(0.70710678118654752);
  switch (m & 15) {
    case 0: return mkc<R>(R(1), R(0));
    case 1: return mkc<R>(c1, -s1);
    case 2: return mkc<R>(c2, -c2);
    case 3: return mkc<R>(s1, -c1);
    case 4: return mkc<R>(R(0), R(-1));
    case 5: return mkc<R>(-s1, -c1);
    case 6: return mkc<R>(-c2, -c2);
    case 7: return mkc<R>(-c1, -s1);
    case 8: return mkc<R>(R(-1), R(0));
    case 9: return mkc<R>(-c1, s1);
    case 10: return mkc<R>(-c2, c2);
    case 11: return mkc<R>(-s1, c1);
    case 12: return mkc<R>(R(0), R(1));
    case 13: return mkc<R>(s1, c1);
    case 14: return mkc<R>(c2, c2);
    default: return mkc<R>(c1, s1);
  }
}

// x * W_16^m (conjugate twiddle when INV), with the trivial multipliers
// (1, -1, -i, +i) done as swaps.
template <typename R, bool INV> __device__ __forceinline__ cplx<R> mul_w16(cplx<R> x, int m) {
  m &= 15;
  if (INV) m = (16 - m) & 15;
  if (m == 0) return x;
  if (m == 8) return mkc<R>(-x.x, -x.y);
  if (m == 4) return mkc<R>(x.y, -x.x);
  if (m == 12) return mkc<R>(-x.y, x.x);
  return cmul(x, w16<R>(m));
}

// In-register DFT of RAD (2..16, power of two) points in natural order:
// Stockham radix-2 steps over the register array, fully unrolled.
template <typename R, int RAD, bool INV> __device__ __forceinline__ void dft_reg(cplx<R>* v) {
  typedef cplx<R> Z;
  Z a[RAD], b[RAD];
#pragma unroll
  for (int r = 0; r < RAD; ++r) a[r] = v[r];
#pragma unroll
  for (int ns = 1; ns < RAD; ns <<= 1) {
#pragma unroll
    for (int j = 0; j < RAD / 2; ++j) {
      const int k = j & (ns - 1);
      const Z x0 = a[j];
      const Z x1 = mul_w16<R, INV>(a[j + RAD / 2], k * (16 / (2 * ns)));
      const int base = ((j - k) << 1) + k;
      b[base] = cadd(x0, x1);
      b[base + ns] = csub(x0, x1);
    }
#pragma unroll
    for (int r = 0; r < RAD; ++r) a[r] = b[r];
  }
#pragma unroll
  for (int r = 0; r < RAD; ++r) v[r] = a[r];
}

// Accessors of a batch held in shared memory with layout [k][b].
template <typename R> struct BufIn {
  const cplx<R>* p;
  int lgB;
  __device__ __forceinline__ cplx<R> operator()(int k, int b) const { return p[(k << lgB) + b]; }
};
template <typename R> struct BufOut {
  cplx<R>* p;
  int lgB;
  __device__ __forceinline__ void operator()(int k, int b, cplx<R> z) const { p[(k << lgB) + b] = z; }
};

// One radix-RAD Stockham stage over B = 2^lgB sequences of length N; Ns is
// the length of the sub-transforms already done.  in(k, b) fetches element k
// of sequence b, out(k, b, z) stores it; each is called once per element.
// tw[k] = e^{-2 pi i k/T}, T >= N a power of two.
template <typename R, bool INV, int RAD, class In, class Out>
__device__ __forceinline__ void fft_stage_f(In& in, Out& out, int N, int Ns, int lgB,
                                            const cplx<R>* __restrict__ tw, int T) {
  typedef cplx<R> Z;
  const int Q = N / RAD;
  const int B = 1 << lgB;
  const int total = Q << lgB;
  const int st = T / (Ns * RAD);
#pragma unroll 1
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int bb = t & (B - 1);
    const int j = t >> lgB;
    const int k = j & (Ns - 1);
    Z v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = in(j + r * Q, bb);
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        Z w = tw[r * k * st];
        if (INV) w = cconj(w);
        v[r] = cmul(v[r], w);
      }
    }
    dft_reg<R, RAD, INV>(v);
    const int base = (j - k) * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) out(base + r * Ns, bb, v[r]);
  }
}

template <typename R, bool INV, class In, class Out>
__device__ __forceinline__ void fft_stage_any(int rad, In& in, Out& out, int N, int Ns, int lgB,
                                              const cplx<R>* __restrict__ tw, int T) {
  switch (rad) {
    case 16: fft_stage_f<R, INV, 16>(in, out, N, Ns, lgB, tw, T); break;
    case 8: fft_stage_f<R, INV, 8>(in, out, N, Ns, lgB, tw, T); break;
    case 4: fft_stage_f<R, INV, 4>(in, out, N, Ns, lgB, tw, T); break;
    default: fft_stage_f<R, INV, 2>(in, out, N, Ns, lgB, tw, T); break;
  }
}

// Number of stages fft_pipe takes for a length-2^lgN transform.
__host__ __device__ __forceinline__ int pipe_stages(int lgN) { return (lgN + 3) >> 2; }

// Batched FFT of length N = 2^lgN (>= 2) in radix-16 Stockham stages, the
// last one of radix 2^(lgN mod 4) when 4 does not divide lgN.  The first
// stage reads through ld, the last writes through st, and the stages in
// between alternate between shared buffers first, second, first, ... (each
// N << lgB elements).  ld must not read `first`, and st must not write the
// buffer the last stage reads (stage s >= 1 writes `first` for odd s).
// Ends with __syncthreads().
template <typename R, bool INV, class Ld, class St>
__device__ __forceinline__ void fft_pipe(int lgN, int lgB, Ld& ld, St& st, cplx<R>* first,
                                         cplx<R>* second, const cplx<R>* __restrict__ tw, int T) {
  const int N = 1 << lgN;
  const int ns = pipe_stages(lgN);
  if (ns == 1) {
    fft_stage_any<R, INV>(N, ld, st, N, 1, lgB, tw, T);
    __syncthreads();
    return;
  }
  {
    BufOut<R> o{first, lgB};
    fft_stage_f<R, INV, 16>(ld, o, N, 1, lgB, tw, T);
    __syncthreads();
  }
  cplx<R>* cur = first;
  cplx<R>* nxt = second;
  int Ns = 16;
#pragma unroll 1
  for (int s = 1; s < ns - 1; ++s) {
    BufIn<R> i{cur, lgB};
    BufOut<R> o{nxt, lgB};
    fft_stage_f<R, INV, 16>(i, o, N, Ns, lgB, tw, T);
    __syncthreads();
    cplx<R>* tmp = cur;
    cur = nxt;
    nxt = tmp;
    Ns <<= 4;
  }
  BufIn<R> i{cur, lgB};
  fft_stage_any<R, INV>(N / Ns, i, st, N, Ns, lgB, tw, T);
  __syncthreads();
}

// ------------------------------------------------------------ reductions
// Block sum of one double per thread; result valid in every thread.
// red: 33 doubles of shared scratch.  Fixed order -> deterministic.
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double x = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (l == 0) red[32] = x;
  }
  __syncthreads();
  return red[32];
}
__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double x = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (l == 0) red[32] = x;
  }
  __syncthreads();
  return red[32];
}

// ------------------------------------------------------- grid barrier
// Barrier over all CTAs of a cooperative launch that can also reduce
// per-CTA partial sums.  Thread 0 of each CTA adds one arrival with an
// acquire-release atomic; the value it returns gives the barrier's epoch
// k = old/G + 1, and the CTA waits (bounded) until the counter reaches k G.
// No CTA has to release the others, so the barrier costs one atomic and the
// polling (measured on GB300 with 304 CTAs: 2.1 us, against 3.7 us for a
// fence / atomic / fence arrival with a separate release word).  Every CTA
// then reduces the requested partial slots itself, in one fixed order, so
// all CTAs see bitwise the same values.  The partials of barrier k live in
// buffer k mod 2 (put_partial writes the buffer of the CTA's next barrier):
// a buffer is rewritten only for barrier k + 2, after every CTA has passed
// barrier k + 1 and so finished reading it.  On a timeout err is set, later
// barriers return false at once and the kernel unwinds.
// red: >= 64 doubles of shared scratch.  out: nred values, in every thread.

// Grid barriers this CTA has passed; grid_epoch_init() clears it at the
// start of every kernel that uses the grid barrier.
static __shared__ unsigned s_grid_epoch;
__device__ __forceinline__ void grid_epoch_init() {
  if (threadIdx.x == 0) s_grid_epoch = 0u;
  __syncthreads();
}
// Partial-sum buffer of the CTA's next barrier (part holds 2 x kSlots x G).
__device__ __forceinline__ double* grid_partials_next(double* part, int G) {
  return part + (size_t)((s_grid_epoch + 1u) & 1u) * kSlots * G;
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ bool grid_sync_red(GridBarrier* gb, long long timeout,
                                              const double* part, int G, int nred,
                                              const int* slots, unsigned maxmask,
                                              double* out, double* red) {
  int* flag = reinterpret_cast<int*>(red + 48);
  __syncthreads();
  if (threadIdx.x == 0) {
    int f = 0;
    if (*(volatile int*)&gb->err == 0) {
      const unsigned old = atom_add_acq_rel(&gb->count, 1u);
      const unsigned k = old / (unsigned)G + 1u;
      const unsigned target = k * (unsigned)G;
      const long long t0 = clock64();
      f = 1;
      while (ld_acquire_u32(&gb->count) < target) {
        if (*(volatile int*)&gb->err != 0) { f = 0; break; }
        if (clock64() - t0 > timeout) {
          atomicOr(&gb->err, 1);
          f = 0;
          break;
        }
        __nanosleep(20);
      }
      s_grid_epoch = k;
    }
    flag[0] = f;
  }
  __syncthreads();
  if (!flag[0]) return false;
  const double* pk = part + (size_t)(s_grid_epoch & 1u) * kSlots * G;
  for (int q = 0; q < nred; ++q) {
    const double* p = pk + slots[q] * G;
    const bool mx = (maxmask >> q) & 1u;
    double v = 0.0;
    for (int c = threadIdx.x; c < G; c += blockDim.x) {
      const double y = __ldcg(p + c);
      v = mx ? fmax(v, y) : v + y;
    }
    out[q] = mx ? block_max(v, red) : block_sum(v, red);
  }
  return true;
}

}  // namespace tsfde
