// dev.cuh -- device primitives for the FIDS hot path on sm_103a:
// complex arithmetic, a bounded grid barrier, a shared-memory Stockham
// radix-4/2 FFT over a batch of short sequences, and deterministic
// block/grid reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "plan.h"

namespace tsfde {

// ----------------------------------------------------------------- complex
template <typename R> struct CT;
template <> struct CT<double> { using T = double2; };
template <> struct CT<float> { using T = float2; };
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

__device__ __forceinline__ bool grid_sync(GridBarrier* gb, long long timeout) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* errp = &gb->err;
    if (*errp == 0) {
      const unsigned g = ld_acquire_u32(&gb->gen);
      __threadfence();
      const unsigned old = atomicAdd(&gb->count, 1u);
      if (old == gridDim.x - 1) {
        atomicExch(&gb->count, 0u);
        __threadfence();
        st_release_u32(&gb->gen, g + 1u);
      } else {
        const long long t0 = clock64();
        while (ld_acquire_u32(&gb->gen) == g) {
          if (*errp != 0) break;
          if (clock64() - t0 > timeout) {
            atomicOr(&gb->err, 1);
            break;
          }
        }
      }
      __threadfence();
    }
  }
  __syncthreads();
  return *(volatile int*)&gb->err == 0;
}

// --------------------------------------------------- shared-memory FFT
// Stockham autosort FFT (radix 4, one radix-2 stage when log2 N is odd) of
// B independent length-N sequences held in shared memory with layout
// [k][b] (element k of sequence b at k*B + b).  `a` holds the input, `b`
// is scratch of the same size; the function returns whichever buffer holds
// the result.  tw[k] = e^{-2 pi i k / T} for k < T, T >= N a power of two.
// INV selects e^{+...}; neither direction normalises.
template <typename R, bool INV>
__device__ __forceinline__ cplx<R>* fft_batch(cplx<R>* a, cplx<R>* b, int N, int lgB,
                                              const cplx<R>* __restrict__ tw, int T) {
  typedef cplx<R> Z;
  Z* in = a;
  Z* out = b;
  const int B = 1 << lgB;
  int Ns = 1;
  while (Ns < N) {
    if (N / Ns >= 4) {
      const int Q = N >> 2;
      const int total = Q << lgB;
      const int st = T / (Ns << 2);
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int bb = t & (B - 1);
        const int j = t >> lgB;
        const int k = j & (Ns - 1);
        Z v0 = in[(j << lgB) + bb];
        Z v1 = in[((j + Q) << lgB) + bb];
        Z v2 = in[((j + 2 * Q) << lgB) + bb];
        Z v3 = in[((j + 3 * Q) << lgB) + bb];
        if (Ns > 1) {
          Z w1 = tw[k * st], w2 = tw[2 * k * st], w3 = tw[3 * k * st];
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
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int bb = t & (B - 1);
        const int j = t >> lgB;
        const int k = j & (Ns - 1);
        Z v0 = in[(j << lgB) + bb];
        Z v1 = in[((j + H) << lgB) + bb];
        if (Ns > 1) {
          Z w = tw[k * st];
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

// Sum (or max) of G per-CTA partials p[0..G), identical in every CTA:
// lane l adds p[l], p[l+32], ... in order, then a fixed xor tree.
template <bool MAX>
__device__ __forceinline__ double grid_reduce(const double* p, int G, double* red) {
  __syncthreads();
  if (threadIdx.x < 32) {
    const int l = threadIdx.x;
    double x = 0.0;
    for (int q = l; q < G; q += 32) {
      double y = __ldcg(p + q);
      x = MAX ? fmax(x, y) : x + y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = MAX ? fmax(x, y) : x + y;
    }
    if (l == 0) red[32] = x;
  }
  __syncthreads();
  return red[32];
}

}  // namespace tsfde
