// dsf.cuh -- double-single arithmetic on the FP32 pipes.
//
// A dsf value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2 (Dekker, "A floating-point technique for extending the
// available precision", Numer. Math. 18, 1971), about 48 significant bits.
// The operations are built from error-free transformations:
//   two_sum      Knuth's TwoSum: s + e == a + b exactly, any a, b;
//   fast_two_sum Dekker's Fast2Sum: the same when |a| >= |b| (or a == 0);
//   two_prod     p + e == a * b exactly, e from one fused multiply-add.
// Addition is the "sloppy" double-single sum (Hida, Li and Bailey, QD
// library report, 2000): the high parts are added exactly, the low parts in
// FP32, and the result renormalised.  Its error is bounded by a few u^2
// (|a| + |b|) with u = 2^-24, i.e. normwise, which is the bound an FFT
// error analysis needs; it is not relatively accurate under cancellation.
// Multiplication adds the two cross terms to the exact error of hi * hi,
// error a few u^2 |a b|.
//
// Every operation here is a handful of FP32 adds and FMAs (add 11, multiply
// 6): on GB300 that runs ~8x faster than the same operation in FP64, whose
// pipe is 1/58 of the FP32 rate.
#pragma once
#include <cuda_runtime.h>

#include "plan.h"

namespace tsfde {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dsf operator+(dsf a, dsf b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  dsf r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dsf operator-(dsf a) { return dsf(-a.hi, -a.lo); }
__device__ __forceinline__ dsf operator-(dsf a, dsf b) { return a + (-b); }

__device__ __forceinline__ dsf operator*(dsf a, dsf b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  dsf r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dsf& operator+=(dsf& a, dsf b) { a = a + b; return a; }
__device__ __forceinline__ dsf& operator-=(dsf& a, dsf b) { a = a - b; return a; }
__device__ __forceinline__ dsf& operator*=(dsf& a, dsf b) { a = a * b; return a; }

// Cache-global loads (L2 only): the work buffers are rewritten by other CTAs
// between grid barriers.
template <typename Z> __device__ __forceinline__ Z ldcg(const Z* p) { return __ldcg(p); }
__device__ __forceinline__ dsf2 ldcg(const dsf2* p) {
  const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
  dsf2 z;
  z.x = dsf(v.x, v.y);
  z.y = dsf(v.z, v.w);
  return z;
}

}  // namespace tsfde
