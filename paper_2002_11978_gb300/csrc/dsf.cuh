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
// Every operation is a handful of FP32 adds and FMAs (add 11, multiply 6,
// dot2 19).  GB300 issues FP32 at 58x its FP64 rate (72.6 against 1.25
// TFLOP/s measured), so a double-single operation costs several times less
// pipe time than the FP64 one it replaces.
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

// a1 b1 + a2 b2 with one renormalisation: both high products exactly
// (two_prod), their sum exactly (two_sum), the product errors and cross
// terms accumulated in FP32.  19 operations against 23 for two products and
// a sum; error a few u^2 (|a1 b1| + |a2 b2|).
__device__ __forceinline__ dsf dot2(dsf a1, dsf b1, dsf a2, dsf b2) {
  const float p1 = __fmul_rn(a1.hi, b1.hi);
  const float e1 = __fmaf_rn(a1.hi, b1.hi, -p1);
  const float p2 = __fmul_rn(a2.hi, b2.hi);
  const float e2 = __fmaf_rn(a2.hi, b2.hi, -p2);
  float s, e;
  two_sum(p1, p2, s, e);
  e = __fadd_rn(e, __fadd_rn(e1, e2));
  e = __fmaf_rn(a1.hi, b1.lo, e);
  e = __fmaf_rn(a1.lo, b1.hi, e);
  e = __fmaf_rn(a2.hi, b2.lo, e);
  e = __fmaf_rn(a2.lo, b2.hi, e);
  dsf r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// Complex products (overloads of the generic ones in dev.cuh): a b and a conj(b).
__device__ __forceinline__ dsf2 cmul(dsf2 a, dsf2 b) {
  dsf2 c;
  c.x = dot2(a.x, b.x, -a.y, b.y);
  c.y = dot2(a.x, b.y, a.y, b.x);
  return c;
}
__device__ __forceinline__ dsf2 cmulc(dsf2 a, dsf2 b) {
  dsf2 c;
  c.x = dot2(a.x, b.x, a.y, b.y);
  c.y = dot2(a.y, b.x, -a.x, b.y);
  return c;
}

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
