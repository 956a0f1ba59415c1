// Double-float ("dd") arithmetic shared by the eigensolver and the batched
// ST-HOSVD kernels.
#pragma once

#include <cuda_runtime.h>

namespace atc {

// A value is an unevaluated sum hi + lo of two floats (48-bit significand, error-free
// transformations with FMA; Dekker, Numer. Math. 18, 1971; the "double-double"
// technique at single-precision width).  On GB300 an FP64 operation has a
// 64-cycle latency and 1/64 of the FP32 rate, while the algorithms here are
// chains of dependent operations, so the pair arithmetic is several times
// faster at an accuracy of about 2^-47 relative per operation.  Callers scale
// their data by powers of two so that the float exponent range is never
// approached.
// (8-byte aligned: a pair moves with one 64-bit load or store)
struct __align__(8) dd {
  float hi, lo;
};
__device__ __forceinline__ dd ddf(float a) { return dd{a, 0.f}; }
__device__ __forceinline__ dd dd_from(double x) {
  const float h = (float)x;
  return dd{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double dd_to(dd a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dd dd_qts(float s, float e) {  // |s| >= |e|
  const float h = s + e;
  return dd{h, e - (h - s)};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  const float s = a.hi + b.hi;
  const float bp = s - a.hi;
  float e = (a.hi - (s - bp)) + (b.hi - bp);
  e += a.lo + b.lo;
  return dd_qts(s, e);
}
__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return dd_qts(p, e);
}
__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) { return dd_add(dd_mul(a, b), c); }
// a / b: float quotient, one correction from the exact residual
__device__ __forceinline__ dd dd_div(dd a, dd b) {
  const float rb = 1.0f / b.hi;
  const float q1 = a.hi * rb;
  const dd r = dd_sub(a, dd_mul(b, ddf(q1)));
  const float q2 = r.hi * rb;
  const dd q = dd_qts(q1, q2);
  const dd r2 = dd_sub(a, dd_mul(b, q));
  return dd_add(q, ddf(r2.hi * rb));
}
// sqrt(a), a >= 0: float root, one Newton correction
__device__ __forceinline__ dd dd_sqrt(dd a) {
  if (a.hi <= 0.f) return dd{0.f, 0.f};
  const float x = sqrtf(a.hi);
  const dd xx = dd_mul(ddf(x), ddf(x));
  const dd r = dd_sub(a, xx);
  return dd_qts(x, r.hi * (0.5f / x));
}
__device__ __forceinline__ bool dd_neg_sign(dd a) { return a.hi < 0.f || (a.hi == 0.f && a.lo < 0.f); }

}  // namespace atc
