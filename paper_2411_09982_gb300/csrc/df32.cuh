// Double-float ("DF32") storage and arithmetic of the split-precision path.
//
// A real number is held as an unevaluated sum hi + lo of two FP32 values with
// |lo| <= ulp(hi)/2 (about 48 significant bits, 2^-47 relative).  A complex
// matrix element is one float4 {re.hi, re.lo, im.hi, im.lo}: 16 bytes, the
// same footprint as an FP64 complex.  All arithmetic below runs on the FP32
// pipe (GB300's FP64 pipe is a small fraction of it): error-free TwoSum and
// FMA-based TwoProd (Dekker / Knuth), which the split GEMM epilogue, the
// digit slicers and the elementwise Taylor/phase kernels share.
#pragma once

#include <cuda_runtime.h>

namespace mg {

struct df32 {
  float hi, lo;
};

__device__ __forceinline__ df32 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ df32 fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = a + b;
  return {s, b - (s - a)};
}

// accurate double-word addition (relative error a few u^2 even under cancellation)
__device__ __forceinline__ df32 df_add(df32 x, df32 y) {
  const df32 s = two_sum(x.hi, y.hi);
  const df32 t = two_sum(x.lo, y.lo);
  df32 r = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(r.hi, t.lo + r.lo);
}

// x * c (c a DF32 constant)
__device__ __forceinline__ df32 df_mul(df32 x, df32 c) {
  const float p = x.hi * c.hi;
  float e = fmaf(x.hi, c.hi, -p);
  e = fmaf(x.hi, c.lo, e);
  e = fmaf(x.lo, c.hi, e);
  return fast_two_sum(p, e);
}

// x * c + y
__device__ __forceinline__ df32 df_fma(df32 x, df32 c, df32 y) { return df_add(df_mul(x, c), y); }

__host__ __device__ __forceinline__ df32 df_from_double(double v) {
  const float hi = (float)v;
  const float lo = (float)(v - (double)hi);
  return {hi, lo};
}

__device__ __forceinline__ double df_to_double(df32 x) { return (double)x.hi + (double)x.lo; }

__device__ __forceinline__ df32 df_neg(df32 x) { return {-x.hi, -x.lo}; }

// exact scaling by 2^k for |k| <= 250 (two steps keep each factor representable)
__device__ __forceinline__ float pow2f_exact(int k) { return __int_as_float((127 + k) << 23); }
__device__ __forceinline__ df32 df_ldexp(df32 x, int k) {
  const int k1 = k / 2, k2 = k - k1;
  const float f1 = pow2f_exact(k1), f2 = pow2f_exact(k2);
  return {(x.hi * f1) * f2, (x.lo * f1) * f2};
}

}  // namespace mg
