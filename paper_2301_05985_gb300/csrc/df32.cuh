// df32.cuh -- double-float ("float-float") arithmetic for kernels whose FP64 work would
// run on GB300's FP64 pipe (1/64 of the FP32 rate).  A value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi) / 2: about 48 significant bits, exponent range
// of float.  Built on the classical error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly, any a, b;
//   Fast2Sum (Dekker 1971): the same when |a| >= |b|, three operations;
//   TwoProduct with a fused multiply-add: p + e = a b exactly, e = fma(a, b, -p).
// The sum carries the low parts' rounding error too (accurate under cancellation, which
// the finite-element differences u_b - u_(1-b) and the element sums produce); the product
// drops lo * lo.  Relative error of one operation: a few 2^-48.
#pragma once

#include <cuda_runtime.h>

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit constexpr df(int x) : hi((float)x), lo(0.0f) {}
  // rounded split of a double (exact for constants folded at compile time)
  __host__ __device__ explicit df(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
};

__host__ __device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df(s, (a - (s - bb)) + (b - bb));
}
__host__ __device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return df(s, b - (s - a));
}
__host__ __device__ __forceinline__ df df_two_prod(float a, float b) {
  const float p = a * b;
  return df(p, fmaf(a, b, -p));
}

__host__ __device__ __forceinline__ df operator+(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  const df t = df_two_sum(a.lo, b.lo);
  s = df_fast_two_sum(s.hi, s.lo + t.hi);
  return df_fast_two_sum(s.hi, s.lo + t.lo);
}
__host__ __device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__host__ __device__ __forceinline__ df operator*(df a, df b) {
  const df p = df_two_prod(a.hi, b.hi);
  return df_fast_two_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}
__host__ __device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__host__ __device__ __forceinline__ df fma(df a, df b, df c) { return a * b + c; }

// 1 / sqrt(x), x > 0: the float estimate refined by two Newton steps y += y (1 - x y^2) / 2,
// each evaluated in double-float (the error of the estimate squares per step)
__device__ __forceinline__ df inv_sqrt(df x) {
  df y(rsqrtf(x.hi), 0.0f);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const df r = df(1.0f, 0.0f) - x * (y * y);
    y = y + y * (r * df(0.5f, 0.0f));
  }
  return y;
}
__device__ __forceinline__ float inv_sqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double inv_sqrt(double x) { return 1.0 / sqrt(x); }

// split of a loaded double; back to double for the output
__device__ __forceinline__ df df_split(double x) {
  const float h = __double2float_rn(x);
  return df(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
