// dw.cuh -- double-word ("double-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// i.e. about 48 significant bits within the FP32 exponent range. On GB300 the
// FP32 pipe issues 128 FMAs per clock per SM and the FP64 pipe 2, so an
// operation built from a few error-free transformations (Dekker 1971, Knuth's
// TwoSum, the FMA-based TwoProd) runs several times faster than the FP64
// instruction it replaces, at a unit roundoff of a few 2^-48.
//
// The algorithms and their error bounds are those of M. Joldes, J.-M. Muller,
// V. Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 44(2), 2017, with u = 2^-24:
//   product (their DWTimesDW3, with FMA)   relative error <= 4 u^2
//   sum (their SloppyDWPlusDW)             error <= 2 u^2 (|x| + |y|)  (no relative
//                                          bound under cancellation, which the
//                                          norm-wise error analyses here do not need)
// Every step is written with _rn intrinsics so that the compiler neither
// contracts nor reassociates them.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace mn {

struct alignas(8) df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ constexpr df(float v) : hi(v), lo(0.0f) {}
  // nearest double-word of a double (two roundings: |d - hi - lo| <= 2^-48 |d|)
  __host__ __device__ df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df dw_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ df dw_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df dw_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df operator-(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df operator+(df x, df y) {
  const df s = dw_two_sum(x.hi, y.hi);
  const float w = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return dw_fast_two_sum(s.hi, w);
}
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__device__ __forceinline__ df operator*(df x, df y) {
  const df c = dw_two_prod(x.hi, y.hi);
  const float t = __fmaf_rn(x.lo, y.hi, __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.lo)));
  return dw_fast_two_sum(c.hi, __fadd_rn(c.lo, t));
}
__device__ __forceinline__ df &operator+=(df &x, df y) { return x = x + y; }
__device__ __forceinline__ df &operator-=(df &x, df y) { return x = x - y; }
__device__ __forceinline__ df &operator*=(df &x, df y) { return x = x * y; }
// a * b + c (one product, one sum: the error bounds above added); the built-in
// fma overloads stay visible inside this namespace
using ::fma;
__device__ __forceinline__ df fma(df a, df b, df c) { return a * b + c; }

// warp shuffles of a double-word, overloaded next to the built-in ones (which
// the using-declarations keep visible inside this namespace)
using ::__shfl_down_sync;
using ::__shfl_xor_sync;
__device__ __forceinline__ df __shfl_down_sync(unsigned mask, df v, unsigned delta, int width = 32) {
  return {::__shfl_down_sync(mask, v.hi, delta, width), ::__shfl_down_sync(mask, v.lo, delta, width)};
}
__device__ __forceinline__ df __shfl_xor_sync(unsigned mask, df v, int lane_mask, int width = 32) {
  return {::__shfl_xor_sync(mask, v.hi, lane_mask, width), ::__shfl_xor_sync(mask, v.lo, lane_mask, width)};
}

using zw = cx<df>;  // complex double-word: 16 bytes, (re.hi, re.lo, im.hi, im.lo)

}  // namespace mn
