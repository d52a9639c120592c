// Unevaluated sums hi + lo of two floats ("double-float"), for reductions that
// must keep far more than FP32's 24 bits without this GPU's narrow FP64 pipe
// (a one-block FP64 reduction of a few thousand partials took ~20 us).
//
// Knuth's TwoSum and Dekker's Fast2Sum error-free transformations; the sum of
// two pairs renormalises twice (the accurate variant, safe under the heavy
// cancellation of force sums), so each addition is good to ~2^-44 relative.
// No multiplications appear, so FMA contraction cannot alter them, and
// without fast-math the compiler keeps every FP32 addition as written.
#pragma once
#include <cuda_runtime.h>

namespace mm {

struct dfloat {
  float hi, lo;
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  const float e = (a - (s - bp)) + (b - bp);
  return {s, e};
}

// |a| >= |b| or a == 0
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  dfloat s = df_two_sum(a.hi, b.hi);
  const dfloat t = df_two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = df_fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dfloat df_shfl_down(dfloat a, int o) {
  return {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}

__device__ __forceinline__ double df_to_double(dfloat a) { return (double)a.hi + (double)a.lo; }

}  // namespace mm
