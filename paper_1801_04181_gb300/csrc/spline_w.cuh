// Cubic B-spline weights of the tricubic evaluation (Sec. III.A, IV.D),
// shared by the gather and its transpose.
#pragma once
#include <cuda_runtime.h>

namespace mm {

__device__ __forceinline__ void bspline_w(float t, float* w) {
  // w[0..3] value, w[4..7] first, w[8..11] second derivative weights at t
  const float s = 1.f - t;
  const float t2 = t * t, t3 = t2 * t;
  w[0] = s * s * s * (1.f / 6.f);
  w[1] = (3.f * t3 - 6.f * t2 + 4.f) * (1.f / 6.f);
  w[2] = (-3.f * t3 + 3.f * t2 + 3.f * t + 1.f) * (1.f / 6.f);
  w[3] = t3 * (1.f / 6.f);
  w[4] = -0.5f * s * s;
  w[5] = 1.5f * t2 - 2.f * t;
  w[6] = -1.5f * t2 + t + 0.5f;
  w[7] = 0.5f * t2;
  w[8] = s;
  w[9] = 3.f * t - 2.f;
  w[10] = -3.f * t + 1.f;
  w[11] = t;
}

}  // namespace mm
