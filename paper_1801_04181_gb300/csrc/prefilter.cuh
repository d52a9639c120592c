// Cubic B-spline prefilter shared by the FFT passes.
//
// Prefilter (Sec. III.A, cubic B-spline coefficients with mirror ends): the
// inverse of (q + 4 + 1/q)/6 factors into a causal and an anticausal
// first-order recursion with pole z1 = sqrt(3) - 2 and gain -6 z1.  On the
// mirror-extended samples each thread runs both recursions over a chunk of
// outputs plus kPrefWarm samples of warm-up on either side; the warm-up error
// is |z1|^14 ~ 1e-8 relative.
#pragma once
#include <cuda_runtime.h>

#include "fft.cuh"

namespace mm {

constexpr int kPrefWarm = 14;
constexpr float kZ1 = -0.26794919243112270f;    // sqrt(3) - 2
constexpr float kPrefGain = 1.6076951545867362f; // -6 z1
// prefilter outputs per thread; odd, so neighbouring threads' table reads
// fall in different shared-memory banks
constexpr int kYChunk = 9;   // y pass (complex)
constexpr int kXChunk = 9;   // x pass (real)
constexpr int kZChunk = 9;   // z pass of thick sources (complex)
// Shared-memory index of the samples the prefilter reads: entry j holds the
// position, in a line of `Q` left in the digit-reversed order of a transform
// (`pos`: its frequency -> position table; natural order when null), of
// box-local node mirror(start - kPrefWarm + j) -- or, when the box is a whole
// period (periodic boundaries), of that node wrapped around the period.
__device__ __forceinline__ void build_pref_table(int* tab, int n, int box_lo, int box_len, int start, int Q,
                                                 const int* __restrict__ pos, bool periodic = false) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    int local;
    if (periodic) {
      local = (start - kPrefWarm + j) % box_len;
      if (local < 0) local += box_len;
    } else {
      local = mirror_index(start - kPrefWarm + j, box_len);
    }
    const int g = wrap_once(box_lo + local, Q);
    tab[j] = pos ? __ldg(pos + g) : g;
  }
}

// Prefilter outputs [k0, k0 + CH) of one line: src(j) = sample at table entry j.
template <int CH, typename T, typename Src, typename Out>
__device__ __forceinline__ void prefilter_chunk(int k0, int r, Src src, Out out) {
  T ybuf[CH + kPrefWarm];
  T y = T();
#pragma unroll
  for (int j = 0; j < CH + 2 * kPrefWarm; ++j) {
    y = src(k0 + j) + kZ1 * y;
    if (j >= kPrefWarm) ybuf[j - kPrefWarm] = y;
  }
  T c = T();
#pragma unroll
  for (int i = CH + kPrefWarm - 1; i >= 0; --i) {
    c = ybuf[i] + kZ1 * c;
    if (i < CH && k0 + i < r) out(k0 + i, kPrefGain * c);
  }
}

struct f2 {  // float2 with the arithmetic the recursion needs
  float x, y;
  __device__ f2() : x(0.f), y(0.f) {}
  __device__ f2(float2 v) : x(v.x), y(v.y) {}
  __device__ f2(float a, float b) : x(a), y(b) {}
};
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ f2 operator*(float s, f2 a) { return f2(s * a.x, s * a.y); }

}  // namespace mm
