// Power bookkeeping (Sec. III, after Eq. (EQForce)): the Gilbert dissipation
// of a magnet needs S = sum_i |m_i x H_eff,i|^2 over its cells,
//   P_diss = gamma0 alpha mu0 V Ms / (1 + alpha^2) S
// (the host applies the prefactor in FP64).  k_mxh2: one thread per cell,
// FP32 products, a double-float block sum written as one double per block;
// k_mxh2_sum: one block adds the block sums in a fixed order in FP64, so the
// result does not depend on scheduling.
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "mm_internal.h"

namespace mm {

constexpr int kPowThreads = 256;

__global__ void __launch_bounds__(kPowThreads) k_mxh2(const float* __restrict__ m, const float* __restrict__ H,
                                                      size_t N, double* __restrict__ partial) {
  __shared__ dfloat red[kPowThreads / 32];
  const size_t i = (size_t)blockIdx.x * kPowThreads + threadIdx.x;
  float c2 = 0.f;
  if (i < N) {
    const float m0 = m[i], m1 = m[N + i], m2 = m[2 * N + i];
    const float h0 = H[i], h1 = H[N + i], h2 = H[2 * N + i];
    const float c0 = m1 * h2 - m2 * h1;
    const float c1 = m2 * h0 - m0 * h2;
    const float cz = m0 * h1 - m1 * h0;
    c2 = c0 * c0 + c1 * c1 + cz * cz;
  }
  dfloat s{c2, 0.f};
  for (int o = 16; o > 0; o >>= 1) s = df_add(s, df_shfl_down(s, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    dfloat t = red[0];
    for (int w = 1; w < kPowThreads / 32; ++w) t = df_add(t, red[w]);
    partial[blockIdx.x] = df_to_double(t);
  }
}

__global__ void __launch_bounds__(kPowThreads) k_mxh2_sum(const double* __restrict__ partial, int n,
                                                          double* __restrict__ out) {
  __shared__ double red[kPowThreads];
  double s = 0.0;
  for (int b = threadIdx.x; b < n; b += kPowThreads) s += partial[b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kPowThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

int power_blocks(size_t N) { return (int)((N + kPowThreads - 1) / kPowThreads); }

cudaError_t launch_mxh2(const float* m, const float* H, size_t N, double* partial, double* out, cudaStream_t st) {
  const int nb = power_blocks(N);
  if (nb == 0) return cudaSuccess;
  k_mxh2<<<nb, kPowThreads, 0, st>>>(m, H, N, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_mxh2_sum<<<1, kPowThreads, 0, st>>>(partial, nb, out);
  return cudaGetLastError();
}

}  // namespace mm
