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

// ------------------------------------------------------------------ div / curl
// Sec. IV.A diagnostics of a field H [3][nz][ny][nx] on cells d: per interior
// cell (both neighbours along every axis of at least three cells) the two-point
// central differences give |div H| and ||curl H||; an axis of fewer than three
// cells contributes no derivative.  Block sums of both in double-float, one
// double each per block; k_sum2 adds them in a fixed order.
__global__ void __launch_bounds__(kPowThreads) k_divcurl(const float* __restrict__ H, int nx, int ny, int nz,
                                                         float idx2, float idy2, float idz2,
                                                         double* __restrict__ partial) {
  __shared__ dfloat red[2][kPowThreads / 32];
  const bool ux = nx >= 3, uy = ny >= 3, uz = nz >= 3;
  const int ix0 = ux, iy0 = uy, iz0 = uz;
  const int mx = nx - 2 * ix0, my = ny - 2 * iy0, mz = nz - 2 * iz0;  // interior extents
  const size_t M = (size_t)mx * my * mz;
  const size_t N = (size_t)nx * ny * nz;
  const size_t t = (size_t)blockIdx.x * kPowThreads + threadIdx.x;
  float dv = 0.f, cv = 0.f;
  if (t < M) {
    const unsigned tt = (unsigned)t;  // interior cells < 2^30
    const unsigned mxy = (unsigned)mx * (unsigned)my;
    const int k = (int)(tt / mxy);
    const unsigned r = tt - (unsigned)k * mxy;
    const int j = (int)(r / (unsigned)mx);
    const int i = (int)(r - (unsigned)j * (unsigned)mx);
    const size_t c = ((size_t)(k + iz0) * ny + (j + iy0)) * nx + (i + ix0);
    const size_t sx = 1, sy = (size_t)nx, sz = (size_t)nx * ny;
    // g[comp][axis] = dH_comp / d axis
    float g[3][3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float* h = H + q * N;
      g[q][0] = ux ? (h[c + sx] - h[c - sx]) * idx2 : 0.f;
      g[q][1] = uy ? (h[c + sy] - h[c - sy]) * idy2 : 0.f;
      g[q][2] = uz ? (h[c + sz] - h[c - sz]) * idz2 : 0.f;
    }
    dv = fabsf(g[0][0] + g[1][1] + g[2][2]);
    const float cx = g[2][1] - g[1][2], cy = g[0][2] - g[2][0], cz = g[1][0] - g[0][1];
    cv = sqrtf(cx * cx + cy * cy + cz * cz);
  }
  dfloat sd{dv, 0.f}, sc{cv, 0.f};
  for (int o = 16; o > 0; o >>= 1) {
    sd = df_add(sd, df_shfl_down(sd, o));
    sc = df_add(sc, df_shfl_down(sc, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sd;
    red[1][threadIdx.x >> 5] = sc;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    dfloat s = red[threadIdx.x][0];
    for (int w = 1; w < kPowThreads / 32; ++w) s = df_add(s, red[threadIdx.x][w]);
    partial[2 * (size_t)blockIdx.x + threadIdx.x] = df_to_double(s);
  }
}

__global__ void __launch_bounds__(kPowThreads) k_sum2(const double* __restrict__ partial, int n,
                                                      double* __restrict__ out) {
  __shared__ double red[2][kPowThreads];
  double s0 = 0.0, s1 = 0.0;
  for (int b = threadIdx.x; b < n; b += kPowThreads) {
    s0 += partial[2 * b];
    s1 += partial[2 * b + 1];
  }
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  __syncthreads();
  for (int w = kPowThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = red[0][0];
    out[1] = red[1][0];
  }
}

size_t divcurl_cells(int nx, int ny, int nz) {
  const int mx = nx >= 3 ? nx - 2 : nx, my = ny >= 3 ? ny - 2 : ny, mz = nz >= 3 ? nz - 2 : nz;
  return (size_t)mx * my * mz;
}
int divcurl_blocks(int nx, int ny, int nz) { return power_blocks(divcurl_cells(nx, ny, nz)); }

cudaError_t launch_divcurl(const float* H, int nx, int ny, int nz, double dx, double dy, double dz,
                           double* partial, double* out, cudaStream_t st) {
  const int nb = divcurl_blocks(nx, ny, nz);
  if (nb == 0) return cudaSuccess;
  k_divcurl<<<nb, kPowThreads, 0, st>>>(H, nx, ny, nz, (float)(0.5 / dx), (float)(0.5 / dy), (float)(0.5 / dz),
                                        partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum2<<<1, kPowThreads, 0, st>>>(partial, nb, out);
  return cudaGetLastError();
}

}  // namespace mm
