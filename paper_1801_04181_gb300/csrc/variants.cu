// Comparison variants of the stray field.
//
// The four-point finite-difference gradient of the interpolated potential
// (Sec. III.A mentions a four-point central difference for the gradient; the
// main path differentiates the spline analytically).  With the B-spline
// coefficients c of the whole box, the interpolant is evaluated at every
// target centre and at the centres up to two cells beyond the target along
// each axis (all share the fractional offset of the displacement), and
//   H_a(i) = -(-phi(i + 2 e_a) + 8 phi(i + e_a) - 8 phi(i - e_a) + phi(i - 2 e_a)) / (12 d_a).
// Box-local node coordinate of target cell i along an axis: i + f + 1 + m
// (f the fractional part of the displacement, m the margin, m >= 2), so the
// 4 x 4 x 4 taps of an extended centre i in [-2, n + 2) start at node i + m.
#include <cuda_runtime.h>

#include "mm_internal.h"
#include "spline_w.cuh"

namespace mm {

// V[(k + 2)][(j + 2)][(i + 2)] = interpolant at extended centre (i, j, k)
__global__ void __launch_bounds__(256) k_spline_values(const float* __restrict__ C, int bx, int by, int bz,
                                                       int nx, int ny, int nz, int m, float fx, float fy,
                                                       float fz, float* __restrict__ V) {
  __shared__ float w[3][12];
  if (threadIdx.x < 3) bspline_w(threadIdx.x == 0 ? fx : (threadIdx.x == 1 ? fy : fz), w[threadIdx.x]);
  __syncthreads();
  const int ex = nx + 4, ey = ny + 4, ez = nz + 4;
  const size_t n = (size_t)ex * ey * ez;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = (int)(t % ex);
  const int j = (int)((t / ex) % ey);
  const int k = (int)(t / ((size_t)ex * ey));
  // extended index e = i means centre i - 2, whose taps start at node i - 2 + m
  const int x0 = i - 2 + m, y0 = j - 2 + m, z0 = k - 2 + m;
  if (x0 < 0 || y0 < 0 || z0 < 0 || x0 + 3 >= bx || y0 + 3 >= by || z0 + 3 >= bz) {
    V[t] = 0.f;  // unreachable for m >= 2 (the host checks); kept in bounds
    return;
  }
  float v = 0.f;
#pragma unroll
  for (int kz = 0; kz < 4; ++kz) {
    float vy = 0.f;
#pragma unroll
    for (int ky = 0; ky < 4; ++ky) {
      const float* row = C + ((size_t)(z0 + kz) * by + (y0 + ky)) * bx + x0;
      const float vx = w[0][0] * row[0] + w[0][1] * row[1] + w[0][2] * row[2] + w[0][3] * row[3];
      vy += w[1][ky] * vx;
    }
    v += w[2][kz] * vy;
  }
  V[t] = v;
}

__global__ void __launch_bounds__(256) k_fd4(const float* __restrict__ V, int nx, int ny, int nz, float sx,
                                             float sy, float sz, float* __restrict__ H) {
  const size_t N = (size_t)nx * ny * nz;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const int i = (int)(t % nx);
  const int j = (int)((t / nx) % ny);
  const int k = (int)(t / ((size_t)nx * ny));
  const int ex = nx + 4, ey = ny + 4;
  const size_t c = ((size_t)(k + 2) * ey + (j + 2)) * ex + (i + 2);
  const size_t dy = (size_t)ex, dz = (size_t)ex * ey;
  // s_a = -1 / (12 d_a)
  H[t] = sx * (-V[c + 2] + 8.f * V[c + 1] - 8.f * V[c - 1] + V[c - 2]);
  H[N + t] = sy * (-V[c + 2 * dy] + 8.f * V[c + dy] - 8.f * V[c - dy] + V[c - 2 * dy]);
  H[2 * N + t] = sz * (-V[c + 2 * dz] + 8.f * V[c + dz] - 8.f * V[c - dz] + V[c - 2 * dz]);
}

// Componentwise field variant (Sec. II.A, the direct method): H_a(i) = the
// B-spline interpolant of component a at target centre i, 64 taps from the
// coefficients of that component on the full box; the taps of centre i start
// at box node i + m along every axis.
__global__ void __launch_bounds__(256) k_field_values(const float* __restrict__ C, int bx, int by, int bz,
                                                      int nx, int ny, int nz, int m, float fx, float fy,
                                                      float fz, float* __restrict__ H) {
  __shared__ float w[3][12];
  if (threadIdx.x < 3) bspline_w(threadIdx.x == 0 ? fx : (threadIdx.x == 1 ? fy : fz), w[threadIdx.x]);
  __syncthreads();
  const size_t N = (size_t)nx * ny * nz;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const int i = (int)(t % nx);
  const int j = (int)((t / nx) % ny);
  const int k = (int)(t / ((size_t)nx * ny));
  const int x0 = i + m, y0 = j + m, z0 = k + m;
  const size_t box = (size_t)bx * by * bz;
  for (int a = 0; a < 3; ++a) {
    float v = 0.f;
    if (x0 + 3 < bx && y0 + 3 < by && z0 + 3 < bz) {  // always true on the full box (host-checked)
#pragma unroll
      for (int kz = 0; kz < 4; ++kz) {
        float vy = 0.f;
#pragma unroll
        for (int ky = 0; ky < 4; ++ky) {
          const float* row = C + a * box + ((size_t)(z0 + kz) * by + (y0 + ky)) * bx + x0;
          const float vx = w[0][0] * row[0] + w[0][1] * row[1] + w[0][2] * row[2] + w[0][3] * row[3];
          vy += w[1][ky] * vx;
        }
        v += w[2][kz] * vy;
      }
    }
    H[a * N + t] = v;
  }
}

cudaError_t launch_field_values(const float* C, const int bdim[3], const int nt[3], int margin,
                                const double frac[3], float* H, cudaStream_t st) {
  const size_t N = (size_t)nt[0] * nt[1] * nt[2];
  if (N == 0) return cudaSuccess;
  k_field_values<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(C, bdim[0], bdim[1], bdim[2], nt[0], nt[1], nt[2],
                                                               margin, (float)frac[0], (float)frac[1],
                                                               (float)frac[2], H);
  return cudaGetLastError();
}

cudaError_t launch_fd4_field(const float* C, const int bdim[3], const int nt[3], int margin, const double frac[3],
                             const double cell[3], float* V, float* H, cudaStream_t st) {
  const size_t ne = (size_t)(nt[0] + 4) * (nt[1] + 4) * (nt[2] + 4);
  const size_t N = (size_t)nt[0] * nt[1] * nt[2];
  if (N == 0) return cudaSuccess;
  k_spline_values<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(C, bdim[0], bdim[1], bdim[2], nt[0], nt[1], nt[2],
                                                                 margin, (float)frac[0], (float)frac[1],
                                                                 (float)frac[2], V);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_fd4<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(V, nt[0], nt[1], nt[2], (float)(-1.0 / (12.0 * cell[0])),
                                                     (float)(-1.0 / (12.0 * cell[1])),
                                                     (float)(-1.0 / (12.0 * cell[2])), H);
  return cudaGetLastError();
}

}  // namespace mm
