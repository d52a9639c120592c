// Tricubic B-spline evaluation of the source potential at the displaced target
// centres, stray field H = -grad phi and the Eq. (EQForce) force / interaction
// energy partial sums (Sec. II.A, III, III.A, IV.D).
//
// The slider moves rigidly, so every target centre has the same fractional
// position f in the source lattice: the 64 weights (cubic B-spline w, w', w''
// per axis at f, full float precision as in Sec. IV.D) are shared by all
// cells and the evaluation is a separable 4-tap filter of the coefficient box.
// A CTA stages a (32 + 3) x (8 + 3) x (nz + 3) coefficient tile in shared
// memory, filters it along x for the three derivative orders, then each thread
// finishes y and z for one (x, y) column of the target.
//
// Per cell it writes H (A/m) and accumulates sum m . grad phi and
// sum_a m_a d_a d_b phi (FP32 within a warp, FP64 across warps and tiles);
// the constants mu0 V Ms_t turn them into E and F (F_t = -mu0 V Ms_t sum Hess(phi) m).
#include <cuda_runtime.h>

#include "mech.cuh"
#include "mm_internal.h"

namespace mm {

constexpr int TX = 32, TY = 8;

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

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// y and z stages for one target column (x, y), all NZ layers.
template <int NZ>
__device__ __forceinline__ void gather_column(const GatherJob& J, const float* A, int a_n,
                                              const float (*w_s)[12], int tx, int ty, int x, int y,
                                              float* acc) {
  constexpr int CZ = NZ + 3;
  float B[6][CZ];
  const float* wy = w_s[1];
#pragma unroll
  for (int zz = 0; zz < CZ; ++zz) {
    float a0[4], a1[4], a2[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int o = (zz * (TY + 3) + ty + k) * TX + tx;
      a0[k] = A[o];
      a1[k] = A[a_n + o];
      a2[k] = A[2 * a_n + o];
    }
    float b00 = 0.f, b10 = 0.f, b01 = 0.f, b20 = 0.f, b02 = 0.f, b11 = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      b00 += wy[k] * a0[k];
      b10 += wy[k] * a1[k];
      b01 += wy[4 + k] * a0[k];
      b20 += wy[k] * a2[k];
      b02 += wy[8 + k] * a0[k];
      b11 += wy[4 + k] * a1[k];
    }
    B[0][zz] = b00; B[1][zz] = b10; B[2][zz] = b01;
    B[3][zz] = b20; B[4][zz] = b02; B[5][zz] = b11;
  }
  const float* wz = w_s[2];
  const float ix = J.inv_d[0], iy = J.inv_d[1], iz = J.inv_d[2];
  const size_t N = (size_t)J.nx * J.ny * NZ;
  float m[3][NZ];
#pragma unroll
  for (int zl = 0; zl < NZ; ++zl) {
    const size_t cell = ((size_t)zl * J.ny + y) * J.nx + x;
    m[0][zl] = __ldg(J.m + cell);
    m[1][zl] = __ldg(J.m + N + cell);
    m[2][zl] = __ldg(J.m + 2 * N + cell);
  }
#pragma unroll
  for (int zl = 0; zl < NZ; ++zl) {
    float gx = 0.f, gy = 0.f, gz = 0.f, hxx = 0.f, hyy = 0.f, hzz = 0.f, hxy = 0.f, hxz = 0.f, hyz = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int zz = zl + k;
      gx += wz[k] * B[1][zz];
      gy += wz[k] * B[2][zz];
      gz += wz[4 + k] * B[0][zz];
      hxx += wz[k] * B[3][zz];
      hyy += wz[k] * B[4][zz];
      hzz += wz[8 + k] * B[0][zz];
      hxy += wz[k] * B[5][zz];
      hxz += wz[4 + k] * B[1][zz];
      hyz += wz[4 + k] * B[2][zz];
    }
    gx *= ix; gy *= iy; gz *= iz;
    hxx *= ix * ix; hyy *= iy * iy; hzz *= iz * iz;
    hxy *= ix * iy; hxz *= ix * iz; hyz *= iy * iz;
    const size_t cell = ((size_t)zl * J.ny + y) * J.nx + x;
    if (J.H) {
      J.H[cell] = -gx;
      J.H[N + cell] = -gy;
      J.H[2 * N + cell] = -gz;
    }
    const float mx = m[0][zl], my = m[1][zl], mz = m[2][zl];
    acc[0] += mx * hxx + my * hxy + mz * hxz;
    acc[1] += mx * hxy + my * hyy + mz * hyz;
    acc[2] += mx * hxz + my * hyz + mz * hzz;
    acc[3] += mx * gx + my * gy + mz * gz;
  }
}

__global__ void __launch_bounds__(TX * TY, 3) k_gather(const Launch<GatherJob> Lc, const MechParams P, int* ticket) {
  extern __shared__ float gsm[];
  __shared__ float w_s[3][12];
  __shared__ int shift_s[3];
  __shared__ double red_s[TX * TY / 32][4];

  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const GatherJob& J = Lc.job[j];
  const int tile = blockIdx.x - Lc.tile_start[j];
  const int ntx = (J.nx + TX - 1) / TX;
  const int x0 = (tile % ntx) * TX;
  const int y0 = (tile / ntx) * TY;
  const int nz = J.nz;
  const int cz = nz + 3;

  if (threadIdx.x < 3) {
    const int a = threadIdx.x;
    // sigma * u in source lattice cells; floor -> integer shift, rest -> weights
    const double su = J.sigma * J.u[a];
    const double fl = floor(su);
    const int U = (int)fl;
    bspline_w((float)(su - fl), w_s[a]);
    int sh = J.guard[a] + (U - J.U0[a]);
    const int need = (a == 0 ? J.nx : a == 1 ? J.ny : J.nz) + 3;
    const int have = a == 0 ? J.rx : a == 1 ? J.ry : J.rz;
    if (sh < 0 || sh + need > have) {
      atomicExch(J.err, 1);
      sh = 0x7fffffff;
    }
    shift_s[a] = sh;
  }
  __syncthreads();
  const bool bad = shift_s[0] == 0x7fffffff || shift_s[1] == 0x7fffffff || shift_s[2] == 0x7fffffff;

  // coefficient tile [cz][TY+3][TX+3]
  float* ct = gsm;
  float* A = gsm + cz * (TY + 3) * (TX + 3);  // [3][cz][TY+3][TX]
  const int tile_n = cz * (TY + 3) * (TX + 3);
  if (!bad) {
    const int sx = shift_s[0], sy = shift_s[1], sz = shift_s[2];
    for (int base = threadIdx.x; base < tile_n; base += 4 * blockDim.x) {
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = base + u * blockDim.x;
        v[u] = 0.f;
        if (idx < tile_n) {
          const int xx = idx % (TX + 3);
          const int rest = idx / (TX + 3);
          const int yy = rest % (TY + 3);
          const int zz = rest / (TY + 3);
          const int gx = x0 + xx + sx, gy = y0 + yy + sy, gz = zz + sz;
          if (gx < J.rx && gy < J.ry && gz < J.rz) v[u] = __ldg(J.C + ((size_t)gz * J.ry + gy) * J.rx + gx);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = base + u * blockDim.x;
        if (idx < tile_n) ct[idx] = v[u];
      }
    }
  }
  __syncthreads();
  const int a_n = cz * (TY + 3) * TX;
  for (int idx = threadIdx.x; idx < a_n; idx += blockDim.x) {
    const int x = idx % TX;
    const int zy = idx / TX;  // zz * (TY+3) + yy
    const float* row = ct + zy * (TX + 3) + x;
    const float c0 = row[0], c1 = row[1], c2 = row[2], c3 = row[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float* w = w_s[0] + 4 * d;
      A[d * a_n + idx] = w[0] * c0 + w[1] * c1 + w[2] * c2 + w[3] * c3;
    }
  }
  __syncthreads();

  const int tx = threadIdx.x % TX;
  const int ty = threadIdx.x / TX;
  const int x = x0 + tx, y = y0 + ty;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  if (!bad && x < J.nx && y < J.ny) {
    switch (nz) {
      case 1: gather_column<1>(J, A, a_n, w_s, tx, ty, x, y, acc); break;
      case 2: gather_column<2>(J, A, a_n, w_s, tx, ty, x, y, acc); break;
      case 3: gather_column<3>(J, A, a_n, w_s, tx, ty, x, y, acc); break;
      default: gather_column<4>(J, A, a_n, w_s, tx, ty, x, y, acc); break;
    }
  }
  // FP32 within a warp (at most 32 x nz cells), FP64 from there on: the FP64
  // pipe of this GPU is narrow, and a warp's partial sum keeps ~1e-6 of the
  // magnitude of its terms, well inside the force tolerance
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float s = acc[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red_s[warp][c] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < TX * TY / 32; ++w) s += red_s[w][threadIdx.x];
    J.partial[(size_t)tile * 4 + threadIdx.x] = s;
  }
  // the last block reduces the forces and, during a step, advances the slider
  if (P.state && last_block(ticket, (int)gridDim.x)) mech_block(P);
}

int gather_tiles(int nx, int ny) { return ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY); }

size_t gather_smem(int nz) {
  const int cz = nz + 3;
  return sizeof(float) * ((size_t)cz * (TY + 3) * (TX + 3) + 3 * (size_t)cz * (TY + 3) * TX);
}

cudaError_t launch_gather(const Launch<GatherJob>& L, int nz_max, const MechParams& P, int* ticket,
                          cudaStream_t st) {
  const size_t smem = gather_smem(nz_max);
  cudaFuncSetAttribute((const void*)k_gather, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaError_t e = cudaFuncSetAttribute(k_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  k_gather<<<grid, TX * TY, smem, st>>>(L, P, ticket);
  return cudaGetLastError();
}

}  // namespace mm
