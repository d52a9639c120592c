// Gradients of the interaction energy (Sec. II.A with Eq. (EQForce)):
//   E = mu0 V Ms_t sum_i m_t(i) . grad phi_s(x_i),  phi_s = spline of (S * M_s).
// E is linear in m_s, so dE/dm_s is the transposed forward path applied to
// the target's weights, run backwards:
//   1. transposed gradient evaluation (k_adj_scatter): every coefficient node
//      collects mu0 V Ms_t m_t,a / d_a times the derivative weights of axis a
//      from the targets whose 64 taps cover it;
//   2. transposed prefilter on the whole box (k_pref_T), per axis: with the
//      mirror band matrix B of the prefilter P = B^-1, B^T = W B W^-1 for
//      W = diag(1/2, 1, ..., 1, 1/2), so P^T = W P W^-1: scale the two end
//      samples by 2, run the mirror recursion, scale the ends by 1/2;
//   3. transposed potential sum Mbar_c(j) = sum_b S_c(b - j) phibar(b): the
//      box is laid on the circular grid at its nodes (k_place), transformed by
//      the x and y forward passes, multiplied by the conjugate S spectra and
//      summed over box planes per source layer (k_zadj), and transformed back
//      by the y and x inverse passes.
// The recursion of step 2 is Unser's exact mirror-boundary one (causal start
// from the mirrored periodic extension, anticausal start in closed form).
#include <cuda_runtime.h>

#include "mm_internal.h"
#include "spline_w.cuh"

namespace mm {

// ------------------------------------------------------------------ 1. scatter
__global__ void __launch_bounds__(256) k_adj_scatter(const AdjScatterJob J) {
  __shared__ float w_s[3][12];
  __shared__ int sh_s[3];
  if (threadIdx.x < 3) {
    // the gather's split of sigma u into a whole-cell shift and weights
    const int a = threadIdx.x;
    const double su = J.sigma * J.u[a];
    const double fl = floor(su);
    bspline_w((float)(su - fl), w_s[a]);
    int sh = J.guard[a] + ((int)fl - J.U0[a]);
    const int need = (a == 0 ? J.nx : a == 1 ? J.ny : J.nz) + 3;
    if (sh < 0 || sh + need > J.r[a]) {
      atomicOr(J.err, 1);
      sh = 0x7fffffff;
    }
    sh_s[a] = sh;
  }
  __syncthreads();
  if (sh_s[0] == 0x7fffffff || sh_s[1] == 0x7fffffff || sh_s[2] == 0x7fffffff) return;
  const size_t nr = (size_t)J.r[0] * J.r[1] * J.r[2];
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nr) return;
  const int xr = (int)(idx % J.r[0]);
  const int yr = (int)((idx / J.r[0]) % J.r[1]);
  const int zr = (int)(idx / ((size_t)J.r[0] * J.r[1]));
  const size_t N = (size_t)J.nx * J.ny * J.nz;
  const float gx = J.escale * J.inv_d[0], gy = J.escale * J.inv_d[1], gz = J.escale * J.inv_d[2];
  float s = 0.f;
  for (int kz = 0; kz < 4; ++kz) {
    const int iz = zr - sh_s[2] - kz;
    if (iz < 0 || iz >= J.nz) continue;
    for (int ky = 0; ky < 4; ++ky) {
      const int iy = yr - sh_s[1] - ky;
      if (iy < 0 || iy >= J.ny) continue;
#pragma unroll
      for (int kx = 0; kx < 4; ++kx) {
        const int ix = xr - sh_s[0] - kx;
        if (ix < 0 || ix >= J.nx) continue;
        const size_t cell = ((size_t)iz * J.ny + iy) * J.nx + ix;
        const float mx = __ldg(J.m + cell), my = __ldg(J.m + N + cell), mz = __ldg(J.m + 2 * N + cell);
        s += gx * mx * w_s[0][4 + kx] * w_s[1][ky] * w_s[2][kz] +
             gy * my * w_s[0][kx] * w_s[1][4 + ky] * w_s[2][kz] +
             gz * mz * w_s[0][kx] * w_s[1][ky] * w_s[2][4 + kz];
      }
    }
  }
  J.box[((size_t)(zr + J.start[2]) * J.bdim[1] + (yr + J.start[1])) * J.bdim[0] + (xr + J.start[0])] = s;
}

cudaError_t launch_adj_scatter(const AdjScatterJob& J, cudaStream_t st) {
  const size_t nr = (size_t)J.r[0] * J.r[1] * J.r[2];
  if (nr == 0) return cudaSuccess;
  k_adj_scatter<<<(unsigned)((nr + 255) / 256), 256, 0, st>>>(J);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ 2. prefilter transpose
constexpr float kZ1a = -0.26794919243112270f;  // sqrt(3) - 2

// One thread per box line along `axis`: P^T = W P W^-1 in place.
__global__ void __launch_bounds__(128) k_pref_T(float* box, int bx, int by, int bz, int axis) {
  const int L = axis == 0 ? bx : (axis == 1 ? by : bz);
  const size_t nlines = (size_t)bx * by * bz / L;
  const size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlines || L < 2) return;
  size_t base, stride;
  if (axis == 0) { base = l * bx; stride = 1; }
  else if (axis == 1) { base = (l / bx) * ((size_t)bx * by) + l % bx; stride = bx; }
  else { base = l; stride = (size_t)bx * by; }
  float* x = box + base;
  const float z = kZ1a;
  auto y = [&](int k) {  // W^-1 x: end samples doubled
    const float v = x[(size_t)k * stride];
    return (k == 0 || k == L - 1) ? 2.f * v : v;
  };
  // causal start: sum_k z^k of the mirrored periodic extension (period 2L - 2)
  const int P = 2 * L - 2;
  const int K = P < 48 ? P : 48;  // |z|^48 ~ 3e-28
  float c0 = 0.f, zk = 1.f;
  for (int k = 0; k < K; ++k) {
    const int kk = k < L ? k : P - k;
    c0 += zk * y(kk);
    zk *= z;
  }
  if (K == P) c0 /= (1.f - zk);  // zk = z^P
  // causal pass, c+ stored in place
  float cp = c0;
  float yprev_cp = 0.f;
  x[0] = cp;
  for (int k = 1; k < L; ++k) {
    const float v = y(k);
    yprev_cp = cp;
    cp = v + z * cp;
    x[(size_t)k * stride] = cp;
  }
  // anticausal pass: c-[L-1] = z / (z^2 - 1) (c+[L-1] + z c+[L-2]); c = 6 c-; W: ends halved
  float cm = z / (z * z - 1.f) * (cp + z * yprev_cp);
  x[(size_t)(L - 1) * stride] = 0.5f * 6.f * cm;
  for (int k = L - 2; k >= 0; --k) {
    cm = z * (cm - x[(size_t)k * stride]);
    x[(size_t)k * stride] = (k == 0 ? 0.5f : 1.f) * 6.f * cm;
  }
}

cudaError_t launch_pref_T(float* box, const int bdim[3], cudaStream_t st) {
  for (int axis = 0; axis < 3; ++axis) {
    const size_t nlines = (size_t)bdim[0] * bdim[1] * bdim[2] / bdim[axis];
    k_pref_T<<<(unsigned)((nlines + 127) / 128), 128, 0, st>>>(box, bdim[0], bdim[1], bdim[2], axis);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------------ 3. place, z sum, scale
// box node (xb, yb, zb) -> grid[zb][(lo_y + yb) mod Qy][(lo_x + xb) mod Qx]
__global__ void k_place(const float* box, int bx, int by, int bz, int lo_x, int lo_y, float* grid, int Qx,
                        int Qy) {
  const size_t n = (size_t)bx * by * bz;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int xb = (int)(i % bx);
  const int yb = (int)((i / bx) % by);
  const int zb = (int)(i / ((size_t)bx * by));
  int gx = (lo_x + xb) % Qx, gy = (lo_y + yb) % Qy;
  if (gx < 0) gx += Qx;
  if (gy < 0) gy += Qy;
  grid[((size_t)zb * Qy + gy) * Qx + gx] = box[i];
}

cudaError_t launch_place(const float* box, const int bdim[3], const int box_lo[3], float* grid, int Qx, int Qy,
                         cudaStream_t st) {
  const size_t n = (size_t)bdim[0] * bdim[1] * bdim[2];
  k_place<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(box, bdim[0], bdim[1], bdim[2], box_lo[0], box_lo[1], grid,
                                                       Qx, Qy);
  return cudaGetLastError();
}

// Thread -> (kx, source plane (c, jz), frequency pair ky, Qy - ky).  The
// stored S_x, S_y are imaginary parts, S_z real; conjugation flips the
// imaginary ones, and S_y is odd in y.
__global__ void __launch_bounds__(256) k_zadj(const ZAdjJob J) {
  const int nch = (J.kyq + 255) / 256;
  const int P3 = 3 * J.nz;
  const int kx = blockIdx.x / (P3 * nch);
  const int rem = blockIdx.x - kx * P3 * nch;
  const int o = rem / nch;
  const int k = (rem - o * nch) * 256 + threadIdx.x;
  if (k >= J.kyq) return;
  const int c = o / J.nz, jz = o - c * J.nz;
  const int Qy = J.Qy;
  const bool two = k != 0 && 2 * k != Qy;
  const int k1 = two ? Qy - k : k;
  const size_t pstride = (size_t)J.kxh * Qy;
  const size_t kstride = (size_t)J.kxh * J.kyq;
  const size_t koff = (size_t)kx * J.kyq + k;
  const float2* in = J.in + (size_t)kx * Qy;
  float2 a0 = make_float2(0.f, 0.f), a1 = a0;
  for (int zb = 0; zb < J.bz; ++zb) {
    const float v = __ldg(J.Sq + ((size_t)(zb - jz + J.nz - 1) * 3 + c) * kstride + koff);
    const float2 p0 = in[(size_t)zb * pstride + k], p1 = in[(size_t)zb * pstride + k1];
    if (c == 2) {  // real, even in y
      a0.x += v * p0.x; a0.y += v * p0.y;
      a1.x += v * p1.x; a1.y += v * p1.y;
    } else {       // conj(i v) = -i v; S_y flips sign at Qy - ky
      const float v1 = c == 1 ? -v : v;
      a0.x += v * p0.y; a0.y -= v * p0.x;
      a1.x += v1 * p1.y; a1.y -= v1 * p1.x;
    }
  }
  float2* dst = J.out + (size_t)o * pstride + (size_t)kx * Qy;
  dst[k] = a0;
  if (two) dst[k1] = a1;
}

cudaError_t launch_zadj(const ZAdjJob& J, cudaStream_t st) {
  const int grid = J.kxh * 3 * J.nz * ((J.kyq + 255) / 256);
  if (grid == 0) return cudaSuccess;
  k_zadj<<<grid, 256, 0, st>>>(J);
  return cudaGetLastError();
}

__global__ void k_scale(const float* in, float* out, size_t n, float s) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = s * in[i];
}

cudaError_t launch_scale(const float* in, float* out, size_t n, float s, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_scale<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n, s);
  return cudaGetLastError();
}

}  // namespace mm
