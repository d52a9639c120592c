// FFT passes of the potential / self-demag convolution (Sec. III.A).
//
// Per source magnet s the circular convolution over a Qx x Qy grid runs as
//   x pass (R2C, two real rows per complex line)  -> X1[plane][kx][y]
//   y pass: forward y FFT, z plane mixing with the kernel spectra, inverse y
//           FFT, y prefilter of the coefficient planes    -> Y[plane][kx][row]
//   x pass (C2R, two rows per line), x prefilter          -> real rows
// Spectra are stored kx-major with y fastest, so every pass reads and writes
// whole contiguous rows or columns of HBM.  Thin films (nz <= 4) take z by a
// direct sum over planes inside the y pass, which saves a third FFT pass.
//
// Kernel spectra are real quarter planes (kx <= Qx/2, ky <= Qy/2): every
// component of S and N is even or odd in x and y, so its spectrum is purely
// real or purely imaginary and even or odd in ky.  Signs and the factor i are
// restored here.
#include "fft.cuh"
#include "mm_internal.h"

namespace mm {

// Cubic B-spline prefilter taps h_i = sqrt(3) z1^|i|, z1 = sqrt(3) - 2: the
// impulse response of the inverse of (z + 4 + 1/z)/6 (Sec. III.A prefilter),
// truncated at |i| <= kFirHalf; applied to the mirror-extended samples this is
// the mirror-end spline to ~1e-8 relative.
__constant__ float c_fir[kFirHalf + 1];

// ------------------------------------------------------------------ x forward
__global__ void __launch_bounds__(256) k_xfwd(const Launch<XFwdJob> Lc) {
  extern __shared__ float2 sm[];
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const XFwdJob& J = Lc.job[j];
  const int tile = blockIdx.x - Lc.tile_start[j];
  const int Q = J.fx.plan.L;
  const int rows = 3 * J.nz * J.ny;
  const int r0 = tile * kRowsPerCta;
  const int nrows = min(kRowsPerCta, rows - r0);
  const int nlines = (nrows + 1) >> 1;

  for (int idx = threadIdx.x; idx < nlines * Q; idx += blockDim.x) {
    const int line = idx / Q;
    const int x = idx - line * Q;
    float a = 0.f, b = 0.f;
    if (x < J.nx) {
      const int ra = r0 + 2 * line;
      a = __ldg(J.m + (size_t)ra * J.nx + x);
      if (2 * line + 1 < nrows) b = __ldg(J.m + (size_t)(ra + 1) * J.nx + x);
    }
    sm[line * Q + x] = make_float2(a, b);
  }
  __syncthreads();
  fft_smem<float2>(sm, Q, nlines, J.fx.plan, J.fx.tw_f, false, 0, blockDim.x);

  // Z = A + iB:  A_k = (Z_k + conj Z_{Q-k}) / 2,  B_k = (Z_k - conj Z_{Q-k}) / (2i)
  for (int idx = threadIdx.x; idx < J.kxh * nrows; idx += blockDim.x) {
    const int kx = idx / nrows;
    const int rl = idx - kx * nrows;
    const int line = rl >> 1;
    const float2 Zk = sm[line * Q + J.fx.pos[kx]];
    const float2 Zm = sm[line * Q + J.fx.pos[kx == 0 ? 0 : Q - kx]];
    float2 v;
    if ((rl & 1) == 0) {
      v = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
    } else {
      v = make_float2(0.5f * (Zk.y + Zm.y), -0.5f * (Zk.x - Zm.x));
    }
    const int row = r0 + rl;
    const int plane = row / J.ny;
    const int y = row - plane * J.ny;
    J.out[((size_t)plane * J.kxh + kx) * J.ny + y] = v;
  }
}

// ------------------------------------------------------------------ y pass
__device__ __forceinline__ float2 kmul(float v, bool imag, float2 m) {
  return imag ? make_float2(-v * m.y, v * m.x) : make_float2(v * m.x, v * m.y);
}

__global__ void __launch_bounds__(256) k_ypass(const Launch<YJob> Lc) {
  extern __shared__ float2 sm[];
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const YJob& J = Lc.job[j];
  const int kx = blockIdx.x - Lc.tile_start[j];
  const int Q = J.fy.plan.L;
  const int nz = J.nz;
  const int Pin = 3 * nz;
  const int nH = J.do_H ? 3 * nz : 0;
  const int Pout = nH + (J.do_C ? J.n_out : 0);

  for (int idx = threadIdx.x; idx < Pin * Q; idx += blockDim.x) {
    const int p = idx / Q;
    const int y = idx - p * Q;
    float2 v = make_float2(0.f, 0.f);
    if (y < J.ny) v = J.in[((size_t)p * J.kxh + kx) * J.ny + y];
    sm[p * Q + y] = v;
  }
  __syncthreads();
  fft_smem<float2>(sm, Q, Pin, J.fy.plan, J.fy.tw_f, false, 0, blockDim.x);

  const size_t kstride = (size_t)J.kxh * J.kyq;  // one stored kernel plane
  for (int q = threadIdx.x; q < Q; q += blockDim.x) {
    const int ky = J.fy.freq[q];
    const bool upper = 2 * ky > Q;
    const int kyq = upper ? Q - ky : ky;
    const float fy = upper ? -1.f : 1.f;     // sign of odd-in-y spectra above Qy/2
    const size_t koff = (size_t)kx * J.kyq + kyq;
    float2 mh[3 * kMaxNz];
    for (int p = 0; p < Pin; ++p) mh[p] = sm[p * Q + q];
    if (J.do_H) {
      // H_a(iz) = sum_jz sum_b Ns_ab(iz - jz) m_b(jz); Ns = -Ms N / (Qx Qy)
      for (int iz = 0; iz < nz; ++iz) {
        float2 acc[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        for (int jz = 0; jz < nz; ++jz) {
          const int dz = iz - jz;
          const int adz = dz < 0 ? -dz : dz;
          const float sz = dz < 0 ? -1.f : 1.f;
          const float* base = J.Nq + (size_t)adz * kstride + koff;
          const float nxx = __ldg(base + 0 * nz * kstride);
          const float nyy = __ldg(base + 1 * nz * kstride);
          const float nzz = __ldg(base + 2 * nz * kstride);
          const float nxy = __ldg(base + 3 * nz * kstride) * fy;
          const float nxz = __ldg(base + 4 * nz * kstride) * sz;
          const float nyz = __ldg(base + 5 * nz * kstride) * sz * fy;
          const float2 mx = mh[0 * nz + jz], my = mh[1 * nz + jz], mz = mh[2 * nz + jz];
          float2 t;
          t = kmul(nxx, false, mx); acc[0].x += t.x; acc[0].y += t.y;
          t = kmul(nxy, false, my); acc[0].x += t.x; acc[0].y += t.y;
          t = kmul(nxz, true, mz);  acc[0].x += t.x; acc[0].y += t.y;
          t = kmul(nxy, false, mx); acc[1].x += t.x; acc[1].y += t.y;
          t = kmul(nyy, false, my); acc[1].x += t.x; acc[1].y += t.y;
          t = kmul(nyz, true, mz);  acc[1].x += t.x; acc[1].y += t.y;
          t = kmul(nxz, true, mx);  acc[2].x += t.x; acc[2].y += t.y;
          t = kmul(nyz, true, my);  acc[2].x += t.x; acc[2].y += t.y;
          t = kmul(nzz, false, mz); acc[2].x += t.x; acc[2].y += t.y;
        }
        for (int a = 0; a < 3; ++a) sm[(a * nz + iz) * Q + q] = acc[a];
      }
    }
    if (J.do_C) {
      // c(o) = sum_jz sum_c T_c(o, jz) m_c(jz); T = Ms W (S spectra) / (Qx Qy)
      for (int o = 0; o < J.n_out; ++o) {
        float2 acc = make_float2(0.f, 0.f);
        for (int jz = 0; jz < nz; ++jz) {
          const float* base = J.Tq + (size_t)((o * nz + jz) * 3) * kstride + koff;
          const float tx = __ldg(base);
          const float ty = __ldg(base + kstride) * fy;
          const float tz = __ldg(base + 2 * kstride);
          float2 t;
          t = kmul(tx, true, mh[0 * nz + jz]);  acc.x += t.x; acc.y += t.y;
          t = kmul(ty, true, mh[1 * nz + jz]);  acc.x += t.x; acc.y += t.y;
          t = kmul(tz, false, mh[2 * nz + jz]); acc.x += t.x; acc.y += t.y;
        }
        sm[(nH + o) * Q + q] = acc;
      }
    }
  }
  __syncthreads();
  fft_smem<float2>(sm, Q, Pout, J.fy.plan, J.fy.tw_f, true, 0, blockDim.x);

  if (J.do_H) {
    for (int idx = threadIdx.x; idx < nH * J.ny; idx += blockDim.x) {
      const int p = idx / J.ny;
      const int y = idx - p * J.ny;
      J.outH[((size_t)p * J.kxh + kx) * J.ny + y] = sm[p * Q + y];
    }
  }
  if (J.do_C) {
    for (int idx = threadIdx.x; idx < J.n_out * J.r; idx += blockDim.x) {
      const int o = idx / J.r;
      const int k = idx - o * J.r;
      const float2* col = sm + (size_t)(nH + o) * Q;
      float2 v;
      if (J.fir) {
        v = make_float2(0.f, 0.f);
        const int c = J.start + k;
#pragma unroll
        for (int i = -kFirHalf; i <= kFirHalf; ++i) {
          const float h = c_fir[i < 0 ? -i : i];
          const float2 s = col[wrap_index((long long)J.box_lo + mirror_index(c - i, J.box_len), Q)];
          v.x += h * s.x;
          v.y += h * s.y;
        }
      } else {
        v = col[wrap_index((long long)J.box_lo + J.start + k, Q)];
      }
      J.outC[((size_t)o * J.kxh + kx) * J.r + k] = v;
    }
  }
}

// ------------------------------------------------------------------ x inverse
__global__ void __launch_bounds__(256) k_xinv(const Launch<XInvJob> Lc) {
  extern __shared__ float2 sm[];
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const XInvJob& J = Lc.job[j];
  const int tile = blockIdx.x - Lc.tile_start[j];
  const int Q = J.fx.plan.L;
  const int rows = J.planes * J.rows_per_plane;
  const int r0 = tile * kRowsPerCta;
  const int nrows = min(kRowsPerCta, rows - r0);
  const int nlines = (nrows + 1) >> 1;

  // Z_k = A_k + i B_k and Z_{Q-k} = conj(A_k) + i conj(B_k), scattered to DIF order
  for (int idx = threadIdx.x; idx < J.kxh * nlines; idx += blockDim.x) {
    const int kx = idx / nlines;
    const int line = idx - kx * nlines;
    const int ra = r0 + 2 * line;
    const int pa = ra / J.rows_per_plane, ya = ra - pa * J.rows_per_plane;
    const float2 A = J.in[((size_t)pa * J.kxh + kx) * J.rows_per_plane + ya];
    float2 B = make_float2(0.f, 0.f);
    if (2 * line + 1 < nrows) {
      const int rb = ra + 1;
      const int pb = rb / J.rows_per_plane, yb = rb - pb * J.rows_per_plane;
      B = J.in[((size_t)pb * J.kxh + kx) * J.rows_per_plane + yb];
    }
    sm[line * Q + J.fx.pos[kx]] = make_float2(A.x - B.y, A.y + B.x);
    if (kx > 0 && 2 * kx != Q) sm[line * Q + J.fx.pos[Q - kx]] = make_float2(A.x + B.y, B.x - A.y);
  }
  __syncthreads();
  fft_smem<float2>(sm, Q, nlines, J.fx.plan, J.fx.tw_f, true, 0, blockDim.x);

  for (int idx = threadIdx.x; idx < nrows * J.out_len; idx += blockDim.x) {
    const int rl = idx / J.out_len;
    const int k = idx - rl * J.out_len;
    const float2* line = sm + (size_t)(rl >> 1) * Q;
    const bool im = rl & 1;
    float v;
    if (J.fir) {
      v = 0.f;
      const int c = J.start + k;
#pragma unroll
      for (int i = -kFirHalf; i <= kFirHalf; ++i) {
        const float2 s = line[wrap_index((long long)J.box_lo + mirror_index(c - i, J.box_len), Q)];
        v += c_fir[i < 0 ? -i : i] * (im ? s.y : s.x);
      }
    } else {
      const float2 s = line[wrap_index((long long)J.box_lo + J.start + k, Q)];
      v = im ? s.y : s.x;
    }
    const int row = r0 + rl;
    J.out[(size_t)row * J.out_len + k] = v;
  }
}

// ------------------------------------------------------------------ host side
static size_t xpass_smem(int Qmax) { return (size_t)(kRowsPerCta / 2) * Qmax * sizeof(float2); }

cudaError_t set_fir_taps(const float* taps) {
  return cudaMemcpyToSymbol(c_fir, taps, sizeof(float) * (kFirHalf + 1));
}

cudaError_t launch_xfwd(const Launch<XFwdJob>& L, int Qmax, cudaStream_t st) {
  const size_t smem = xpass_smem(Qmax);
  cudaError_t e = cudaFuncSetAttribute(k_xfwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  k_xfwd<<<grid, 256, smem, st>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_ypass(const Launch<YJob>& L, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_ypass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  k_ypass<<<grid, 256, smem, st>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_xinv(const Launch<XInvJob>& L, int Qmax, cudaStream_t st) {
  const size_t smem = xpass_smem(Qmax);
  cudaError_t e = cudaFuncSetAttribute(k_xinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  k_xinv<<<grid, 256, smem, st>>>(L);
  return cudaGetLastError();
}

}  // namespace mm
