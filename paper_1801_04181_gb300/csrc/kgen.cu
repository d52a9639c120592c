// One-time FP64 generation of the convolution kernels and their spectra
// (Sec. III.A: kernels are computed once, Fourier transformed, kept resident).
//
// S: scalar-potential kernel, S(r_i - r_j) = (1/4pi) int_{V_j} grad'(1/|r - r'|),
//    target at the cell centre.  Closed form: each component is the difference
//    of the potentials of the two opposite faces of the source cell; a face
//    potential is the four-corner sum of the rectangle primitive
//        F(y, z) = y asinh(z / sqrt(xi^2+y^2)) + z asinh(y / sqrt(xi^2+z^2))
//                  - xi atan(y z / (xi R)).
// N: demagnetisation tensor, Newell-Williams-Dunlop f / g functions under the
//    27-point second difference, divided by 4 pi V.
// Beyond kFarCells (max-norm, in cells) both switch to 3-point Gauss-Legendre
// quadrature of the point kernel (source cell for S; source and target cells
// for N), where the closed forms lose digits to cancellation.
//
// Spectra: the real-space kernel of one z offset is laid on the circular
// Qx x Qy grid (window |d| <= W, zero elsewhere), transformed by the FP64
// shared-memory FFT along x, transposed, transformed along y, and the real or
// imaginary part of the kx <= Qx/2, ky <= Qy/2 quarter is kept.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "fft.cuh"
#include "mm_internal.h"

namespace mm {

constexpr int kFarCells = 16;
constexpr double kPi = 3.14159265358979323846;

cudaError_t init_fft_constants_kgen() { return upload_roots(); }

// 3-point Gauss-Legendre on [-1, 1]
__constant__ double c_gl_x[3] = {-0.77459666924148337704, 0.0, 0.77459666924148337704};
__constant__ double c_gl_w[3] = {0.55555555555555555556, 0.88888888888888888889,
                                 0.55555555555555555556};

__device__ __forceinline__ double asinh_ratio(double num, double den2) {
  return den2 > 0.0 ? asinh(num / sqrt(den2)) : 0.0;
}

__device__ double rect_F(double xi, double y, double z) {
  const double R = sqrt(xi * xi + y * y + z * z);
  double v = y * asinh_ratio(z, xi * xi + y * y) + z * asinh_ratio(y, xi * xi + z * z);
  const double den = xi * R;
  if (den != 0.0) v -= xi * atan(y * z / den);
  return v;
}

__device__ double rect_pot(double xi, double y1, double y2, double z1, double z2) {
  return rect_F(xi, y2, z2) - rect_F(xi, y1, z2) - rect_F(xi, y2, z1) + rect_F(xi, y1, z1);
}

__device__ void S_closed(double X, double Y, double Z, double a, double b, double c, double* S) {
  const double k = 1.0 / (4.0 * kPi);
  S[0] = k * (rect_pot(X - 0.5 * a, Y - 0.5 * b, Y + 0.5 * b, Z - 0.5 * c, Z + 0.5 * c) -
              rect_pot(X + 0.5 * a, Y - 0.5 * b, Y + 0.5 * b, Z - 0.5 * c, Z + 0.5 * c));
  S[1] = k * (rect_pot(Y - 0.5 * b, X - 0.5 * a, X + 0.5 * a, Z - 0.5 * c, Z + 0.5 * c) -
              rect_pot(Y + 0.5 * b, X - 0.5 * a, X + 0.5 * a, Z - 0.5 * c, Z + 0.5 * c));
  S[2] = k * (rect_pot(Z - 0.5 * c, X - 0.5 * a, X + 0.5 * a, Y - 0.5 * b, Y + 0.5 * b) -
              rect_pot(Z + 0.5 * c, X - 0.5 * a, X + 0.5 * a, Y - 0.5 * b, Y + 0.5 * b));
}

__device__ void S_far(double X, double Y, double Z, double a, double b, double c, double* S) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) {
        const double w = c_gl_w[i] * c_gl_w[j] * c_gl_w[k] * 0.125;
        const double dx = X - 0.5 * a * c_gl_x[i];
        const double dy = Y - 0.5 * b * c_gl_x[j];
        const double dz = Z - 0.5 * c * c_gl_x[k];
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double ir3 = 1.0 / (r2 * sqrt(r2));
        s0 += w * dx * ir3;
        s1 += w * dy * ir3;
        s2 += w * dz * ir3;
      }
  const double k = a * b * c / (4.0 * kPi);
  S[0] = k * s0; S[1] = k * s1; S[2] = k * s2;
}

__device__ double newell_f(double x, double y, double z) {
  const double x2 = x * x, y2 = y * y, z2 = z * z;
  const double R = sqrt(x2 + y2 + z2);
  double v = 0.5 * y * (z2 - x2) * asinh_ratio(y, x2 + z2) + 0.5 * z * (y2 - x2) * asinh_ratio(z, x2 + y2);
  const double den = x * R;
  if (den != 0.0) v -= x * y * z * atan(y * z / den);
  v += (2.0 * x2 - y2 - z2) * R / 6.0;
  return v;
}

__device__ double newell_g(double x, double y, double z) {
  const double x2 = x * x, y2 = y * y, z2 = z * z;
  const double R = sqrt(x2 + y2 + z2);
  double v = x * y * z * asinh_ratio(z, x2 + y2) + y * (3.0 * z2 - y2) * asinh_ratio(x, y2 + z2) / 6.0 +
             x * (3.0 * z2 - x2) * asinh_ratio(y, x2 + z2) / 6.0;
  double den = z * R;
  if (den != 0.0) v -= z2 * z * atan(x * y / den) / 6.0;
  den = y * R;
  if (den != 0.0) v -= 0.5 * z * y2 * atan(x * z / den);
  den = x * R;
  if (den != 0.0) v -= 0.5 * z * x2 * atan(y * z / den);
  v -= x * y * R / 3.0;
  return v;
}

// comp: 0 xx, 1 yy, 2 zz, 3 xy, 4 xz, 5 yz
__device__ double N_closed(int comp, double X, double Y, double Z, double a, double b, double c) {
  double sum = 0.0;
  for (int ex = -1; ex <= 1; ++ex) {
    const double wx = ex == 0 ? 2.0 : -1.0;
    const double x = X + ex * a;
    for (int ey = -1; ey <= 1; ++ey) {
      const double wy = ey == 0 ? 2.0 : -1.0;
      const double y = Y + ey * b;
      for (int ez = -1; ez <= 1; ++ez) {
        const double wz = ez == 0 ? 2.0 : -1.0;
        const double z = Z + ez * c;
        double f;
        switch (comp) {
          case 0: f = newell_f(x, y, z); break;
          case 1: f = newell_f(y, x, z); break;
          case 2: f = newell_f(z, x, y); break;
          case 3: f = newell_g(x, y, z); break;
          case 4: f = newell_g(x, z, y); break;
          default: f = newell_g(y, z, x); break;
        }
        sum += wx * wy * wz * f;
      }
    }
  }
  return sum / (4.0 * kPi * a * b * c);
}

__device__ void N_far(double X, double Y, double Z, double a, double b, double c, double* N) {
  // average over target and source GL points of the point-dipole tensor; the
  // 9 (target, source) pairs per axis collapse to 5 distinct differences
  double t[5], wt[5];
  {
    const double g = c_gl_x[2];
    const double w0 = c_gl_w[0] * 0.5, w1 = c_gl_w[1] * 0.5;
    t[0] = -2.0 * g; wt[0] = w0 * w0;
    t[1] = -g;       wt[1] = 2.0 * w0 * w1;
    t[2] = 0.0;      wt[2] = 2.0 * w0 * w0 + w1 * w1;
    t[3] = g;        wt[3] = 2.0 * w0 * w1;
    t[4] = 2.0 * g;  wt[4] = w0 * w0;
  }
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j)
      for (int k = 0; k < 5; ++k) {
        const double w = wt[i] * wt[j] * wt[k];
        const double dx = X + 0.5 * a * t[i];
        const double dy = Y + 0.5 * b * t[j];
        const double dz = Z + 0.5 * c * t[k];
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double ir5 = 1.0 / (r2 * r2 * sqrt(r2));
        acc[0] += w * (3.0 * dx * dx - r2) * ir5;
        acc[1] += w * (3.0 * dy * dy - r2) * ir5;
        acc[2] += w * (3.0 * dz * dz - r2) * ir5;
        acc[3] += w * 3.0 * dx * dy * ir5;
        acc[4] += w * 3.0 * dx * dz * ir5;
        acc[5] += w * 3.0 * dy * dz * ir5;
      }
  const double k = -a * b * c / (4.0 * kPi);
  for (int q = 0; q < 6; ++q) N[q] = k * acc[q];
}

__device__ __forceinline__ bool is_far(double ix, double iy, double iz) {
  return fmax(fabs(ix), fmax(fabs(iy), fabs(iz))) > kFarCells + 1e-9;
}

// acc += w K(offset (ix, iy, iz) cells): S (3 values) or N (6 values)
__device__ __forceinline__ void add_kernel(int kind, double ix, double iy, int iz, double a, double b,
                                           double c, double w, double* acc) {
  const double X = ix * a, Y = iy * b, Z = iz * c;
  if (kind == 0) {
    double S[3];
    if (is_far(ix, iy, iz)) S_far(X, Y, Z, a, b, c, S);
    else S_closed(X, Y, Z, a, b, c, S);
    for (int q = 0; q < 3; ++q) acc[q] += w * S[q];
  } else {
    double N[6];
    if (is_far(ix, iy, iz)) N_far(X, Y, Z, a, b, c, N);
    else
      for (int q = 0; q < 6; ++q) N[q] = N_closed(q, X, Y, Z, a, b, c);
    for (int q = 0; q < 6; ++q) acc[q] += w * N[q];
  }
}

// Real-space kernel of one z offset on the circular grid, as complex (re, 0).
// kind 0: S (ncomp 3), kind 1: N (ncomp 6).  out[comp][y][x].  An open axis
// keeps the offsets |d| <= W; a periodic one (px, py) keeps every offset of the
// period and sums the images d + i Q, |i| <= R; at the Nyquist offset Q/2 of an
// even period it averages the image sums of +Q/2 and -Q/2, so the periodic
// kernel stays exactly even or odd along that axis.
__global__ void k_gen_plane(double2* out, int kind, int Qx, int Qy, int Wx, int Wy, int dz, double a,
                            double b, double c, int px, int py, int R) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= Qx) return;
  const int sx = 2 * x > Qx ? x - Qx : x;
  const int sy = 2 * y > Qy ? y - Qy : y;
  const size_t plane = (size_t)Qx * Qy;
  const size_t o = (size_t)y * Qx + x;
  const bool inside = (px || (sx >= -Wx && sx <= Wx)) && (py || (sy >= -Wy && sy <= Wy));
  const int ncomp = kind == 0 ? 3 : 6;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  if (inside) {
    const bool nyx = px && 2 * x == Qx, nyy = py && 2 * y == Qy;
    const int Rx = px ? R : 0, Ry = py ? R : 0;
    const double w = (nyx ? 0.5 : 1.0) * (nyy ? 0.5 : 1.0);
    for (int fx = 0; fx <= (nyx ? 1 : 0); ++fx)
      for (int fy = 0; fy <= (nyy ? 1 : 0); ++fy) {
        const int bx = fx ? -sx : sx, by = fy ? -sy : sy;
        for (int i = -Rx; i <= Rx; ++i)
          for (int j = -Ry; j <= Ry; ++j)
            add_kernel(kind, (double)bx + (double)i * Qx, (double)by + (double)j * Qy, dz, a, b, c, w, acc);
      }
  }
  for (int q = 0; q < ncomp; ++q) out[q * plane + o] = make_double2(acc[q], 0.0);
}

// Point evaluation of S (3) or N (6) at listed offsets (metres), for tests.
__global__ void k_eval_points(int kind, int n, const double* off, double a, double b, double c,
                              double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double X = off[3 * i], Y = off[3 * i + 1], Z = off[3 * i + 2];
  const bool far = is_far(X / a, Y / b, Z / c);
  if (kind == 0) {
    double S[3];
    if (far) S_far(X, Y, Z, a, b, c, S);
    else S_closed(X, Y, Z, a, b, c, S);
    for (int q = 0; q < 3; ++q) out[3 * i + q] = S[q];
  } else {
    double N[6];
    if (far) N_far(X, Y, Z, a, b, c, N);
    else
      for (int q = 0; q < 6; ++q) N[q] = N_closed(q, X, Y, Z, a, b, c);
    for (int q = 0; q < 6; ++q) out[6 * i + q] = N[q];
  }
}

// Forward FFT of contiguous lines, natural-order output (FP64, setup only).
__global__ void __launch_bounds__(256) k_fft_lines_d(double2* data, int nlines, FftTables T) {
  extern __shared__ double2 smd[];
  const int L = T.plan.L;
  const int line = blockIdx.x;
  if (line >= nlines) return;
  double2* g = data + (size_t)line * L;
  for (int i = threadIdx.x; i < L; i += blockDim.x) smd[i] = g[i];
  __syncthreads();
  fft_smem<kFwdDif, double2>(smd, L, 1, T.plan, T.tw_d, 0, blockDim.x);
  for (int k = threadIdx.x; k < L; k += blockDim.x) g[k] = smd[T.pos[k]];
}

__global__ void k_transpose_d(const double2* in, double2* out, int rows, int cols) {
  __shared__ double2 tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = by + i, c = bx + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = bx + i, r = by + threadIdx.x;
    if (r < rows && c < cols) out[(size_t)c * rows + r] = tile[threadIdx.x][i];
  }
}

// spec is [kx][ky] (Qx x Qy); keep kx <= Qx/2, ky <= Qy/2, real or imaginary part
__global__ void k_extract_quarter(const double2* spec, double* out, int Qx, int Qy, int kxh, int kyq,
                                  int take_imag) {
  const int ky = blockIdx.x * blockDim.x + threadIdx.x;
  const int kx = blockIdx.y;
  if (ky >= kyq || kx >= kxh) return;
  const double2 v = spec[(size_t)kx * Qy + ky];
  out[(size_t)kx * kyq + ky] = take_imag ? v.y : v.x;
}

// T[o][jz][c] = scale * sum_zb W[o][zb] Sq[(zb - jz) - dz_lo][c]  (quarter planes)
__global__ void k_mix_T(const double* Sq, const double* W, float* T, int n_out, int nz, int bz,
                        int dz_first_plane_offset, size_t qsize, double scale) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= qsize) return;
  const int c = blockIdx.y;
  const int oj = blockIdx.z;  // o * nz + jz
  const int o = oj / nz, jz = oj - o * nz;
  double acc = 0.0;
  for (int zb = 0; zb < bz; ++zb) {
    const double w = W[o * bz + zb];
    if (w == 0.0) continue;
    const int plane = zb - jz + dz_first_plane_offset;
    acc += w * Sq[((size_t)plane * 3 + c) * qsize + i];
  }
  T[((size_t)oj * 3 + c) * qsize + i] = (float)(scale * acc);
}

// Componentwise field variant: TN[(a n_out + o) nz + jz][b] = scale * sum_zb
// W[o][zb] N_ab((zb - jz) - dz_lo), from the six N components of every z
// offset (Nq6 [plane][6][qsize], xx yy zz xy xz yz).
__global__ void k_mix_TN(const double* Nq6, const double* W, float* T, int n_out, int nz, int bz,
                         size_t qsize, double scale) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= qsize) return;
  const int a = blockIdx.y / 3, b = blockIdx.y - 3 * (blockIdx.y / 3);
  const int comp = a == b ? a : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5));
  const int oj = blockIdx.z;  // o * nz + jz
  const int o = oj / nz, jz = oj - o * nz;
  double acc = 0.0;
  for (int zb = 0; zb < bz; ++zb) {
    const double w = W[o * bz + zb];
    if (w == 0.0) continue;
    const int plane = zb - jz + nz - 1;
    acc += w * Nq6[((size_t)plane * 6 + comp) * qsize + i];
  }
  T[((((size_t)a * n_out + o) * nz + jz) * 3 + b) * qsize + i] = (float)(scale * acc);
}

__global__ void k_scale_to_float(const double* in, float* out, size_t n, double scale) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)(scale * in[i]);
}

// ------------------------------------------------------------------ host

cudaError_t eval_points_fp64(int kind, int n, const double* off_dev, double a, double b, double c,
                             double* out_dev, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_eval_points<<<(n + 127) / 128, 128, 0, st>>>(kind, n, off_dev, a, b, c, out_dev);
  return cudaGetLastError();
}

// Spectrum quarters of `ncomp` kernel components for one z offset.
// work: 2 * ncomp * Qx * Qy double2; out_q: ncomp quarter planes (double).
static cudaError_t plane_spectra(int kind, int ncomp, const KernelPlan& K, int dz, double a,
                                 double b, double c, const FftTables& fx, const FftTables& fy,
                                 double2* work, double* out_q, const int* take_imag, cudaStream_t st) {
  const int Qx = K.Qx, Qy = K.Qy;
  const size_t plane = (size_t)Qx * Qy;
  double2* A = work;
  double2* B = work + ncomp * plane;
  dim3 g((Qx + 127) / 128, Qy);
  k_gen_plane<<<g, 128, 0, st>>>(A, kind, Qx, Qy, K.Wx, K.Wy, dz, a, b, c, K.px, K.py, K.R);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int kxh = Qx / 2 + 1, kyq = Qy / 2 + 1;
  for (int q = 0; q < ncomp; ++q) {
    size_t smem = sizeof(double2) * Qx;
    cudaFuncSetAttribute(k_fft_lines_d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double2) * (Qx > Qy ? Qx : Qy)));
    k_fft_lines_d<<<Qy, 256, smem, st>>>(A + q * plane, Qy, fx);
    dim3 tg((Qx + 31) / 32, (Qy + 31) / 32);
    k_transpose_d<<<tg, dim3(32, 8), 0, st>>>(A + q * plane, B + q * plane, Qy, Qx);
    smem = sizeof(double2) * Qy;
    k_fft_lines_d<<<Qx, 256, smem, st>>>(B + q * plane, Qx, fy);
    dim3 eg((kyq + 127) / 128, kxh);
    k_extract_quarter<<<eg, 128, 0, st>>>(B + q * plane, out_q + (size_t)q * kxh * kyq, Qx, Qy, kxh, kyq,
                                          take_imag[q]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t build_N_spectra(const KernelPlan& K, const FftTables& fx, const FftTables& fy, double a,
                            double b, double c, double scale, float* Nq, double2* work, double* qbuf,
                            cudaStream_t st) {
  const int kxh = K.Qx / 2 + 1, kyq = K.Qy / 2 + 1;
  const size_t qsize = (size_t)kxh * kyq;
  static const int imag6[6] = {0, 0, 0, 0, 1, 1};
  for (int dz = 0; dz < K.nz; ++dz) {
    cudaError_t e = plane_spectra(1, 6, K, dz, a, b, c, fx, fy, work, qbuf, imag6, st);
    if (e != cudaSuccess) return e;
    // Nq layout [6][nz][kxh][kyq]
    for (int q = 0; q < 6; ++q) {
      const size_t n = qsize;
      k_scale_to_float<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
          qbuf + q * qsize, Nq + ((size_t)q * K.nz + dz) * qsize, n, scale);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t build_T_spectra(const KernelPlan& K, const FftTables& fx, const FftTables& fy, double a,
                            double b, double c, double scale, int box_lo_z, int bz, int n_out,
                            const double* W_dev, float* Tq, double2* work, double* Sq,
                            cudaStream_t st) {
  const int kxh = K.Qx / 2 + 1, kyq = K.Qy / 2 + 1;
  const size_t qsize = (size_t)kxh * kyq;
  static const int imag3[3] = {1, 1, 0};
  const int dz_lo = box_lo_z - (K.nz - 1);
  const int nplanes = bz + K.nz - 1;
  for (int p = 0; p < nplanes; ++p) {
    cudaError_t e = plane_spectra(0, 3, K, dz_lo + p, a, b, c, fx, fy, work,
                                  Sq + (size_t)p * 3 * qsize, imag3, st);
    if (e != cudaSuccess) return e;
  }
  // plane index of offset dz = (box_lo_z + zb) - jz is (zb - jz) + (nz - 1)
  dim3 g((unsigned)((qsize + 255) / 256), 3, n_out * K.nz);
  k_mix_T<<<g, 256, 0, st>>>(Sq, W_dev, Tq, n_out, K.nz, bz, K.nz - 1, qsize, scale);
  return cudaGetLastError();
}

cudaError_t build_TN_spectra(const KernelPlan& K, const FftTables& fx, const FftTables& fy, double a,
                             double b, double c, double scale, int box_lo_z, int bz, int n_out,
                             const double* W_dev, float* TN, double2* work, double* Nq6, cudaStream_t st) {
  const size_t qsize = (size_t)(K.Qx / 2 + 1) * (K.Qy / 2 + 1);
  static const int imag6[6] = {0, 0, 0, 0, 1, 1};
  const int dz_lo = box_lo_z - (K.nz - 1);
  const int nplanes = bz + K.nz - 1;
  for (int p = 0; p < nplanes; ++p) {
    cudaError_t e = plane_spectra(1, 6, K, dz_lo + p, a, b, c, fx, fy, work,
                                  Nq6 + (size_t)p * 6 * qsize, imag6, st);
    if (e != cudaSuccess) return e;
  }
  dim3 g((unsigned)((qsize + 255) / 256), 9, n_out * K.nz);
  k_mix_TN<<<g, 256, 0, st>>>(Nq6, W_dev, TN, n_out, K.nz, bz, qsize, scale);
  return cudaGetLastError();
}

cudaError_t build_S_planes(const KernelPlan& K, const FftTables& fx, const FftTables& fy, double a, double b,
                           double c, double scale, int dz_lo, int nplanes, float* Sq, double2* work,
                           double* qtmp, cudaStream_t st) {
  static const int imag3[3] = {1, 1, 0};
  const size_t qsize = (size_t)(K.Qx / 2 + 1) * (K.Qy / 2 + 1);
  for (int p = 0; p < nplanes; ++p) {
    cudaError_t e = plane_spectra(0, 3, K, dz_lo + p, a, b, c, fx, fy, work, qtmp, imag3, st);
    if (e != cudaSuccess) return e;
    const size_t n = 3 * qsize;
    k_scale_to_float<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(qtmp, Sq + (size_t)p * n, n, scale);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------------ 3D spectra
// q2 [Qz][qsize] (real) -> z lines [qsize][Qz] (complex; the 2D value was the
// real or the imaginary part of the 2D spectrum)
__global__ void k_zlines(const double* q2, double2* zl, int Qz, size_t qsize, int imag2d) {
  __shared__ double tile[32][33];
  const size_t i0 = (size_t)blockIdx.x * 32;
  const int z0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int z = z0 + r;
    const size_t i = i0 + threadIdx.x;
    tile[r][threadIdx.x] = (z < Qz && i < qsize) ? q2[(size_t)z * qsize + i] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const size_t i = i0 + r;
    const int z = z0 + threadIdx.x;
    if (i < qsize && z < Qz) {
      const double v = tile[threadIdx.x][r];
      zl[i * Qz + z] = imag2d ? make_double2(0.0, v) : make_double2(v, 0.0);
    }
  }
}

// z-transformed lines [qsize][Qz] -> out [qsize][kzq] (real or imaginary part, scaled)
__global__ void k_extract_kz(const double2* zl, float* out, int Qz, int kzq, size_t qsize, int take_imag,
                             double scale) {
  const size_t n = qsize * kzq;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t q = i / kzq;
  const int kz = (int)(i - q * kzq);
  const double2 v = zl[q * Qz + kz];
  out[i] = (float)(scale * (take_imag ? v.y : v.x));
}

// 3D spectra: the 2D quarter spectra of every z offset |dz| <= Wz (laid on
// the circular z grid), transformed along z in FP64; kz <= Qz/2 is kept.
cudaError_t build_spectra_3d(int kind, const KernelPlan3& K, const FftTables& fx, const FftTables& fy,
                             const FftTables& fz, double a, double b, double c, double scale, float* out,
                             double2* work, double* q2, double* qtmp, double2* zl, cudaStream_t st) {
  const int ncomp = kind == 0 ? 3 : 6;
  static const int imagS[3] = {1, 1, 0};           // 2D: S_x, S_y odd in-plane
  static const int imagN[6] = {0, 0, 0, 0, 1, 1};  // 2D: N_xz, N_yz odd in x or y alone
  const int* imag2d = kind == 0 ? imagS : imagN;
  const int take_imag3 = kind == 0 ? 1 : 0;        // S imaginary, N real in 3D
  const int kxh = K.Qx / 2 + 1, kyq = K.Qy / 2 + 1, kzq = K.Qz / 2 + 1;
  const size_t qsize = (size_t)kxh * kyq;
  cudaError_t e = cudaMemsetAsync(q2, 0, sizeof(double) * ncomp * (size_t)K.Qz * qsize, st);
  if (e != cudaSuccess) return e;
  KernelPlan K2{};  // open boundaries: sources thicker than the direct z sum are not periodic
  K2.Qx = K.Qx; K2.Qy = K.Qy; K2.Wx = K.Wx; K2.Wy = K.Wy;
  for (int dz = -K.Wz; dz <= K.Wz; ++dz) {
    e = plane_spectra(kind, ncomp, K2, dz, a, b, c, fx, fy, work, qtmp, imag2d, st);
    if (e != cudaSuccess) return e;
    const int zs = dz < 0 ? dz + K.Qz : dz;
    for (int q = 0; q < ncomp; ++q) {
      e = cudaMemcpyAsync(q2 + ((size_t)q * K.Qz + zs) * qsize, qtmp + (size_t)q * qsize, sizeof(double) * qsize,
                          cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
  }
  cudaFuncSetAttribute(k_fft_lines_d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(sizeof(double2) * std::max(K.Qz, std::max(K.Qx, K.Qy))));
  for (int q = 0; q < ncomp; ++q) {
    dim3 tg((unsigned)((qsize + 31) / 32), (K.Qz + 31) / 32);
    k_zlines<<<tg, dim3(32, 8), 0, st>>>(q2 + (size_t)q * K.Qz * qsize, zl, K.Qz, qsize, imag2d[q]);
    k_fft_lines_d<<<(unsigned)qsize, 256, sizeof(double2) * K.Qz, st>>>(zl, (int)qsize, fz);
    const size_t n = qsize * kzq;
    k_extract_kz<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(zl, out + (size_t)q * n, K.Qz, kzq, qsize,
                                                              take_imag3, scale);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace mm
