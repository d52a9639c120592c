// Eddy currents of a conducting magnet (Sec. III.B, the Torres method): the
// cell kernels of the electric-potential step and of the current.
//
// E_sol (step 1) and H_eddy (step 4) are cross products with the kernel S of
// the scalar potential, sum_j V(r_j) x S(r_i - r_j); each component of such a
// product is a dot product of S with a rearranged field,
//   (V x S)_x = S . (0, -V_z, V_y),  (V x S)_y = S . (V_z, 0, -V_x),
//   (V x S)_z = S . (-V_y, V_x, 0),
// so the host runs the potential path three times (k_cross_input builds the
// inputs, k_scale_into collects the outputs).
//
// Step 2, Laplace's equation for phi_E in the magnet with d phi / dn = E_sol . n
// on its surface, cell-centred: in every cell the sum over axes of
// w_a sum_{neighbours present} (phi_nb - phi) equals b = the surface fluxes,
// w_a = 1 / d_a^2, b = -sum_{a: + face on the surface} E_sol,a / d_a
// + sum_{a: - face on the surface} E_sol,a / d_a, with the mean of b removed
// (compatibility).  Solved by red-black successive over-relaxation in FP64
// (phi stored in FP32 would leave a residual floor of ~n 2e-7 of the source,
// too coarse to certify convergence); the host checks the residual every few
// sweeps, bounds the number of sweeps, and removes the mean of phi at the end.
#include <cuda_runtime.h>

#include "mm_internal.h"

namespace mm {

struct CellIdx {
  int x, y, z;
};

__device__ __forceinline__ CellIdx cell_of(size_t i, int nx, int ny) {
  const unsigned nxy = (unsigned)nx * (unsigned)ny;
  const int z = (int)((unsigned)i / nxy);
  const unsigned rem = (unsigned)i - (unsigned)z * nxy;
  const int y = (int)(rem / (unsigned)nx);
  return CellIdx{(int)(rem - (unsigned)y * (unsigned)nx), y, z};
}

__global__ void __launch_bounds__(256) k_cross_input(const float* __restrict__ V, size_t N, int comp,
                                                     float* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float vx = V[i], vy = V[N + i], vz = V[2 * N + i];
  float a = 0.f, b = 0.f, c = 0.f;
  if (comp == 0) { b = -vz; c = vy; }
  else if (comp == 1) { a = vz; c = -vx; }
  else { a = -vy; b = vx; }
  out[i] = a; out[N + i] = b; out[2 * N + i] = c;
}

__global__ void __launch_bounds__(256) k_scale_into(const float* __restrict__ in, size_t N, float s,
                                                    float* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) out[i] = s * in[i];
}

__global__ void __launch_bounds__(256) k_accumulate(const float* __restrict__ in, size_t N,
                                                    float* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) out[i] += in[i];
}

// b of every cell and per-block sums of b (for its mean)
__global__ void __launch_bounds__(256) k_eddy_source(const float* __restrict__ E, int nx, int ny, int nz,
                                                     double idx_, double idy, double idz, double* __restrict__ b,
                                                     double* __restrict__ part) {
  __shared__ double red[256];
  const size_t N = (size_t)nx * ny * nz;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < N) {
    const CellIdx c = cell_of(i, nx, ny);
    const double ex = E[i], ey = E[N + i], ez = E[2 * N + i];
    if (c.x == nx - 1) v -= ex * idx_;
    if (c.x == 0) v += ex * idx_;
    if (c.y == ny - 1) v -= ey * idy;
    if (c.y == 0) v += ey * idy;
    if (c.z == nz - 1) v -= ez * idz;
    if (c.z == 0) v += ez * idz;
    b[i] = v;
  }
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// fixed-order sum of nparts doubles into *out (one block)
__global__ void __launch_bounds__(256) k_sum_parts(const double* __restrict__ part, int nparts, double scale,
                                                   double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) s += part[k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int t = 128; t > 0; t >>= 1) {
    if (threadIdx.x < t) red[threadIdx.x] += red[threadIdx.x + t];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = scale * red[0];
}

// one colour of a red-black SOR sweep: cells with (x + y + z) % 2 == colour
__global__ void __launch_bounds__(256) k_sor(double* __restrict__ phi, const double* __restrict__ b,
                                             const double* __restrict__ bmean, int nx, int ny, int nz, double wx,
                                             double wy, double wz, double omega, int colour) {
  const size_t N = (size_t)nx * ny * nz;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const CellIdx c = cell_of(i, nx, ny);
  if (((c.x + c.y + c.z) & 1) != colour) return;
  double s = 0.0, w = 0.0;
  if (c.x > 0) { s += wx * phi[i - 1]; w += wx; }
  if (c.x < nx - 1) { s += wx * phi[i + 1]; w += wx; }
  if (c.y > 0) { s += wy * phi[i - nx]; w += wy; }
  if (c.y < ny - 1) { s += wy * phi[i + nx]; w += wy; }
  if (c.z > 0) { s += wz * phi[i - (size_t)nx * ny]; w += wz; }
  if (c.z < nz - 1) { s += wz * phi[i + (size_t)nx * ny]; w += wz; }
  if (w == 0.0) return;  // a single cell: phi = 0
  const double gs = (s - (b[i] - *bmean)) / w;
  phi[i] += omega * (gs - phi[i]);
}

// per-block max |A phi - b'| and max |b'|, and the block sum of phi (its mean)
__global__ void __launch_bounds__(256) k_sor_residual(const double* __restrict__ phi, const double* __restrict__ b,
                                                      const double* __restrict__ bmean, int nx, int ny, int nz,
                                                      double wx, double wy, double wz, double* __restrict__ part) {
  __shared__ double rmax[256], bmax[256], psum[256];
  const size_t N = (size_t)nx * ny * nz;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double r = 0.0, bb = 0.0, p = 0.0;
  if (i < N) {
    const CellIdx c = cell_of(i, nx, ny);
    const double f = phi[i];
    double s = 0.0;
    if (c.x > 0) s += wx * (phi[i - 1] - f);
    if (c.x < nx - 1) s += wx * (phi[i + 1] - f);
    if (c.y > 0) s += wy * (phi[i - nx] - f);
    if (c.y < ny - 1) s += wy * (phi[i + nx] - f);
    if (c.z > 0) s += wz * (phi[i - (size_t)nx * ny] - f);
    if (c.z < nz - 1) s += wz * (phi[i + (size_t)nx * ny] - f);
    const double bi = b[i] - *bmean;
    r = fabs(s - bi);
    bb = fabs(bi);
    p = f;
  }
  rmax[threadIdx.x] = r;
  bmax[threadIdx.x] = bb;
  psum[threadIdx.x] = p;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      rmax[threadIdx.x] = fmax(rmax[threadIdx.x], rmax[threadIdx.x + s]);
      bmax[threadIdx.x] = fmax(bmax[threadIdx.x], bmax[threadIdx.x + s]);
      psum[threadIdx.x] += psum[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = rmax[0];
    part[3 * blockIdx.x + 1] = bmax[0];
    part[3 * blockIdx.x + 2] = psum[0];
  }
}

// out[0] = max residual, out[1] = max |b'|, out[2] = mean phi (one block)
__global__ void __launch_bounds__(256) k_residual_reduce(const double* __restrict__ part, int nparts, double invN,
                                                         double* __restrict__ out) {
  __shared__ double rmax[256], bmax[256], psum[256];
  double r = 0.0, bb = 0.0, p = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) {
    r = fmax(r, part[3 * k]);
    bb = fmax(bb, part[3 * k + 1]);
    p += part[3 * k + 2];
  }
  rmax[threadIdx.x] = r;
  bmax[threadIdx.x] = bb;
  psum[threadIdx.x] = p;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      rmax[threadIdx.x] = fmax(rmax[threadIdx.x], rmax[threadIdx.x + s]);
      bmax[threadIdx.x] = fmax(bmax[threadIdx.x], bmax[threadIdx.x + s]);
      psum[threadIdx.x] += psum[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = rmax[0];
    out[1] = bmax[0];
    out[2] = psum[0] * invN;
  }
}

// E_irrot = -grad (phi - mean phi) with the boundary condition's ghost values,
// J = sigma (E_sol + E_irrot)
__global__ void __launch_bounds__(256) k_eddy_current(const double* __restrict__ phi, const double* __restrict__ stats,
                                                      const float* __restrict__ E, int nx, int ny, int nz, double dx,
                                                      double dy, double dz, double sigma, float* __restrict__ J) {
  const size_t N = (size_t)nx * ny * nz;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const CellIdx c = cell_of(i, nx, ny);
  const double mean = stats[2];
  const double f = phi[i] - mean;
  const double ex = E[i], ey = E[N + i], ez = E[2 * N + i];
  const double xp = c.x < nx - 1 ? phi[i + 1] - mean : f + dx * ex;
  const double xm = c.x > 0 ? phi[i - 1] - mean : f - dx * ex;
  const double yp = c.y < ny - 1 ? phi[i + nx] - mean : f + dy * ey;
  const double ym = c.y > 0 ? phi[i - nx] - mean : f - dy * ey;
  const size_t sz = (size_t)nx * ny;
  const double zp = c.z < nz - 1 ? phi[i + sz] - mean : f + dz * ez;
  const double zm = c.z > 0 ? phi[i - sz] - mean : f - dz * ez;
  J[i] = (float)(sigma * (ex - (xp - xm) / (2.0 * dx)));
  J[N + i] = (float)(sigma * (ey - (yp - ym) / (2.0 * dy)));
  J[2 * N + i] = (float)(sigma * (ez - (zp - zm) / (2.0 * dz)));
}

// Coupling into the time step: B = mu0 (H_demag + H_stray + H_ext + Ms y) of
// the step's last evaluation; with a previous B, dB/dt = (B - B_prev) / dt;
// then B_prev = B.
__global__ void __launch_bounds__(256) k_flux_rate(const float* __restrict__ Hself, const float* __restrict__ Hstray,
                                                   const float* __restrict__ y, size_t N, float hx, float hy, float hz,
                                                   float Ms, float mu0, float inv_dt, int have_prev,
                                                   float* __restrict__ Bprev, float* __restrict__ Bdot) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float he[3] = {hx, hy, hz};
  for (int c = 0; c < 3; ++c) {
    const size_t k = c * N + i;
    const float B = mu0 * (Hself[k] + Hstray[k] + he[c] + Ms * y[k]);
    if (have_prev) Bdot[k] = (B - Bprev[k]) * inv_dt;
    Bprev[k] = B;
  }
}

static unsigned blocks(size_t N) { return (unsigned)((N + 255) / 256); }

cudaError_t launch_flux_rate(const float* Hself, const float* Hstray, const float* y, size_t N, const double hext[3],
                             double Ms, double dt, int have_prev, float* Bprev, float* Bdot, cudaStream_t st) {
  k_flux_rate<<<blocks(N), 256, 0, st>>>(Hself, Hstray, y, N, (float)hext[0], (float)hext[1], (float)hext[2],
                                         (float)Ms, (float)(4e-7 * 3.14159265358979323846), (float)(1.0 / dt),
                                         have_prev, Bprev, Bdot);
  return cudaGetLastError();
}

cudaError_t launch_cross_input(const float* V, size_t N, int comp, float* out, cudaStream_t st) {
  k_cross_input<<<blocks(N), 256, 0, st>>>(V, N, comp, out);
  return cudaGetLastError();
}

cudaError_t launch_scale_into(const float* in, size_t N, float s, float* out, cudaStream_t st) {
  k_scale_into<<<blocks(N), 256, 0, st>>>(in, N, s, out);
  return cudaGetLastError();
}

cudaError_t launch_accumulate(const float* in, size_t N, float* out, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  k_accumulate<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(in, N, out);
  return cudaGetLastError();
}

int eddy_blocks(size_t N) { return (int)blocks(N); }

cudaError_t launch_eddy_source(const float* E, int nx, int ny, int nz, const double d[3], double* b, double* part,
                               double* bmean, cudaStream_t st) {
  const size_t N = (size_t)nx * ny * nz;
  k_eddy_source<<<blocks(N), 256, 0, st>>>(E, nx, ny, nz, 1.0 / d[0], 1.0 / d[1], 1.0 / d[2], b, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_parts<<<1, 256, 0, st>>>(part, (int)blocks(N), 1.0 / (double)N, bmean);
  return cudaGetLastError();
}

cudaError_t launch_sor_sweeps(double* phi, const double* b, const double* bmean, int nx, int ny, int nz,
                              const double d[3], double omega, int sweeps, cudaStream_t st) {
  const size_t N = (size_t)nx * ny * nz;
  const double wx = 1.0 / (d[0] * d[0]), wy = 1.0 / (d[1] * d[1]), wz = 1.0 / (d[2] * d[2]);
  for (int k = 0; k < sweeps; ++k)
    for (int colour = 0; colour < 2; ++colour)
      k_sor<<<blocks(N), 256, 0, st>>>(phi, b, bmean, nx, ny, nz, wx, wy, wz, omega, colour);
  return cudaGetLastError();
}

cudaError_t launch_sor_residual(const double* phi, const double* b, const double* bmean, int nx, int ny, int nz,
                                const double d[3], double* part, double* stats, cudaStream_t st) {
  const size_t N = (size_t)nx * ny * nz;
  const double wx = 1.0 / (d[0] * d[0]), wy = 1.0 / (d[1] * d[1]), wz = 1.0 / (d[2] * d[2]);
  k_sor_residual<<<blocks(N), 256, 0, st>>>(phi, b, bmean, nx, ny, nz, wx, wy, wz, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_residual_reduce<<<1, 256, 0, st>>>(part, (int)blocks(N), 1.0 / (double)N, stats);
  return cudaGetLastError();
}

cudaError_t launch_eddy_current(const double* phi, const double* stats, const float* E, int nx, int ny, int nz,
                                const double d[3], double sigma, float* J, cudaStream_t st) {
  const size_t N = (size_t)nx * ny * nz;
  k_eddy_current<<<blocks(N), 256, 0, st>>>(phi, stats, E, nx, ny, nz, d[0], d[1], d[2], sigma, J);
  return cudaGetLastError();
}

}  // namespace mm
