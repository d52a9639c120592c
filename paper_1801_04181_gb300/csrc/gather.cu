// Tricubic B-spline evaluation of the source potential at the displaced target
// centres, stray field H = -grad phi and the Eq. (EQForce) force / interaction
// energy partial sums (Sec. II.A, III, III.A, IV.D).
//
// The slider moves rigidly, so every target centre has the same fractional
// position f in the source lattice: the 64 weights (cubic B-spline w, w', w''
// per axis at f, full float precision as in Sec. IV.D) are shared by all
// cells and the evaluation is a separable 4-tap filter of the coefficient box.
// A CTA takes 32 x 8 target columns and up to four layers (thick targets
// are split into chunks of four): it filters the (32 + 3) x (8 + 3) x
// (layers + 3) coefficient tile along x for the three derivative orders (into
// shared memory), then each thread finishes y and z for one (x, y) column.
//
// Per cell it writes H (A/m) and accumulates sum m . grad phi and
// sum_a m_a d_a d_b phi (FP32 within a warp, double-float across warps and tiles);
// the constants mu0 V Ms_t turn them into E and F (F_t = -mu0 V Ms_t sum Hess(phi) m).
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "mm_internal.h"
#include "spline_w.cuh"

namespace mm {

constexpr int TX = 32, TY = 8;

// y and z stages for one target column (x, y), the NZ layers z0 .. z0 + NZ - 1.
template <int NZ>
__device__ __forceinline__ void gather_column(const GatherJob& J, const float* A, int a_n,
                                              const float (*w_s)[12], int tx, int ty, int x, int y, int z0,
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
  const size_t N = (size_t)J.nx * J.ny * J.nz;
  float m[3][NZ];
#pragma unroll
  for (int zl = 0; zl < NZ; ++zl) {
    const size_t cell = ((size_t)(z0 + zl) * J.ny + y) * J.nx + x;
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
    const size_t cell = ((size_t)(z0 + zl) * J.ny + y) * J.nx + x;
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

// WRAP: some job has a periodic x or y (the taps wrap around the period);
// open boundaries run the instantiation without the wrapping arithmetic.
template <bool WRAP>
__global__ void __launch_bounds__(TX * TY, 4) k_gather(const Launch<GatherJob> Lc) {
  extern __shared__ float gsm[];
  __shared__ float w_s[3][12];
  __shared__ float red_s[TX * TY / 32][4];

  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const GatherJob& J = Lc.job[j];
  const int tile = blockIdx.x - Lc.tile_start[j];
  // tile -> (x tile, y tile, chunk of up to kMaxNz layers)
  const int ntx = (J.nx + TX - 1) / TX, nty = (J.ny + TY - 1) / TY;
  const int zc = tile / (ntx * nty);
  const int txy = tile - zc * ntx * nty;
  const int x0 = (txy % ntx) * TX;
  const int y0 = (txy / ntx) * TY;
  const int z0 = zc * kMaxNz;
  const int nz = min(kMaxNz, J.nz - z0);
  const int cz = nz + 3;

  // Every thread finds the integer tap shifts itself, so the coefficient
  // loads below are in flight before the barrier that publishes the weights.
  // sigma u in source lattice cells arrives split: floor(sigma u) -> integer
  // shift, the rest -> weights.
  int sh[3];
  bool bad = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int U = J.ucell[a];
    if (threadIdx.x == a) bspline_w(J.ufrac[a], w_s[a]);
    if (WRAP && a < 2 && J.wrapP[a] > 0) {
      // periodic axis: the coefficients span the period, the taps wrap
      const int P = J.wrapP[a];
      sh[a] = (J.tap0[a] + (U % P + P) % P) % P;
    } else {
      sh[a] = J.guard[a] + (U - J.U0[a]);
      const int need = (a == 0 ? J.nx : a == 1 ? J.ny : J.nz) + 3;
      const int have = a == 0 ? J.rx : a == 1 ? J.ry : J.rz;
      bad = bad || sh[a] < 0 || sh[a] + need > have;
    }
  }
  if (bad && threadIdx.x == 0) atomicOr(J.err, 1);

  // x-filtered coefficient rows A[d][zz][yy][x] (d: w, w', w''), one warp per
  // (zz, yy) row, filtered straight from global memory: a warp's four tap
  // loads are four coalesced 128-byte reads of one coefficient row (L1 hits
  // after the first).  Lanes past the target's edge read clamped, in-box
  // positions and their results are never used.  kRowBatch rows per warp
  // are loaded at once (all of them for open targets of up to two layers).
  float* A = gsm;
  const int a_n = cz * (TY + 3) * TX;
  const int sx = sh[0], sy = sh[1], sz = sh[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // column of each of the four x taps (wrapped around a periodic x)
  const int P0 = WRAP ? J.wrapP[0] : 0, P1 = WRAP ? J.wrapP[1] : 0;
  const int xb = min(x0 + lane, J.nx - 1) + sx;
  int xt[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) xt[k] = P0 > 0 ? (xb + k) % P0 : xb + k;
  const int nrow = cz * (TY + 3);
  constexpr int kWarps = TX * TY / 32;
  constexpr int kRowBatch = WRAP ? 2 : 7;  // the wrapped taps take registers of their own
  // every warp has rows in the first batch (nrow >= 44 > kWarps), so the
  // barrier that publishes the weights sits in that batch, after its loads
  for (int r0 = warp; r0 < nrow; r0 += kRowBatch * kWarps) {
    float c[kRowBatch][4];
    if (!bad) {
#pragma unroll
      for (int b = 0; b < kRowBatch; ++b) {
        const int r = min(r0 + b * kWarps, nrow - 1);
        const int zz = r / (TY + 3), yy = r - zz * (TY + 3);
        // rows past the target's last support row are clamped in the box
        // (a periodic y wraps them around the period instead)
        const int gy = P1 > 0 ? (y0 + yy + sy) % P1 : min(y0 + yy, J.ny + 2) + sy;
        const float* src = J.C + ((size_t)(z0 + zz + sz) * J.ry + gy) * J.rx;
#pragma unroll
        for (int k = 0; k < 4; ++k) c[b][k] = __ldg(src + xt[k]);
      }
    }
    if (r0 == warp) __syncthreads();  // the weights
    if (!bad) {
      const float w0 = w_s[0][0], w1 = w_s[0][1], w2 = w_s[0][2], w3 = w_s[0][3];
      const float d0 = w_s[0][4], d1 = w_s[0][5], d2 = w_s[0][6], d3 = w_s[0][7];
      const float e0 = w_s[0][8], e1 = w_s[0][9], e2 = w_s[0][10], e3 = w_s[0][11];
#pragma unroll
      for (int b = 0; b < kRowBatch; ++b) {
        const int r = r0 + b * kWarps;
        if (r >= nrow) break;
        const int o = r * TX + lane;
        A[o] = w0 * c[b][0] + w1 * c[b][1] + w2 * c[b][2] + w3 * c[b][3];
        A[a_n + o] = d0 * c[b][0] + d1 * c[b][1] + d2 * c[b][2] + d3 * c[b][3];
        A[2 * a_n + o] = e0 * c[b][0] + e1 * c[b][1] + e2 * c[b][2] + e3 * c[b][3];
      }
    }
  }
  __syncthreads();

  const int tx = threadIdx.x % TX;
  const int ty = threadIdx.x / TX;
  const int x = x0 + tx, y = y0 + ty;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  if (!bad && x < J.nx && y < J.ny) {
    switch (nz) {
      case 1: gather_column<1>(J, A, a_n, w_s, tx, ty, x, y, z0, acc); break;
      case 2: gather_column<2>(J, A, a_n, w_s, tx, ty, x, y, z0, acc); break;
      case 3: gather_column<3>(J, A, a_n, w_s, tx, ty, x, y, z0, acc); break;
      default: gather_column<4>(J, A, a_n, w_s, tx, ty, x, y, z0, acc); break;
    }
  }
  // FP32 within a warp (at most 32 x nz cells), FP64 from there on: the FP64
  // pipe of this GPU is narrow, and a warp's partial sum keeps ~1e-6 of the
  // magnitude of its terms, well inside the force tolerance
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float s = acc[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red_s[warp][q] = s;
  }
  __syncthreads();
  if (warp != 0) return;
  // the tile's four sums: lane c adds the warps in a fixed order in
  // double-float; the fixed-order reduction over tiles runs in a later launch
  if (lane < 4) {
    dfloat s = {0.f, 0.f};
    for (int w = 0; w < TX * TY / 32; ++w) s = df_add(s, dfloat{red_s[w][lane], 0.f});
    J.partial[(size_t)tile * 4 + lane] = make_float2(s.hi, s.lo);
  }
}

int gather_tiles(int nx, int ny, int nz) {
  return ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY) * ((nz + kMaxNz - 1) / kMaxNz);
}

size_t gather_smem(int nz) {
  const int cz = min(nz, kMaxNz) + 3;  // one chunk of layers
  return sizeof(float) * 3 * (size_t)cz * (TY + 3) * TX;
}

cudaError_t launch_gather(const Launch<GatherJob>& L, int nz_max, cudaStream_t st) {
  const size_t smem = gather_smem(nz_max);
  bool wrap = false;
  for (int i = 0; i < L.njobs; ++i) wrap = wrap || L.job[i].wrapP[0] > 0 || L.job[i].wrapP[1] > 0;
  auto k = wrap ? k_gather<true> : k_gather<false>;
  cudaFuncSetAttribute((const void*)k, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  k<<<grid, TX * TY, smem, st>>>(L);
  return cudaGetLastError();
}

}  // namespace mm
