// LLG right-hand side, Dormand-Prince stage combination and the slider's
// equation of motion (Sec. II eq. 1, Sec. III, Sec. IV.B).
//
// k_stage: one thread per cell.  Effective field = own demag + stray field of
// the other magnet (both produced upstream) + 6-neighbour exchange (free
// ends) + uniaxial anisotropy + uniform Zeeman (+ the eddy field of a
// conducting magnet); torque in Landau-Lifshitz
// form  dm/dt = -gamma0/(1+alpha^2) [m x H + alpha m x (m x H)];  then the
// next stage input y + dt sum_j a_{i+1,j} k_j (or, at the last stage, the
// max-norm of the embedded 5(4) error).
// k_mech: one block.  Reduces the Eq. (EQForce) tile partials of both
// directions in a fixed order (deterministic, double-float) and advances the
// slider state
// m x'' = k (v_d t + x0 - x) - gamma_v m x' + F . e with the same tableau.
#include <cuda_runtime.h>

#include "mech.cuh"
#include "mm_internal.h"

namespace mm {

__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// WRAP: some job has periodic x or y (exchange neighbours wrap around the
// period); open boundaries run the instantiation without the wrap tests.
// EDDY: some job is a conducting magnet carrying an eddy field; the plain
// instantiation has no load of it (and no extra register pressure).
// SG > 0: every job is RK stage SG of mode 0 (the combination unrolls, its k
// loads can overlap); SG = 0: stage and mode of the job, at run time.
template <bool WRAP, bool EDDY, int SG>
__global__ void __launch_bounds__(256, 6) k_stage(const Launch<StageJob> Lc, const MechParams Perr, int* ticket) {
  __shared__ float red[8];
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const StageJob& J = Lc.job[j];
  const int tile = blockIdx.x - Lc.tile_start[j];
  const int nx = J.nx, ny = J.ny, nz = J.nz;
  const size_t N = (size_t)nx * ny * nz;
  const size_t idx = (size_t)tile * blockDim.x + threadIdx.x;
  float emax = 0.f;
  if (idx < N) {
    // 32-bit index arithmetic: a magnet holds at most 2^30 cells
    const unsigned nxy = (unsigned)nx * (unsigned)ny;
    const unsigned i32 = (unsigned)idx;
    const int z = (int)(i32 / nxy);
    const unsigned rem = i32 - (unsigned)z * nxy;
    const int y = (int)(rem / (unsigned)nx);
    const int x = (int)(rem - (unsigned)y * (unsigned)nx);
    const float* m = J.ys;
    const float m0 = m[idx], m1 = m[N + idx], m2 = m[2 * N + idx];
    float h0 = J.Hself[idx] + J.Hstray[idx] + J.hext[0];
    float h1 = J.Hself[N + idx] + J.Hstray[N + idx] + J.hext[1];
    float h2 = J.Hself[2 * N + idx] + J.Hstray[2 * N + idx] + J.hext[2];
    if (EDDY && J.Heddy) {  // conducting magnet: the eddy field of the last accepted step
      h0 += J.Heddy[idx];
      h1 += J.Heddy[N + idx];
      h2 += J.Heddy[2 * N + idx];
    }
    // exchange, free ends: only neighbours inside the magnet contribute;
    // periodic x / y: the neighbours wrap around the period
    float e0 = 0.f, e1 = 0.f, e2 = 0.f;
#define MM_NB(cond, off, coef)                                          \
    if (cond) {                                                         \
      const size_t q = idx + (off);                                     \
      e0 += (coef) * (m[q] - m0);                                       \
      e1 += (coef) * (m[N + q] - m1);                                   \
      e2 += (coef) * (m[2 * N + q] - m2);                               \
    }
    if constexpr (WRAP) {
      const bool wx = J.wrap[0] && nx > 1, wy = J.wrap[1] && ny > 1;
      MM_NB(x > 0 || wx, x > 0 ? -1 : (ptrdiff_t)nx - 1, J.ex[0])
      MM_NB(x < nx - 1 || wx, x < nx - 1 ? 1 : -((ptrdiff_t)nx - 1), J.ex[0])
      MM_NB(y > 0 || wy, y > 0 ? -(ptrdiff_t)nx : (ptrdiff_t)nx * (ny - 1), J.ex[1])
      MM_NB(y < ny - 1 || wy, y < ny - 1 ? (ptrdiff_t)nx : -(ptrdiff_t)nx * (ny - 1), J.ex[1])
    } else {
      MM_NB(x > 0, -1, J.ex[0])
      MM_NB(x < nx - 1, 1, J.ex[0])
      MM_NB(y > 0, -(ptrdiff_t)nx, J.ex[1])
      MM_NB(y < ny - 1, (ptrdiff_t)nx, J.ex[1])
    }
    MM_NB(z > 0, -(ptrdiff_t)nx * ny, J.ex[2])
    MM_NB(z < nz - 1, (ptrdiff_t)nx * ny, J.ex[2])
#undef MM_NB
    h0 += e0; h1 += e1; h2 += e2;
    const float proj = J.an * (m0 * J.ku[0] + m1 * J.ku[1] + m2 * J.ku[2]);
    h0 += proj * J.ku[0]; h1 += proj * J.ku[1]; h2 += proj * J.ku[2];
    if (J.Heff) {
      J.Heff[idx] = h0; J.Heff[N + idx] = h1; J.Heff[2 * N + idx] = h2;
    }
    // m x H and m x (m x H)
    const float c0 = m1 * h2 - m2 * h1;
    const float c1 = m2 * h0 - m0 * h2;
    const float c2 = m0 * h1 - m1 * h0;
    const float d0 = m1 * c2 - m2 * c1;
    const float d1 = m2 * c0 - m0 * c2;
    const float d2 = m0 * c1 - m1 * c0;
    const float k0 = J.pref * (c0 + J.alpha * d0);
    const float k1 = J.pref * (c1 + J.alpha * d1);
    const float k2 = J.pref * (c2 + J.alpha * d2);
    const int stage = SG > 0 ? SG : J.stage;
    const int mode = SG > 0 ? 0 : J.mode;
    float* ko = J.k[stage - 1];
    ko[idx] = k0; ko[N + idx] = k1; ko[2 * N + idx] = k2;
    if (mode == 0 && stage < 7) {
      float s0 = J.y[idx], s1 = J.y[N + idx], s2 = J.y[2 * N + idx];
      if constexpr (SG > 0) {
        // every a_ij below the diagonal enters (a zero one adds an exact zero)
#pragma unroll
        for (int jj = 0; jj < SG - 1; ++jj) {
          const float a = J.comb[jj];
          const float* kj = J.k[jj];
          s0 += a * kj[idx]; s1 += a * kj[N + idx]; s2 += a * kj[2 * N + idx];
        }
      } else {
        for (int jj = 0; jj < stage - 1; ++jj) {
          const float a = J.comb[jj];
          if (a != 0.f) {
            const float* kj = J.k[jj];
            s0 += a * kj[idx]; s1 += a * kj[N + idx]; s2 += a * kj[2 * N + idx];
          }
        }
      }
      const float a = J.comb[stage - 1];
      s0 += a * k0; s1 += a * k1; s2 += a * k2;
      J.ys_next[idx] = s0; J.ys_next[N + idx] = s1; J.ys_next[2 * N + idx] = s2;
    } else if (mode == 0 && stage == 7) {
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
      if constexpr (SG > 0) {
#pragma unroll
        for (int jj = 0; jj < 6; ++jj) {
          const float a = J.ecoef[jj];
          if (a != 0.f) {
            const float* kj = J.k[jj];
            s0 += a * kj[idx]; s1 += a * kj[N + idx]; s2 += a * kj[2 * N + idx];
          }
        }
      } else {
        for (int jj = 0; jj < 6; ++jj) {
          const float a = J.ecoef[jj];
          if (a != 0.f) {
            const float* kj = J.k[jj];
            s0 += a * kj[idx]; s1 += a * kj[N + idx]; s2 += a * kj[2 * N + idx];
          }
        }
      }
      s0 += J.ecoef[6] * k0; s1 += J.ecoef[6] * k1; s2 += J.ecoef[6] * k2;
      emax = fmaxf(fabsf(s0), fmaxf(fabsf(s1), fabsf(s2)));
    }
  }
  if ((SG > 0 ? SG == 7 : J.mode == 0 && J.stage == 7)) {
    emax = warp_max(emax);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = emax;
    __syncthreads();
    if (threadIdx.x == 0) {
      float v = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmaxf(v, red[w]);
      J.err_partial[tile] = v;
    }
    // the last block reduces the error norm of the attempt
    if (Perr.state && last_block(ticket, (int)gridDim.x)) err_block(Perr);
  }
}

// y_next = y + sum_j comb[j] k_j   (stage input built from stored k only)
__global__ void __launch_bounds__(256) k_combine(const Launch<CombineJob> Lc) {
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const CombineJob& J = Lc.job[j];
  const size_t i = (size_t)(blockIdx.x - Lc.tile_start[j]) * blockDim.x + threadIdx.x;
  const size_t n3 = 3 * J.n;
  if (i >= n3) return;
  float s = J.y[i];
  for (int jj = 0; jj < J.nk; ++jj) s += J.comb[jj] * J.k[jj][i];
  J.out[i] = s;
}

// y = normalise(src)  (accepted step)
__global__ void __launch_bounds__(256) k_normalise(const Launch<CombineJob> Lc) {
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const CombineJob& J = Lc.job[j];
  const size_t i = (size_t)(blockIdx.x - Lc.tile_start[j]) * blockDim.x + threadIdx.x;
  if (i >= J.n) return;
  const float a = J.y[i], b = J.y[J.n + i], c = J.y[2 * J.n + i];
  const float inv = rsqrtf(a * a + b * b + c * c);
  J.out[i] = a * inv; J.out[J.n + i] = b * inv; J.out[2 * J.n + i] = c * inv;
}

__global__ void __launch_bounds__(256) k_mech(const MechParams P) { mech_block(P); }

cudaError_t launch_stage(const Launch<StageJob>& L, const MechParams& Perr, int* ticket, cudaStream_t st) {
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  bool wrap = false, eddy = false;
  for (int i = 0; i < L.njobs; ++i) {
    wrap = wrap || L.job[i].wrap[0] || L.job[i].wrap[1];
    eddy = eddy || L.job[i].Heddy != nullptr;
  }
  // one RK stage of mode 0 for every job: the build for that stage (open
  // boundaries, no eddy field), else the run-time one
  int sg = L.job[0].mode == 0 ? L.job[0].stage : 0;
  for (int i = 1; i < L.njobs; ++i)
    if (L.job[i].mode != 0 || L.job[i].stage != sg) sg = 0;
  if (wrap || eddy) sg = 0;
  switch (sg) {
    case 1: k_stage<false, false, 1><<<grid, 256, 0, st>>>(L, Perr, ticket); break;
    case 2: k_stage<false, false, 2><<<grid, 256, 0, st>>>(L, Perr, ticket); break;
    case 3: k_stage<false, false, 3><<<grid, 256, 0, st>>>(L, Perr, ticket); break;
    case 4: k_stage<false, false, 4><<<grid, 256, 0, st>>>(L, Perr, ticket); break;
    case 5: k_stage<false, false, 5><<<grid, 256, 0, st>>>(L, Perr, ticket); break;
    case 6: k_stage<false, false, 6><<<grid, 256, 0, st>>>(L, Perr, ticket); break;
    case 7: k_stage<false, false, 7><<<grid, 256, 0, st>>>(L, Perr, ticket); break;
    default:
      if (wrap && eddy) k_stage<true, true, 0><<<grid, 256, 0, st>>>(L, Perr, ticket);
      else if (wrap) k_stage<true, false, 0><<<grid, 256, 0, st>>>(L, Perr, ticket);
      else if (eddy) k_stage<false, true, 0><<<grid, 256, 0, st>>>(L, Perr, ticket);
      else k_stage<false, false, 0><<<grid, 256, 0, st>>>(L, Perr, ticket);
  }
  return cudaGetLastError();
}
cudaError_t launch_combine(const Launch<CombineJob>& L, cudaStream_t st) {
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  k_combine<<<grid, 256, 0, st>>>(L);
  return cudaGetLastError();
}
cudaError_t launch_normalise(const Launch<CombineJob>& L, cudaStream_t st) {
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  k_normalise<<<grid, 256, 0, st>>>(L);
  return cudaGetLastError();
}
cudaError_t launch_mech(const MechParams& P, cudaStream_t st) {
  k_mech<<<1, 256, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace mm
