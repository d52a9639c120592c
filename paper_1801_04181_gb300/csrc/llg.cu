// LLG right-hand side, Dormand-Prince stage combination and the slider's
// equation of motion (Sec. II eq. 1, Sec. III, Sec. IV.B).
//
// k_stage: one thread per cell.  Effective field = own demag + stray field of
// the other magnet (both produced upstream) + 6-neighbour exchange (free
// ends) + uniaxial anisotropy + uniform Zeeman; torque in Landau-Lifshitz
// form  dm/dt = -gamma0/(1+alpha^2) [m x H + alpha m x (m x H)];  then the
// next stage input y + dt sum_j a_{i+1,j} k_j (or, at the last stage, the
// max-norm of the embedded 5(4) error).
// k_mech: one block.  Reduces the Eq. (EQForce) partial sums of both
// directions in a fixed order (deterministic, FP64) and advances the slider
// state m x'' = k (v_d t + x0 - x) - gamma_v m x' + F . e with the same tableau.
#include <cuda_runtime.h>

#include "mm_internal.h"

namespace mm {

__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

__global__ void __launch_bounds__(256) k_stage(const Launch<StageJob> Lc) {
  __shared__ float red[8];
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const StageJob& J = Lc.job[j];
  const int tile = blockIdx.x - Lc.tile_start[j];
  const int nx = J.nx, ny = J.ny, nz = J.nz;
  const size_t N = (size_t)nx * ny * nz;
  const size_t idx = (size_t)tile * blockDim.x + threadIdx.x;
  float emax = 0.f;
  if (idx < N) {
    const int x = (int)(idx % nx);
    const int y = (int)((idx / nx) % ny);
    const int z = (int)(idx / ((size_t)nx * ny));
    const float* m = J.ys;
    const float m0 = m[idx], m1 = m[N + idx], m2 = m[2 * N + idx];
    float h0 = J.Hself[idx] + J.Hstray[idx] + J.hext[0];
    float h1 = J.Hself[N + idx] + J.Hstray[N + idx] + J.hext[1];
    float h2 = J.Hself[2 * N + idx] + J.Hstray[2 * N + idx] + J.hext[2];
    // exchange, free ends: only neighbours inside the magnet contribute
    float e0 = 0.f, e1 = 0.f, e2 = 0.f;
#define MM_NB(cond, off, coef)                                          \
    if (cond) {                                                         \
      const size_t q = idx + (off);                                     \
      e0 += (coef) * (m[q] - m0);                                       \
      e1 += (coef) * (m[N + q] - m1);                                   \
      e2 += (coef) * (m[2 * N + q] - m2);                               \
    }
    MM_NB(x > 0, -1, J.ex[0])
    MM_NB(x < nx - 1, 1, J.ex[0])
    MM_NB(y > 0, -(ptrdiff_t)nx, J.ex[1])
    MM_NB(y < ny - 1, (ptrdiff_t)nx, J.ex[1])
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
    float* ko = J.k[J.stage - 1];
    ko[idx] = k0; ko[N + idx] = k1; ko[2 * N + idx] = k2;
    if (J.mode == 0 && J.stage < 7) {
      float s0 = J.y[idx], s1 = J.y[N + idx], s2 = J.y[2 * N + idx];
      for (int jj = 0; jj < J.stage - 1; ++jj) {
        const float a = J.comb[jj];
        if (a != 0.f) {
          const float* kj = J.k[jj];
          s0 += a * kj[idx]; s1 += a * kj[N + idx]; s2 += a * kj[2 * N + idx];
        }
      }
      const float a = J.comb[J.stage - 1];
      s0 += a * k0; s1 += a * k1; s2 += a * k2;
      J.ys_next[idx] = s0; J.ys_next[N + idx] = s1; J.ys_next[2 * N + idx] = s2;
    } else if (J.mode == 0 && J.stage == 7) {
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
      for (int jj = 0; jj < 6; ++jj) {
        const float a = J.ecoef[jj];
        if (a != 0.f) {
          const float* kj = J.k[jj];
          s0 += a * kj[idx]; s1 += a * kj[N + idx]; s2 += a * kj[2 * N + idx];
        }
      }
      s0 += J.ecoef[6] * k0; s1 += J.ecoef[6] * k1; s2 += J.ecoef[6] * k2;
      emax = fmaxf(fabsf(s0), fmaxf(fabsf(s1), fabsf(s2)));
    }
  }
  if (J.mode == 0 && J.stage == 7) {
    emax = warp_max(emax);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = emax;
    __syncthreads();
    if (threadIdx.x == 0) {
      float v = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmaxf(v, red[w]);
      J.err_partial[tile] = v;
    }
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

__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  __syncthreads();
  return s;  // valid in thread 0
}

__global__ void __launch_bounds__(256) k_mech(const MechParams P) {
  __shared__ double sh[8][9];
  MechState* S = P.state;
  // Eq. (EQForce) reductions in a fixed order: thread t sums tiles t, t+256, ...
  // then a fixed warp-shuffle and cross-warp order (deterministic)
  double v[9];
  for (int d = 0; d < 2; ++d) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (P.partial[d]) {
      const double4* pp = reinterpret_cast<const double4*>(P.partial[d]);
      for (int t = threadIdx.x; t < P.ntiles[d]; t += blockDim.x) {
        const double4 q = pp[t];
        a0 += q.x; a1 += q.y; a2 += q.z; a3 += q.w;
      }
    }
    v[4 * d + 0] = a0; v[4 * d + 1] = a1; v[4 * d + 2] = a2; v[4 * d + 3] = a3;
  }
  float emax = 0.f;
  if (P.mode == 0 && P.stage == 7)
    for (int d = 0; d < 2; ++d)
      if (P.err_partial[d])
        for (int t = threadIdx.x; t < P.nerr[d]; t += blockDim.x) emax = fmaxf(emax, P.err_partial[d][t]);
  v[8] = emax;
#pragma unroll
  for (int c = 0; c < 8; ++c)
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
  for (int o = 16; o > 0; o >>= 1) v[8] = fmax(v[8], __shfl_down_sync(0xffffffffu, v[8], o));
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int c = 0; c < 9; ++c) sh[threadIdx.x >> 5][c] = v[c];
  __syncthreads();
  if (threadIdx.x != 0) return;
  double red[2][4];
  for (int c = 0; c < 8; ++c) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w][c];
    red[c / 4][c % 4] = s;
  }
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) emax = fmaxf(emax, (float)sh[w][8]);

  if (P.mode == 0 || P.mode == 1) {
    for (int c = 0; c < 3; ++c) {
      if (P.partial[0]) S->F_slider[c] = P.Fscale[0] * red[0][c];
      if (P.partial[1]) S->F_base[c] = P.Fscale[1] * red[1][c];
    }
    if (P.partial[0]) S->E_slider = P.Escale[0] * red[0][3];
    if (P.partial[1]) S->E_base = P.Escale[1] * red[1][3];
  }
  const double dt = P.dt;
  if (P.mode == 0) {
    const int i = P.stage;
    const double Fe = S->F_slider[0] * P.e[0] + S->F_slider[1] * P.e[1] + S->F_slider[2] * P.e[2];
    if (P.move) {
      S->kx[i - 1] = S->vs;
      S->kv[i - 1] = (P.k_spring * (P.v_drive * S->ts + P.x0_spring - S->xs) -
                      P.gamma_v * P.mass * S->vs + Fe) / P.mass;
    } else {
      S->kx[i - 1] = 0.0;
      S->kv[i - 1] = 0.0;
    }
    if (i < 7) {
      double xs = S->x, vs = S->v;
      for (int jj = 0; jj < i; ++jj) {
        xs += dt * P.a[jj] * S->kx[jj];
        vs += dt * P.a[jj] * S->kv[jj];
      }
      S->xs = xs; S->vs = vs; S->ts = S->t + P.c_next * dt;
    } else {
      S->err = emax;
    }
  } else if (P.mode == 2) {  // stage 2 input from a stored k1
    S->xs = S->x + dt * P.a[0] * S->kx[0];
    S->vs = S->v + dt * P.a[0] * S->kv[0];
    S->ts = S->t + P.c_next * dt;
  } else if (P.mode == 3) {  // accept: stage-7 input is the 5th-order solution
    S->x = S->xs; S->v = S->vs; S->t = S->t + dt;
    S->kx[0] = S->kx[6]; S->kv[0] = S->kv[6];
    S->xs = S->x; S->vs = S->v; S->ts = S->t;
  } else if (P.mode == 4) {  // restart an attempt from the accepted state
    S->xs = S->x; S->vs = S->v; S->ts = S->t;
  }
  if (P.mode != 1)
    for (int c = 0; c < 3; ++c) S->u[c] = P.u_base[c] + S->xs * P.e[c] * P.inv_d[c];
}

cudaError_t launch_stage(const Launch<StageJob>& L, cudaStream_t st) {
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  k_stage<<<grid, 256, 0, st>>>(L);
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
