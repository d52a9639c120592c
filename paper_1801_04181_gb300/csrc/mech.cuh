// Force / energy reduction and the slider's Dormand-Prince update, run by one
// block of 256 threads: a dedicated one-block launch (step-level updates) or
// the last block of a gather / LLG stage launch (per-stage updates).
//
// Eq. (EQForce) partial sums of both directions are reduced in a fixed order
// (thread t takes tiles t, t + 256, ..., then a fixed warp-shuffle and
// cross-warp order), so results are deterministic.  The slider obeys
// m x'' = k (v_d t + x0 - x) - gamma_v m x' + F . e (Sec. IV.B).
#pragma once
#include <cuda_runtime.h>

#include "mm_internal.h"

namespace mm {

__device__ __forceinline__ void mech_block(const MechParams& P) {
  __shared__ double mech_sh[8][9];
  MechState* S = P.state;
  double v[9];
  for (int d = 0; d < 2; ++d) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (P.partial[d]) {
      // read through L2: other blocks of the same launch wrote these
      const double2* pp = reinterpret_cast<const double2*>(P.partial[d]);
      for (int t = threadIdx.x; t < P.ntiles[d]; t += blockDim.x) {
        const double2 q0 = __ldcg(pp + 2 * t), q1 = __ldcg(pp + 2 * t + 1);
        a0 += q0.x; a1 += q0.y; a2 += q1.x; a3 += q1.y;
      }
    }
    v[4 * d + 0] = a0; v[4 * d + 1] = a1; v[4 * d + 2] = a2; v[4 * d + 3] = a3;
  }
  float emax = 0.f;
  for (int d = 0; d < 2; ++d)
    if (P.err_partial[d])
      for (int t = threadIdx.x; t < P.nerr[d]; t += blockDim.x) emax = fmaxf(emax, __ldcg(P.err_partial[d] + t));
  v[8] = emax;
#pragma unroll
  for (int c = 0; c < 8; ++c)
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
  for (int o = 16; o > 0; o >>= 1) v[8] = fmax(v[8], __shfl_down_sync(0xffffffffu, v[8], o));
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int c = 0; c < 9; ++c) mech_sh[threadIdx.x >> 5][c] = v[c];
  __syncthreads();
  if (threadIdx.x != 0) return;
  double red[2][4];
  for (int c = 0; c < 8; ++c) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += mech_sh[w][c];
    red[c / 4][c % 4] = s;
  }
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) emax = fmaxf(emax, (float)mech_sh[w][8]);

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
  } else if (P.mode == 5) {  // embedded error norm of the finished attempt
    S->err = emax;
  }
  if (P.mode == 0 || P.mode == 2 || P.mode == 3 || P.mode == 4)
    for (int c = 0; c < 3; ++c) S->u[c] = P.u_base[c] + S->xs * P.e[c] * P.inv_d[c];
}

// True in every thread of the block that finishes last among the `total`
// blocks sharing *ticket (which it resets for the next launch).  Each block
// calls it once, after its partial results are written.
__device__ __forceinline__ bool last_block(int* ticket, int total) {
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const int t = atomicAdd(ticket, 1);
    is_last = (t == total - 1);
    if (is_last) *ticket = 0;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

}  // namespace mm
