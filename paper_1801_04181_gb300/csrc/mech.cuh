// Force / energy reduction and the slider's Dormand-Prince update (modes 0-4),
// run by a one-block launch (during a step on a second stream, beside the LLG
// stage launch), and the embedded error norm of a step attempt (mode 5), run
// by the last block of the final stage launch.
//
// Eq. (EQForce) tile partials of both directions are reduced in double-float
// in a fixed order (thread t takes tiles t, t + 256, ..., then a fixed
// warp-shuffle and cross-warp order), so results are deterministic; the slider
// update itself is FP64, one thread.  The slider obeys
// m x'' = k (v_d t + x0 - x) - gamma_v m x' + F . e (Sec. IV.B).
#pragma once
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "mm_internal.h"

namespace mm {

// Every field of the state except the error norm (written by err_block alone,
// which can run at the same time in the last block of a stage launch).
__device__ __forceinline__ void store_state(MechState* d, const MechState& s) {
  d->x = s.x; d->v = s.v; d->t = s.t;
  d->xs = s.xs; d->vs = s.vs; d->ts = s.ts;
  for (int i = 0; i < 7; ++i) { d->kx[i] = s.kx[i]; d->kv[i] = s.kv[i]; }
  for (int c = 0; c < 3; ++c) { d->u[c] = s.u[c]; d->F_slider[c] = s.F_slider[c]; d->F_base[c] = s.F_base[c]; }
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c) { d->ucell[r][c] = s.ucell[r][c]; d->ufrac[r][c] = s.ufrac[r][c]; }
  d->E_slider = s.E_slider;
  d->E_base = s.E_base;
}

__device__ __forceinline__ void mech_block(const MechParams& P) {
  __shared__ dfloat mech_sh[8][8];
  // thread 0 updates a shared-memory copy of the state, read here so that its
  // loads overlap the reduction, and writes it back once
  __shared__ MechState Sc;
  if (threadIdx.x == 0) Sc = *P.state;
  dfloat v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = dfloat{0.f, 0.f};
  {
    // both directions, kBatch tiles per thread loaded before any is added
    // (one L2 round trip per batch instead of one per tile)
    constexpr int kBatch = 4;
    const float4* pp[2] = {reinterpret_cast<const float4*>(P.partial[0]),
                           reinterpret_cast<const float4*>(P.partial[1])};
    const int n[2] = {pp[0] ? P.nparts[0] : 0, pp[1] ? P.nparts[1] : 0};
    const int nmax = n[0] > n[1] ? n[0] : n[1];
    for (int base = threadIdx.x; base < nmax; base += kBatch * blockDim.x) {
      float4 q[kBatch][2][2];
#pragma unroll
      for (int u = 0; u < kBatch; ++u)
#pragma unroll
        for (int d = 0; d < 2; ++d) {
          const int t = base + u * blockDim.x;
          const bool ok = t < n[d];
          q[u][d][0] = ok ? __ldcg(pp[d] + 2 * t) : make_float4(0.f, 0.f, 0.f, 0.f);
          q[u][d][1] = ok ? __ldcg(pp[d] + 2 * t + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
      for (int u = 0; u < kBatch; ++u)
#pragma unroll
        for (int d = 0; d < 2; ++d) {
          if (base + u * blockDim.x >= n[d]) continue;
          v[4 * d + 0] = df_add(v[4 * d + 0], dfloat{q[u][d][0].x, q[u][d][0].y});
          v[4 * d + 1] = df_add(v[4 * d + 1], dfloat{q[u][d][0].z, q[u][d][0].w});
          v[4 * d + 2] = df_add(v[4 * d + 2], dfloat{q[u][d][1].x, q[u][d][1].y});
          v[4 * d + 3] = df_add(v[4 * d + 3], dfloat{q[u][d][1].z, q[u][d][1].w});
        }
    }
  }
#pragma unroll
  for (int c = 0; c < 8; ++c)
    for (int o = 16; o > 0; o >>= 1) v[c] = df_add(v[c], df_shfl_down(v[c], o));
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int c = 0; c < 8; ++c) mech_sh[threadIdx.x >> 5][c] = v[c];
  __syncthreads();
  if (threadIdx.x >= 32) return;
  // lanes 0-7 of warp 0 each finish one of the eight sums
  __shared__ double red_sh[8];
  if (threadIdx.x < 8) {
    dfloat s = {0.f, 0.f};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = df_add(s, mech_sh[w][threadIdx.x]);
    red_sh[threadIdx.x] = df_to_double(s);
  }
  __syncwarp();
  if (threadIdx.x != 0) return;
  double red[2][4];
  for (int c = 0; c < 8; ++c) red[c / 4][c % 4] = red_sh[c];

  MechState* S = &Sc;
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
      // 1 / m from the host: an FP64 division is ~600 cycles on this GPU
      S->kv[i - 1] = (P.k_spring * (P.v_drive * S->ts + P.x0_spring - S->xs) -
                      P.gamma_v * P.mass * S->vs + Fe) * P.inv_mass;
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
  }
  if (P.mode == 0 || P.mode == 2 || P.mode == 3 || P.mode == 4) {
    for (int c = 0; c < 3; ++c) S->u[c] = P.u_base[c] + S->xs * P.e[c] * P.inv_d[c];
    split_displacement(S->u, S->ucell, S->ufrac);
  }
  store_state(P.state, Sc);
}

// Mode 5 alone, for the last block of the final stage launch: the embedded
// error norm (max over both magnets' tile partials) into the state.  Kept
// apart from mech_block so the stage kernel does not carry its registers.
__device__ __forceinline__ void err_block(const MechParams& P) {
  __shared__ float em_s[32];
  float emax = 0.f;
  for (int d = 0; d < 2; ++d)
    if (P.err_partial[d])
      for (int t = threadIdx.x; t < P.nerr[d]; t += blockDim.x) emax = fmaxf(emax, __ldcg(P.err_partial[d] + t));
  for (int o = 16; o > 0; o >>= 1) emax = fmaxf(emax, __shfl_down_sync(0xffffffffu, emax, o));
  if ((threadIdx.x & 31) == 0) em_s[threadIdx.x >> 5] = emax;
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) emax = fmaxf(emax, em_s[w]);
  P.state->err = emax;
}

// True in every thread of the block that finishes last among the `total`
// blocks sharing *ticket (which it resets for the next launch).  Each block
// calls it once, after thread 0 alone has written the block's results: its
// fence orders them before the ticket.
__device__ __forceinline__ bool last_block(int* ticket, int total) {
  __shared__ int is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const int t = atomicAdd(ticket, 1);
    is_last = (t == total - 1);
    if (is_last) *ticket = 0;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

}  // namespace mm
