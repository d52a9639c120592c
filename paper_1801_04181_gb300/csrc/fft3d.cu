// FFT passes for thick magnets (nz > 4): the convolution of Sec. III.A with z
// by FFT, on a Qx x Qy x Qz circular grid.
//
//   x pass (k_xfwd, shared with thin films)          -> X1[plane][kx][y]
//   y forward (k_yfwd3): y FFT of each column        -> Y3[kx][ypos][plane]
//   z pass (k_zpass3): per (kx, y position) the z FFT of the three components,
//       H = -N.M and phi = S.M against the 3D kernel spectra, the inverse z
//       FFT, and the z prefilter of phi on the box  -> Z[plane][kx][ypos]
//   or, for sources of up to kMaxNzDirect layers, the direct z sum (k_zmix3)
//       with thin-film spectra (z prefilter folded in), y in natural order
//   y inverse (k_yinv3): inverse y FFT, demag rows and y prefilter
//                                                    -> Y[plane][kx][row]
//   x pass (k_xinv, shared)                          -> real rows
//
// Planes are (component, z layer) = c nz + z.  Y3 keeps the planes of one
// (kx, y position) contiguous so the z pass reads them as whole runs, and Z
// keeps y positions contiguous for the y inverse.  y positions stay in the
// DIF order of the forward transform; the inverse (DIT) takes them back.
//
// Kernel spectra (FP32, generated once in FP64) are stored for kx <= Qx/2,
// ky <= Qy/2, kz <= Qz/2.  Every component of N and S has a parity in each
// axis: the six N spectra are real (each off-diagonal is odd in exactly two
// axes), the three S spectra imaginary (each odd in one); mirrored ky or kz
// flips the sign of the components odd in that axis.
#include <algorithm>

#include "fft.cuh"
#include "mm_internal.h"
#include "prefilter.cuh"
#include "umma.cuh"

namespace mm {

// this translation unit's copy of the small-DFT roots (see fft.cuh)
cudaError_t init_fft_constants_3d() { return upload_roots(); }

// ------------------------------------------------------------------ y forward
// FIXP > 0: every job's y plan is fixed plan FIXP, run with its lengths as constants.
template <unsigned RSET, int FIXP>
__global__ void __launch_bounds__(256, 3) k_yfwd3(const Launch<YFwdJob> Lc) {
  extern __shared__ float2 sm[];
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const YFwdJob& J = Lc.job[j];
  const int tile = blockIdx.x - Lc.tile_start[j];
  const int ng = (J.planes + J.group - 1) / J.group;
  const int kx = tile / ng;
  const int p0 = (tile - kx * ng) * J.group;
  const int np = min(J.group, J.planes - p0);
  const int Q = FIXP ? FixedPlan<FIXP ? FIXP : 1>::L : J.fy.plan.L;
  const int ldl = Q + 1;  // odd stride: the plane-fastest reads below spread over the banks
  for (int l = 0; l < np; ++l) {
    const float2* col = J.in + ((size_t)(p0 + l) * J.kxh + kx) * J.ny;
    for (int y = threadIdx.x; y < Q; y += blockDim.x)
      sm[l * ldl + y] = y < J.ny ? col[y] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  if constexpr (FIXP > 0)
    fft_smem_plan<kFwdDif, FIXP, FixedPlan<FIXP>::L + 1>(sm, np, J.fy.plan, J.fy.tw_f, 0, blockDim.x);
  else
    fft_smem<kFwdDif, float2, RSET>(sm, ldl, np, J.fy.plan, J.fy.tw_f, 0, blockDim.x);
  if (J.natural) {
    // frequency ky read from its DIF position: whole contiguous output rows
    for (int l = 0; l < np; ++l) {
      float2* row = J.out + ((size_t)(p0 + l) * J.kxh + kx) * Q;
      for (int k = threadIdx.x; k < Q; k += blockDim.x) row[k] = sm[l * ldl + __ldg(J.fy.pos + k)];
    }
    return;
  }
  float2* dst = J.out + (size_t)kx * Q * J.planes + p0;
  for (int i = threadIdx.x; i < Q * np; i += blockDim.x) {
    const int p = i / np, l = i - p * np;
    dst[(size_t)p * J.planes + l] = sm[l * ldl + p];
  }
}

// ------------------------------------------------------------------ z pass
__device__ __forceinline__ float2 c_i_times(float2 m) { return make_float2(-m.y, m.x); }

template <unsigned RSET>
__global__ void __launch_bounds__(256, 2) k_zpass3(const Launch<ZJob> Lc) {
  extern __shared__ float2 sm[];
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const ZJob& J = Lc.job[j];
  const int tile = blockIdx.x - Lc.tile_start[j];
  const int Qy = J.fy.plan.L, Qz = J.fz.plan.L;
  const int zt = J.ztile;
  const int npt = (Qy + zt - 1) / zt;
  const int kx = tile / npt;
  const int y0 = (tile - kx * npt) * zt;
  const int nt = min(zt, Qy - y0);
  const int nz = J.nz, P3 = 3 * nz;
  const int ldz = Qz + 1;
  // lines: t * 3 + c (input, then H in place) for t < nt; phi line t at 3 zt + t
  float2* phi = sm + 3 * zt * ldz;
  int* tab = reinterpret_cast<int*>(sm + 4 * zt * ldz);

  const float2* src = J.in + ((size_t)kx * Qy + y0) * P3;
  for (int i = threadIdx.x; i < nt * P3; i += blockDim.x) {
    const int t = i / P3, q = i - t * P3;
    const int c = q / nz, z = q - c * nz;
    sm[(t * 3 + c) * ldz + z] = src[i];
  }
  const int pad = Qz - nz;
  for (int i = threadIdx.x; i < nt * 3 * pad; i += blockDim.x) {
    const int l = i / pad, z = nz + (i - l * pad);
    sm[l * ldz + z] = make_float2(0.f, 0.f);
  }
  if (J.do_C) build_pref_table(tab, J.r + 2 * kPrefWarm + kZChunk, J.box_lo, J.box_len, J.start, Qz, nullptr);
  __syncthreads();
  fft_smem<kFwdDif, float2, RSET>(sm, ldz, 3 * nt, J.fz.plan, J.fz.tw_f, 0, blockDim.x);

  // spectral products at the pair (kz, Qz - kz) of every y position of the tile
  const int half = Qz >> 1;
  const size_t kstride = (size_t)J.kxh * J.kyq * J.kzq;
  for (int i = threadIdx.x; i < nt * (half + 1); i += blockDim.x) {
    const int t = i / (half + 1), kz = i - t * (half + 1);
    const int ky = fft_freq(y0 + t, J.fy.plan);
    const bool ym = 2 * ky > Qy;
    const int kys = ym ? Qy - ky : ky;
    const bool two = kz != 0 && 2 * kz != Qz;
    const int q0 = fft_pos(kz, J.fz.plan);
    const int q1 = two ? fft_pos(Qz - kz, J.fz.plan) : q0;
    const size_t koff = ((size_t)kx * J.kyq + kys) * J.kzq + kz;
    float nv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, sv[3] = {0.f, 0.f, 0.f};
    if (J.do_H)
#pragma unroll
      for (int c = 0; c < 6; ++c) nv[c] = __ldg(J.N3 + c * kstride + koff);
    if (J.do_C)
#pragma unroll
      for (int c = 0; c < 3; ++c) sv[c] = __ldg(J.S3 + c * kstride + koff);
    const float sy = ym ? -1.f : 1.f;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      if (side == 1 && !two) break;
      const int q = side ? q1 : q0;
      const float sz = side ? -1.f : 1.f;
      const float2 mx = sm[(t * 3 + 0) * ldz + q], my = sm[(t * 3 + 1) * ldz + q],
                   mz = sm[(t * 3 + 2) * ldz + q];
      if (J.do_C) {
        // phi = i (Sx mx + Sy my + Sz mz); Sy odd in y, Sz odd in z
        const float ax = sv[0], ay = sy * sv[1], az = sz * sv[2];
        phi[t * ldz + q] = c_i_times(make_float2(ax * mx.x + ay * my.x + az * mz.x,
                                                 ax * mx.y + ay * my.y + az * mz.y));
      }
      if (J.do_H) {
        // N real: xy odd in y, xz odd in z, yz odd in both
        const float nxx = nv[0], nyy = nv[1], nzz = nv[2];
        const float nxy = sy * nv[3], nxz = sz * nv[4], nyz = sy * sz * nv[5];
        sm[(t * 3 + 0) * ldz + q] = make_float2(nxx * mx.x + nxy * my.x + nxz * mz.x,
                                                nxx * mx.y + nxy * my.y + nxz * mz.y);
        sm[(t * 3 + 1) * ldz + q] = make_float2(nxy * mx.x + nyy * my.x + nyz * mz.x,
                                                nxy * mx.y + nyy * my.y + nyz * mz.y);
        sm[(t * 3 + 2) * ldz + q] = make_float2(nxz * mx.x + nyz * my.x + nzz * mz.x,
                                                nxz * mx.y + nyz * my.y + nzz * mz.y);
      }
    }
  }
  __syncthreads();
  if (J.do_H) fft_smem<kInvDit, float2, RSET>(sm, ldz, 3 * nt, J.fz.plan, J.fz.tw_f, 0, blockDim.x);
  if (J.do_C) fft_smem<kInvDit, float2, RSET>(phi, ldz, nt, J.fz.plan, J.fz.tw_f, 0, blockDim.x);

  if (J.do_H) {
    for (int i = threadIdx.x; i < P3 * nt; i += blockDim.x) {
      const int q = i / nt, t = i - q * nt;
      const int c = q / nz, z = q - c * nz;
      J.outH[((size_t)q * J.kxh + kx) * Qy + y0 + t] = sm[(t * 3 + c) * ldz + z];
    }
  }
  if (J.do_C) {
    const int r = J.r;
    if (J.fir) {
      const int nch = (r + kZChunk - 1) / kZChunk;
      for (int i = threadIdx.x; i < nt * nch; i += blockDim.x) {
        const int t = i / nch;
        const int k0 = (i - t * nch) * kZChunk;
        const float2* line = phi + t * ldz;
        prefilter_chunk<kZChunk, f2>(
            k0, r, [&](int jj) { return f2(line[tab[jj]]); },
            [&](int k, f2 v) { J.outC[((size_t)k * J.kxh + kx) * Qy + y0 + t] = make_float2(v.x, v.y); });
      }
    } else {
      for (int i = threadIdx.x; i < nt * r; i += blockDim.x) {
        const int k = i / nt, t = i - k * nt;
        J.outC[((size_t)k * J.kxh + kx) * Qy + y0 + t] = phi[t * ldz + tab[k + kPrefWarm]];
      }
    }
  }
}

// ------------------------------------------------------------------ y inverse
template <unsigned RSET, int FIXP>
__global__ void __launch_bounds__(256, 3) k_yinv3(const Launch<YInvJob> Lc) {
  extern __shared__ float2 sm[];
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const YInvJob& J = Lc.job[j];
  const int tile = blockIdx.x - Lc.tile_start[j];
  const int ng = (J.planes + J.group - 1) / J.group;
  const int kx = tile / ng;
  const int p0 = (tile - kx * ng) * J.group;
  const int np = min(J.group, J.planes - p0);
  const int Q = FIXP ? FixedPlan<FIXP ? FIXP : 1>::L : J.fy.plan.L;
  const int ldl = Q + 1;
  int* tab = reinterpret_cast<int*>(sm + J.group * ldl);
  for (int l = 0; l < np; ++l) {
    const float2* col = J.in + ((size_t)(p0 + l) * J.kxh + kx) * Q;
    for (int p = threadIdx.x; p < Q; p += blockDim.x) sm[l * ldl + p] = col[p];
  }
  // natural-order input: DIF stages of the inverse leave the rows in DIF
  // order, read back through the position table; DIF-order input: DIT stages
  // leave natural order
  if (J.is_C)
    build_pref_table(tab, J.r + 2 * kPrefWarm + kYChunk, J.box_lo, J.box_len, J.start, Q,
                     J.natural ? J.fy.pos : nullptr, J.periodic != 0);
  __syncthreads();
  if constexpr (FIXP > 0) {
    if (J.natural) fft_smem_plan<kInvDif, FIXP, FixedPlan<FIXP>::L + 1>(sm, np, J.fy.plan, J.fy.tw_f, 0, blockDim.x);
    else fft_smem_plan<kInvDit, FIXP, FixedPlan<FIXP>::L + 1>(sm, np, J.fy.plan, J.fy.tw_f, 0, blockDim.x);
  } else {
    if (J.natural) fft_smem<kInvDif, float2, RSET>(sm, ldl, np, J.fy.plan, J.fy.tw_f, 0, blockDim.x);
    else fft_smem<kInvDit, float2, RSET>(sm, ldl, np, J.fy.plan, J.fy.tw_f, 0, blockDim.x);
  }
  if (!J.is_C) {
    for (int l = 0; l < np; ++l) {
      float2* dst = J.outH + ((size_t)(p0 + l) * J.kxh + kx) * J.ny;
      for (int y = threadIdx.x; y < J.ny; y += blockDim.x)
        dst[y] = sm[l * ldl + (J.natural ? __ldg(J.fy.pos + y) : y)];
    }
    return;
  }
  const int r = J.r;
  if (J.fir) {
    const int nch = (r + kYChunk - 1) / kYChunk;
    for (int i = threadIdx.x; i < np * nch; i += blockDim.x) {
      const int l = i / nch;
      const int k0 = (i - l * nch) * kYChunk;
      const float2* line = sm + l * ldl;
      float2* dst = J.outC + ((size_t)(p0 + l) * J.kxh + kx) * r;
      prefilter_chunk<kYChunk, f2>(
          k0, r, [&](int jj) { return f2(line[tab[jj]]); },
          [&](int k, f2 v) { dst[k] = make_float2(v.x, v.y); });
    }
  } else {
    for (int l = 0; l < np; ++l) {
      float2* dst = J.outC + ((size_t)(p0 + l) * J.kxh + kx) * r;
      for (int k = threadIdx.x; k < r; k += blockDim.x) dst[k] = sm[l * ldl + tab[k + kPrefWarm]];
    }
  }
}

// dynamic shared memory of a launch, with the carveout set to shared memory
static cudaError_t prep(const void* f, size_t smem) {
  cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// ------------------------------------------------------------------ direct z sum
// The thin-film plane mixing of Sec. III.A for sources of up to kMaxNzDirect
// layers.  CTA -> (kx, a chunk of kZMixChunk frequency pairs ky, Qy - ky): the
// input planes of the chunk are staged in shared memory once, then each warp
// takes one output plane at a time with one frequency pair per lane, so the
// kernel-spectrum loads and the output stores are coalesced runs and the
// inputs are read from shared memory instead of again from L2 for every
// output plane.  (Staging inputs and looping over all outputs inside one
// thread measured 1.3-2.7x slower than streaming; this layout keeps a warp
// per output plane.)
constexpr int kZMixThreads = 128;
constexpr int kZMixChunk = 32;  // frequency pairs per CTA, one per lane

// Sums of one output plane at frequency k (acc0) and Qy - k (acc1).  Terms
// whose kernel spectrum is real and those whose spectrum is imaginary are
// summed apart (r*, i*) and the factor i is applied once at the end, so a
// term is one load of the spectrum, two shared-memory loads and four FMAs;
// every parity below is a compile-time constant of the output component A.
struct ZAcc {
  float2 r0, r1, i0, i1;
  __device__ ZAcc() : r0(make_float2(0.f, 0.f)), r1(r0), i0(r0), i1(r0) {}
  __device__ __forceinline__ void add(bool imag, float v0, float v1, float2 m0, float2 m1) {
    float2& a0 = imag ? i0 : r0;
    float2& a1 = imag ? i1 : r1;
    a0.x = fmaf(v0, m0.x, a0.x); a0.y = fmaf(v0, m0.y, a0.y);
    a1.x = fmaf(v1, m1.x, a1.x); a1.y = fmaf(v1, m1.y, a1.y);
  }
  __device__ __forceinline__ float2 out0() const { return make_float2(r0.x - i0.y, r0.y + i0.x); }
  __device__ __forceinline__ float2 out1() const { return make_float2(r1.x - i1.y, r1.y + i1.x); }
};

// H_A(iz) = sum_jz sum_b Ns_Ab(iz - jz) m_b(jz): xz, yz odd in dz and
// imaginary, xy and yz odd in y (Nq holds dz >= 0)
template <int A>
__device__ __forceinline__ ZAcc zmix_demag(const ZMixJob& J, int iz, const float* __restrict__ nq,
                                           const float2* s0, const float2* s1, size_t kstride) {
  ZAcc acc;
  const int nz = J.nz;
  for (int jz = 0; jz < nz; ++jz) {
    const int adz = iz >= jz ? iz - jz : jz - iz;
    const float sz = iz >= jz ? 1.f : -1.f;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int comp = A == b ? A : (A + b == 1 ? 3 : (A + b == 2 ? 4 : 5));
      const bool imag = comp >= 4;               // xz, yz
      const bool odd_y = comp == 3 || comp == 5; // xy, yz
      const float v = (imag ? sz : 1.f) * __ldg(nq + (size_t)(comp * nz + adz) * kstride);
      acc.add(imag, v, odd_y ? -v : v, s0[(b * nz + jz) * kZMixChunk], s1[(b * nz + jz) * kZMixChunk]);
    }
  }
  return acc;
}

// c(o) = sum_jz sum_c T_c(o, jz) m_c(jz), T_x, T_y imaginary, T_y odd in y
// (A = 2: rows with the parities of S); field variant: H_A(o) with the rows
// of -N, imaginary when odd in x (xz, zx) or y (yz, zy), odd in y for xy,
// yx, yz, zy
template <int A>
__device__ __forceinline__ ZAcc zmix_coef(const ZMixJob& J, int oc, const float* __restrict__ tq,
                                          const float2* s0, const float2* s1, size_t kstride) {
  ZAcc acc;
  const int nz = J.nz;
  for (int jz = 0; jz < nz; ++jz) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const bool imag = (A == 2) != (c == 2);
      const bool odd_y = (A == 1) != (c == 1);
      const float v = __ldg(tq + (size_t)((oc * nz + jz) * 3 + c) * kstride);
      acc.add(imag, v, odd_y ? -v : v, s0[(c * nz + jz) * kZMixChunk], s1[(c * nz + jz) * kZMixChunk]);
    }
  }
  return acc;
}

__global__ void __launch_bounds__(kZMixThreads) k_zmix3(const Launch<ZMixJob> Lc) {
  extern __shared__ float2 zs[];  // [2][3 nz][kZMixChunk]: inputs at ky, then at Qy - ky
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const ZMixJob& J = Lc.job[j];
  const int tile = blockIdx.x - Lc.tile_start[j];
  const int nch = (J.kyq + kZMixChunk - 1) / kZMixChunk;
  const int kx = tile / nch;
  const int k0 = (tile - kx * nch) * kZMixChunk;
  const int nk = min(kZMixChunk, J.kyq - k0);
  const int Qy = J.Qy, nz = J.nz, P3 = 3 * nz;
  const size_t pstride = (size_t)J.kxh * Qy;  // one input / output plane
  const float2* inb = J.in + (size_t)kx * Qy;
  for (int i = threadIdx.x; i < P3 * kZMixChunk; i += blockDim.x) {
    const int p = i / kZMixChunk, l = i - p * kZMixChunk;
    if (l < nk) {
      const int k = k0 + l;
      const bool two = k != 0 && 2 * k != Qy;
      const float2* row = inb + (size_t)p * pstride;
      zs[i] = row[k];
      zs[P3 * kZMixChunk + i] = row[two ? Qy - k : k];
    }
  }
  __syncthreads();
  const int l = threadIdx.x % kZMixChunk;
  if (l >= nk) return;
  const int k = k0 + l;
  const bool two = k != 0 && 2 * k != Qy;
  const size_t kstride = (size_t)J.kxh * J.kyq;  // one stored kernel plane
  const size_t koff = (size_t)kx * J.kyq + k;
  const float2* s0 = zs + l;
  const float2* s1 = zs + P3 * kZMixChunk + l;
  const int planes = J.nH + J.n_out;
  // one output plane per warp at a time (warp-uniform branches below)
  for (int o = threadIdx.x / kZMixChunk; o < planes; o += kZMixThreads / kZMixChunk) {
    ZAcc acc;
    float2* dst;
    uint16_t* pk;
    int prow;  // row (plane, kx) of the packed output
    if (o < J.nH) {
      const int a = o / nz, iz = o - a * nz;
      const float* nq = J.Nq + koff;
      if (a == 0) acc = zmix_demag<0>(J, iz, nq, s0, s1, kstride);
      else if (a == 1) acc = zmix_demag<1>(J, iz, nq, s0, s1, kstride);
      else acc = zmix_demag<2>(J, iz, nq, s0, s1, kstride);
      dst = J.outH + (size_t)o * pstride + (size_t)kx * Qy;
      pk = J.pkH;
      prow = o * J.kxh + kx;
    } else {
      const int oc = o - J.nH;
      const int a = J.field_nbox > 0 ? oc / J.field_nbox : 2;  // row z of N has the parities of S
      const float* tq = J.Tq + koff;
      if (a == 0) acc = zmix_coef<0>(J, oc, tq, s0, s1, kstride);
      else if (a == 1) acc = zmix_coef<1>(J, oc, tq, s0, s1, kstride);
      else acc = zmix_coef<2>(J, oc, tq, s0, s1, kstride);
      dst = J.outC + (size_t)oc * pstride + (size_t)kx * Qy;
      pk = J.pkC;
      prow = oc * J.kxh + kx;
    }
    if (pk) {  // reduced precision: straight into the inverse DFT's split operand
      const int kch = (Qy + (int)(kKChunk / 2) - 1) / (int)(kKChunk / 2);
      store_split(pk, kch, prow, k, acc.out0());
      if (two) store_split(pk, kch, prow, Qy - k, acc.out1());
    } else {
      dst[k] = acc.out0();
      if (two) dst[Qy - k] = acc.out1();
    }
  }
}

// CTAs per kx (the output planes are covered inside each CTA)
int zmix_tiles(int kyq, int planes) {
  (void)planes;
  return (kyq + kZMixChunk - 1) / kZMixChunk;
}

cudaError_t launch_zmix3(const Launch<ZMixJob>& L, cudaStream_t st) {
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  int nzmax = 1;
  for (int i = 0; i < L.njobs; ++i) nzmax = max(nzmax, L.job[i].nz);
  const size_t smem = sizeof(float2) * 2 * 3 * (size_t)nzmax * kZMixChunk;
  k_zmix3<<<grid, kZMixThreads, smem, st>>>(L);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ host side
// about 80 KB of lines per CTA (two CTAs per SM), at least 8 y positions:
// short z grids get many positions, which spreads the per-CTA set-up
int zpass_tile(int Qz) { return std::max(8, (80 * 1024) / (4 * (Qz + 1) * (int)sizeof(float2))); }
int zpass_tiles(int Qy, int ztile) { return (Qy + ztile - 1) / ztile; }

// every job's y plan is 1080 = 12 6 15 (fixed plan 2: the 512 x 512 films)
template <typename JobT> static bool y_fixed_1080(const Launch<JobT>& L) {
  for (int i = 0; i < L.njobs; ++i)
    if (fixed_plan_id(L.job[i].fy.plan) != 2) return false;
  return L.njobs > 0;
}

cudaError_t launch_yfwd3(const Launch<YFwdJob>& L, cudaStream_t st) {
  size_t smem = 0;
  for (int i = 0; i < L.njobs; ++i)
    smem = std::max(smem, sizeof(float2) * (size_t)L.job[i].group * (L.job[i].fy.plan.L + 1));
  unsigned rs = 0;
  for (int i = 0; i < L.njobs; ++i) rs |= plan_radix_set(L.job[i].fy.plan);
  auto k = y_fixed_1080(L) ? k_yfwd3<kAllRadices, 2>
           : (rs & ~kRadixSetA) == 0u ? k_yfwd3<kRadixSetA, 0> : k_yfwd3<kAllRadices, 0>;
  cudaError_t e = prep((const void*)k, smem);
  if (e != cudaSuccess) return e;
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  k<<<grid, 256, smem, st>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_zpass3(const Launch<ZJob>& L, cudaStream_t st) {
  size_t smem = 0;
  for (int i = 0; i < L.njobs; ++i) {
    const ZJob& J = L.job[i];
    const size_t lines = sizeof(float2) * 4 * J.ztile * (size_t)(J.fz.plan.L + 1);
    const size_t tab = sizeof(int) * (size_t)(J.do_C ? J.r + 2 * kPrefWarm + kZChunk : 0);
    smem = std::max(smem, lines + tab);
  }
  unsigned rs = 0;
  for (int i = 0; i < L.njobs; ++i) rs |= plan_radix_set(L.job[i].fz.plan);
  auto k = (rs & ~kRadixSetA) == 0u ? k_zpass3<kRadixSetA> : k_zpass3<kAllRadices>;
  cudaError_t e = prep((const void*)k, smem);
  if (e != cudaSuccess) return e;
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  k<<<grid, 256, smem, st>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_yinv3(const Launch<YInvJob>& L, cudaStream_t st) {
  size_t smem = 0;
  for (int i = 0; i < L.njobs; ++i) {
    const YInvJob& J = L.job[i];
    const size_t lines = sizeof(float2) * (size_t)J.group * (J.fy.plan.L + 1);
    const size_t tab = sizeof(int) * (size_t)(J.is_C ? J.r + 2 * kPrefWarm + kYChunk : 0);
    smem = std::max(smem, lines + tab);
  }
  unsigned rs = 0;
  for (int i = 0; i < L.njobs; ++i) rs |= plan_radix_set(L.job[i].fy.plan);
  auto k = y_fixed_1080(L) ? k_yinv3<kAllRadices, 2>
           : (rs & ~kRadixSetA) == 0u ? k_yinv3<kRadixSetA, 0> : k_yinv3<kAllRadices, 0>;
  cudaError_t e = prep((const void*)k, smem);
  if (e != cudaSuccess) return e;
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  k<<<grid, 256, smem, st>>>(L);
  return cudaGetLastError();
}

}  // namespace mm
