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
// restored here; one thread handles the pair (ky, Qy - ky), which shares the
// stored values, and walks ky in natural order so those loads coalesce.
// Thicker magnets (nz > 4) take z by an FFT pass of its own (fft3d.cu).
#include "fft.cuh"
#include "mm_internal.h"
#include "prefilter.cuh"
#include "umma.cuh"

namespace mm {

constexpr int kLines = kRowsPerCta / 2;  // complex lines per CTA in the x passes
// threads per CTA of the x passes (multiples of kLines)
constexpr int kXFwdThreads = 256;
constexpr int kXInvThreads = 256;
constexpr int kLinePad = 4;              // float2 between lines of an x-pass CTA

cudaError_t init_fft_constants_passes() { return upload_roots(); }

// ------------------------------------------------------------------ x forward
// FIXP > 0: every job's x plan is fixed plan FIXP, run with its lengths as constants.
template <unsigned RSET, int FIXP>
__global__ void __launch_bounds__(kXFwdThreads, 3) k_xfwd(const Launch<XFwdJob> Lc) {
  extern __shared__ float2 sm[];
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const XFwdJob& J = Lc.job[j];
  const int tile = blockIdx.x - Lc.tile_start[j];
  const int Q = FIXP ? FixedPlan<FIXP ? FIXP : 1>::L : J.fx.plan.L;
  const int ldl = Q + kLinePad;  // padded line stride: the lines start in different banks
  const int rows = 3 * J.nz * J.ny;
  const int r0 = tile * kRowsPerCta;
  const int nrows = min(kRowsPerCta, rows - r0);
  const int nlines = (nrows + 1) >> 1;
  const int nx = J.nx;
  const float* row0 = J.m + (size_t)r0 * nx;

  if ((nx & 3) == 0) {
    // all rows of the CTA per thread and step: 2 kLines float4 loads in flight
    const int n4 = nx >> 2;
    for (int x4 = threadIdx.x; x4 < n4; x4 += blockDim.x) {
      float4 v[kRowsPerCta];
#pragma unroll
      for (int r = 0; r < kRowsPerCta; ++r)
        v[r] = r < nrows ? __ldg(reinterpret_cast<const float4*>(row0 + r * nx) + x4)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int l = 0; l < kLines; ++l) {
        if (l < nlines) {
          float2* d = sm + l * ldl + 4 * x4;
          const float4 a = v[2 * l], b = v[2 * l + 1];
          d[0] = make_float2(a.x, b.x);
          d[1] = make_float2(a.y, b.y);
          d[2] = make_float2(a.z, b.z);
          d[3] = make_float2(a.w, b.w);
        }
      }
    }
  } else {
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      float v[kRowsPerCta];
#pragma unroll
      for (int r = 0; r < kRowsPerCta; ++r) v[r] = r < nrows ? __ldg(row0 + r * nx + x) : 0.f;
#pragma unroll
      for (int l = 0; l < kLines; ++l)
        if (l < nlines) sm[l * ldl + x] = make_float2(v[2 * l], v[2 * l + 1]);
    }
  }
  // entries [nx, Q) are zero padding: the first stage takes them as zero unread
  // DIF positions of k and Q - k for every kx <= Q/2
  ushort2* ptab = reinterpret_cast<ushort2*>(sm + kLines * ldl);  // Q < 65536
  for (int kx = threadIdx.x; kx < J.kxh; kx += blockDim.x)
    ptab[kx] = make_ushort2((unsigned short)__ldg(J.fx.pos + kx),
                            (unsigned short)__ldg(J.fx.pos + (kx == 0 ? 0 : Q - kx)));
  __syncthreads();
  if constexpr (FIXP > 0)
    fft_smem_plan<kFwdDif, FIXP, FixedPlan<FIXP>::L + kLinePad>(sm, nlines, J.fx.plan, J.fx.tw_f, 0, blockDim.x, nx);
  else
    fft_smem<kFwdDif, float2, RSET>(sm, ldl, nlines, J.fx.plan, J.fx.tw_f, 0, blockDim.x, nx);

  // Z = A + iB:  A_k = (Z_k + conj Z_{Q-k}) / 2,  B_k = (Z_k - conj Z_{Q-k}) / (2i)
  // thread -> (kx, line) with the line fastest: a warp writes 8 runs of 64 bytes
  const int ny = J.ny;
  const int pa0 = r0 / ny;
  const bool pairs = (ny & 1) == 0 && (nrows & 1) == 0;  // both rows of a line in one plane, 16-B aligned
  if (pairs && nlines == kLines) {
    // full tile: blockDim is a multiple of kLines, so every thread keeps one
    // line and its output row pair for all its kx
    const int l = threadIdx.x % kLines;
    int pa = pa0, ya = r0 + 2 * l - pa0 * ny;
    while (ya >= ny) { ++pa; ya -= ny; }
    float2* dst0 = J.out + (size_t)pa * J.kxh * ny + ya;
    const float2* line = sm + l * ldl;
    const int kch = (ny + (int)(kKChunk / 2) - 1) / (int)(kKChunk / 2);
    for (int kx = threadIdx.x / kLines; kx < J.kxh; kx += blockDim.x / kLines) {
      const ushort2 pp = ptab[kx];
      const float2 Zk = line[pp.x];
      const float2 Zm = line[pp.y];
      if (J.pk) {  // reduced precision: straight into the forward DFT's split operand
        store_split(J.pk, kch, pa * J.kxh + kx, ya, make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y)));
        store_split(J.pk, kch, pa * J.kxh + kx, ya + 1, make_float2(0.5f * (Zk.y + Zm.y), -0.5f * (Zk.x - Zm.x)));
      } else {
        *reinterpret_cast<float4*>(dst0 + (size_t)kx * ny) =
            make_float4(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y), 0.5f * (Zk.y + Zm.y), -0.5f * (Zk.x - Zm.x));
      }
    }
    return;
  }
  const int n = J.kxh * nlines;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int kx = nlines == kLines ? idx / kLines : idx / nlines;
    const int l = idx - kx * nlines;
    const ushort2 pp = ptab[kx];
    const float2 Zk = sm[l * ldl + pp.x];
    const float2 Zm = sm[l * ldl + pp.y];
    const float2 A = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
    const float2 B = make_float2(0.5f * (Zk.y + Zm.y), -0.5f * (Zk.x - Zm.x));
    int pa = pa0, ya = r0 + 2 * l - pa0 * ny;
    while (ya >= ny) { ++pa; ya -= ny; }
    if (J.pk) {
      const int kch = (ny + (int)(kKChunk / 2) - 1) / (int)(kKChunk / 2);
      store_split(J.pk, kch, pa * J.kxh + kx, ya, A);
      if (2 * l + 1 < nrows) {
        int pb = pa, yb = ya + 1;
        if (yb >= ny) { ++pb; yb -= ny; }
        store_split(J.pk, kch, pb * J.kxh + kx, yb, B);
      }
      continue;
    }
    float2* dst = J.out + ((size_t)pa * J.kxh + kx) * ny + ya;
    if (pairs) {
      *reinterpret_cast<float4*>(dst) = make_float4(A.x, A.y, B.x, B.y);
    } else {
      *dst = A;
      if (2 * l + 1 < nrows) {
        int pb = pa, yb = ya + 1;
        if (yb >= ny) { ++pb; yb -= ny; }
        J.out[((size_t)pb * J.kxh + kx) * ny + yb] = B;
      }
    }
  }
}

// ------------------------------------------------------------------ y pass
__device__ __forceinline__ float2 kmul(float v, bool imag, float2 m) {
  return imag ? make_float2(-v * m.y, v * m.x) : make_float2(v * m.x, v * m.y);
}
__device__ __forceinline__ void cacc(float2& a, float2 b) { a.x += b.x; a.y += b.y; }

template <int NZ>
__device__ __forceinline__ void load_pair(const float2* sm, int Q, int p0, int p1, float2 (*mh)[3][NZ]) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int z = 0; z < NZ; ++z) {
      mh[0][c][z] = sm[(c * NZ + z) * Q + p0];
      mh[1][c][z] = sm[(c * NZ + z) * Q + p1];
    }
}

// Spectral products at every (ky, Qy - ky) pair of one kx column.  The
// potential planes land beyond the input planes whenever the demag planes are
// produced too; those overwrite the inputs in place.  A thread owns the two
// positions of its pair in every plane, so it reads the inputs once and writes
// both products without any barrier.  Kernel-spectrum loads are issued in
// batches before the arithmetic that uses them.
template <int NZ>
__device__ __forceinline__ void ypass_mix(const YJob& J, float2* sm, int kx, int Q, int nH) {
  // output planes per batch of kernel loads (about 30 values in flight)
  constexpr int OB = 30 / (3 * NZ) > 0 ? 30 / (3 * NZ) : 1;
  const int kstride = J.kxh * J.kyq;  // one stored kernel plane (< 2^31 values in all)
  const int half = Q >> 1;
  for (int kyq = threadIdx.x; kyq <= half; kyq += blockDim.x) {
    // the two frequencies ky = kyq and Qy - kyq share every stored kernel value;
    // the second has the odd-in-y components negated
    const bool two = kyq != 0 && 2 * kyq != Q;
    const int koff = kx * J.kyq + kyq;
    const int p0 = fft_pos(kyq, J.fy.plan);
    const int p1 = two ? fft_pos(Q - kyq, J.fy.plan) : p0;
    float2 mh[2][3][NZ];
    load_pair<NZ>(sm, Q, p0, p1, mh);
    if (J.do_C) {
      const float* Tk = J.Tq + koff;
      for (int ob = 0; ob < J.n_out; ob += OB) {
        float tv[OB][NZ][3];
#pragma unroll
        for (int o = 0; o < OB; ++o)
#pragma unroll
          for (int jz = 0; jz < NZ; ++jz)
#pragma unroll
            for (int c = 0; c < 3; ++c)
              tv[o][jz][c] = ob + o < J.n_out ? __ldg(Tk + (((ob + o) * NZ + jz) * 3 + c) * kstride) : 0.f;
        // c(o) = sum_jz sum_c T_c(o, jz) m_c(jz); T = Ms W (S spectra) / (Qx Qy)
#pragma unroll
        for (int o = 0; o < OB; ++o) {
          if (ob + o >= J.n_out) break;
          float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0;
#pragma unroll
          for (int jz = 0; jz < NZ; ++jz) {
            const float tx = tv[o][jz][0], ty = tv[o][jz][1], tz = tv[o][jz][2];
            cacc(acc0, kmul(tx, true, mh[0][0][jz]));
            cacc(acc0, kmul(ty, true, mh[0][1][jz]));
            cacc(acc0, kmul(tz, false, mh[0][2][jz]));
            cacc(acc1, kmul(tx, true, mh[1][0][jz]));
            cacc(acc1, kmul(-ty, true, mh[1][1][jz]));
            cacc(acc1, kmul(tz, false, mh[1][2][jz]));
          }
          sm[(nH + ob + o) * Q + p0] = acc0;
          if (two) sm[(nH + ob + o) * Q + p1] = acc1;
        }
      }
    }
    if (J.do_H) {
      // H_a(iz) = sum_jz sum_b Ns_ab(iz - jz) m_b(jz); Ns = -Ms N / (Qx Qy)
      const float* Nk = J.Nq + koff;
      float nv[6][NZ];
#pragma unroll
      for (int comp = 0; comp < 6; ++comp)
#pragma unroll
        for (int dz = 0; dz < NZ; ++dz) nv[comp][dz] = __ldg(Nk + (comp * NZ + dz) * kstride);
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const float fy = side ? -1.f : 1.f;
        const int p = side ? p1 : p0;
        if (side == 1 && !two) break;
#pragma unroll
        for (int iz = 0; iz < NZ; ++iz) {
          float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0;
#pragma unroll
          for (int jz = 0; jz < NZ; ++jz) {
            const int adz = iz >= jz ? iz - jz : jz - iz;
            const float sz = iz >= jz ? 1.f : -1.f;
            const float nxx = nv[0][adz], nyy = nv[1][adz], nzz = nv[2][adz];
            const float nxy = nv[3][adz] * fy, nxz = nv[4][adz] * sz, nyz = nv[5][adz] * sz * fy;
            const float2 mx = mh[side][0][jz], my = mh[side][1][jz], mz = mh[side][2][jz];
            cacc(a0, kmul(nxx, false, mx)); cacc(a0, kmul(nxy, false, my)); cacc(a0, kmul(nxz, true, mz));
            cacc(a1, kmul(nxy, false, mx)); cacc(a1, kmul(nyy, false, my)); cacc(a1, kmul(nyz, true, mz));
            cacc(a2, kmul(nxz, true, mx));  cacc(a2, kmul(nyz, true, my));  cacc(a2, kmul(nzz, false, mz));
          }
          sm[(0 * NZ + iz) * Q + p] = a0;
          sm[(1 * NZ + iz) * Q + p] = a1;
          sm[(2 * NZ + iz) * Q + p] = a2;
        }
      }
    }
  }
}

// One CTA per kx; every job of a launch has NZ layers.  kYThreads = 288 (nine
// warps) covers the 271 frequency pairs of a 540-point line in one round of
// the spectral products.
constexpr int kYThreads = 288;
// FIX540: every job's y plan is 540 = 4 9 15, run with its lengths as constants.
template <int NZ, unsigned RSET, bool FIX540>
__global__ void __launch_bounds__(kYThreads, NZ <= 2 ? 3 : 2) k_ypass(const Launch<YJob> Lc) {
  constexpr int Pin = 3 * NZ;
  extern __shared__ float2 sm[];
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const YJob& J = Lc.job[j];
  const int kx = blockIdx.x - Lc.tile_start[j];
  const int Q = J.fy.plan.L;
  const int nH = J.do_H ? Pin : 0;
  const int Pout = nH + (J.do_C ? J.n_out : 0);
  int* tab = reinterpret_cast<int*>(sm + max(Pin, Pout) * Q);
  const int ny = J.ny;
  const float2* col0 = J.in + (size_t)kx * ny;
  const size_t pstride = (size_t)J.kxh * ny;  // one input plane

  // The kernel spectra of this kx column are read only after the forward FFT:
  // start moving their lines into L2 now (one prefetch per 128-byte line).
  {
    const size_t kstride = (size_t)J.kxh * J.kyq;
    const int lines = (J.kyq + 31) / 32;
    const int nN = J.do_H ? 6 * NZ : 0;
    const int nT = J.do_C ? 3 * NZ * J.n_out : 0;
    for (int i = threadIdx.x; i < (nN + nT) * lines; i += blockDim.x) {
      const int row = i / lines, ln = i - row * lines;
      const float* p = row < nN ? J.Nq + (size_t)row * kstride : J.Tq + (size_t)(row - nN) * kstride;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(p + (size_t)kx * J.kyq + 32 * ln));
    }
  }

  if ((ny & 1) == 0) {
    // one float4 (two complex rows) of every plane per thread and step
    const int n2 = ny >> 1;
    for (int y2 = threadIdx.x; y2 < n2; y2 += blockDim.x) {
      float4 v[Pin];
#pragma unroll
      for (int p = 0; p < Pin; ++p) v[p] = *(reinterpret_cast<const float4*>(col0 + p * pstride) + y2);
#pragma unroll
      for (int p = 0; p < Pin; ++p) {
        sm[p * Q + 2 * y2] = make_float2(v[p].x, v[p].y);
        sm[p * Q + 2 * y2 + 1] = make_float2(v[p].z, v[p].w);
      }
    }
  } else {
    for (int y = threadIdx.x; y < ny; y += blockDim.x) {
      float2 v[Pin];
#pragma unroll
      for (int p = 0; p < Pin; ++p) v[p] = col0[p * pstride + y];
#pragma unroll
      for (int p = 0; p < Pin; ++p) sm[p * Q + y] = v[p];
    }
  }
  // (taking the zero rows as zero unread in the first stage measured slower here)
  for (int y = ny + threadIdx.x; y < Q; y += blockDim.x)
#pragma unroll
    for (int p = 0; p < Pin; ++p) sm[p * Q + y] = make_float2(0.f, 0.f);
  if (J.do_C)
    build_pref_table(tab, J.r + 2 * kPrefWarm + kYChunk, J.box_lo, J.box_len, J.start, Q, nullptr, J.periodic != 0);
  __syncthreads();
  if constexpr (FIX540) fft_smem_fixed<kFwdDif, float2, 4, 9, 15>(sm, Pin, J.fy.plan, J.fy.tw_f, 0, blockDim.x);
  else fft_smem<kFwdDif, float2, RSET>(sm, Q, Pin, J.fy.plan, J.fy.tw_f, 0, blockDim.x);
  ypass_mix<NZ>(J, sm, kx, Q, nH);
  __syncthreads();
  if constexpr (FIX540) fft_smem_fixed<kInvDit, float2, 4, 9, 15>(sm, Pout, J.fy.plan, J.fy.tw_f, 0, blockDim.x);
  else fft_smem<kInvDit, float2, RSET>(sm, Q, Pout, J.fy.plan, J.fy.tw_f, 0, blockDim.x);

  if (J.do_H) {
    float2* out0 = J.outH + (size_t)kx * ny;
    for (int y = threadIdx.x; y < ny; y += blockDim.x)
#pragma unroll
      for (int p = 0; p < Pin; ++p) out0[p * pstride + y] = sm[p * Q + y];
  }
  if (J.do_C) {
    const int r = J.r;
    float2* out0 = J.outC + (size_t)kx * r;
    const size_t ostride = (size_t)J.kxh * r;
    if (J.fir) {
      const int nch = (r + kYChunk - 1) / kYChunk;
      for (int idx = threadIdx.x; idx < J.n_out * nch; idx += blockDim.x) {
        const int o = idx / nch;
        const int k0 = (idx - o * nch) * kYChunk;
        const float2* col = sm + (nH + o) * Q;
        float2* dst = out0 + o * ostride;
        prefilter_chunk<kYChunk, f2>(
            k0, r, [&](int jj) { return f2(col[tab[jj]]); },
            [&](int k, f2 v) { dst[k] = make_float2(v.x, v.y); });
      }
    } else {
      for (int k = threadIdx.x; k < r; k += blockDim.x) {
        const int t = tab[k + kPrefWarm];
        for (int o = 0; o < J.n_out; ++o) out0[o * ostride + k] = sm[(nH + o) * Q + t];
      }
    }
  }
}

// ------------------------------------------------------------------ x inverse
__device__ __forceinline__ void xinv_put(float2* sm, int off, int Q, int kx, float2 A, float2 B) {
  // Z_k = A_k + i B_k and Z_{Q-k} = conj(A_k) + i conj(B_k), natural order; off = line start
  sm[off + kx] = make_float2(A.x - B.y, A.y + B.x);
  if (kx > 0 && 2 * kx != Q) sm[off + Q - kx] = make_float2(A.x + B.y, B.x - A.y);
}

template <unsigned RSET, int FIXP>
__global__ void __launch_bounds__(kXInvThreads, 3) k_xinv(const Launch<XInvJob> Lc) {
  extern __shared__ float2 sm[];
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const XInvJob& J = Lc.job[j];
  const int tile = blockIdx.x - Lc.tile_start[j];
  const int Q = FIXP ? FixedPlan<FIXP ? FIXP : 1>::L : J.fx.plan.L;
  const int ldl = Q + kLinePad;  // padded line stride: the lines start in different banks
  const int rpp = J.rows_per_plane;
  const int rows = J.planes * rpp;
  const int r0 = tile * kRowsPerCta;
  const int nrows = min(kRowsPerCta, rows - r0);
  const int nlines = (nrows + 1) >> 1;
  int* tab = reinterpret_cast<int*>(sm + kLines * ldl);

  // input row r of this CTA (its kx = 0 element)
  const int pa0 = r0 / rpp;
  auto rowptr = [&](int r) {
    int p = pa0, y = min(r0 + r, rows - 1) - pa0 * rpp;
    while (y >= rpp) { ++p; y -= rpp; }
    return J.in + (size_t)p * J.kxh * rpp + y;
  };
  const bool paired = (rpp & 1) == 0 && (nrows & 1) == 0;  // row pairs adjacent, 16-byte aligned
  const int n = J.kxh * nlines;
  if (paired && nlines == kLines) {
    // full tile: blockDim is a multiple of kLines, so every thread keeps one
    // line (its input row pair) for all its kx; kBatchX reads in flight (three
    // rounds of loads for a 2160-point line)
    constexpr int kBatchX = 6;
    const int l = threadIdx.x % kLines;
    const float2* src = rowptr(2 * l);
    const int step = blockDim.x / kLines;
    for (int kx0 = threadIdx.x / kLines; kx0 < J.kxh; kx0 += kBatchX * step) {
      float4 v[kBatchX];
#pragma unroll
      for (int u = 0; u < kBatchX; ++u) {
        const int kx = kx0 + u * step;
        if (kx < J.kxh) v[u] = *reinterpret_cast<const float4*>(src + (size_t)kx * rpp);
      }
#pragma unroll
      for (int u = 0; u < kBatchX; ++u) {
        const int kx = kx0 + u * step;
        if (kx < J.kxh) xinv_put(sm, l * ldl, Q, kx, make_float2(v[u].x, v[u].y), make_float2(v[u].z, v[u].w));
      }
    }
  } else if (paired) {
    // thread -> (kx, line), line fastest: a warp reads 8 runs of 64 bytes;
    // kBatchX such reads in flight per thread
    constexpr int kBatchX = 4;
    for (int base = threadIdx.x; base < n; base += kBatchX * blockDim.x) {
      float4 v[kBatchX];
#pragma unroll
      for (int u = 0; u < kBatchX; ++u) {
        const int idx = base + u * blockDim.x;
        if (idx < n) {
          const int kx = idx / nlines, l = idx - kx * nlines;
          v[u] = *reinterpret_cast<const float4*>(rowptr(2 * l) + (size_t)kx * rpp);
        }
      }
#pragma unroll
      for (int u = 0; u < kBatchX; ++u) {
        const int idx = base + u * blockDim.x;
        if (idx < n) {
          const int kx = idx / nlines, l = idx - kx * nlines;
          xinv_put(sm, l * ldl, Q, kx, make_float2(v[u].x, v[u].y), make_float2(v[u].z, v[u].w));
        }
      }
    }
  } else {
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const int kx = idx / nlines, l = idx - kx * nlines;
      const size_t off = (size_t)kx * rpp;
      const float2 a = rowptr(2 * l)[off];
      const float2 b = 2 * l + 1 < nrows ? rowptr(2 * l + 1)[off] : make_float2(0.f, 0.f);
      xinv_put(sm, l * ldl, Q, kx, a, b);
    }
  }
  build_pref_table(tab, J.out_len + 2 * kPrefWarm + kXChunk, J.box_lo, J.box_len, J.start, Q, J.fx.pos,
                   J.periodic != 0);
  __syncthreads();
  // natural-order input, digit-reversed output: the table above maps through it
  if constexpr (FIXP > 0)
    fft_smem_plan<kInvDif, FIXP, FixedPlan<FIXP>::L + kLinePad>(sm, nlines, J.fx.plan, J.fx.tw_f, 0, blockDim.x);
  else
    fft_smem<kInvDif, float2, RSET>(sm, ldl, nlines, J.fx.plan, J.fx.tw_f, 0, blockDim.x);

  const int r = J.out_len;
  float* out0 = J.out + (size_t)r0 * r;
  if (J.fir) {
    const int nch = (r + kXChunk - 1) / kXChunk;
    for (int idx = threadIdx.x; idx < nrows * nch; idx += blockDim.x) {
      const int rl = idx / nch;
      const int k0 = (idx - rl * nch) * kXChunk;
      const float* line = reinterpret_cast<const float*>(sm + (rl >> 1) * ldl) + (rl & 1);
      float* dst = out0 + rl * r;
      prefilter_chunk<kXChunk, float>(
          k0, r, [&](int jj) { return line[2 * tab[jj]]; }, [&](int k, float v) { dst[k] = v; });
    }
  } else {
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
      const int t = 2 * tab[k + kPrefWarm];
      const float* base = reinterpret_cast<const float*>(sm) + t;
#pragma unroll
      for (int rl = 0; rl < kRowsPerCta; ++rl)
        if (rl < nrows) out0[rl * r + k] = base[(rl >> 1) * 2 * ldl + (rl & 1)];
    }
  }
}

// ------------------------------------------------------------------ host side
size_t ypass_table_bytes(int r) { return sizeof(int) * (size_t)(r + 2 * kPrefWarm + kYChunk); }

static size_t xinv_smem(int Qmax, int out_max) {
  return (size_t)kLines * (Qmax + kLinePad) * sizeof(float2) +
         sizeof(int) * (size_t)(out_max + 2 * kPrefWarm + kXChunk);
}

// the fixed plan every job's x plan is (fixed_plan_id), 0 if they differ or none is
template <typename JobT> static int x_fixed_plan(const Launch<JobT>& L) {
  int id = L.njobs > 0 ? fixed_plan_id(L.job[0].fx.plan) : 0;
  for (int i = 1; i < L.njobs; ++i)
    if (fixed_plan_id(L.job[i].fx.plan) != id) id = 0;
  return id;
}

static void max_carveout(const void* f) {
  cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

cudaError_t launch_xfwd(const Launch<XFwdJob>& L, int Qmax, cudaStream_t st) {
  const size_t smem =
      (size_t)kLines * (Qmax + kLinePad) * sizeof(float2) + sizeof(ushort2) * (size_t)(Qmax / 2 + 1);
  unsigned rs = 0;
  for (int i = 0; i < L.njobs; ++i) rs |= plan_radix_set(L.job[i].fx.plan);
  const int fx = x_fixed_plan(L);
  auto k = fx == 1 ? k_xfwd<kRadixSetA, 1>
           : fx == 2 ? k_xfwd<kAllRadices, 2>
           : (rs & ~kRadixSetA) == 0u ? k_xfwd<kRadixSetA, 0> : k_xfwd<kAllRadices, 0>;
  max_carveout((const void*)k);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  k<<<grid, kXFwdThreads, smem, st>>>(L);
  return cudaGetLastError();
}

template <int NZ>
static cudaError_t launch_ypass_nz(const Launch<YJob>& L, size_t smem, cudaStream_t st) {
  unsigned rs = 0;
  bool fix540 = true;
  for (int i = 0; i < L.njobs; ++i) {
    rs |= plan_radix_set(L.job[i].fy.plan);
    fix540 = fix540 && fixed_plan_id(L.job[i].fy.plan) == 3;
  }
  auto k = fix540 ? k_ypass<NZ, kRadixSetA, true>
                  : (rs & ~kRadixSetA) == 0u ? k_ypass<NZ, kRadixSetA, false> : k_ypass<NZ, kAllRadices, false>;
  max_carveout((const void*)k);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  k<<<grid, kYThreads, smem, st>>>(L);
  return cudaGetLastError();
}

// Jobs of different layer counts go to separate launches of the matching kernel.
cudaError_t launch_ypass(const Launch<YJob>& L, size_t smem, cudaStream_t st) {
  for (int nz = 1; nz <= kMaxNz; ++nz) {
    Launch<YJob> S{};
    int tiles = 0;
    for (int i = 0; i < L.njobs; ++i) {
      if (L.job[i].nz != nz) continue;
      S.job[S.njobs] = L.job[i];
      S.tile_start[S.njobs] = tiles;
      tiles += L.tile_start[i + 1] - L.tile_start[i];
      ++S.njobs;
    }
    if (S.njobs == 0) continue;
    S.tile_start[S.njobs] = tiles;
    cudaError_t e = nz == 1   ? launch_ypass_nz<1>(S, smem, st)
                    : nz == 2 ? launch_ypass_nz<2>(S, smem, st)
                    : nz == 3 ? launch_ypass_nz<3>(S, smem, st)
                              : launch_ypass_nz<4>(S, smem, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_xinv(const Launch<XInvJob>& L, int Qmax, cudaStream_t st) {
  int out_max = 0;
  for (int i = 0; i < L.njobs; ++i) out_max = max(out_max, L.job[i].out_len);
  const size_t smem = xinv_smem(Qmax, out_max);
  unsigned rs = 0;
  for (int i = 0; i < L.njobs; ++i) rs |= plan_radix_set(L.job[i].fx.plan);
  const int fx = x_fixed_plan(L);
  auto k = fx == 1 ? k_xinv<kRadixSetA, 1>
           : fx == 2 ? k_xinv<kAllRadices, 2>
           : (rs & ~kRadixSetA) == 0u ? k_xinv<kRadixSetA, 0> : k_xinv<kAllRadices, 0>;
  max_carveout((const void*)k);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  k<<<grid, kXInvThreads, smem, st>>>(L);
  return cudaGetLastError();
}

}  // namespace mm
