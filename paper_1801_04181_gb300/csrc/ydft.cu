// Reduced-precision form of the y stage (Sec. III.A convolutions): the y
// transforms as complex DFT-matrix products on the 5th-generation tensor
// cores, BF16 operands split into hi + lo parts, FP32 accumulation in TMEM.
//
//   forward:  Y[row][ky] = sum_{y < ny} X[row][y] e^{-2 pi i ky y / Q}
//   inverse:  H[row][y]  = sum_ky Z[row][ky] e^{+2 pi i ky y / Q},  y < ny
//   inverse with the y prefilter folded in:
//             C[row][k]  = sum_ky Z[row][ky] G[k][ky],
//             G[k][ky]   = sum_d h(d) e^{+2 pi i ky g(k, d) / Q}
//   where h(d) = -6 z1 z1^|d| / (1 - z1^2) is the impulse response of the
//   cubic B-spline prefilter (z1 = sqrt(3) - 2) and g(k, d) the grid row of
//   box node start + k + d with mirror ends (or wrapped around the period).
//
// A row is one (plane, kx) line; the rows of a launch are independent, so one
// CTA takes 128 rows (the MMA's M) and one tile of at most 160 real output
// columns (its N, FP32 accumulators in TMEM).  In real form a complex product
// is [re im] . [[c, s], [-s, c]]; each complex matrix entry becomes four real
// ones, so K = 2 Kc and N = 2 Nc.  The split product keeps three of the four
// BF16 products, hi.hi + hi.lo + lo.hi (the dropped lo.lo is ~2^-18 of the
// terms), which gives ~2^-16 relative per dot product.
#include <cuda_bf16.h>

#include "fft.cuh"
#include "mm_internal.h"
#include "umma.cuh"

namespace mm {

constexpr int kDftThreads = 256;
constexpr int kDftRows = 128;     // MMA M: rows per CTA
constexpr int kDftMaxN = 160;     // MMA N: real columns per CTA (a multiple of 16)
constexpr uint32_t kDftTmemCols = 256;  // TMEM allocation: the power of two >= kDftMaxN
constexpr int kDftStages = 3;     // K chunks in flight per CTA (two CTAs share an SM)
constexpr uint32_t kDftStageA = kTileSplitBytes;          // one split of A, bytes
constexpr uint32_t kDftStageB = kDftMaxN * kKChunk * 2;  // one split of B, bytes
constexpr uint32_t kDftStageBytes = 2 * kDftStageA + 2 * kDftStageB;
constexpr size_t kDftSmem = (size_t)kDftStages * kDftStageBytes + 128;  // + barriers, TMEM slot
// about one second at the SM clock: a wait on the tensor core or a bulk copy
// never takes this long unless something is wrong
constexpr long long kDftSpinCycles = 2000000000LL;
constexpr int kDftErrBit = 2;
// per-warp epilogue staging: 32 rows x 16 floats, row pitch 20 (the float4
// stores of 8 lanes fall in distinct banks)
constexpr int kDftEpiPitch = 20;

// Product pass.  Thread 0 alone runs the main loop: bulk copies of the A and
// B blocks of each K chunk into a stage (completing on full[s]), the MMAs of
// the chunk once they landed (their completion committed to empty[s]), and
// the refill of a stage once its MMAs are done.  The other warps wait at the
// barrier before the epilogue; two CTAs share an SM, so one's epilogue runs
// beside the other's main loop.
__global__ void __launch_bounds__(kDftThreads, 2) k_ydft(const Launch<DftJob> Lc) {
  extern __shared__ __align__(128) uint8_t sm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + kDftStages * kDftStageBytes);  // a stage's copies landed
  uint64_t* empty = full + kDftStages;                                            // a stage's MMAs done
  uint32_t* slot = reinterpret_cast<uint32_t*>(empty + kDftStages);
  __shared__ int ok;
  const int j = find_job(Lc.tile_start, Lc.njobs, blockIdx.x);
  const DftJob& J = Lc.job[j];
  const int tile = blockIdx.x - Lc.tile_start[j];
  const int mt = tile / J.ntiles, nt = tile - mt * J.ntiles;
  const int row0 = mt * kDftRows;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    tmem_alloc(slot, kDftTmemCols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kDftStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    ok = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const int K = J.kchunks;

  if (threadIdx.x == 0) {
    const uint32_t idesc = idesc_bf16_f32(kDftRows, J.ntile);
    const uint32_t bbytes = (uint32_t)J.ntile * kKChunk * 2u;  // one split of one (N tile, K chunk) block
    const size_t bblock = (size_t)J.ntile * kKChunk;            // its BF16 values
    const uint8_t* Ablk = reinterpret_cast<const uint8_t*>(J.Apk) + (size_t)mt * K * 2 * kDftStageA;
    auto issue = [&](int c) {
      uint8_t* st = sm + (c % kDftStages) * kDftStageBytes;
      uint64_t* bar = &full[c % kDftStages];
      const size_t off = ((size_t)nt * K + c) * bblock;
      mbar_expect_tx(bar, 2u * kDftStageA + 2u * bbytes);
      bulk_g2s(st, Ablk + (size_t)c * 2 * kDftStageA, 2u * kDftStageA, bar);
      bulk_g2s(st + 2 * kDftStageA, J.Bhi + off, bbytes, bar);
      bulk_g2s(st + 2 * kDftStageA + kDftStageB, J.Blo + off, bbytes, bar);
    };
    int n_issued = 0, n_committed = 0;
    bool good = true;
    for (; n_issued < min(kDftStages, K); ++n_issued) issue(n_issued);
    for (int c = 0; c < K && good; ++c) {
      const int s = c % kDftStages;
      if (!mbar_wait(&full[s], (uint32_t)(c / kDftStages) & 1u, kDftSpinCycles)) {
        good = false;
        break;
      }
      tc_fence_after();
      const uint32_t aB = smem_u32(sm + s * kDftStageBytes), bB = aB + 2 * kDftStageA;
#pragma unroll
      for (int q = 0; q < (int)kKChunk / 16; ++q) {
        const uint32_t off = (uint32_t)q * 2u * kCoreBytes;  // 16 K values = two core matrices
        const uint64_t ah = smem_desc(aB + off, kCoreBytes, kRowGroupBytes);
        const uint64_t al = smem_desc(aB + kDftStageA + off, kCoreBytes, kRowGroupBytes);
        const uint64_t bh = smem_desc(bB + off, kCoreBytes, kRowGroupBytes);
        const uint64_t bl = smem_desc(bB + kDftStageB + off, kCoreBytes, kRowGroupBytes);
        umma_bf16(tmem, ah, bh, idesc, (c > 0 || q > 0) ? 1u : 0u);
        umma_bf16(tmem, ah, bl, idesc, 1u);
        umma_bf16(tmem, al, bh, idesc, 1u);
      }
      umma_commit(&empty[s]);
      n_committed = c + 1;
      // refill the stage of chunk c - 1 once its MMAs are done (the MMAs of
      // chunk c keep the tensor core busy meanwhile)
      if (c >= 1 && c - 1 + kDftStages < K) {
        const int cp = c - 1;
        if (!mbar_wait(&empty[cp % kDftStages], (uint32_t)(cp / kDftStages) & 1u, kDftSpinCycles)) {
          good = false;
          break;
        }
        issue(cp + kDftStages);
        ++n_issued;
      }
    }
    if (good) {
      const int c = K - 1;  // its commit completes after every MMA issued before it
      good = mbar_wait(&empty[c % kDftStages], (uint32_t)(c / kDftStages) & 1u, kDftSpinCycles);
    }
    if (!good) {
      atomicOr(J.err, kDftErrBit);
      // drain, each wait bounded: copies into this CTA's shared memory and
      // MMAs on its TMEM that may still be in flight
      for (int c = max(0, n_issued - kDftStages); c < n_issued; ++c)
        mbar_wait(&full[c % kDftStages], (uint32_t)(c / kDftStages) & 1u, kDftSpinCycles / 8);
      if (n_committed > 0) {
        const int c = n_committed - 1;
        mbar_wait(&empty[c % kDftStages], (uint32_t)(c / kDftStages) & 1u, kDftSpinCycles / 8);
      }
      ok = 0;
    }
  }
  __syncthreads();
  tc_fence_after();
  if (ok) {
    // TMEM -> per-warp staging (the stage buffers are free now) -> row
    // segments of 8 complex (64 bytes).  Warps w and w + 4 share TMEM lanes
    // 32 (w % 4) .. and take alternate 16-column blocks.
    float* W = reinterpret_cast<float*>(sm) + warp * 32 * kDftEpiPitch;
    const int q = warp & 3, half = warp >> 2;
    const int cc0 = (nt * J.ntile) >> 1;  // first complex column of the tile
    for (int c0 = 16 * half; c0 < J.ntile; c0 += 32) {
      float o[16];
      tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, o);
#pragma unroll
      for (int i = 0; i < 16; i += 4)
        *reinterpret_cast<float4*>(W + lane * kDftEpiPitch + i) = make_float4(o[i], o[i + 1], o[i + 2], o[i + 3]);
      __syncwarp();
      const int cc = cc0 + (c0 >> 1) + (lane & 7);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int rr = 4 * i + (lane >> 3);
        const int row = row0 + 32 * q + rr;
        if (row < J.rows && cc < J.Nc)
          J.D[(size_t)row * J.ldd + cc] = *reinterpret_cast<const float2*>(W + rr * kDftEpiPitch + 2 * (lane & 7));
      }
      __syncwarp();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kDftTmemCols);
}

// ------------------------------------------------------------------ matrices
// FP64 entries, rounded to BF16 hi and lo = BF16(v - hi).  One thread per
// complex entry (n, k) writes its four real entries.
__device__ __forceinline__ void dft_entry(const DftSpec& P, int n, int k, double* cr, double* ci) {
  const long long Q = P.Q;
  if (P.kind == kDftForward) {  // n = ky, k = y
    double s, c;
    sincospi(2.0 * (double)(((long long)n * k) % Q) / (double)Q, &s, &c);
    *cr = c;
    *ci = -s;  // e^{-i theta}
    return;
  }
  if (P.kind == kDftInverse) {  // n = y, k = ky
    double s, c;
    sincospi(2.0 * (double)(((long long)n * k) % Q) / (double)Q, &s, &c);
    *cr = c;
    *ci = s;
    return;
  }
  // inverse with the prefilter: n = box coefficient row, k = ky
  const double z1 = -0.26794919243112270;  // sqrt(3) - 2
  const double g0 = -6.0 * z1 / (1.0 - z1 * z1);
  const int D = P.fir ? kDftPrefTaps : 0;
  double sr = 0.0, si = 0.0, hd = g0;
  for (int d = 0; d <= D; ++d) {
    const double h = P.fir ? hd : 1.0;
    for (int sgn = (d == 0 ? 1 : -1); sgn <= 1; sgn += 2) {
      const int node = P.start + n + sgn * d;
      int local;
      if (P.periodic) {
        local = node % P.box_len;
        if (local < 0) local += P.box_len;
      } else {
        local = mirror_index(node, P.box_len);
      }
      const int g = wrap_once(P.box_lo + local, P.Q);
      double s, c;
      sincospi(2.0 * (double)(((long long)g * k) % Q) / (double)Q, &s, &c);
      sr += h * c;
      si += h * s;
    }
    hd *= z1;
  }
  *cr = sr;
  *ci = si;
}

__device__ __forceinline__ void put_bf16(uint16_t* hi, uint16_t* lo, size_t at, double v) {
  const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
  const __nv_bfloat16 l = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
  hi[at] = *reinterpret_cast<const uint16_t*>(&h);
  lo[at] = *reinterpret_cast<const uint16_t*>(&l);
}

__global__ void __launch_bounds__(256) k_dft_pack(const DftSpec P, int ntile, int ntiles, int kchunks, uint16_t* hi,
                                                  uint16_t* lo) {
  // one thread per complex (n, k) pair of the padded matrix
  const int ncp = ntiles * ntile / 2, kcp = kchunks * (int)kKChunk / 2;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)ncp * kcp) return;
  const int n = (int)(idx / kcp), k = (int)(idx - (long long)n * kcp);
  double cr = 0.0, ci = 0.0;
  if (n < P.Nc && k < P.Kc) dft_entry(P, n, k, &cr, &ci);
  // D[.][2n + a] = sum_k A[.][2k + b] B[2n + a][2k + b]:
  //   re out: (re in) cr - (im in) ci;  im out: (re in) ci + (im in) cr
  const double e[2][2] = {{cr, -ci}, {ci, cr}};
  for (int a = 0; a < 2; ++a) {
    const int nr = 2 * n + a;
    const int t = nr / ntile, nl = nr - t * ntile;
    for (int b = 0; b < 2; ++b) {
      const int kr = 2 * k + b;
      const int c = kr / (int)kKChunk, kl = kr - c * (int)kKChunk;
      const size_t blk = ((size_t)t * kchunks + c) * (size_t)ntile * kKChunk;
      const size_t at = blk + (size_t)((nl >> 3) * (int)(kRowGroupBytes / 2) + (kl >> 3) * (int)(kCoreBytes / 2) +
                                       (nl & 7) * 8 + (kl & 7));
      put_bf16(hi, lo, at, e[a][b]);
    }
  }
}

DftShape dft_shape(int Nc, int Kc) {
  DftShape s;
  const int nreal = 2 * Nc;
  s.ntiles = (nreal + kDftMaxN - 1) / kDftMaxN;
  const int per = (nreal + s.ntiles - 1) / s.ntiles;
  s.ntile = (per + 15) / 16 * 16;
  s.kchunks = (2 * Kc + (int)kKChunk - 1) / (int)kKChunk;
  return s;
}

size_t dft_matrix_elems(const DftShape& s) { return (size_t)s.ntiles * s.ntile * s.kchunks * kKChunk; }

cudaError_t launch_dft_pack(const DftSpec& P, const DftShape& s, uint16_t* hi, uint16_t* lo, cudaStream_t st) {
  const long long n = (long long)(s.ntiles * s.ntile / 2) * (s.kchunks * (int)kKChunk / 2);
  if (n == 0) return cudaSuccess;
  k_dft_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, s.ntile, s.ntiles, s.kchunks, hi, lo);
  return cudaGetLastError();
}

// no CTAs for an empty product (the kernel needs at least one K chunk)
int dft_tiles(int rows, const DftShape& s) {
  if (rows <= 0 || s.kchunks <= 0 || s.ntiles <= 0) return 0;
  return (rows + kDftRows - 1) / kDftRows * s.ntiles;
}

size_t dft_a_bytes(int rows, const DftShape& s) {
  if (rows <= 0 || s.kchunks <= 0) return 0;
  return (size_t)((rows + kDftRows - 1) / kDftRows) * s.kchunks * 2 * kDftStageA;
}

cudaError_t launch_ydft(const Launch<DftJob>& L, cudaStream_t st) {
  const int grid = L.tile_start[L.njobs];
  if (grid == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_ydft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDftSmem);
  if (e != cudaSuccess) return e;
  k_ydft<<<grid, kDftThreads, kDftSmem, st>>>(L);
  return cudaGetLastError();
}

}  // namespace mm
