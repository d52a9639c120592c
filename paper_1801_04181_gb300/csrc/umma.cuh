// 5th-generation tensor core (tcgen05) helpers for sm_103a: TMEM allocation,
// shared-memory matrix descriptors, the BF16 MMA with FP32 accumulation in
// TMEM, completion through an mbarrier, and the TMEM -> register load.
//
// Operand layout used throughout: K-major, no swizzle.  A "core matrix" is 8
// rows x 16 bytes (8 BF16 values of K) stored as 128 contiguous bytes, row i
// at byte 16 i.  A tile of R rows x 32 K (one pipeline stage) keeps the 4 core
// matrices of a row group contiguous: core (row group g, K group c) at byte
// g * 512 + c * 128.  The descriptor's leading byte offset is then the stride
// between core matrices along K (128) and its stride byte offset the stride
// between row groups (512).  (Measured on GB300: back-to-back MMAs on this
// layout run at the tensor core's full rate, as with the 128-byte swizzle.)
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mm {

constexpr uint32_t kCoreBytes = 128;      // one 8 x 16-byte core matrix
constexpr uint32_t kKChunk = 32;          // BF16 K values per pipeline stage
constexpr uint32_t kRowGroupBytes = 512;  // 8 rows x 32 K x 2 bytes

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) of a stage tile (see the layout above)
__device__ __forceinline__ uint32_t tile_offset(int row, int k) {
  return (uint32_t)(row >> 3) * kRowGroupBytes + (uint32_t)(k >> 3) * kCoreBytes + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}

// Packed split operand: rows of complex values stored as BF16 hi | lo blocks,
// one block per (128-row tile, K chunk of 16 complex): the hi tile (8 KB, the
// layout above) followed by the lo tile, so a stage loads it by one bulk copy.
constexpr int kTileRows = 128;
constexpr uint32_t kTileSplitBytes = kTileRows * kKChunk * 2;  // one split of one block

// v = (re, im) of row `row`, complex column `kc`, into the packed operand
// with `kchunks` K chunks per 128-row tile: hi = BF16(v), lo = BF16(v - hi)
__device__ __forceinline__ void store_split(void* packed, int kchunks, int row, int kc, float2 v) {
  const int cpx = (int)(kKChunk / 2);
  uint8_t* blk = reinterpret_cast<uint8_t*>(packed) +
                 ((size_t)(row / kTileRows) * kchunks + kc / cpx) * 2 * kTileSplitBytes;
  const uint32_t off = tile_offset(row % kTileRows, 2 * (kc % cpx));
  const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
  *reinterpret_cast<__nv_bfloat162*>(blk + off) = h;
  *reinterpret_cast<__nv_bfloat162*>(blk + kTileSplitBytes + off) = l;
}

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (all in 16-byte units), descriptor version 1 (bits 46-47), base
// offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16: D in FP32 (bits 4-5 = 1), A and B in
// BF16 (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// TMEM: one whole warp allocates ncols columns (a power of two, 32..512); the
// base address is written to *slot in shared memory
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core's reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// the arrival of the thread that starts `bytes` of bulk copies completing on *bar
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// bulk copy (TMA, untiled) of `bytes` from global to this CTA's shared memory,
// completing on *bar; both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Wait until the phase of parity `parity` of *bar has completed, for at most
// `max_cycles` SM clocks; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long max_cycles) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > max_cycles) return false;
  }
}

// D[tmem] (+)= A[desc] * B[desc]^T, M x N x 16, issued by one thread
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive once on *bar when every MMA this thread issued so far has completed
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive FP32 columns of the TMEM lane this thread's warp owns
// (warp w of a warpgroup reads lanes 32 (w % 4) .. 32 (w % 4) + 31)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace mm
