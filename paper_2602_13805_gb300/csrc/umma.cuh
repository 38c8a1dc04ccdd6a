// BF16 tensor-core GEMM for sm_103a: tcgen05.mma with TMEM accumulators, operands staged in
// shared memory by TMA (cp.async.bulk.tensor, 128-byte swizzle), an mbarrier ring between
// one producer thread and one MMA-issuing thread.
//
//   C[z][m][n] = sum_{k in split z} A[m][k] * B[n][k]          (fp32 accumulate)
//   split_bf16: A = A_hi + A_lo, B = B_hi + B_lo (bf16 each) and the product is taken as
//               A_hi B_hi + A_hi B_lo + A_lo B_hi, which carries ~16 mantissa bits.
//
// A and B are K-major bf16 row arrays; the tile is 128 (m) x 128 (n) x 64 (k) per stage,
// one CTA of 128 threads per output tile and K split.  Every wait is bounded (about a second
// of clock cycles); on timeout the kernel raises *err, skips the remaining work, and still
// releases its TMEM.
#pragma once

#include <cuda.h>

#include "common.cuh"

#define UMMA_BM 128
#define UMMA_BN 128
#define UMMA_BK 64
#define UMMA_STAGES 3
#define UMMA_TILE_BYTES (UMMA_BM * UMMA_BK * 2)           // 16 KB: 128 rows x 128 B
#define UMMA_STAGE_BYTES (4 * UMMA_TILE_BYTES)             // A_hi, B_hi, A_lo, B_lo
#define UMMA_SMEM_BYTES (UMMA_STAGES * UMMA_STAGE_BYTES + 1024)

struct UmmaArgs {
  int m_rows, n_rows, k;     // A [m_rows][k], B [n_rows][k]
  int kb_per_split;          // 64-wide k-blocks per split (blockIdx.z)
  int split_bf16;            // 1: three-product split-BF16
  float* C;                  // [split][m_rows][ldc]
  int ldc;
  long long split_stride;    // elements between consecutive splits of C
  int* err;                  // raised on a wait timeout
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok;
}
// Bounded wait on phase `parity`; false (and *err = 1) after ~2^31 cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err) {
  if (mbar_try_wait(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(b, parity)) {
    if (clock64() - t0 > (1ll << 31)) {
      atomicExch(err, 1);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile of 128-byte rows with the 128-byte swizzle,
// 8-row atoms 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;      // stride byte offset
  d |= (uint64_t)1 << 46;                // version
  d |= (uint64_t)2 << 61;                // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both K-major, M = 128, N = UMMA_BN.
__host__ __device__ constexpr uint32_t umma_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(UMMA_BN >> 3) << 17) | ((uint32_t)(UMMA_BM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// 8 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3);
  v[4] = __uint_as_float(r4);
  v[5] = __uint_as_float(r5);
  v[6] = __uint_as_float(r6);
  v[7] = __uint_as_float(r7);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct UmmaOperand {
  CUtensorMap hi, lo;
  int rows, k;
};

// Encodes the tensor maps of a bf16 [rows][k] K-major array pair (k * 2 bytes must be a
// multiple of 16, pointers 16-byte aligned).  lo may equal hi when the split is not used.
pdf_status umma_operand(UmmaOperand* op, const void* hi, const void* lo, int rows, int k);
// Launches the GEMM over C (see UmmaArgs); nsplit K splits (clamped to the k-block count).
pdf_status umma_gemm(const UmmaOperand& A, const UmmaOperand& B, int split_bf16, int nsplit, float* C, int ldc,
                     long long split_stride, int* err, cudaStream_t st);
int umma_kblocks(int k);
