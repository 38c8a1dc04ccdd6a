// Host side of the tcgen05 GEMM: tensor-map encoding (driver entry point looked up through the
// runtime, no link against libcuda) and the launcher.
#include <cudaTypedefs.h>

#include <mutex>
#include <string>

#include "problem.cuh"
#include "umma.cuh"

__global__ void __launch_bounds__(128, 1)
    k_umma_gemm(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tB_hi,
                const __grid_constant__ CUtensorMap tA_lo, const __grid_constant__ CUtensorMap tB_lo, UmmaArgs g) {
  extern __shared__ uint8_t umma_smem_raw[];
  __shared__ __align__(8) uint64_t full[UMMA_STAGES], empty[UMMA_STAGES], done;
  __shared__ uint32_t tmem_slot;
  uint8_t* smem = (uint8_t*)(((uintptr_t)umma_smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * UMMA_BM, n0 = blockIdx.y * UMMA_BN;
  const int kb_total = (g.k + UMMA_BK - 1) / UMMA_BK;
  const int kb0 = blockIdx.z * g.kb_per_split;
  const int kb1 = min(kb0 + g.kb_per_split, kb_total);
  const int nkb = max(kb1 - kb0, 0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < UMMA_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) tmem_alloc(&tmem_slot, UMMA_BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = tmem_slot;

  if (warp == 0 && lane == 0 && nkb > 0) {
    // TMA producer
    const uint32_t bytes = (g.split_bf16 ? 4u : 2u) * UMMA_TILE_BYTES;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % UMMA_STAGES;
      if (i >= UMMA_STAGES && !mbar_wait(&empty[s], ((i / UMMA_STAGES) - 1) & 1, g.err)) break;
      uint8_t* st = smem + s * UMMA_STAGE_BYTES;
      mbar_arrive_expect_tx(&full[s], bytes);
      const int kx = (kb0 + i) * UMMA_BK;
      tma_load_2d(st, &tA_hi, &full[s], kx, m0);
      tma_load_2d(st + UMMA_TILE_BYTES, &tB_hi, &full[s], kx, n0);
      if (g.split_bf16) {
        tma_load_2d(st + 2 * UMMA_TILE_BYTES, &tA_lo, &full[s], kx, m0);
        tma_load_2d(st + 3 * UMMA_TILE_BYTES, &tB_lo, &full[s], kx, n0);
      }
    }
  } else if (warp == 1 && lane == 0 && nkb > 0) {
    // MMA issuer
    const uint32_t idesc = umma_idesc();
    for (int i = 0; i < nkb; ++i) {
      const int s = i % UMMA_STAGES;
      if (!mbar_wait(&full[s], (i / UMMA_STAGES) & 1, g.err)) break;
      tc_fence_after();
      const uint32_t a_hi = smem_u32(smem + s * UMMA_STAGE_BYTES);
      const uint32_t b_hi = a_hi + UMMA_TILE_BYTES, a_lo = a_hi + 2 * UMMA_TILE_BYTES, b_lo = a_hi + 3 * UMMA_TILE_BYTES;
#pragma unroll
      for (int kk = 0; kk < UMMA_BK / 16; ++kk) {
        const uint32_t off = kk * 32;   // 16 bf16 along K inside the swizzled 128-byte row
        umma_bf16(taddr, umma_sdesc(a_hi + off), umma_sdesc(b_hi + off), idesc, (i | kk) != 0);
        if (g.split_bf16) {
          umma_bf16(taddr, umma_sdesc(a_hi + off), umma_sdesc(b_lo + off), idesc, 1);
          umma_bf16(taddr, umma_sdesc(a_lo + off), umma_sdesc(b_hi + off), idesc, 1);
        }
      }
      umma_commit(&empty[s]);
    }
    umma_commit(&done);
  }
  __syncwarp();
  // epilogue: warp w owns accumulator rows 32w .. 32w + 31 (TMEM lanes)
  bool have = nkb > 0 ? mbar_wait(&done, 0, g.err) : false;
  have = __all_sync(0xffffffffu, have);
  tc_fence_after();
  const int row = m0 + warp * 32 + lane;
  float* crow = g.C + (long long)blockIdx.z * g.split_stride + (long long)row * g.ldc;
  for (int c0 = 0; c0 < UMMA_BN; c0 += 8) {
    float v[8];
    if (have) {
      tmem_ld8(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = 0.f;
    }
    if (row < g.m_rows) {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (n0 + c0 + j < g.n_rows) crow[n0 + c0 + j] = v[j];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) tmem_dealloc(taddr, UMMA_BN);
}


static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static pdf_status get_encode() {
  static std::once_flag once;
  static cudaError_t status = cudaSuccess;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    status = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (status == cudaSuccess && q == cudaDriverEntryPointSuccess) g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  if (!g_encode) return set_err(PDF_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
  return PDF_OK;
}

static pdf_status encode(CUtensorMap* m, const void* ptr, int rows, int k) {
  if (((uintptr_t)ptr & 15) || ((k * 2) % 16)) return set_err(PDF_EINVAL, "TMA operand misaligned");
  cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)k * 2};
  cuuint32_t box[2] = {UMMA_BK, UMMA_BM};
  cuuint32_t es[2] = {1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_err(PDF_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return PDF_OK;
}

pdf_status umma_operand(UmmaOperand* op, const void* hi, const void* lo, int rows, int k) {
  pdf_status s = get_encode();
  if (s != PDF_OK) return s;
  if ((s = encode(&op->hi, hi, rows, k)) != PDF_OK) return s;
  if ((s = encode(&op->lo, lo ? lo : hi, rows, k)) != PDF_OK) return s;
  op->rows = rows;
  op->k = k;
  return PDF_OK;
}

int umma_kblocks(int k) { return (k + UMMA_BK - 1) / UMMA_BK; }

pdf_status umma_gemm(const UmmaOperand& A, const UmmaOperand& B, int split_bf16, int nsplit, float* C, int ldc,
                     long long split_stride, int* err, cudaStream_t st) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_umma_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, UMMA_SMEM_BYTES);
  });
  if (A.k != B.k) return set_err(PDF_EINVAL, "GEMM operands disagree on K");
  const int kb = umma_kblocks(A.k);
  if (nsplit < 1) nsplit = 1;
  if (nsplit > kb) nsplit = kb;
  const int per = (kb + nsplit - 1) / nsplit;
  nsplit = (kb + per - 1) / per;
  UmmaArgs g;
  g.m_rows = A.rows;
  g.n_rows = B.rows;
  g.k = A.k;
  g.kb_per_split = per;
  g.split_bf16 = split_bf16;
  g.C = C;
  g.ldc = ldc;
  g.split_stride = split_stride;
  g.err = err;
  dim3 grid((A.rows + UMMA_BM - 1) / UMMA_BM, (B.rows + UMMA_BN - 1) / UMMA_BN, nsplit);
  k_umma_gemm<<<grid, 128, UMMA_SMEM_BYTES, st>>>(A.hi, B.hi, A.lo, B.lo, g);
  pdf_count_launch(1);
  PDF_LAUNCHED("tcgen05 GEMM");
  return PDF_OK;
}
