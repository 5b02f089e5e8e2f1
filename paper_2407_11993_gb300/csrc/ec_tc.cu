// BF16 tensor-core GEMM on tcgen05 for the reduced-precision variant of the
// modal form's dense contractions (projections U^T [R_D | L_D | M_0], U^T (C K)^T
// and the snapshot reconstruction U X), FP32 accumulation, FP64 output.
//
//   C[i, j] = alpha * sum_k A[i, k] B[j, k]      (A: M x K, B: N x K, both K-major bf16)
//
// One CTA computes a 128 x 128 tile of C:
//   * warp 0 / lane 0 streams 128 x 64 tiles of A and B into shared memory with
//     TMA (cp.async.bulk.tensor, 128-byte swizzle) through a 4-stage ring guarded
//     by mbarriers;
//   * warp 1 / lane 0 issues tcgen05.mma (kind::f16, M = 128, N = 128, K = 16) into
//     a 128-column FP32 accumulator in tensor memory and returns each stage to the
//     producer with tcgen05.commit;
//   * all four warps then read the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32w .. 32w+31 = rows of the tile) and store FP64 results.
// Every mbarrier wait is bounded; a wait that runs out records EC_ERR_TIMEOUT in
// the status block and the kernel skips its remaining work and frees its TMEM.

#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "ec_async.cuh"
#include "ec_internal.h"
#include "ec_tc.h"

namespace ec {

namespace {

constexpr int TM = 128, TN = 128, TK = 64, STAGES = 4;
constexpr int A_BYTES = TM * TK * 2;   // 16 KB
constexpr int B_BYTES = TN * TK * 2;   // 16 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;   // + alignment slack
constexpr long long WAIT_LIMIT = 1ll << 26;

using dev::mbar_expect_tx;
using dev::mbar_init;
using dev::mbar_try_wait;
using dev::smem_u32;

// Bounded wait; false (and the status set) when the bound runs out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, DevStatus* st,
                                          int where) {
  return dev::mbar_wait(bar, parity, st, where, WAIT_LIMIT);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile, rows of 128 bytes, 128-byte
// swizzle, 8-row groups 1024 bytes apart, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint64_t addr = smem_u32(p);
  return ((addr & 0x3FFFFull) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, N = TN, M = TM.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__global__ void __launch_bounds__(128) tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                                                      const __grid_constant__ CUtensorMap mapB,
                                                      int M, int N, int K, double alpha,
                                                      double beta, double* C, int64_t ldc,
                                                      DevStatus* st) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, issued, consumed;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  const int nk = (K + TK - 1) / TK;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    issued = 0;
    consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t use = kb / STAGES;
      if (kb >= STAGES && !mbar_wait(&empty_bar[s], (use - 1) & 1, st, 21)) {
        abort_flag = 1;
        break;
      }
      uint8_t* a = smem + s * STAGE_BYTES;
      uint8_t* b = a + A_BYTES;
      mbar_expect_tx(&full_bar[s], STAGE_BYTES);
      tma_load_2d(a, &mapA, &full_bar[s], kb * TK, m0);
      tma_load_2d(b, &mapB, &full_bar[s], kb * TK, n0);
      *(volatile int*)&issued = kb + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(&full_bar[s], (kb / STAGES) & 1, st, 22)) {
        abort_flag = 1;
        break;
      }
      *(volatile int*)&consumed = kb + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint8_t* a = smem + s * STAGE_BYTES;
      const uint8_t* b = a + A_BYTES;
      const uint64_t da = smem_desc(a), db = smem_desc(b);
#pragma unroll
      for (int kk = 0; kk < TK / 16; ++kk)
        mma_bf16(tmem, da + 2 * kk, db + 2 * kk, (kb > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty_bar[s]);
    }
    // always committed: arrives once every MMA this thread issued has completed
    mma_commit(&done_bar);
  }
  __syncwarp();
  __syncthreads();
  // wait for the accumulator; on an aborted pipeline also drain the TMA loads that were
  // issued but never consumed, so no copy is still writing shared memory at exit
  if (threadIdx.x == 0) {
    if (!mbar_wait(&done_bar, 0, st, 23)) abort_flag = 1;
    if (abort_flag)
      for (int kb = consumed; kb < issued; ++kb)
        mbar_wait(&full_bar[kb % STAGES], (kb / STAGES) & 1, st, 24);
  }
  __syncthreads();
  const bool good = (abort_flag == 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (good) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < TN; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c0 + j;
          if (col < N) {
            double* c = C + (int64_t)row + (int64_t)col * ldc;
            const double d = alpha * (double)__uint_as_float(r[j]);
            *c = (beta != 0.0) ? fma(beta, *c, d) : d;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN)
                 : "memory");
}

// dst (bf16): element (i, k) of an M x K operand, K-major with leading dimension ld
// (ld >= K, multiple of 8; the padding is zeroed).  src (FP64) is column-major with
// leading dimension lds and holds either the operand (trans = 0: src[i + k lds]) or
// its transpose (trans = 1: src[k + i lds]).
// lo (optional) receives bf16(v - hi): hi + lo carries about 16 significant bits.
__global__ void to_bf16_kernel(int64_t M, int64_t K, const double* src, int64_t lds, int trans,
                               __nv_bfloat16* dst, __nv_bfloat16* lo, int64_t ld) {
  const int64_t tot = M * ld;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / ld, k = idx % ld;
    double v = 0.0;
    if (k < K) v = trans ? src[k + i * lds] : src[i + k * lds];
    const __nv_bfloat16 h = __double2bfloat16(v);
    dst[idx] = h;
    if (lo) lo[idx] = __double2bfloat16(v - (double)__bfloat162float(h));
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    cudaGetLastError();
  });
  return fn;
}

bool make_map(CUtensorMap* map, const __nv_bfloat16* base, int64_t rows, int64_t K, int64_t ld,
              int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

void* tensor_map_encode_fn() { return (void*)encode_fn(); }

int64_t bf16_ld(int64_t K) { return (K + 7) / 8 * 8; }

void to_bf16(cudaStream_t s, int64_t M, int64_t K, const double* src, int64_t lds, int trans,
             __nv_bfloat16* dst, int64_t ld, __nv_bfloat16* lo) {
  const int64_t tot = M * ld;
  int64_t g = (tot + 255) / 256;
  if (g > (int64_t)num_sms() * 16) g = num_sms() * 16;
  if (g < 1) g = 1;
  to_bf16_kernel<<<(unsigned)g, 256, 0, ::ec::counted(s)>>>(M, K, src, lds, trans, dst, lo, ld);
}

ec_status tc_gemm_bf16(cudaStream_t s, int64_t M, int64_t N, int64_t K, double alpha,
                       const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb,
                       double beta, double* C, int64_t ldc, DevStatus* st) {
  if (M <= 0 || N <= 0) return EC_OK;
  if (K <= 0 || (lda % 8) || (ldb % 8) || lda < K || ldb < K) return EC_ERR_ARG;
  if (((uintptr_t)A | (uintptr_t)B) & 15) return EC_ERR_ARG;
  if (M > (1ll << 31) - TM || N > (1ll << 31) - TN || K > (1ll << 31)) return EC_ERR_UNSUPPORTED;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, K, lda, TM) || !make_map(&mb, B, N, K, ldb, TN)) return EC_ERR_CUDA;
  static std::atomic<unsigned long long> attr_set{0};
  if (first_on_device(attr_set))
    cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  dim3 grid((unsigned)((M + TM - 1) / TM), (unsigned)((N + TN - 1) / TN));
  tc_gemm_kernel<<<grid, 128, SMEM_BYTES, ::ec::counted(s)>>>(ma, mb, (int)M, (int)N, (int)K,
                                                              alpha, beta, C, ldc, st);
  return cudaGetLastError() == cudaSuccess ? EC_OK : EC_ERR_CUDA;
}

ec_status tc_gemm_bf16x3(cudaStream_t s, int64_t M, int64_t N, int64_t K, double alpha,
                         const __nv_bfloat16* Ah, const __nv_bfloat16* Al, int64_t lda,
                         const __nv_bfloat16* Bh, const __nv_bfloat16* Bl, int64_t ldb, double* C,
                         int64_t ldc, DevStatus* st) {
  ec_status rc = tc_gemm_bf16(s, M, N, K, alpha, Al, lda, Bh, ldb, 0.0, C, ldc, st);
  if (rc == EC_OK) rc = tc_gemm_bf16(s, M, N, K, alpha, Ah, lda, Bl, ldb, 1.0, C, ldc, st);
  if (rc == EC_OK) rc = tc_gemm_bf16(s, M, N, K, alpha, Ah, lda, Bh, ldb, 1.0, C, ldc, st);
  return rc;
}

}  // namespace ec

extern "C" ec_status ec_gemm_bf16(int64_t M, int64_t N, int64_t K, const double* A,
                                  const double* B, double* C, void* stream) {
  using namespace ec;
  if (!A || !B || !C || M < 0 || N < 0 || K < 1) return EC_ERR_ARG;
  if (M == 0 || N == 0) return EC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t ld = bf16_ld(K);
  __nv_bfloat16 *a = nullptr, *b = nullptr;
  DevStatus* st = nullptr;
  if (cudaMalloc((void**)&a, sizeof(__nv_bfloat16) * M * ld) != cudaSuccess ||
      cudaMalloc((void**)&b, sizeof(__nv_bfloat16) * N * ld) != cudaSuccess ||
      cudaMalloc((void**)&st, sizeof(DevStatus)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(a);
    cudaFree(b);
    return EC_ERR_OOM;
  }
  cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
  to_bf16(s, M, K, A, M, 0, a, ld);
  to_bf16(s, N, K, B, K, 1, b, ld);
  ec_status rc = tc_gemm_bf16(s, M, N, K, 1.0, a, ld, b, ld, 0.0, C, M, st);
  cudaError_t e = cudaStreamSynchronize(s);
  DevStatus h{};
  if (e == cudaSuccess) e = cudaMemcpy(&h, st, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(a);
  cudaFree(b);
  cudaFree(st);
  if (rc != EC_OK) return rc;
  if (e != cudaSuccess) return EC_ERR_CUDA;
  return h.code ? (ec_status)h.code : EC_OK;
}
