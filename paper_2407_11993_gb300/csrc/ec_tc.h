// BF16 tcgen05 GEMM (reduced-precision variant of the modal projections and
// reconstruction).
#pragma once

#include <cuda_bf16.h>

#include "ec_internal.h"

namespace ec {

// cuTensorMapEncodeTiled, resolved once through the runtime's driver entry-point
// query (nullptr when unavailable).
void* tensor_map_encode_fn();

// Leading dimension (elements) of a K-major bf16 operand: K rounded up to 8 (16 bytes).
int64_t bf16_ld(int64_t K);
// dst[i * ld + k] = bf16(src element (i, k)), zero for k >= K; src column-major (lds),
// holding the operand (trans = 0: src[i + k lds]) or its transpose (trans = 1: src[k + i lds]).
// lo (optional): bf16 of the rounding remainder, so that hi + lo holds ~16 significant bits.
void to_bf16(cudaStream_t s, int64_t M, int64_t K, const double* src, int64_t lds, int trans,
             __nv_bfloat16* dst, int64_t ld, __nv_bfloat16* lo = nullptr);
// C[i + j ldc] = alpha sum_k A[i * lda + k] B[j * ldb + k] + beta C  (FP32 accumulation in TMEM)
ec_status tc_gemm_bf16(cudaStream_t s, int64_t M, int64_t N, int64_t K, double alpha,
                       const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb,
                       double beta, double* C, int64_t ldc, DevStatus* st);

// Split-BF16 product: with A = Ah + Al and B = Bh + Bl,
// C = alpha (Ah Bh + Ah Bl + Al Bh) (three tensor-core products summed in FP64).
ec_status tc_gemm_bf16x3(cudaStream_t s, int64_t M, int64_t N, int64_t K, double alpha,
                         const __nv_bfloat16* Ah, const __nv_bfloat16* Al, int64_t lda,
                         const __nv_bfloat16* Bh, const __nv_bfloat16* Bl, int64_t ldb, double* C,
                         int64_t ldc, DevStatus* st);

}  // namespace ec
