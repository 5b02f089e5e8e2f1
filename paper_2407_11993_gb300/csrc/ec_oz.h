// FP64-accurate dense products on the tensor cores (Ozaki-type integer slices in
// BF16, tcgen05 MMAs, exact per-diagonal accumulation); see ec_oz.cu.
#pragma once

#include <cuda_bf16.h>

#include "ec_internal.h"

namespace ec {

// K handled by one launch (longer K runs as consecutive launches accumulating in C).
constexpr int OZ_KCHUNK = 192;

// Device workspace of the emulated products: the BF16 slices of one panel of each
// operand, their power-of-two exponents, and a scratch of row maxima.  Grown on demand
// (through device_alloc) and kept until oz_free; cap_elems bounds the slices (BF16
// elements), which makes large operands go through in panels.
struct OzWork {
  __nv_bfloat16* slices = nullptr;
  int64_t slices_cap = 0;
  int* exps = nullptr;
  unsigned long long* maxb = nullptr;
  int64_t rows_cap = 0;
  int64_t cap_elems = 2ll << 30;        // 4 GB of slices
};

int64_t oz_kchunk();
void oz_free(OzWork* w);

// C = alpha op(A) op(B) + beta C with FP64 inputs and output, column-major, computed
// on the tensor cores from eight 8-bit slices per operand.  tri = 1 (M == N) updates
// only the lower triangle of C.  Error: below 2^-60 max_k|a_ik| max_k|b_kj| sqrt(K)
// per entry (the scales are per row of op(A) and per column of op(B)) plus one FP64
// rounding of each 192-long K chunk's contribution.  Enqueued on s; needs w.
ec_status oz_gemm(cudaStream_t s, Op ta, Op tb, int64_t M, int64_t N, int64_t K, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                  double* C, int64_t ldc, int tri, OzWork* w, DevStatus* st);

// The slices of a fixed left operand op(A) (R x K, rows scaled by their own powers of
// two), cut once and reused by every later product with it: a product with few right
// columns then reads 16 bytes per entry of A instead of splitting A again (24 bytes of
// traffic per entry on top).  Layout: blocks of 128 rows x 32 K (64 KB, all eight slices)
// stored as the tensor-core kernel's shared-memory image (64-byte swizzle applied), so
// that each block arrives with one contiguous bulk copy.  Memory: 16 x (R rounded up to
// 128) x (K rounded up to 32) bytes.
struct OzSplit {
  uint8_t* blocks = nullptr;            // [row tile][K block][slice][128 rows][64 B]
  int* exps = nullptr;                  // R
  int64_t R = 0, K = 0, nkb = 0;        // nkb: K blocks of 32
};
// EC_ERR_OOM when the slices do not fit (out stays empty).
ec_status oz_presplit(cudaStream_t s, Op ta, int64_t R, int64_t K, const double* A, int64_t lda,
                      OzSplit* out);
void oz_split_free(OzSplit* a);
// C = op(A)[:, :kuse] op(B) with op(A) from `a` (kuse <= a.K), op(B) kuse x N; C is
// overwritten (beta = 0).  Column groups of up to 32, one stream-K launch each.
ec_status oz_gemm_presplit(cudaStream_t s, const OzSplit& a, int64_t kuse, Op tb, int64_t N,
                           const double* B, int64_t ldb, double* C, int64_t ldc, OzWork* w,
                           DevStatus* st);

}  // namespace ec
