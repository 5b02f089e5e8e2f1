// FP32 and FP32-pair products of the modal form's mode matrix U with a few columns
// (EC_PREC_FP32 / EC_PREC_FP32X2 of the modal form): the snapshot reconstruction
// U X (Sec. 3.2, Eq. modal_decomposition_discrete) and the projections U^T Y.
#pragma once

#include "ec_kernels.h"

namespace ec {

// Element layout of a reduced-precision copy of U: FP32 (4 bytes) or an FP32 hi/lo
// pair (8 bytes, hi = fp32(u), lo = fp32(u - hi)).
struct U32 {
  void* data = nullptr;      // column-major, ld rows per column (ld % 4 == 0), rows >= n0 zero
  int64_t ld = 0;
  int pair = 0;              // 0: float, 1: float2 pair
  int eU = 0;                // U32 holds U * 2^-eU (a power of two: exact)
};

// Rounds the FP64 matrix U (n0 x n0, ldu) into u (allocated here with device_alloc).
// Returns EC_ERR_OOM when the copy does not fit.
ec_status u32_build(cudaStream_t s, int64_t n0, const double* U, int64_t ldu, int pair, U32* u);
void u32_free(U32* u);

// Scratch of the products: the right operand rounded column by column (with a power
// of two per column) and the K-split partial sums.
struct Skinny32Work {
  void* y = nullptr;
  size_t ycap = 0;           // bytes
  int* yexp = nullptr;
  size_t ecap = 0;           // entries
  double* part = nullptr;
  size_t pcap = 0;           // doubles
};
void skinny32_free(Skinny32Work* w);

// C (n0 x N, ldc) = U[:, :K] Y (trans = 0, Y K x N, ldy) or U^T Y (trans = 1, K = n0,
// Y n0 x N).  FP32: operands rounded to FP32, FP32 products and FP32 sums within each
// K segment, the segments added in FP64.  Pair: compensated FP32 arithmetic (exact
// hi*hi products by FMA, the two cross terms, float-float sums) with FP64 sums every
// 64 products.  Returns EC_ERR_OOM when the scratch cannot grow.
ec_status skinny32_product(cudaStream_t s, const U32& u, int64_t n0, int trans, int64_t N,
                           int64_t K, const double* Y, int64_t ldy, double* C, int64_t ldc,
                           Skinny32Work* w, const DevStatus* st);

}  // namespace ec
