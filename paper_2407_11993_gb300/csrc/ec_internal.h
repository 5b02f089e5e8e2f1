// Internal declarations shared by the translation units of the eddy-current
// theta-method library.  Not part of the C ABI (that is include/eddy_theta.h).
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/eddy_theta.h"

namespace ec {

// Device-side status block.  Kernels write the first error they see and later
// kernels of the same pipeline return early once it is set.
struct DevStatus {
  int code;        // ec_status value, 0 = OK
  int info;        // e.g. the global index of a non-positive pivot
  int where;       // which kernel / wait gave up (diagnostics)
  int pad;
};

constexpr int NB = 64;              // block size of every blocked FP64 algorithm here
constexpr int GEMM_TILE = 64;       // output tile of the FP64 GEMM kernel
constexpr int GEMM_KC = 16;         // K chunk staged through shared memory

enum Op { N_ = 0, T_ = 1 };

struct OzWork;   // workspace of the FP64-accurate tensor-core products (ec_oz.h)

// ---- FP64 dense kernels (ec_blas.cu); all column-major -------------------
// C[MxN] = alpha op(A) op(B) + beta C.  tri = 1 restricts work to the lower
// triangle of C (tiles above the diagonal skipped, diagonal tiles masked).
// Products with at most 16 columns (or, for A^T B, at most 16 rows) go to streaming
// kernels instead of 64 x 64 tiles, and a last column tile of at most 16 columns is
// split off the same way (no FMAs spent on padding).
void dgemm(cudaStream_t s, Op ta, Op tb, int64_t M, int64_t N, int64_t K, double alpha,
           const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
           double* C, int64_t ldc, int tri, const DevStatus* st);

// Same product, dispatched: with a tensor-core workspace `oz` and a product large enough
// to gain from it, the FP64-accurate tensor-core path (ec_oz.cu); otherwise dgemm.
void gemm_auto(cudaStream_t s, OzWork* oz, Op ta, Op tb, int64_t M, int64_t N, int64_t K,
               double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
               double beta, double* C, int64_t ldc, int tri, const DevStatus* st);

// C (M x N, ld ldc) = A^T B for a short output (M <= 64) and long K, with K split
// into `splits` slices whose partial products (ws: splits x M x N) are summed in
// slice order; dgemm_tn_splits picks the slice count that fills the GPU.
int dgemm_tn_splits(int64_t M, int64_t N, int64_t K);
void dgemm_tn_split(cudaStream_t s, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double* C, int64_t ldc, double* ws, int splits,
                    const DevStatus* st);

// Divide-and-conquer merge products: for each merge z (rows / columns [z bs,
// min((z+1) bs, n))), the top and bottom children's diagonal blocks of Qin times the
// matching rows of Wm, into the same rows of Qout (columns of the whole merge).
void dgemm_halves(cudaStream_t s, int64_t n, int64_t bs, int64_t groups, const double* Qin,
                  const double* Wm, double* Qout, int64_t ld, const DevStatus* st);

// The blocked drivers below take an optional tensor-core workspace: with it, their
// trailing updates and panel products run through gemm_auto's FP64-accurate
// tensor-core path; without it, on the FP64 CUDA cores.
//
// Blocked right-looking Cholesky of the lower triangle of A (n x n, ld lda), in
// place.  Dinv receives, per NB block, the inverse of the diagonal block of the
// factor (NB x NB column-major, zero above the diagonal).  A non-positive pivot
// sets st->code = EC_ERR_NOT_SPD and st->info = its global index.
void potrf(cudaStream_t s, int64_t n, double* A, int64_t lda, double* Dinv, DevStatus* st,
           OzWork* oz = nullptr);

// B <- Lfac^{-1} B  (left, lower, no transpose); B is n x nrhs.
void trsm_left_lower(cudaStream_t s, int64_t n, int64_t nrhs, const double* Lfac, int64_t ldl,
                     const double* Dinv, double* B, int64_t ldb, const DevStatus* st,
                     OzWork* oz = nullptr);
// B <- Lfac^{-T} B  (left, lower factor, transposed = upper solve).
void trsm_left_lower_t(cudaStream_t s, int64_t n, int64_t nrhs, const double* Lfac, int64_t ldl,
                       const double* Dinv, double* B, int64_t ldb, const DevStatus* st,
                       OzWork* oz = nullptr);
// Lower triangle of B <- B Lfac^{-T} for square B whose result is symmetric
// (n x n); the strict upper triangle is not written.
void trsm_right_lower_t_sym(cudaStream_t s, int64_t n, const double* Lfac, int64_t ldl,
                            const double* Dinv, double* B, int64_t ldb, const DevStatus* st,
                            OzWork* oz = nullptr);

// Symmetrise: copy the lower triangle onto the upper one.
void symmetrize_lower(cudaStream_t s, int64_t n, double* A, int64_t lda);
// A <- A + alpha B on the lower triangle (n x n).
void add_lower(cudaStream_t s, int64_t n, double* A, int64_t lda, const double* B, int64_t ldb,
               double alpha);
void copy_matrix(cudaStream_t s, int64_t m, int64_t n, const double* A, int64_t lda, double* B,
                 int64_t ldb);

// ---- persistent blocked triangular solves (ec_trsv.cu) --------------------
struct TrsvSync {
  int* flags_fwd;     // one per NB block: epoch of the last published block
  int* flags_bwd;
  unsigned* tickets;  // [0] forward, [1] backward
  int* epoch;         // device epoch, bumped once per solve pair
};
// Lfac y = b then Lfac^T x = y, x and y of length n.  b and x may alias.
// ev (optional, 3 events): recorded before the forward solve, between the two
// solves and after the backward solve.
void trsv_pair(cudaStream_t s, int64_t n, const double* Lfac, int64_t ldl, const double* Dinv,
               const double* b, double* y, double* x, const TrsvSync& sync, int grid,
               long long spin_limit, DevStatus* st, cudaEvent_t* ev = nullptr);
void trsv_begin(cudaStream_t s, const TrsvSync& sync);   // resets tickets, bumps epoch

// ---- inverse-factor solves (ec_trmv.cu) ----------------------------------
// W = C^{-1} for the lower Cholesky factor C (n x n); W's diagonal 64 x 64 blocks
// hold zeros above the diagonal, blocks above the block diagonal are not written.
void trtri_lower(cudaStream_t s, int64_t n, const double* C, int64_t ldc, const double* Dinv,
                 double* W, int64_t ldw, const DevStatus* st,
                 OzWork* oz = nullptr);
int trmv_chunks(int64_t n, int chunk);
// y = W b (part1: trmv_chunks x n partials, summed into y), then x = W^T y as
// trmv_chunks x n partials in part2 (the consumer sums them in order).
void trmv_pair(cudaStream_t s, int64_t n, const double* W, int64_t ldw, const double* b,
               double* part1, double* y, double* part2, int chunk, const DevStatus* st,
               cudaEvent_t* ev = nullptr);

// out[i] = sum_q part[q * n + i], q = 0 .. nin-1 (fixed order)
void sum_partials(cudaStream_t s, int64_t n, int nin, const double* part, double* out);

// Test hook: a wait on a flag nothing sets, bounded by spin_limit.
void wait_timeout_probe(cudaStream_t s, int* flag, long long spin_limit, DevStatus* st);

int num_sms();

// Every device allocation the library makes for a context goes through here
// (cudaMalloc, or a reported failure while the test hook set by
// ec_selftest_fail_alloc is armed and has run out).
cudaError_t device_alloc(void** p, size_t bytes);

// True the first time it is called with `mask` while a given device is current (one bit
// per device; devices past 63 always get true).  For per-device one-time setup such as
// raising a kernel's dynamic shared-memory limit.
inline bool first_on_device(std::atomic<unsigned long long>& mask) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return true;
  const unsigned long long bit = 1ull << dev;
  return (mask.fetch_or(bit) & bit) == 0;
}

// Every kernel launch of the library passes its stream through counted(), which
// increments the process-wide launch counter reported by ec_launch_count().
void note_launch();
inline cudaStream_t counted(cudaStream_t s) {
  note_launch();
  return s;
}

}  // namespace ec

namespace ec {
// B <- B + alpha A  (m x n blocks).
void axpy_matrix(cudaStream_t s, int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                 double* B, int64_t ldb);
}  // namespace ec
