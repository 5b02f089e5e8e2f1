// Symmetric eigensolver stages: tridiagonalisation, back-transformation and the
// divide-and-conquer tridiagonal eigensolver.
#pragma once

#include "ec_internal.h"

namespace ec {

// A (n x n, full symmetric, column-major) -> d (n), e (n-1), tau (n-2); reflector
// tails stored below the subdiagonal of A.  v, w: n-vectors; partial: scratch of
// partial_cap doubles (at least n).
void sytrd_lower(cudaStream_t s, int64_t n, double* A, int64_t lda, double* d, double* e,
                 double* tau, double* v, double* w, double* partial, int64_t partial_cap,
                 const DevStatus* st);

// Y (n x ncol) <- Q Y with Q = H_0 ... H_{n-3} from sytrd_lower.  Scratch: V (n x 64),
// G, T (64 x 64), W, W2 (64 x ncol), ws (ws_cap doubles, for the split-K product
// V^T Y; up to dgemm_tn_splits(64, ncol, n) x 64 x ncol are used).
void ormtr_lower(cudaStream_t s, int64_t n, const double* A, int64_t lda, const double* tau,
                 double* Y, int64_t ldy, int64_t ncol, double* V, double* G, double* T,
                 double* W, double* W2, double* ws, int64_t ws_cap, const DevStatus* st);

// Divide-and-conquer eigensolver of the symmetric tridiagonal (d, e):
// lam (n, ascending) and Q (n x n, column-major, ld n) with T = Q diag(lam) Q^T.
struct DcWork;
DcWork* dc_alloc(int64_t n, cudaError_t (*alloc)(void**, size_t));
void dc_free(DcWork* w);
// Q must be an n x n buffer; Qtmp and W two more n x n scratch buffers.
ec_status dc_solve(cudaStream_t s, int64_t n, const double* d, const double* e, double* lam,
                   double* Q, double* Qtmp, double* W, DcWork* wk, DevStatus* st);

}  // namespace ec
