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

// Same reduction, blocked in panels of 64 columns (the LAPACK LATRD scheme): inside a
// panel each column is brought up to date with the panel's earlier reflectors, the
// symmetric product uses the panel-start trailing matrix plus low-rank corrections,
// and the panel's rank-2 updates are applied together as one rank-128 update of the
// trailing lower triangle through gemm_auto (tensor cores with `oz`).  The symmetric
// product reads each element of the trailing triangle once (64 x 64 tiles, both
// contributions per element, partials summed in a fixed order).  Identical reflectors
// in exact arithmetic.  Scratch: V, W (n x 64), y (128), partial
// (sytrd_blocked_scratch(n) doubles).  pair_symv = 1 runs the symmetric product in
// compensated FP32 (FP64 entries split into FP32 hi/lo pairs, about 2^-46 relative per
// product; reflectors, updates and everything else stay FP64-accurate).
int64_t sytrd_blocked_scratch(int64_t n);
void sytrd_lower_blocked(cudaStream_t s, int64_t n, double* A, int64_t lda, double* d, double* e,
                         double* tau, double* V, double* W, double* y, double* partial,
                         OzWork* oz, const DevStatus* st, int pair_symv = 0);

// Y (n x ncol) <- Q Y with Q = H_0 ... H_{n-3} from sytrd_lower.  Scratch: V (n x 64),
// G, T (64 x 64), W, W2 (64 x ncol), ws (ws_cap doubles, for the split-K product
// V^T Y; up to dgemm_tn_splits(64, ncol, n) x 64 x ncol are used).
void ormtr_lower(cudaStream_t s, int64_t n, const double* A, int64_t lda, const double* tau,
                 double* Y, int64_t ldy, int64_t ncol, double* V, double* G, double* T,
                 double* W, double* W2, double* ws, int64_t ws_cap, const DevStatus* st);

// Same application of Q in compact-WY groups of gsize reflectors (a multiple of 64):
// per group one V (n x gsize), T (gsize x gsize) and three large products, so that Y is
// read once per group; the products go through gemm_auto (tensor cores with `oz`).
// Scratch: V (n x gsize), G, T (gsize x gsize), X (gsize x 64), W, W2 (gsize x ncol).
void ormtr_lower_grouped(cudaStream_t s, int64_t n, const double* A, int64_t lda,
                         const double* tau, double* Y, int64_t ldy, int64_t ncol, int64_t gsize,
                         double* V, double* G, double* T, double* X, double* W, double* W2,
                         OzWork* oz, const DevStatus* st);

// Divide-and-conquer eigensolver of the symmetric tridiagonal (d, e):
// lam (n, ascending) and Q (n x n, column-major, ld n) with T = Q diag(lam) Q^T.
struct DcWork;
DcWork* dc_alloc(int64_t n, cudaError_t (*alloc)(void**, size_t));
void dc_free(DcWork* w);
// Q must be an n x n buffer; Qtmp and W two more n x n scratch buffers.
// With a tensor-core workspace `oz`, merges of DC_TC_MIN or more rows multiply their
// eigenvector blocks on the FP64-accurate tensor-core path.
constexpr int64_t DC_TC_MIN = 1024;
ec_status dc_solve(cudaStream_t s, int64_t n, const double* d, const double* e, double* lam,
                   double* Q, double* Qtmp, double* W, DcWork* wk, DevStatus* st,
                   OzWork* oz = nullptr);

}  // namespace ec
