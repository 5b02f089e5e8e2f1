// FP64 dense kernels: a register-tiled GEMM and the blocked Cholesky /
// triangular-solve drivers built on it.  All matrices are column-major.
//
// On GB300 the FP64 pipe retires about two DFMA per SM per clock (1.2 TFLOP/s
// for the GPU), so every FP64 contraction here is arithmetic-bound: a 64 x 64
// output tile with a 16-deep shared-memory stage reads 2 x 8 KB per 16 K of
// DFMA work, far below what HBM or L2 deliver.  The design goal is simply to
// keep the DFMA pipe busy: 16 independent accumulators per thread and a
// register prefetch of the next K chunk while the current one is consumed.

#include <cmath>
#include <cstdio>

#include "ec_internal.h"

namespace ec {

namespace {

__device__ __forceinline__ bool failed(const DevStatus* st) {
  return st != nullptr && *(volatile const int*)&st->code != 0;
}

// Lower-triangle tile enumeration: t -> (i, j) with i >= j.
__device__ __forceinline__ void tri_tile(int64_t t, int64_t& i, int64_t& j) {
  int64_t r = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (r * (r + 1) / 2 > t) --r;
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  i = r;
  j = t - r * (r + 1) / 2;
}

template <int TA, int TB>
__device__ __forceinline__ void gemm_tile(int64_t M, int64_t N, int64_t K, double alpha,
                                          const double* A, int64_t lda, const double* B,
                                          int64_t ldb, double beta, double* C, int64_t ldc,
                                          int tri, int64_t tm, int64_t tn) {
  const int64_t row0 = tm * GEMM_TILE, col0 = tn * GEMM_TILE;
  __shared__ double As[GEMM_KC][GEMM_TILE + 1];
  __shared__ double Bs[GEMM_KC][GEMM_TILE + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  double ra[4], rb[4];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int idx = tid + 256 * q;
      int r, kk;
      if (TA == 0) { r = idx & 63; kk = idx >> 6; } else { r = idx >> 4; kk = idx & 15; }
      int64_t gr = row0 + r, gk = k0 + kk;
      double v = 0.0;
      if (gr < M && gk < K) v = (TA == 0) ? A[gr + gk * lda] : A[gk + gr * lda];
      ra[q] = v;
      int c;
      if (TB == 0) { kk = idx & 15; c = idx >> 4; } else { c = idx & 63; kk = idx >> 6; }
      int64_t gc = col0 + c;
      gk = k0 + kk;
      v = 0.0;
      if (gc < N && gk < K) v = (TB == 0) ? B[gk + gc * ldb] : B[gc + gk * ldb];
      rb[q] = v;
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int idx = tid + 256 * q;
      int r, kk, c;
      if (TA == 0) { r = idx & 63; kk = idx >> 6; } else { r = idx >> 4; kk = idx & 15; }
      As[kk][r] = ra[q];
      if (TB == 0) { kk = idx & 15; c = idx >> 4; } else { c = idx & 63; kk = idx >> 6; }
      Bs[kk][c] = rb[q];
    }
  };

  if (K > 0) load(0);
  for (int64_t k0 = 0; k0 < K; k0 += GEMM_KC) {
    stash();
    __syncthreads();
    if (k0 + GEMM_KC < K) load(k0 + GEMM_KC);
#pragma unroll
    for (int kk = 0; kk < GEMM_KC; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int64_t gc = col0 + ty + 16 * j;
    if (gc >= N) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int64_t gr = row0 + tx + 16 * i;
      if (gr >= M || (tri && gr < gc)) continue;
      double* p = C + gr + gc * ldc;
      double v = alpha * acc[i][j];
      if (beta != 0.0) v = fma(beta, *p, v);
      *p = v;
    }
  }
}

template <int TA, int TB>
__global__ void __launch_bounds__(256) dgemm_kernel(int64_t M, int64_t N, int64_t K, double alpha,
                                                    const double* A, int64_t lda, const double* B,
                                                    int64_t ldb, double beta, double* C,
                                                    int64_t ldc, int tri, const DevStatus* st) {
  if (failed(st)) return;
  int64_t tm, tn;
  if (tri) {
    tri_tile(blockIdx.x, tm, tn);
  } else {
    tm = blockIdx.x;
    tn = blockIdx.y;
  }
  gemm_tile<TA, TB>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tri, tm, tn);
}

// Split-K partial products for C = A^T B with a short output (M <= 64 rows): slice z of
// the K range [z kc, (z+1) kc) goes to ws + z M N (ld M).
__global__ void __launch_bounds__(256) dgemm_tn_split_kernel(int64_t M, int64_t N, int64_t K,
                                                             int64_t kc, const double* A,
                                                             int64_t lda, const double* B,
                                                             int64_t ldb, double* ws,
                                                             const DevStatus* st) {
  if (failed(st)) return;
  const int64_t k0 = (int64_t)blockIdx.z * kc;
  const int64_t kl = (K - k0) < kc ? (K - k0) : kc;
  double* C = ws + (int64_t)blockIdx.z * M * N;
  gemm_tile<1, 0>(M, N, kl > 0 ? kl : 0, 1.0, A + k0, lda, B + k0, ldb, 0.0, C, M, 0, blockIdx.x,
                  blockIdx.y);
}

__global__ void split_sum_kernel(int64_t M, int64_t N, int splits, const double* ws, double* C,
                                 int64_t ldc) {
  const int64_t tot = M * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int z = 0; z < splits; ++z) v += ws[(int64_t)z * tot + idx];
    C[(idx % M) + (idx / M) * ldc] = v;
  }
}

// Merge products of divide and conquer: group z covers [s, s + nb), s = z bs, with the
// children's blocks [s, s + bs/2) and [s + bs/2, s + nb) of the block-diagonal Qin;
//   Qout[top rows, s : s + nb]    = Qin[top, top]       Wm[top rows, s : s + nb]
//   Qout[bottom rows, s : s + nb] = Qin[bottom, bottom] Wm[bottom rows, s : s + nb]
// blockIdx.z = 2 (z - z0) + (0: top, 1: bottom) for merges z0, z0 + 1, ...
__global__ void __launch_bounds__(256) dgemm_halves_kernel(int64_t n, int64_t bs, int64_t z0,
                                                           const double* Qin, const double* Wm,
                                                           double* Qout, int64_t ld,
                                                           const DevStatus* st) {
  if (failed(st)) return;
  const int64_t s0 = (z0 + (int64_t)(blockIdx.z >> 1)) * bs;
  const int64_t nb = (n - s0) < bs ? (n - s0) : bs;
  const int64_t half = bs / 2;
  const int64_t off = (blockIdx.z & 1) ? half : 0;
  const int64_t M = (blockIdx.z & 1) ? nb - half : half;
  if (M <= 0 || (int64_t)blockIdx.x * GEMM_TILE >= M || (int64_t)blockIdx.y * GEMM_TILE >= nb)
    return;
  const int64_t r0 = s0 + off;
  gemm_tile<0, 0>(M, nb, M, 1.0, Qin + r0 + r0 * ld, ld, Wm + r0 + s0 * ld, ld, 0.0,
                  Qout + r0 + s0 * ld, ld, 0, blockIdx.x, blockIdx.y);
}

// Cholesky of one diagonal block (kb <= 64) in shared memory, plus the inverse
// of the resulting lower-triangular factor.  One CTA of 256 threads.
__global__ void __launch_bounds__(256) potf2_diag_kernel(double* A, int64_t lda, int kb,
                                                         double* Dinv, DevStatus* st,
                                                         int64_t gk) {
  if (failed(st)) return;
  extern __shared__ double sm[];
  double* S = sm;                 // S[c * 65 + r] = L(r, c)
  double* X = sm + 64 * 65;       // X[c * 65 + r] = Linv(r, c)
  __shared__ int bad;
  __shared__ double rpiv;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kb * kb; idx += blockDim.x) {
    int r = idx % kb, c = idx / kb;
    S[c * 65 + r] = (r >= c) ? A[r + (int64_t)c * lda] : 0.0;
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (tid == 0) {
      double d = S[j * 65 + j];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
        if (atomicCAS(&st->code, 0, (int)EC_ERR_NOT_SPD) == 0) st->info = (int)(gk + j);
      } else {
        double p = sqrt(d);
        S[j * 65 + j] = p;
        rpiv = 1.0 / p;
      }
    }
    __syncthreads();
    if (bad) return;
    for (int r = j + 1 + tid; r < kb; r += blockDim.x) S[j * 65 + r] *= rpiv;
    __syncthreads();
    const int n2 = kb - j - 1;
    for (int idx = tid; idx < n2 * n2; idx += blockDim.x) {
      int c = j + 1 + idx / n2, r = j + 1 + idx % n2;
      if (r >= c) S[c * 65 + r] = fma(-S[j * 65 + r], S[j * 65 + c], S[c * 65 + r]);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < kb * kb; idx += blockDim.x) {
    int r = idx % kb, c = idx / kb;
    if (r >= c) A[r + (int64_t)c * lda] = S[c * 65 + r];
  }
  // Inverse by forward substitution, one column per thread.
  if (tid < kb) {
    const int c = tid;
    for (int r = 0; r < c; ++r) X[c * 65 + r] = 0.0;
    X[c * 65 + c] = 1.0 / S[c * 65 + c];
    for (int r = c + 1; r < kb; ++r) {
      double s0 = 0.0, s1 = 0.0;
      int k = c;
      for (; k + 1 < r; k += 2) {
        s0 = fma(S[k * 65 + r], X[c * 65 + k], s0);
        s1 = fma(S[(k + 1) * 65 + r], X[c * 65 + k + 1], s1);
      }
      if (k < r) s0 = fma(S[k * 65 + r], X[c * 65 + k], s0);
      X[c * 65 + r] = -(s0 + s1) / S[r * 65 + r];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    int r = idx % NB, c = idx / NB;
    Dinv[idx] = (r < kb && c < kb && r >= c) ? X[c * 65 + r] : 0.0;
  }
}

__global__ void symmetrize_kernel(int64_t n, double* A, int64_t lda) {
  int64_t c = blockIdx.y * (int64_t)blockDim.y + threadIdx.y;
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < n && c < n && r < c) A[r + c * lda] = A[c + r * lda];
}

__global__ void add_lower_kernel(int64_t n, double* A, int64_t lda, const double* B, int64_t ldb,
                                 double alpha) {
  for (int64_t c = blockIdx.y; c < n; c += gridDim.y)
    for (int64_t r = c + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
      A[r + c * lda] = fma(alpha, B[r + c * ldb], A[r + c * lda]);
}

__global__ void copy_kernel(int64_t m, int64_t n, const double* A, int64_t lda, double* B,
                            int64_t ldb) {
  for (int64_t c = blockIdx.y; c < n; c += gridDim.y)
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
         r += (int64_t)gridDim.x * blockDim.x)
      B[r + c * ldb] = A[r + c * lda];
}

__global__ void axpy_kernel(int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                            double* B, int64_t ldb) {
  for (int64_t c = blockIdx.y; c < n; c += gridDim.y)
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
         r += (int64_t)gridDim.x * blockDim.x)
      B[r + c * ldb] = fma(alpha, A[r + c * lda], B[r + c * ldb]);
}

}  // namespace

void axpy_matrix(cudaStream_t s, int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                 double* B, int64_t ldb) {
  if (m <= 0 || n <= 0) return;
  dim3 grid((unsigned)((m + 255) / 256 < 64 ? (m + 255) / 256 : 64),
            (unsigned)(n < 65535 ? n : 65535));
  axpy_kernel<<<grid, 256, 0, ::ec::counted(s)>>>(m, n, alpha, A, lda, B, ldb);
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// Products with few columns (N <= SKINNY_N: initial modal state, projections, a few
// snapshots): a 64 x 64 output tile would spend most of its FMAs on padding, so these
// stream A once with all N accumulators per output row.
constexpr int SKINNY_N = 16;

// C = alpha A B + beta C, A: M x K.  Block: 64 rows x 4 K-groups; each thread sums
// every 4th K index of its row, the four partial sums are added in a fixed order.
__global__ void __launch_bounds__(256) skinny_nn_kernel(int64_t M, int N, int64_t K, double alpha,
                                                        const double* A, int64_t lda,
                                                        const double* B, int64_t ldb, double beta,
                                                        double* C, int64_t ldc, const DevStatus* st) {
  if (failed(st)) return;
  __shared__ double red[4][SKINNY_N][64];
  const int tr = threadIdx.x & 63, g = threadIdx.x >> 6;
  const int64_t r = (int64_t)blockIdx.x * 64 + tr;
  double acc[SKINNY_N];
#pragma unroll
  for (int j = 0; j < SKINNY_N; ++j) acc[j] = 0.0;
  if (r < M) {
    for (int64_t k = g; k < K; k += 4) {
      const double a = A[r + k * lda];
#pragma unroll
      for (int j = 0; j < SKINNY_N; ++j)
        if (j < N) acc[j] = fma(a, B[k + j * ldb], acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < SKINNY_N; ++j) red[g][j][tr] = acc[j];
  __syncthreads();
  if (g == 0 && r < M) {
    for (int j = 0; j < N; ++j) {
      const double v = alpha * ((red[0][j][tr] + red[1][j][tr]) + (red[2][j][tr] + red[3][j][tr]));
      double* c = C + r + j * ldc;
      *c = beta != 0.0 ? fma(beta, *c, v) : v;
    }
  }
}

// C = alpha A^T B + beta C, A: K x M.  One warp per output row: lanes stride down the
// contiguous column A[:, r], then a shuffle reduction per output column.  With ct = 1
// the result is stored transposed (C[j + r ldc]), which serves a short A^T B computed
// as (B^T A)^T.
__global__ void __launch_bounds__(256) skinny_tn_kernel(int64_t M, int N, int64_t K, double alpha,
                                                        const double* A, int64_t lda,
                                                        const double* B, int64_t ldb, double beta,
                                                        double* C, int64_t ldc, int ct,
                                                        const DevStatus* st) {
  if (failed(st)) return;
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= M) return;
  const double* col = A + r * lda;
  double acc[SKINNY_N];
#pragma unroll
  for (int j = 0; j < SKINNY_N; ++j) acc[j] = 0.0;
  for (int64_t k = lane; k < K; k += 32) {
    const double a = col[k];
#pragma unroll
    for (int j = 0; j < SKINNY_N; ++j)
      if (j < N) acc[j] = fma(a, B[k + j * ldb], acc[j]);
  }
#pragma unroll
  for (int j = 0; j < SKINNY_N; ++j) {
    double v = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && j < N) {
      double* c = ct ? C + j + r * ldc : C + r + j * ldc;
      *c = beta != 0.0 ? fma(beta, *c, alpha * v) : alpha * v;
    }
  }
}

void dgemm(cudaStream_t s, Op ta, Op tb, int64_t M, int64_t N, int64_t K, double alpha,
           const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
           int64_t ldc, int tri, const DevStatus* st) {
  if (M <= 0 || N <= 0) return;
  if (!tri && tb == N_ && N <= SKINNY_N && K >= 4 * GEMM_TILE) {
    if (ta == N_)
      skinny_nn_kernel<<<(unsigned)((M + 63) / 64), 256, 0, ::ec::counted(s)>>>(
          M, (int)N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
    else
      skinny_tn_kernel<<<(unsigned)((M + 7) / 8), 256, 0, ::ec::counted(s)>>>(
          M, (int)N, K, alpha, A, lda, B, ldb, beta, C, ldc, 0, st);
    return;
  }
  if (!tri && ta == T_ && tb == N_ && M <= SKINNY_N && K >= 4 * GEMM_TILE) {
    // few output rows: C^T = B^T A, one warp per column of C, stored transposed
    skinny_tn_kernel<<<(unsigned)((N + 7) / 8), 256, 0, ::ec::counted(s)>>>(
        N, (int)M, K, alpha, B, ldb, A, lda, beta, C, ldc, 1, st);
    return;
  }
  if (!tri && tb == N_ && N > GEMM_TILE && N % GEMM_TILE != 0 && N % GEMM_TILE <= SKINNY_N &&
      K >= 4 * GEMM_TILE) {
    // a ragged last column tile would be mostly padding: full tiles + a skinny remainder
    const int64_t r = N % GEMM_TILE, Nf = N - r;
    dgemm(s, ta, tb, M, Nf, K, alpha, A, lda, B, ldb, beta, C, ldc, 0, st);
    dgemm(s, ta, tb, M, r, K, alpha, A, lda, B + Nf * ldb, ldb, beta, C + Nf * ldc, ldc, 0, st);
    return;
  }
  dim3 grid;
  if (tri) {
    int64_t nt = (M + GEMM_TILE - 1) / GEMM_TILE;
    grid = dim3((unsigned)(nt * (nt + 1) / 2), 1, 1);
  } else {
    grid = dim3((unsigned)((M + GEMM_TILE - 1) / GEMM_TILE), (unsigned)((N + GEMM_TILE - 1) / GEMM_TILE), 1);
  }
  if (ta == N_ && tb == N_)
    dgemm_kernel<0, 0><<<grid, 256, 0, ::ec::counted(s)>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tri, st);
  else if (ta == N_ && tb == T_)
    dgemm_kernel<0, 1><<<grid, 256, 0, ::ec::counted(s)>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tri, st);
  else if (ta == T_ && tb == N_)
    dgemm_kernel<1, 0><<<grid, 256, 0, ::ec::counted(s)>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tri, st);
  else
    dgemm_kernel<1, 1><<<grid, 256, 0, ::ec::counted(s)>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tri, st);
}

int dgemm_tn_splits(int64_t M, int64_t N, int64_t K) {
  const int64_t tiles = ((M + GEMM_TILE - 1) / GEMM_TILE) * ((N + GEMM_TILE - 1) / GEMM_TILE);
  int64_t sp = (4 * (int64_t)num_sms() + tiles - 1) / tiles;
  if (sp > 64) sp = 64;
  if (sp > K / 256) sp = K / 256;
  return sp < 1 ? 1 : (int)sp;
}

void dgemm_tn_split(cudaStream_t s, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double* C, int64_t ldc, double* ws, int splits,
                    const DevStatus* st) {
  if (M <= 0 || N <= 0) return;
  if (splits <= 1 || !ws) {
    dgemm(s, T_, N_, M, N, K, 1.0, A, lda, B, ldb, 0.0, C, ldc, 0, st);
    return;
  }
  int64_t kc = (K + splits - 1) / splits;
  kc = (kc + GEMM_KC - 1) / GEMM_KC * GEMM_KC;
  const int sp = (int)((K + kc - 1) / kc);
  dim3 grid((unsigned)((M + GEMM_TILE - 1) / GEMM_TILE), (unsigned)((N + GEMM_TILE - 1) / GEMM_TILE),
            (unsigned)sp);
  dgemm_tn_split_kernel<<<grid, 256, 0, ::ec::counted(s)>>>(M, N, K, kc, A, lda, B, ldb, ws, st);
  const int64_t g = (M * N + 255) / 256 < 2048 ? (M * N + 255) / 256 : 2048;
  split_sum_kernel<<<(unsigned)g, 256, 0, ::ec::counted(s)>>>(M, N, sp, ws, C, ldc);
}

void dgemm_halves(cudaStream_t s, int64_t n, int64_t bs, int64_t groups, const double* Qin,
                  const double* Wm, double* Qout, int64_t ld, const DevStatus* st) {
  if (groups <= 0) return;
  const int64_t half = bs / 2;
  const unsigned tm = (unsigned)((half + GEMM_TILE - 1) / GEMM_TILE);
  const unsigned tn = (unsigned)((bs + GEMM_TILE - 1) / GEMM_TILE);
  // gridDim.z is limited to 65535: at most 32767 merges (two halves each) per launch
  constexpr int64_t ZMAX = 32767;
  for (int64_t z0 = 0; z0 < groups; z0 += ZMAX) {
    const int64_t g = (groups - z0) < ZMAX ? (groups - z0) : ZMAX;
    dgemm_halves_kernel<<<dim3(tm, tn, (unsigned)(2 * g)), 256, 0, ::ec::counted(s)>>>(
        n, bs, z0, Qin, Wm, Qout, ld, st);
  }
}

// Two-level blocking: the 64-wide diagonal steps of each PW-wide panel update only the
// panel's own columns (rows) with rank-64 products; the trailing part of the matrix is
// then updated once per panel with a rank-PW product.  PW = 192 is one K chunk of the
// tensor-core path, whose rank-64 updates would be bound by the read-modify-write of C
// rather than by the tensor work.
constexpr int64_t PW = 192;
static_assert(PW % NB == 0, "panel width must be a multiple of the block size");

// Lower-triangle update of an m x w column panel, rows r0.. of C (the first w rows
// form the diagonal square): C -= X Y^T with X (m x kb), Y (w x kb).
void panel_update_lower(cudaStream_t s, OzWork* oz, int64_t m, int64_t w, int kb, const double* X,
                        int64_t ldx, const double* Y, int64_t ldy, double* C, int64_t ldc,
                        const DevStatus* st) {
  if (m <= 0 || w <= 0) return;
  gemm_auto(s, oz, N_, T_, w, w, kb, -1.0, X, ldx, Y, ldy, 1.0, C, ldc, 1, st);
  if (m > w)
    gemm_auto(s, oz, N_, T_, m - w, w, kb, -1.0, X + w, ldx, Y, ldy, 1.0, C + w, ldc, 0, st);
}

void potrf(cudaStream_t s, int64_t n, double* A, int64_t lda, double* Dinv, DevStatus* st,
           OzWork* oz) {
  static std::atomic<unsigned long long> attr_set{0};
  const int smem = 2 * 64 * 65 * (int)sizeof(double);
  if (first_on_device(attr_set))
    cudaFuncSetAttribute(potf2_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  for (int64_t k0 = 0; k0 < n; k0 += PW) {
    const int64_t pe = (k0 + PW) < n ? (k0 + PW) : n;     // panel columns [k0, pe)
    for (int64_t k = k0; k < pe; k += NB) {
      const int kb = (int)((n - k) < NB ? (n - k) : NB);
      double* Akk = A + k + k * lda;
      double* Dk = Dinv + (k / NB) * NB * NB;
      potf2_diag_kernel<<<1, 256, smem, ::ec::counted(s)>>>(Akk, lda, kb, Dk, st, k);
      const int64_t rest = n - k - kb;
      if (rest > 0) {
        double* P = A + (k + kb) + k * lda;
        // panel: P <- P Lkk^{-T}  (in place; each CTA owns whole rows of the panel)
        gemm_auto(s, oz, N_, T_, rest, kb, kb, 1.0, P, lda, Dk, NB, 0.0, P, lda, 0, st);
        // the panel's remaining columns [k + kb, pe), lower part
        panel_update_lower(s, oz, rest, pe - k - kb, kb, P, lda, P, lda,
                           A + (k + kb) + (k + kb) * lda, lda, st);
      }
    }
    const int64_t rest = n - pe;
    if (rest > 0) {   // trailing lower update: A22 <- A22 - P P^T, rank pe - k0
      const double* P = A + pe + k0 * lda;
      gemm_auto(s, oz, N_, T_, rest, rest, pe - k0, -1.0, P, lda, P, lda, 1.0, A + pe + pe * lda,
                lda, 1, st);
    }
  }
}

void trsm_left_lower(cudaStream_t s, int64_t n, int64_t nrhs, const double* Lf, int64_t ldl,
                     const double* Dinv, double* B, int64_t ldb, const DevStatus* st, OzWork* oz) {
  for (int64_t k0 = 0; k0 < n; k0 += PW) {
    const int64_t pe = (k0 + PW) < n ? (k0 + PW) : n;
    for (int64_t k = k0; k < pe; k += NB) {
      const int kb = (int)((n - k) < NB ? (n - k) : NB);
      const double* Dk = Dinv + (k / NB) * NB * NB;
      double* Bk = B + k;
      gemm_auto(s, oz, N_, N_, kb, nrhs, kb, 1.0, Dk, NB, Bk, ldb, 0.0, Bk, ldb, 0, st);
      const int64_t inner = pe - k - kb;
      if (inner > 0)
        gemm_auto(s, oz, N_, N_, inner, nrhs, kb, -1.0, Lf + (k + kb) + k * ldl, ldl, Bk, ldb,
                  1.0, B + k + kb, ldb, 0, st);
    }
    const int64_t rest = n - pe;
    if (rest > 0)
      gemm_auto(s, oz, N_, N_, rest, nrhs, pe - k0, -1.0, Lf + pe + k0 * ldl, ldl, B + k0, ldb,
                1.0, B + pe, ldb, 0, st);
  }
}

void trsm_left_lower_t(cudaStream_t s, int64_t n, int64_t nrhs, const double* Lf, int64_t ldl,
                       const double* Dinv, double* B, int64_t ldb, const DevStatus* st,
                       OzWork* oz) {
  if (n <= 0) return;
  for (int64_t k0 = (n - 1) / PW * PW; k0 >= 0; k0 -= PW) {
    const int64_t pe = (k0 + PW) < n ? (k0 + PW) : n;     // panel rows [k0, pe)
    for (int64_t k = (pe - 1) / NB * NB; k >= k0; k -= NB) {
      const int kb = (int)((n - k) < NB ? (n - k) : NB);
      const double* Dk = Dinv + (k / NB) * NB * NB;
      double* Bk = B + k;
      gemm_auto(s, oz, T_, N_, kb, nrhs, kb, 1.0, Dk, NB, Bk, ldb, 0.0, Bk, ldb, 0, st);
      if (k > k0)  // B[k0:k] -= L[k:k+kb, k0:k]^T B_k
        gemm_auto(s, oz, T_, N_, k - k0, nrhs, kb, -1.0, Lf + k + k0 * ldl, ldl, Bk, ldb, 1.0,
                  B + k0, ldb, 0, st);
    }
    if (k0 > 0)  // B[0:k0] -= L[k0:pe, 0:k0]^T B[k0:pe]
      gemm_auto(s, oz, T_, N_, k0, nrhs, pe - k0, -1.0, Lf + k0, ldl, B + k0, ldb, 1.0, B, ldb, 0,
                st);
  }
}

// Lower triangle of B Lf^{-T} for a square B (n x n) whose product is symmetric (the
// two-sided reduction C^{-1} L C^{-T}): block column k needs only rows >= k, and the
// trailing update only the lower triangle of the trailing block, a third of the
// flops of the full solve.  The strict upper triangle is left stale.
void trsm_right_lower_t_sym(cudaStream_t s, int64_t n, const double* Lf, int64_t ldl,
                            const double* Dinv, double* B, int64_t ldb, const DevStatus* st,
                            OzWork* oz) {
  for (int64_t k0 = 0; k0 < n; k0 += PW) {
    const int64_t pe = (k0 + PW) < n ? (k0 + PW) : n;
    for (int64_t k = k0; k < pe; k += NB) {
      const int kb = (int)((n - k) < NB ? (n - k) : NB);
      const double* Dk = Dinv + (k / NB) * NB * NB;
      double* Bk = B + k * ldb;
      gemm_auto(s, oz, N_, T_, n - k, kb, kb, 1.0, Bk + k, ldb, Dk, NB, 0.0, Bk + k, ldb, 0, st);
      // the panel's remaining columns [k + kb, pe), rows below their diagonal:
      // B[k+kb:, k+kb:pe] -= B[k+kb:, k:k+kb] L[k+kb:pe, k:k+kb]^T
      panel_update_lower(s, oz, n - k - kb, pe - k - kb, kb, Bk + k + kb, ldb,
                         Lf + (k + kb) + k * ldl, ldl, B + (k + kb) + (k + kb) * ldb, ldb, st);
    }
    const int64_t rest = n - pe;
    if (rest > 0)  // lower(B[pe:, pe:]) -= B[pe:, k0:pe] L[pe:, k0:pe]^T
      gemm_auto(s, oz, N_, T_, rest, rest, pe - k0, -1.0, B + pe + k0 * ldb, ldb,
                Lf + pe + k0 * ldl, ldl, 1.0, B + pe + pe * ldb, ldb, 1, st);
  }
}

void symmetrize_lower(cudaStream_t s, int64_t n, double* A, int64_t lda) {
  dim3 blk(32, 8);
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 7) / 8));
  symmetrize_kernel<<<grid, blk, 0, ::ec::counted(s)>>>(n, A, lda);
}

void add_lower(cudaStream_t s, int64_t n, double* A, int64_t lda, const double* B, int64_t ldb,
               double alpha) {
  if (n <= 0) return;
  dim3 grid((unsigned)((n + 255) / 256 < 64 ? (n + 255) / 256 : 64),
            (unsigned)(n < 65535 ? n : 65535));
  add_lower_kernel<<<grid, 256, 0, ::ec::counted(s)>>>(n, A, lda, B, ldb, alpha);
}

void copy_matrix(cudaStream_t s, int64_t m, int64_t n, const double* A, int64_t lda, double* B,
                 int64_t ldb) {
  if (m <= 0 || n <= 0) return;
  dim3 grid((unsigned)((m + 255) / 256 < 64 ? (m + 255) / 256 : 64),
            (unsigned)(n < 65535 ? n : 65535));
  copy_kernel<<<grid, 256, 0, ::ec::counted(s)>>>(m, n, A, lda, B, ldb);
}

}  // namespace ec
