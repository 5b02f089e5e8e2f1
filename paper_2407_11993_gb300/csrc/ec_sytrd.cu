// Householder tridiagonalisation A = Q T Q^T of a symmetric matrix (lower
// reflectors, the first stage of the standard symmetric eigensolver used for
// the pencil of Sec. 3.2 after its reduction to standard form) and the
// application of Q to a block of vectors with compact-WY blocks of 64
// reflectors.
//
// Column j: reflector H_j = I - tau_j v_j v_j^T with v_j = 0 above row j+1,
// v_j[j+1] = 1, annihilating A[j+2:, j]; then
//   p = tau A22 v,  w = p - (tau/2)(p^T v) v,  A22 <- A22 - v w^T - w v^T.
// Blocking (delaying the rank-2 updates into a GEMM) does not pay on GB300: the
// update is FP64-bound either way (2 FMAs per element per column), and FP64 GEMM
// runs at the same ~1.2 TFLOP/s as the streamed rank-2 update.
// Only the lower triangle is kept up to date (half the FP64 work of the rank-2
// update); A22 v is read from it as a row part and a column part, both coalesced.
// v_j[j+2:] is stored back into A[j+2:, j].

#include <cmath>

#include "ec_ff.h"
#include "ec_internal.h"
#include "ec_sytrd.h"

namespace ec {

namespace {

constexpr int HT = 1024;

__device__ double block_sum1024(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

__global__ void __launch_bounds__(HT) house_col_kernel(int64_t n, double* A, int64_t lda,
                                                       int64_t j, double* v, double* d, double* e,
                                                       double* tau, const DevStatus* st) {
  if (st->code) return;
  __shared__ double sh[40];
  __shared__ double s_scale;
  double* col = A + j * lda;
  double sig = 0.0;
  for (int64_t i = j + 2 + threadIdx.x; i < n; i += HT) sig = fma(col[i], col[i], sig);
  sig = block_sum1024(sig, sh);
  const double alpha = col[j + 1];
  double beta, t, scale;
  if (sig == 0.0) {
    beta = alpha;
    t = 0.0;
    scale = 0.0;
  } else {
    const double nx = sqrt(alpha * alpha + sig);
    beta = alpha >= 0.0 ? -nx : nx;
    t = (beta - alpha) / beta;
    scale = 1.0 / (alpha - beta);
  }
  if (threadIdx.x == 0) {
    d[j] = col[j];
    e[j] = beta;
    tau[j] = t;
    s_scale = scale;
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += HT) {
    double vi;
    if (i <= j) vi = 0.0;
    else if (i == j + 1) vi = 1.0;
    else {
      vi = col[i] * s_scale;
      col[i] = vi;
    }
    v[i] = vi;
  }
}

// Only the lower triangle of the trailing matrix is kept up to date, so A22 v is
// split into its row part and its column part:
//   partial[c * n + i] = sum over column chunk c of A[i, k] v[k], k <= i   (row part)
//   colpart[i]         = sum_{k > i} A[k, i] v[k]                        (column part)
__global__ void __launch_bounds__(256) symv_partial_kernel(int64_t n, const double* A, int64_t lda,
                                                           int64_t j, const double* v,
                                                           double* partial, int64_t kc) {
  const int64_t i = j + 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t k0 = j + 1 + blockIdx.y * kc;
  int64_t k1 = k0 + kc;
  if (k1 > n) k1 = n;
  if (k1 > i + 1) k1 = i + 1;
  if (i >= n) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int64_t k = k0;
  for (; k + 3 < k1; k += 4) {
    s0 = fma(A[i + k * lda], v[k], s0);
    s1 = fma(A[i + (k + 1) * lda], v[k + 1], s1);
    s2 = fma(A[i + (k + 2) * lda], v[k + 2], s2);
    s3 = fma(A[i + (k + 3) * lda], v[k + 3], s3);
  }
  for (; k < k1; ++k) s0 = fma(A[i + k * lda], v[k], s0);
  partial[blockIdx.y * n + i] = (s0 + s1) + (s2 + s3);
}

// One warp per column i: colpart[i] = sum_{k > i} A[k, i] v[k] (coalesced down the column).
__global__ void __launch_bounds__(256) symv_col_kernel(int64_t n, const double* A, int64_t lda,
                                                       int64_t j, const double* v, double* colpart) {
  const int64_t i = j + 1 + blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const double* col = A + i * lda;
  double s0 = 0.0, s1 = 0.0;
  int64_t k = i + 1 + lane;
  for (; k + 32 < n; k += 64) {
    s0 = fma(col[k], v[k], s0);
    s1 = fma(col[k + 32], v[k + 32], s1);
  }
  if (k < n) s0 = fma(col[k], v[k], s0);
  double t = s0 + s1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) colpart[i] = t;
}

// p = tau A22 v from the row and column partials (rows j+1 .. n-1), then
// w = p - f v with f = (tau/2) p^T v: each CTA owns a contiguous row range and writes
// its part of p^T v; the last CTA to finish sums the parts in CTA order and turns p
// into w in place.
__global__ void __launch_bounds__(256) p_kernel(int64_t n, int64_t j, const double* v,
                                                const double* tau, const double* partial,
                                                int nchunk, const double* colpart, double* p,
                                                double* dots, unsigned* counter) {
  __shared__ double sh[9];
  __shared__ bool last;
  const double t = tau[j];
  const int64_t len = n - j - 1;
  const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = j + 1 + blockIdx.x * chunk;
  const int64_t r1 = (r0 + chunk < n) ? r0 + chunk : n;
  double dot = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    double q = colpart[i];
    for (int c = 0; c < nchunk; ++c) q += partial[c * n + i];
    q *= t;
    p[i] = q;
    dot = fma(q, v[i], dot);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  if (lane == 0) sh[w] = dot;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) b += sh[q];
    dots[blockIdx.x] = b;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < 32) {
    double b = 0.0;
    for (unsigned q = threadIdx.x; q < gridDim.x; q += 32) b += __ldcg(dots + q);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    if (threadIdx.x == 0) {
      sh[8] = 0.5 * t * b;
      *counter = 0u;
    }
  }
  __syncthreads();
  const double f = sh[8];
  for (int64_t i = j + 1 + threadIdx.x; i < n; i += blockDim.x) p[i] = fma(-f, v[i], p[i]);
}

// lower(A22) <- lower(A22 - v w^T - w v^T).
__global__ void syr2_kernel(int64_t n, double* A, int64_t lda, int64_t j, const double* v,
                            const double* w, const double* tau) {
  if (tau[j] == 0.0) return;
  const int64_t len = n - j - 1;
  for (int64_t kk = blockIdx.y; kk < len; kk += gridDim.y) {
    const int64_t k = j + 1 + kk;
    const double vk = v[k], wk = w[k];
    double* colk = A + k * lda;
    for (int64_t i = k + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
      colk[i] = fma(-v[i], wk, fma(-w[i], vk, colk[i]));
  }
}

__global__ void tail_kernel(int64_t n, const double* A, int64_t lda, double* d, double* e) {
  if (n >= 2) {
    d[n - 2] = A[(n - 2) + (n - 2) * lda];
    d[n - 1] = A[(n - 1) + (n - 1) * lda];
    e[n - 2] = A[(n - 1) + (n - 2) * lda];
  } else if (n == 1) {
    d[0] = A[0];
  }
}

// V (n x kb): column c = v_{b+c}: zero above row b+c+1, one at b+c+1, stored tail below.
__global__ void form_v_kernel(int64_t n, const double* A, int64_t lda, int64_t b, int kb,
                              double* V) {
  const int c = blockIdx.y;
  const int64_t j = b + c;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double x;
    if (i <= j) x = 0.0;
    else if (i == j + 1) x = 1.0;
    else x = A[i + j * lda];
    V[i + (int64_t)c * n] = x;
  }
}

// T (kb x kb upper, ld ldt) of Q_b = H_b ... H_{b+kb-1} = I - V T V^T from G = V^T V
// (ld ldg).
__global__ void form_t_kernel(int kb, const double* G, int64_t ldg, const double* tau, int64_t b,
                              double* T, int64_t ldt) {
  __shared__ double Ts[64][65];
  __shared__ double g[64];
  const int a = threadIdx.x;
  for (int i = 0; i < kb; ++i) {
    if (a < kb) g[a] = G[a + i * ldg];
    __syncthreads();
    const double ti = tau[b + i];
    if (a < i) {
      double s = 0.0;
      for (int c = a; c < i; ++c) s = fma(Ts[a][c], g[c], s);
      Ts[a][i] = -ti * s;
    } else if (a == i) {
      Ts[a][i] = ti;
    } else if (a < kb) {
      Ts[a][i] = 0.0;
    }
    __syncthreads();
  }
  for (int i = 0; i < kb; ++i)
    if (a < kb) T[a + i * ldt] = Ts[a][i];
}

}  // namespace

void sytrd_lower(cudaStream_t s, int64_t n, double* A, int64_t lda, double* d, double* e,
                 double* tau, double* v, double* w, double* partial, int64_t partial_cap,
                 const DevStatus* st) {
  const int sms = num_sms();
  const int pgrid = 2 * sms;
  // the tail of the partial buffer: per-CTA parts of p^T v and the last-CTA counter
  double* dots = partial + partial_cap - (pgrid + 2);
  unsigned* counter = reinterpret_cast<unsigned*>(dots + pgrid);
  partial_cap -= pgrid + 2 + n;
  double* colpart = partial + partial_cap;   // n entries before the tail
  cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  for (int64_t j = 0; j + 2 < n; ++j) {
    const int64_t len = n - j - 1;
    house_col_kernel<<<1, HT, 0, ::ec::counted(s)>>>(n, A, lda, j, v, d, e, tau, st);
    const int64_t rb = (len + 255) / 256;
    int64_t nchunk = (4 * sms + rb - 1) / rb;
    if (nchunk < 1) nchunk = 1;
    if (nchunk > (len + 63) / 64) nchunk = (len + 63) / 64;
    while (nchunk * n > partial_cap) --nchunk;
    const int64_t kc = (len + nchunk - 1) / nchunk;
    nchunk = (len + kc - 1) / kc;
    symv_partial_kernel<<<dim3((unsigned)rb, (unsigned)nchunk), 256, 0, ::ec::counted(s)>>>(n, A, lda, j, v,
                                                                             partial, kc);
    symv_col_kernel<<<(unsigned)((len + 7) / 8), 256, 0, ::ec::counted(s)>>>(n, A, lda, j, v,
                                                                              colpart);
    const int64_t pg = (len + 255) / 256 < pgrid ? (len + 255) / 256 : pgrid;
    p_kernel<<<(unsigned)pg, 256, 0, ::ec::counted(s)>>>(n, j, v, tau, partial, (int)nchunk,
                                                         colpart, w, dots, counter);
    // a few CTAs per SM, each sweeping many columns: the per-column work of the lower
    // triangle is too small to amortise one CTA launch per column
    const int64_t gy = len < 4 * (int64_t)sms ? len : 4 * (int64_t)sms;
    dim3 g2((unsigned)((len + 255) / 256 < 4 ? (len + 255) / 256 : 4), (unsigned)gy);
    syr2_kernel<<<g2, 256, 0, ::ec::counted(s)>>>(n, A, lda, j, v, w, tau);
  }
  tail_kernel<<<1, 1, 0, ::ec::counted(s)>>>(n, A, lda, d, e);
}

void ormtr_lower(cudaStream_t s, int64_t n, const double* A, int64_t lda, const double* tau,
                 double* Y, int64_t ldy, int64_t ncol, double* V, double* G, double* T,
                 double* W, double* W2, double* ws, int64_t ws_cap, const DevStatus* st) {
  const int64_t nref = n - 2;
  if (nref <= 0) return;
  const int64_t nblk = (nref + NB - 1) / NB;
  for (int64_t bi = nblk - 1; bi >= 0; --bi) {
    const int64_t b = bi * NB;
    const int kb = (int)((nref - b) < NB ? (nref - b) : NB);
    form_v_kernel<<<dim3(32, kb), 256, 0, ::ec::counted(s)>>>(n, A, lda, b, kb, V);
    const int64_t r0 = b + 1, len = n - r0;
    // G = V^T V: one 64 x 64 output over a long K; one CTA would carry it alone
    int spg = dgemm_tn_splits(kb, kb, len);
    while (spg > 1 && (int64_t)spg * kb * kb > ws_cap) --spg;
    dgemm_tn_split(s, kb, kb, len, V + r0, n, V + r0, n, G, kb, ws, spg, st);
    form_t_kernel<<<1, 64, 0, ::ec::counted(s)>>>(kb, G, kb, tau, b, T, kb);
    // W = V^T Y: a 64-row output with a long K, split over K to fill the GPU
    int sp = dgemm_tn_splits(kb, ncol, len);
    while (sp > 1 && (int64_t)sp * kb * ncol > ws_cap) --sp;
    dgemm_tn_split(s, kb, ncol, len, V + r0, n, Y + r0, ldy, W, kb, ws, sp, st);
    dgemm(s, N_, N_, kb, ncol, kb, 1.0, T, kb, W, kb, 0.0, W2, kb, 0, st);
    dgemm(s, N_, N_, len, ncol, kb, -1.0, V + r0, n, W2, kb, 1.0, Y + r0, ldy, 0, st);
  }
}

void ormtr_lower_grouped(cudaStream_t s, int64_t n, const double* A, int64_t lda,
                         const double* tau, double* Y, int64_t ldy, int64_t ncol, int64_t gsize,
                         double* V, double* G, double* T, double* X, double* W, double* W2,
                         OzWork* oz, const DevStatus* st) {
  const int64_t nref = n - 2;
  if (nref <= 0) return;
  const int64_t ngroups = (nref + gsize - 1) / gsize;
  for (int64_t gi = ngroups - 1; gi >= 0; --gi) {
    const int64_t b0 = gi * gsize;
    const int64_t gb = (nref - b0) < gsize ? (nref - b0) : gsize;
    const int64_t r0 = b0 + 1, len = n - r0;
    // V: the group's reflectors, 64 columns at a time
    for (int64_t c = 0; c < gb; c += NB) {
      const int kb = (int)((gb - c) < NB ? (gb - c) : NB);
      form_v_kernel<<<dim3(32, kb), 256, 0, ::ec::counted(s)>>>(n, A, lda, b0 + c, kb,
                                                                V + c * n);
    }
    // G = V^T V, then T block by block: diagonal blocks from G's diagonal blocks, and
    // T[0:c, c:c+kb] = -T[0:c, 0:c] G[0:c, c:c+kb] T[c:c+kb, c:c+kb]
    gemm_auto(s, oz, T_, N_, gb, gb, len, 1.0, V + r0, n, V + r0, n, 0.0, G, gb, 0, st);
    cudaMemsetAsync(T, 0, sizeof(double) * (size_t)gb * gb, s);
    for (int64_t c = 0; c < gb; c += NB) {
      const int kb = (int)((gb - c) < NB ? (gb - c) : NB);
      form_t_kernel<<<1, 64, 0, ::ec::counted(s)>>>(kb, G + c + c * gb, gb, tau, b0 + c,
                                                    T + c + c * gb, gb);
      if (c > 0) {
        gemm_auto(s, oz, N_, N_, c, kb, c, 1.0, T, gb, G + c * gb, gb, 0.0, X, gb, 0, st);
        gemm_auto(s, oz, N_, N_, c, kb, kb, -1.0, X, gb, T + c + c * gb, gb, 0.0, T + c * gb, gb,
                  0, st);
      }
    }
    // Y[r0:, :] <- (I - V T V^T) Y[r0:, :]
    gemm_auto(s, oz, T_, N_, gb, ncol, len, 1.0, V + r0, n, Y + r0, ldy, 0.0, W, gb, 0, st);
    gemm_auto(s, oz, N_, N_, gb, ncol, gb, 1.0, T, gb, W, gb, 0.0, W2, gb, 0, st);
    gemm_auto(s, oz, N_, N_, len, ncol, gb, -1.0, V + r0, n, W2, gb, 1.0, Y + r0, ldy, 0, st);
  }
}

namespace {

// Blocked tridiagonalisation, column j = b + i of a panel starting at column b:
// A[j:, j] -= V[j:, 0:i] W[j, 0:i]^T + W[j:, 0:i] V[j, 0:i]^T  (the panel's earlier
// reflectors, not yet applied to the trailing matrix).
__global__ void __launch_bounds__(256) latrd_col_kernel(int64_t n, double* A, int64_t lda,
                                                        int64_t j, const double* V,
                                                        const double* W, int64_t ldv, int i) {
  __shared__ double wj[64], vj[64];
  if (threadIdx.x < i) {
    wj[threadIdx.x] = W[j + threadIdx.x * ldv];
    vj[threadIdx.x] = V[j + threadIdx.x * ldv];
  }
  __syncthreads();
  const int64_t r = j + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  double a0 = A[r + j * lda], a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int c = 0;
  for (; c + 1 < i; c += 2) {
    a0 = fma(-V[r + c * ldv], wj[c], a0);
    a1 = fma(-W[r + c * ldv], vj[c], a1);
    a2 = fma(-V[r + (c + 1) * ldv], wj[c + 1], a2);
    a3 = fma(-W[r + (c + 1) * ldv], vj[c + 1], a3);
  }
  if (c < i) {
    a0 = fma(-V[r + c * ldv], wj[c], a0);
    a1 = fma(-W[r + c * ldv], vj[c], a1);
  }
  A[r + j * lda] = (a0 + a1) + (a2 + a3);
}

// y1[c] = W[j+1:, c] . v[j+1:],  y2[c] = V[j+1:, c] . v[j+1:]  for c < i (one CTA per c).
__global__ void __launch_bounds__(256) latrd_dots_kernel(int64_t n, int64_t j, const double* V,
                                                         const double* W, int64_t ldv,
                                                         const double* v, double* y) {
  __shared__ double sh[2][8];
  const int c = blockIdx.x;
  double a1 = 0.0, a2 = 0.0;
  for (int64_t r = j + 1 + threadIdx.x; r < n; r += blockDim.x) {
    const double vr = v[r];
    a1 = fma(W[r + c * ldv], vr, a1);
    a2 = fma(V[r + c * ldv], vr, a2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][w] = a1;
    sh[1][w] = a2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s1 = 0.0, s2 = 0.0;
    for (int q = 0; q < 8; ++q) {
      s1 += sh[0][q];
      s2 += sh[1][q];
    }
    y[c] = s1;
    y[64 + c] = s2;
  }
}

// Symmetric product over the trailing lower triangle A22 = A[s0:, s0:] (s0 = j + 1,
// m = n - s0), each element read once and used for both of its contributions, in
// 64 x 64 tiles (I, J), I >= J, by column strips: CTA (k, J) takes the tiles (I, J) with
// I in [J + k SEG, J + (k+1) SEG) of the 64-column strip J, loads each tile with
// asynchronous 8-byte copies while the previous one is used, writes the row part of
// every tile (prow[J][rows of I]) and keeps the column part of its whole segment in
// registers, written once (pcol[k][columns of J]).  For a row r of block B:
//   (A22 v)[r] = sum_{J <= B} prow[J][r] + sum_{k < nseg(B)} pcol[k][r],
// nseg(B) = ceil((nbk - B) / SEG); p_latrd_kernel adds them in a fixed order (eight
// interleaved partial sums, then those in order).
constexpr int SEG = 16;

__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(valid ? 8 : 0)
               : "memory");
}

// PAIR: the same products in compensated FP32 (each FP64 entry split into hi + lo
// FP32 parts by integer operations once per tile, float-float sums, partials stored as
// FP32 pairs in the same 8-byte slots): on GB300 this moves the product from the FP64
// pipe (2 FMAs per SM per clock) to the FP32 and integer pipes, leaving the tile reads
// from HBM as its bound; about 2^-46 relative per product.
template <bool PAIR>
__global__ void __launch_bounds__(256) symv_strip_kernel(int64_t n, const double* A, int64_t lda,
                                                         int64_t j, const double* v, double* prow,
                                                         double* pcol, int64_t mp) {
  extern __shared__ double sbuf[];                  // two tiles, As[b][c][r] stride 65
  __shared__ double vr[2][64], vc[64];
  __shared__ double red[4][64];
  __shared__ float2 vrp[2][64], vcp[64];
  const int64_t s0 = j + 1, m = n - s0;
  const int64_t nbk = (m + 63) / 64;
  const int64_t J = blockIdx.y, k = blockIdx.x;
  const int64_t I0 = J + k * SEG;
  if (I0 >= nbk) return;
  const int64_t I1 = (I0 + SEG < nbk) ? I0 + SEG : nbk;
  const int tid = threadIdx.x, lo = tid & 63, qt = tid >> 6;
  const int64_t c0 = J * 64;
  if (tid < 64) {
    vc[tid] = (c0 + tid < m) ? v[s0 + c0 + tid] : 0.0;
    if (PAIR) vcp[tid] = ff::split(vc[tid]);
  }
  auto load = [&](int64_t I, int b) {
    double* As = sbuf + b * 64 * 65;
    const int64_t r0 = I * 64;
    if (PAIR && I != J) {
      // the FP32 pair of A[r, c] (r > c) is kept at position (c, r): read it transposed,
      // consecutive threads along c
      for (int q = tid; q < 64 * 64; q += 256) {
        const int cc = q & 63, rr = q >> 6;
        const int64_t r = r0 + rr, c = c0 + cc;
        const bool ok = r < m && c < m;
        cp_async8(&As[cc * 65 + rr], ok ? (const void*)(A + (s0 + c) + (s0 + r) * lda)
                                        : (const void*)A, ok);
      }
    } else {
      for (int q = tid; q < 64 * 64; q += 256) {
        const int rr = q & 63, cc = q >> 6;
        const int64_t r = r0 + rr, c = c0 + cc;
        const bool ok = r < m && c < m && (I != J || rr >= cc);
        cp_async8(&As[cc * 65 + rr], ok ? (const void*)(A + (s0 + r) + (s0 + c) * lda)
                                        : (const void*)A, ok);
      }
    }
    if (tid < 64) {
      vr[b][tid] = (r0 + tid < m) ? v[s0 + r0 + tid] : 0.0;
      if (PAIR) vrp[b][tid] = ff::split(vr[b][tid]);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  double colacc = 0.0;     // column part of (lo, qt) over the segment
  float ch0 = 0.f, cl0 = 0.f, ch1 = 0.f, cl1 = 0.f;   // the same, PAIR
  float2* red2 = reinterpret_cast<float2*>(&red[0][0]);
  load(I0, 0);
  for (int64_t I = I0; I < I1; ++I) {
    const int b = (int)((I - I0) & 1);
    if (I + 1 < I1) {
      load(I + 1, b ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const double* As = sbuf + b * 64 * 65;
    const int64_t r0 = I * 64;
    if constexpr (PAIR) {
      if (I == J) {
        // the diagonal tile comes from the FP64 lower triangle: split it in place (each
        // 8-byte slot becomes its FP32 pair); the others arrived as pairs
        double* Aw = sbuf + b * 64 * 65;
        float2* A2w = reinterpret_cast<float2*>(Aw);
        for (int q = tid; q < 64 * 64; q += 256) {
          const int idx = (q >> 6) * 65 + (q & 63);
          A2w[idx] = ff::split_fast(Aw[idx]);
        }
        __syncthreads();
      }
      const float2* A2 = reinterpret_cast<const float2*>(As);
      float rh0 = 0.f, rl0 = 0.f, rh1 = 0.f, rl1 = 0.f;
#pragma unroll
      for (int cc = 0; cc < 16; cc += 2) {
        const float2 x0 = A2[(qt * 16 + cc) * 65 + lo], y0 = vcp[qt * 16 + cc];
        const float2 x1 = A2[(qt * 16 + cc + 1) * 65 + lo], y1 = vcp[qt * 16 + cc + 1];
        ff::madd(rh0, rl0, x0.x, x0.y, y0.x, y0.y);
        ff::madd(rh1, rl1, x1.x, x1.y, y1.x, y1.y);
      }
#pragma unroll
      for (int rr = 0; rr < 16; rr += 2) {
        const int ra = qt * 16 + rr, rb = ra + 1;
        const float2 xa = (I != J || ra > lo) ? A2[lo * 65 + ra] : make_float2(0.f, 0.f);
        const float2 xb = (I != J || rb > lo) ? A2[lo * 65 + rb] : make_float2(0.f, 0.f);
        ff::madd(ch0, cl0, xa.x, xa.y, vrp[b][ra].x, vrp[b][ra].y);
        ff::madd(ch1, cl1, xb.x, xb.y, vrp[b][rb].x, vrp[b][rb].y);
      }
      ff::add(rh0, rl0, rh1, rl1);
      red2[qt * 64 + lo] = make_float2(rh0, rl0);
      __syncthreads();
      if (tid < 64 && r0 + tid < m) {
        float h = red2[tid].x, l = red2[tid].y;
        ff::add(h, l, red2[64 + tid].x, red2[64 + tid].y);
        ff::add(h, l, red2[128 + tid].x, red2[128 + tid].y);
        ff::add(h, l, red2[192 + tid].x, red2[192 + tid].y);
        reinterpret_cast<float2*>(prow)[J * mp + r0 + tid] = make_float2(h, l);
      }
      __syncthreads();                             // red and the buffer are reused
    } else {
      // row part: thread (row lo, quarter qt of the columns)
      double a0 = 0.0, a1 = 0.0;
#pragma unroll
      for (int cc = 0; cc < 16; cc += 2) {
        a0 = fma(As[(qt * 16 + cc) * 65 + lo], vc[qt * 16 + cc], a0);
        a1 = fma(As[(qt * 16 + cc + 1) * 65 + lo], vc[qt * 16 + cc + 1], a1);
      }
      // column part: thread (column lo, quarter qt of the rows); the diagonal tile's
      // diagonal is counted once (in the row part)
      double b0 = 0.0, b1 = 0.0;
#pragma unroll
      for (int rr = 0; rr < 16; rr += 2) {
        const int ra = qt * 16 + rr, rb = ra + 1;
        const double xa = (I != J || ra > lo) ? As[lo * 65 + ra] : 0.0;
        const double xb = (I != J || rb > lo) ? As[lo * 65 + rb] : 0.0;
        b0 = fma(xa, vr[b][ra], b0);
        b1 = fma(xb, vr[b][rb], b1);
      }
      colacc += b0 + b1;
      red[qt][lo] = a0 + a1;
      __syncthreads();
      if (tid < 64 && r0 + tid < m)
        prow[J * mp + r0 + tid] = (red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]);
      __syncthreads();                             // red and the buffer are reused
    }
  }
  if constexpr (PAIR) {
    ff::add(ch0, cl0, ch1, cl1);
    red2[qt * 64 + lo] = make_float2(ch0, cl0);
    __syncthreads();
    if (tid < 64 && c0 + tid < m) {
      float h = red2[tid].x, l = red2[tid].y;
      ff::add(h, l, red2[64 + tid].x, red2[64 + tid].y);
      ff::add(h, l, red2[128 + tid].x, red2[128 + tid].y);
      ff::add(h, l, red2[192 + tid].x, red2[192 + tid].y);
      reinterpret_cast<float2*>(pcol)[k * mp + c0 + tid] = make_float2(h, l);
    }
  } else {
    red[qt][lo] = colacc;
    __syncthreads();
    if (tid < 64 && c0 + tid < m)
      pcol[k * mp + c0 + tid] = (red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]);
  }
}

// FP32 pair copies of the trailing lower triangle A[t0:, t0:] for the compensated
// symmetric product: the pair of A[r, c] (r > c) is written to the free upper position
// (c, r), through a shared-memory transpose so that both sides are coalesced.  One CTA
// per 64 x 64 tile (I, J), I >= J, of the trailing block.
__global__ void __launch_bounds__(256) pair_upper_kernel(int64_t n, double* A, int64_t lda,
                                                         int64_t t0) {
  __shared__ float2 T2[64][65];
  const int64_t I = blockIdx.x, J = blockIdx.y;
  if (I < J) return;
  const int64_t m = n - t0, r0 = t0 + I * 64, c0 = t0 + J * 64;
  const int tid = threadIdx.x;
  for (int q = tid; q < 64 * 64; q += 256) {
    const int rr = q & 63, cc = q >> 6;                 // read down the columns
    const int64_t r = r0 + rr, c = c0 + cc;
    if (r - t0 < m && c - t0 < m && r > c) T2[cc][rr] = ff::split_fast(A[r + c * lda]);
  }
  __syncthreads();
  float2* A2 = reinterpret_cast<float2*>(A);
  for (int q = tid; q < 64 * 64; q += 256) {
    const int cc = q & 63, rr = q >> 6;                 // write along the rows
    const int64_t r = r0 + rr, c = c0 + cc;
    if (r - t0 < m && c - t0 < m && r > c) A2[c + r * lda] = T2[cc][rr];
  }
}

// As p_kernel, with the panel's corrections: for rows r > j,
//   p_r = tau ( (A22 v)_r - V[r, 0:i] y1 - W[r, 0:i] y2 ),
// then w = p - (tau/2)(p^T v) v by the last CTA.
template <bool PAIR>
__global__ void __launch_bounds__(256) p_latrd_kernel(int64_t n, int64_t j, const double* v,
                                                      const double* tau, const double* prow,
                                                      const double* pcol, int64_t mp,
                                                      const double* V, const double* W,
                                                      int64_t ldv, int i, const double* y,
                                                      double* p, double* dots, unsigned* counter) {
  __shared__ double sh[9];
  __shared__ double ys[128];
  __shared__ bool last;
  if (threadIdx.x < 2 * i) ys[threadIdx.x < i ? threadIdx.x : 64 + threadIdx.x - i] =
      y[threadIdx.x < i ? threadIdx.x : 64 + threadIdx.x - i];
  __syncthreads();
  const double t = tau[j];
  const int64_t len = n - j - 1;
  double dot = 0.0;
  const int64_t nbk = (len + 63) / 64;
  // 32 rows per pass: the 8 warps split each row's partials (warp q takes partials
  // q, q + 8, ...), their sums are added in warp order, and warp 0 finishes the rows
  __shared__ double part[8][32];
  const int rlane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  for (int64_t g0 = (int64_t)blockIdx.x * 32; g0 < len; g0 += (int64_t)gridDim.x * 32) {
    const int64_t rl = g0 + rlane;
    double acc = 0.0;
    if (rl < len) {
      const int64_t blk = rl >> 6;
      const int64_t nseg = (nbk - blk + SEG - 1) / SEG;
      if constexpr (PAIR) {
        const float2* pr2 = reinterpret_cast<const float2*>(prow);
        const float2* pc2 = reinterpret_cast<const float2*>(pcol);
        float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
        int64_t b = wq;
        for (; b + 8 <= blk; b += 16) {
          const float2 x0 = pr2[b * mp + rl], x1 = pr2[(b + 8) * mp + rl];
          ff::add(h0, l0, x0.x, x0.y);
          ff::add(h1, l1, x1.x, x1.y);
        }
        if (b <= blk) ff::add(h0, l0, pr2[b * mp + rl].x, pr2[b * mp + rl].y);
        b = wq;
        for (; b + 8 < nseg; b += 16) {
          const float2 x0 = pc2[b * mp + rl], x1 = pc2[(b + 8) * mp + rl];
          ff::add(h0, l0, x0.x, x0.y);
          ff::add(h1, l1, x1.x, x1.y);
        }
        if (b < nseg) ff::add(h0, l0, pc2[b * mp + rl].x, pc2[b * mp + rl].y);
        acc = ((double)h0 + (double)l0) + ((double)h1 + (double)l1);
      } else {
        double q0 = 0.0, q1 = 0.0;
        int64_t b = wq;
        for (; b + 8 <= blk; b += 16) {
          q0 += prow[b * mp + rl];
          q1 += prow[(b + 8) * mp + rl];
        }
        if (b <= blk) q0 += prow[b * mp + rl];
        b = wq;
        for (; b + 8 < nseg; b += 16) {
          q0 += pcol[b * mp + rl];
          q1 += pcol[(b + 8) * mp + rl];
        }
        if (b < nseg) q0 += pcol[b * mp + rl];
        acc = q0 + q1;
      }
    }
    part[wq][rlane] = acc;
    __syncthreads();
    if (wq == 0 && rl < len) {
      double q = part[0][rlane];
#pragma unroll
      for (int w2 = 1; w2 < 8; ++w2) q += part[w2][rlane];
      const int64_t r = j + 1 + rl;
      double e0 = 0.0, e1 = 0.0;
      for (int c = 0; c < i; ++c) {
        e0 = fma(V[r + c * ldv], ys[c], e0);
        e1 = fma(W[r + c * ldv], ys[64 + c], e1);
      }
      q = (q - e0) - e1;
      q *= t;
      p[r] = q;
      dot = fma(q, v[r], dot);
    }
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  if (lane == 0) sh[w] = dot;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) b += sh[q];
    dots[blockIdx.x] = b;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < 32) {
    double b = 0.0;
    for (unsigned q = threadIdx.x; q < gridDim.x; q += 32) b += __ldcg(dots + q);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    if (threadIdx.x == 0) {
      sh[8] = 0.5 * t * b;
      *counter = 0u;
    }
  }
  __syncthreads();
  const double f = sh[8];
  for (int64_t r = j + 1 + threadIdx.x; r < n; r += blockDim.x) p[r] = fma(-f, v[r], p[r]);
  // rows above j + 1 of the panel's w column are zero (v is zero there)
  for (int64_t r = threadIdx.x; r <= j; r += blockDim.x) p[r] = 0.0;
}

}  // namespace

int64_t sytrd_blocked_scratch(int64_t n) {
  const int64_t nbk = (n + 63) / 64;
  return 2 * nbk * n + 2 * (int64_t)num_sms() + 8;
}

constexpr int STRIP_SMEM = 2 * 64 * 65 * (int)sizeof(double);

void sytrd_lower_blocked(cudaStream_t s, int64_t n, double* A, int64_t lda, double* d, double* e,
                         double* tau, double* V, double* W, double* y, double* partial,
                         OzWork* oz, const DevStatus* st, int pair_symv) {
  static std::atomic<unsigned long long> attr_set{0};
  if (first_on_device(attr_set)) {
    cudaFuncSetAttribute(symv_strip_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         STRIP_SMEM);
    cudaFuncSetAttribute(symv_strip_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         STRIP_SMEM);
  }
  const int sms = num_sms();
  const int pgrid = 2 * sms;
  const int64_t mp = n;                            // stride of the per-block partials
  const int64_t nbk_max = (n + 63) / 64;
  double* prow = partial;
  double* pcol = partial + nbk_max * mp;
  double* dots = pcol + nbk_max * mp;
  unsigned* counter = reinterpret_cast<unsigned*>(dots + pgrid);
  cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  const int64_t jend = n - 2;                      // columns 0 .. n-3 carry a reflector
  auto refresh_pairs = [&](int64_t t0) {
    const int64_t tb = (n - t0 + 63) / 64;
    if (pair_symv && tb > 0)
      pair_upper_kernel<<<dim3((unsigned)tb, (unsigned)tb), 256, 0, ::ec::counted(s)>>>(n, A, lda,
                                                                                        t0);
  };
  refresh_pairs(0);
  for (int64_t b = 0; b < jend; b += NB) {
    const int nb = (int)((jend - b) < NB ? (jend - b) : NB);
    for (int i = 0; i < nb; ++i) {
      const int64_t j = b + i;
      const int64_t len = n - j - 1;
      double* vj = V + (int64_t)i * n;
      double* wj = W + (int64_t)i * n;
      if (i > 0)
        latrd_col_kernel<<<(unsigned)((n - j + 255) / 256), 256, 0, ::ec::counted(s)>>>(
            n, A, lda, j, V, W, n, i);
      house_col_kernel<<<1, HT, 0, ::ec::counted(s)>>>(n, A, lda, j, vj, d, e, tau, st);
      const int64_t nbk = (len + 63) / 64;
      const dim3 sg((unsigned)((nbk + SEG - 1) / SEG), (unsigned)nbk);
      if (pair_symv)
        symv_strip_kernel<true><<<sg, 256, STRIP_SMEM, ::ec::counted(s)>>>(n, A, lda, j, vj, prow,
                                                                          pcol, mp);
      else
        symv_strip_kernel<false><<<sg, 256, STRIP_SMEM, ::ec::counted(s)>>>(n, A, lda, j, vj,
                                                                           prow, pcol, mp);
      if (i > 0)
        latrd_dots_kernel<<<(unsigned)i, 256, 0, ::ec::counted(s)>>>(n, j, V, W, n, vj, y);
      const int64_t pg = (len + 31) / 32 < pgrid ? (len + 31) / 32 : pgrid;
      if (pair_symv)
        p_latrd_kernel<true><<<(unsigned)pg, 256, 0, ::ec::counted(s)>>>(
            n, j, vj, tau, prow, pcol, mp, V, W, n, i, y, wj, dots, counter);
      else
        p_latrd_kernel<false><<<(unsigned)pg, 256, 0, ::ec::counted(s)>>>(
            n, j, vj, tau, prow, pcol, mp, V, W, n, i, y, wj, dots, counter);
    }
    // the panel's rank-2nb update of the trailing lower triangle
    const int64_t t0 = b + nb, m = n - t0;
    if (m > 0) {
      gemm_auto(s, oz, N_, T_, m, m, nb, -1.0, V + t0, n, W + t0, n, 1.0, A + t0 + t0 * lda, lda,
                1, st);
      gemm_auto(s, oz, N_, T_, m, m, nb, -1.0, W + t0, n, V + t0, n, 1.0, A + t0 + t0 * lda, lda,
                1, st);
      refresh_pairs(t0);
    }
  }
  tail_kernel<<<1, 1, 0, ::ec::counted(s)>>>(n, A, lda, d, e);
}

}  // namespace ec
