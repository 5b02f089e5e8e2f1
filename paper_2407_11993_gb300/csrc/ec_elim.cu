// Constraint elimination (Sec. 3.1, Eq. current_electrodes and
// discrete_version_2) and the O(N)-per-step helpers shared by both forms.
//
// K, the orthonormal basis of ker E, comes from a Householder QR of E^T:
// E^T = Q [Rr; 0] with Q = H_0 ... H_{m-1} = I - V T V^T (compact WY form).
// K is the last N - m columns of Q, and the particular field is
// E^T (E E^T)^{-1} = Q [Rr^{-T}; 0].  Every projected matrix of
// Eq. discrete_version_2 is a block of Q^T A Q, which is obtained from A by a
// rank-2m symmetric update, so nothing N x N0 is ever formed explicitly.

#include <cmath>

#include "ec_internal.h"
#include "ec_kernels.h"

namespace ec {

namespace {

constexpr int HT = 1024;  // threads of the single-CTA Householder kernel

__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// Householder QR of E^T (n x m, given as E row-major m x n); writes V (n x m,
// unit lower trapezoidal), T (m x m upper), Rr^{-T} (m x m lower), all
// column-major.  Rank deficiency -> EC_ERR_RANK.
__global__ void __launch_bounds__(HT) house_kernel(int64_t n, int m, const double* E, double* V,
                                                   double* Tm, double* RrinvT, DevStatus* st) {
  __shared__ double sh[40];
  __shared__ double Rr[MAXM][MAXM];
  __shared__ double tauv[MAXM];
  __shared__ double G[MAXM][MAXM];
  const int tid = threadIdx.x;
  for (int64_t i = tid; i < n * m; i += HT) {
    int64_t r = i % n, c = i / n;
    V[r + c * n] = E[c * n + r];
  }
  __syncthreads();
  double fro = 0.0;
  for (int64_t i = tid; i < n * m; i += HT) fro += V[i] * V[i];
  fro = sqrt(block_sum(fro, sh));
  for (int j = 0; j < m; ++j) {
    double* vj = V + (int64_t)j * n;
    double sig = 0.0;
    for (int64_t i = j + 1 + tid; i < n; i += HT) sig += vj[i] * vj[i];
    sig = block_sum(sig, sh);
    const double alpha = vj[j];
    const double nx = sqrt(alpha * alpha + sig);
    if (!(nx > 1e-12 * fro)) {
      if (tid == 0 && atomicCAS(&st->code, 0, (int)EC_ERR_RANK) == 0) st->info = j;
      return;
    }
    const double beta = alpha >= 0.0 ? -nx : nx;
    const double tau = (beta - alpha) / beta;
    const double scale = 1.0 / (alpha - beta);
    for (int c = j + 1; c < m; ++c) {
      double* vc = V + (int64_t)c * n;
      double d = 0.0;
      for (int64_t i = j + 1 + tid; i < n; i += HT) d += vj[i] * vc[i];
      d = vc[j] + scale * block_sum(d, sh);
      const double f = tau * d;
      for (int64_t i = j + 1 + tid; i < n; i += HT) vc[i] -= f * scale * vj[i];
      __syncthreads();
      if (tid == 0) vc[j] -= f;
      __syncthreads();
    }
    if (tid == 0) {
      Rr[j][j] = beta;
      for (int c = j + 1; c < m; ++c) Rr[j][c] = V[j + (int64_t)c * n];
      tauv[j] = tau;
    }
    __syncthreads();
    for (int64_t i = tid; i < n; i += HT) {
      if (i < j) vj[i] = 0.0;
      else if (i == j) vj[i] = 1.0;
      else vj[i] *= scale;
    }
    __syncthreads();
  }
  // Gram matrix V^T V for the T factor
  for (int a = 0; a < m; ++a)
    for (int b = 0; b <= a; ++b) {
      double d = 0.0;
      for (int64_t i = tid; i < n; i += HT) d += V[i + (int64_t)a * n] * V[i + (int64_t)b * n];
      d = block_sum(d, sh);
      if (tid == 0) { G[a][b] = d; G[b][a] = d; }
    }
  __syncthreads();
  if (tid == 0) {
    double T[MAXM][MAXM];
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) T[a][b] = 0.0;
    for (int j = 0; j < m; ++j) {
      T[j][j] = tauv[j];
      // T[0:j, j] = -tau_j T[0:j, 0:j] (V[:, 0:j]^T v_j)
      for (int a = 0; a < j; ++a) {
        double s = 0.0;
        for (int b = a; b < j; ++b) s += T[a][b] * G[b][j];
        T[a][j] = -tauv[j] * s;
      }
    }
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) Tm[a + b * m] = T[a][b];
    // Rr^{-T}: lower triangular inverse of Rr^T by forward substitution
    double X[MAXM][MAXM];
    for (int c = 0; c < m; ++c) {
      for (int r = 0; r < m; ++r) {
        if (r < c) { X[r][c] = 0.0; continue; }
        double s = (r == c) ? 1.0 : 0.0;
        for (int k = c; k < r; ++k) s -= Rr[k][r] * X[k][c];   // (Rr^T)[r][k] = Rr[k][r]
        X[r][c] = s / Rr[r][r];
      }
    }
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) RrinvT[a + b * m] = X[a][b];
  }
}

// Copy the upper triangle (column-major) onto the lower one.
__global__ void sym_from_upper_kernel(int64_t n, double* A, int64_t lda) {
  const int64_t c = blockIdx.y * (int64_t)blockDim.y + threadIdx.y;
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < n && c < n && r > c) A[r + c * lda] = A[c + r * lda];
}

// CSR of a symmetric dense matrix (column i read as row i).
__global__ void csr_count_kernel(int64_t n, const double* A, int64_t lda, int* cnt) {
  const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* col = A + row * lda;
  int c = 0;
  for (int64_t j = lane; j < n; j += 32) c += (col[j] != 0.0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[row] = c;
}

__global__ void __launch_bounds__(1024) exclusive_scan_kernel(int64_t n, const int* cnt,
                                                              long long* ptr) {
  __shared__ long long part[1024];
  const int tid = threadIdx.x;
  const int64_t chunk = (n + 1023) / 1024;
  const int64_t b = tid * chunk, e = (b + chunk < n) ? b + chunk : n;
  long long s = 0;
  for (int64_t i = b; i < e; ++i) s += cnt[i];
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    long long acc = 0;
    for (int i = 0; i < 1024; ++i) { long long t = part[i]; part[i] = acc; acc += t; }
    ptr[n] = acc;
  }
  __syncthreads();
  s = part[tid];
  for (int64_t i = b; i < e; ++i) { ptr[i] = s; s += cnt[i]; }
}

__global__ void csr_fill_kernel(int64_t n, const double* A, int64_t lda, const long long* ptr,
                                int* colidx, double* val) {
  const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* col = A + row * lda;
  long long pos = ptr[row];
  for (int64_t j0 = 0; j0 < n; j0 += 32) {
    const int64_t j = j0 + lane;
    const double v = (j < n) ? col[j] : 0.0;
    const unsigned mask = __ballot_sync(0xffffffffu, v != 0.0);
    if (v != 0.0) {
      const long long at = pos + __popc(mask & ((1u << lane) - 1u));
      colidx[at] = (int)j;
      val[at] = v;
    }
    pos += __popc(mask);
  }
}

}  // namespace

void house_qr(cudaStream_t s, int64_t n, int m, const double* E, double* V, double* T,
              double* RrinvT, DevStatus* st) {
  house_kernel<<<1, HT, 0, ::ec::counted(s)>>>(n, m, E, V, T, RrinvT, st);
}

void sym_from_upper(cudaStream_t s, int64_t n, double* A, int64_t lda) {
  dim3 blk(32, 8);
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 7) / 8));
  sym_from_upper_kernel<<<grid, blk, 0, ::ec::counted(s)>>>(n, A, lda);
}

void two_sided_update(cudaStream_t s, int64_t n, int m, double* A, const double* V,
                      const double* T, double* Y, double* X, double* Sm, double* Zm,
                      const DevStatus* st) {
  // Q^T A Q = A - W V^T - V W^T,  X = A V T,  W = X - 1/2 V (T^T V^T X)
  dgemm(s, N_, N_, n, m, n, 1.0, A, n, V, n, 0.0, Y, n, 0, st);       // Y = A V
  dgemm(s, N_, N_, n, m, m, 1.0, Y, n, T, m, 0.0, X, n, 0, st);       // X = Y T
  dgemm(s, T_, N_, m, m, n, 1.0, V, n, X, n, 0.0, Sm, m, 0, st);      // S = V^T X
  dgemm(s, T_, N_, m, m, m, 1.0, T, m, Sm, m, 0.0, Zm, m, 0, st);     // Z = T^T S
  dgemm(s, N_, N_, n, m, m, -0.5, V, n, Zm, m, 1.0, X, n, 0, st);     // W = X - V Z / 2
  dgemm(s, N_, T_, n, n, m, -1.0, X, n, V, n, 1.0, A, n, 0, st);      // A -= W V^T
  dgemm(s, N_, T_, n, n, m, -1.0, V, n, X, n, 1.0, A, n, 0, st);      // A -= V W^T
}

void one_sided_qt(cudaStream_t s, int64_t n, int m, double* B, int64_t ncol, const double* V,
                  const double* T, double* S1, double* S2, const DevStatus* st) {
  if (ncol <= 0) return;
  // Q^T B = B - V T^T (V^T B)
  dgemm(s, T_, N_, m, ncol, n, 1.0, V, n, B, n, 0.0, S1, m, 0, st);
  dgemm(s, T_, N_, m, ncol, m, 1.0, T, m, S1, m, 0.0, S2, m, 0, st);
  dgemm(s, N_, N_, n, ncol, m, -1.0, V, n, S2, m, 1.0, B, n, 0, st);
}

void one_sided_q(cudaStream_t s, int64_t n, int m, double* B, int64_t ncol, const double* V,
                 const double* T, double* S1, double* S2, const DevStatus* st) {
  if (ncol <= 0) return;
  // Q B = B - V T (V^T B)
  dgemm(s, T_, N_, m, ncol, n, 1.0, V, n, B, n, 0.0, S1, m, 0, st);
  dgemm(s, N_, N_, m, ncol, m, 1.0, T, m, S1, m, 0.0, S2, m, 0, st);
  dgemm(s, N_, N_, n, ncol, m, -1.0, V, n, S2, m, 1.0, B, n, 0, st);
}

ec_status build_csr(cudaStream_t s, int64_t n, const double* A, Csr& out,
                    cudaError_t (*alloc)(void**, size_t)) {
  int* cnt = nullptr;
  if (alloc((void**)&cnt, sizeof(int) * n) != cudaSuccess) return EC_ERR_OOM;
  if (alloc((void**)&out.ptr, sizeof(long long) * (n + 1)) != cudaSuccess) {
    cudaFree(cnt);
    return EC_ERR_OOM;
  }
  const int wpb = 8;
  const unsigned grid = (unsigned)((n + wpb - 1) / wpb);
  csr_count_kernel<<<grid, 32 * wpb, 0, ::ec::counted(s)>>>(n, A, n, cnt);
  exclusive_scan_kernel<<<1, 1024, 0, ::ec::counted(s)>>>(n, cnt, out.ptr);
  long long nnz = 0;
  cudaMemcpyAsync(&nnz, out.ptr + n, sizeof(long long), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  cudaFree(cnt);
  out.nnz = nnz;
  if (alloc((void**)&out.col, sizeof(int) * (nnz > 0 ? nnz : 1)) != cudaSuccess) return EC_ERR_OOM;
  if (alloc((void**)&out.val, sizeof(double) * (nnz > 0 ? nnz : 1)) != cudaSuccess) return EC_ERR_OOM;
  csr_fill_kernel<<<grid, 32 * wpb, 0, ::ec::counted(s)>>>(n, A, n, out.ptr, out.col, out.val);
  return EC_OK;
}

}  // namespace ec
