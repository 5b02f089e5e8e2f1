// Per-step kernels of the plain (Cholesky) form, Sec. 3.3.1, Eq. time_integration:
//
//   (L_i + dt theta R_i) dI = -dt R_i I_i^k - dt R_D i_D^k - (L_D + dt theta R_D) d i_D - M_0 d i_0
//
// The right-hand side needs R_i I_i = [Q^T R Q x]_{m:} with x = [0; I_i].  R
// is applied from its CSR (sparse for the FEM / synthetic R) and Q^T R Q - R
// is the rank-2m correction  -WR T (V^T x) - V T^T (WR^T x) + V T^T (V^T WR) T (V^T x),
// WR = R V.  The 2m dot products V^T x, WR^T x are produced, together with the
// probe outputs C K I_i, by the update kernel of the previous step, with a
// deterministic two-level reduction (per-CTA partials summed in CTA order by
// the last CTA to finish).

#include "ec_kernels.h"

namespace ec {

namespace {

__device__ __forceinline__ double src_at(const double* a, int64_t T, int row, int64_t k) {
  return a[(int64_t)row * (T + 1) + k];
}

// alpha = -T p, beta = T^T (-q + (V^T WR) T p) for the rank-2m part of Q^T R Q.
__device__ void lowrank_coefs(const StepArgs& a, double* alpha, double* beta) {
  const int m = a.m, P = a.P;
  {
    {
      const double* p = a.dots + P;
      const double* q = a.dots + P + m;
      double Tp[MAXM], u[MAXM];
      for (int i = 0; i < m; ++i) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += a.Tm[i + j * m] * p[j];
        Tp[i] = s;
        alpha[i] = -s;
      }
      for (int i = 0; i < m; ++i) {
        double s = -q[i];
        for (int j = 0; j < m; ++j) s += a.VtWR[i + j * m] * Tp[j];
        u[i] = s;
      }
      for (int i = 0; i < m; ++i) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += a.Tm[j + i * m] * u[j];   // T^T u
        beta[i] = s;
      }
    }
  }
}

// (R_i I_i)_i for internal row i: CSR of R on x = [0; I_i] plus the rank-2m correction.
__device__ __forceinline__ double ri_row(const StepArgs& a, int64_t i, const double* alpha,
                                         const double* beta) {
  const int m = a.m;
  const int64_t row = i + m;
  double s = 0.0;
  for (long long e = a.R.ptr[row]; e < a.R.ptr[row + 1]; ++e) {
    const int c = a.R.col[e];
    if (c >= m) s = fma(a.R.val[e], a.Ii[c - m], s);
  }
  for (int j = 0; j < m; ++j)
    s = fma(a.WR[row + (int64_t)j * a.n], alpha[j], fma(a.V[row + (int64_t)j * a.n], beta[j], s));
  return s;
}

// Body of the right-hand-side kernel for CTA bx of gx (batched launches pass the
// instance's arguments and the CTA index within the instance).
__device__ __forceinline__ void plain_rhs_body(const StepArgs& a, unsigned bx, unsigned gx) {
  __shared__ double alpha[MAXM], beta[MAXM], coef[2 * MAXM + 64];
  const int64_t k = *a.kstep;
  if (bx == 0 && threadIdx.x == 0) {
    a.tickets[0] = 0u;
    a.tickets[1] = 0u;
    *a.epoch = *a.epoch + 1;
  }
  const int m = a.m;
  const int ncoef = 2 * m + a.S;
  if (threadIdx.x == 0) {
    if (m > 0) lowrank_coefs(a, alpha, beta);
    for (int j = 0; j < m; ++j) {
      const double d0 = src_at(a.iD, a.T, j, k), d1 = src_at(a.iD, a.T, j, k + 1);
      coef[j] = -a.dt * d0;
      coef[m + j] = -(d1 - d0);
    }
    for (int l = 0; l < a.S; ++l)
      coef[2 * m + l] = -(src_at(a.src, a.T, l, k + 1) - src_at(a.src, a.T, l, k));
  }
  __syncthreads();
  for (int64_t i = bx * (int64_t)blockDim.x + threadIdx.x; i < a.n0;
       i += (int64_t)gx * blockDim.x) {
    double b = -a.dt * ri_row(a, i, alpha, beta);
    for (int c = 0; c < ncoef; ++c) b = fma(coef[c], a.Gsrc[i + (int64_t)c * a.n0], b);
    a.work[i] = b;
  }
}

__global__ void __launch_bounds__(256) plain_rhs_kernel(StepArgs a) {
  plain_rhs_body(a, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) plain_rhs_batch_kernel(const StepArgs* A) {
  plain_rhs_body(A[blockIdx.y], blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) ri_apply_kernel(StepArgs a, double* out) {
  __shared__ double alpha[MAXM], beta[MAXM];
  if (threadIdx.x == 0 && a.m > 0) lowrank_coefs(a, alpha, beta);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n0;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = ri_row(a, i, alpha, beta);
}

// I_i += dI (mode 0), then the D dot products of the new state: per-CTA partials
// (each warp reduces its rows with shuffles, one barrier for all D), summed by the
// last CTA with one warp per dot product (lanes stride over the CTA partials).
__device__ __forceinline__ void plain_update_body(const StepArgs& a, int mode, unsigned bx,
                                                  unsigned nb) {
  __shared__ double sh[8][MAXD];
  __shared__ bool last;
  const int64_t n0 = a.n0;
  const int64_t chunk = (n0 + nb - 1) / nb;
  const int64_t b0 = bx * chunk;
  const int64_t b1 = (b0 + chunk < n0) ? b0 + chunk : n0;
  if (mode == 0) {
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) a.Ii[i] += a.work[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // Dot products in batches of 8 columns: the 8 loads of a row are issued before
  // any of them is used, so the latency is paid once per batch, not per column.
  for (int d0 = 0; d0 < a.D; d0 += 8) {
    double s[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) s[j] = 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
      const double x = a.Ii[i];
      double c[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) c[j] = (d0 + j < a.D) ? a.Dmat[i + (int64_t)(d0 + j) * n0] : 0.0;
#pragma unroll
      for (int j = 0; j < 8; ++j) s[j] = fma(c[j], x, s[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s[j] += __shfl_xor_sync(0xffffffffu, s[j], o);
      if (lane == 0 && d0 + j < a.D) sh[w][d0 + j] = s[j];
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < a.D; d += blockDim.x) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q][d];
    a.partial[(int64_t)bx * a.D + d] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(a.counter, 1u);
    last = (prev == nb - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int64_t k = *a.kstep;   // this update produces state k + 1 (mode 0)
  for (int d = w; d < a.D; d += (int)(blockDim.x >> 5)) {
    double t = 0.0;
    for (unsigned b = lane; b < nb; b += 32) t += __ldcg(a.partial + (int64_t)b * a.D + d);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) {
      a.dots[d] = t;
      if (mode == 0 && d < a.P && a.probes != nullptr) {
        double y = t;
        for (int j = 0; j < a.m; ++j) y = fma(a.CPE[d + (int64_t)j * a.P], src_at(a.iD, a.T, j, k + 1), y);
        a.probes[k * a.P + d] = y;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *a.counter = 0u;
    if (mode == 0) *a.kstep = k + 1;
  }
}

__global__ void __launch_bounds__(256) plain_update_kernel(StepArgs a, int mode) {
  plain_update_body(a, mode, blockIdx.x, gridDim.x);
}

// blockIdx.y = instance; CTAs past the instance's own update grid leave at once,
// so every instance reduces exactly as its own launch does.
__global__ void __launch_bounds__(256) plain_update_batch_kernel(const StepArgs* A) {
  const StepArgs& a = A[blockIdx.y];
  if (blockIdx.x >= (unsigned)a.ugrid) return;
  plain_update_body(a, 0, blockIdx.x, (unsigned)a.ugrid);
}

__device__ __forceinline__ void plain_snapshot_body(const StepArgs& a, unsigned bx, unsigned gx) {
  const int64_t k = *a.kstep;
  if (a.snap_stride <= 0 || a.snaps == nullptr || k == 0 || k % a.snap_stride != 0) return;
  const int64_t j = k / a.snap_stride - 1;
  __shared__ double Tp[MAXM], iDk[MAXM];
  const int m = a.m;
  if (threadIdx.x == 0) {
    for (int i = 0; i < m; ++i) {
      double s = 0.0;
      for (int c = 0; c < m; ++c) s += a.Tm[i + c * m] * a.dots[a.P + c];
      Tp[i] = s;
      iDk[i] = src_at(a.iD, a.T, i, k);
    }
  }
  __syncthreads();
  for (int64_t i = bx * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gx * blockDim.x) {
    double v = (i >= m) ? a.Ii[i - m] : 0.0;
    for (int c = 0; c < m; ++c)
      v = fma(-a.V[i + (int64_t)c * a.n], Tp[c], fma(a.PE[i + (int64_t)c * a.n], iDk[c], v));
    a.snaps[j * a.n + i] = v;
  }
}

__global__ void plain_snapshot_kernel(StepArgs a) { plain_snapshot_body(a, blockIdx.x, gridDim.x); }

__global__ void plain_snapshot_batch_kernel(const StepArgs* A) {
  plain_snapshot_body(A[blockIdx.y], blockIdx.x, gridDim.x);
}

// FP64 residual of the step equation for an approximate solution x (no electrodes,
// so R_i = R):  r = b - Z x,  Z x = (t1 + t2) + theta dt R x,  t1 + t2 = L x.
__global__ void __launch_bounds__(256) plain_residual_kernel(StepArgs a, const double* b,
                                                             const double* x, const double* t1,
                                                             const double* t2, double* r) {
  const double tdt = a.theta * a.dt;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n0;
       i += (int64_t)gridDim.x * blockDim.x) {
    double rx = 0.0;
    for (long long e = a.R.ptr[i]; e < a.R.ptr[i + 1]; ++e) rx = fma(a.R.val[e], x[a.R.col[e]], rx);
    r[i] = fma(-tdt, rx, b[i] - (t1[i] + t2[i]));
  }
}

int rows_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

namespace {

// Independent trajectories, no electrodes: out[:, r] = -dt R I_r - M_0[:, r] (s_r^{k+1} - s_r^k).
__global__ void __launch_bounds__(256) plain_rhs_multi_kernel(StepArgs a, int64_t k, const double* I,
                                                              double* out) {
  const int r = blockIdx.y;
  const double ds = a.src[(int64_t)r * (a.T + 1) + k + 1] - a.src[(int64_t)r * (a.T + 1) + k];
  const double* Ir = I + (int64_t)r * a.n0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n0;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (long long e = a.R.ptr[i]; e < a.R.ptr[i + 1]; ++e) v = fma(a.R.val[e], Ir[a.R.col[e]], v);
    out[i + (int64_t)r * a.n0] = fma(-a.dt, v, -a.Gsrc[i + (int64_t)r * a.n0] * ds);
  }
}

// probes[r] = C[:, r] . I[:, r]  (paired read-out), C column-major n0 x S (leading dim ldc)
__global__ void __launch_bounds__(256) paired_probe_kernel(int64_t n0, const double* C, int64_t ldc,
                                                           const double* I, double* out) {
  const int r = blockIdx.x;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n0; i += blockDim.x)
    acc = fma(C[i + (int64_t)r * ldc], I[i + (int64_t)r * n0], acc);
  __shared__ double sh[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    out[r] = t;
  }
}

}  // namespace

void plain_rhs_multi(cudaStream_t s, const StepArgs& a, int64_t k, const double* I, double* out) {
  plain_rhs_multi_kernel<<<dim3(rows_grid(a.n0), a.S), 256, 0, ::ec::counted(s)>>>(a, k, I, out);
}

void paired_probes(cudaStream_t s, int64_t n0, int S, const double* C, int64_t ldc,
                   const double* I, double* out) {
  paired_probe_kernel<<<S, 256, 0, ::ec::counted(s)>>>(n0, C, ldc, I, out);
}

void plain_rhs(cudaStream_t s, const StepArgs& a) {
  plain_rhs_kernel<<<rows_grid(a.n0), 256, 0, ::ec::counted(s)>>>(a);
}

void plain_update(cudaStream_t s, const StepArgs& a, int grid, int mode) {
  plain_update_kernel<<<grid, 256, 0, ::ec::counted(s)>>>(a, mode);
}

void ri_apply(cudaStream_t s, const StepArgs& a, double* out) {
  ri_apply_kernel<<<rows_grid(a.n0), 256, 0, ::ec::counted(s)>>>(a, out);
}

void plain_snapshot(cudaStream_t s, const StepArgs& a) {
  plain_snapshot_kernel<<<rows_grid(a.n), 256, 0, ::ec::counted(s)>>>(a);
}

void plain_residual(cudaStream_t s, const StepArgs& a, const double* b, const double* x,
                    const double* t1, const double* t2, double* r) {
  plain_residual_kernel<<<rows_grid(a.n0), 256, 0, ::ec::counted(s)>>>(a, b, x, t1, t2, r);
}

void plain_rhs_batch(cudaStream_t s, const StepArgs* dA, int count, int64_t max_n0) {
  plain_rhs_batch_kernel<<<dim3(rows_grid(max_n0), count), 256, 0, ::ec::counted(s)>>>(dA);
}

void plain_update_batch(cudaStream_t s, const StepArgs* dA, int count, int max_grid) {
  plain_update_batch_kernel<<<dim3(max_grid, count), 256, 0, ::ec::counted(s)>>>(dA);
}

void plain_snapshot_batch(cudaStream_t s, const StepArgs* dA, int count, int64_t max_n) {
  plain_snapshot_batch_kernel<<<dim3(rows_grid(max_n), count), 256, 0, ::ec::counted(s)>>>(dA);
}

}  // namespace ec
