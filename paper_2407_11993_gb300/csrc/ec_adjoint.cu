// Discrete adjoint of the plain theta-method for the probe misfit
//   J = sum_{k=1..T} || C I^k - v^k ||^2
// (no electrodes; the forward recurrence is Eq. time_integration of Sec. 3.3.1,
// Z I^{k+1} = A I^k - M (s^{k+1} - s^k), Z = L + theta dt R, A = Z - dt R).
//
// Backward recurrence, k = T .. 1, lambda^{T+1} = 0:
//   Z lambda^k = A lambda^{k+1} + 2 C^T (C I^k - v^k).
// Because Z lambda^{k+1} is the previous right-hand side, A lambda^{k+1} =
// rhs^{k+1} - dt R lambda^{k+1}: each backward step costs one sparse R product
// and one solve with the same inverse factor the forward steps use -- no dense
// product with A.  Gradients accumulated on the way:
//   dJ/dR_ee = - dt sum_k lambda^k_e (theta I^k_e + (1 - theta) I^{k-1}_e)
//   mu^k     = M^T lambda^k,   dJ/ds^j = mu^{j+1} - mu^j.

#include "ec_kernels.h"

namespace ec {

namespace {

__global__ void __launch_bounds__(256) adj_rhs_kernel(int64_t n, int P, double dt, Csr R,
                                                      const double* lam_next, double* rhs,
                                                      const double* probes_row,
                                                      const double* v_row, const double* Ct) {
  __shared__ double r[MAXD];
  if (threadIdx.x < P) r[threadIdx.x] = 2.0 * (probes_row[threadIdx.x] - v_row[threadIdx.x]);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double rl = 0.0;
    for (long long e = R.ptr[i]; e < R.ptr[i + 1]; ++e) rl = fma(R.val[e], lam_next[R.col[e]], rl);
    double v = fma(-dt, rl, rhs[i]);
    for (int p = 0; p < P; ++p) v = fma(Ct[i + (int64_t)p * n], r[p], v);
    rhs[i] = v;
  }
}

// gR += -dt lambda (theta I^k + (1-theta) I^{k-1});  mu[s] = M[:, s]^T lambda
// (per-CTA partials summed in CTA order by the last CTA).
__global__ void __launch_bounds__(256) adj_accum_kernel(int64_t n, int S, double dt, double theta,
                                                        const double* lam, const double* Ik,
                                                        const double* Ikm1, double* gR,
                                                        const double* M, double* partial,
                                                        unsigned* counter, double* mu_out,
                                                        int64_t mu_stride) {
  __shared__ double sh[33];
  __shared__ bool last;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = blockIdx.x * chunk;
  const int64_t b1 = (b0 + chunk < n) ? b0 + chunk : n;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x)
    gR[i] = fma(-dt * lam[i], fma(theta, Ik[i], (1.0 - theta) * Ikm1[i]), gR[i]);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int s = 0; s < S; ++s) {
    double acc = 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) acc = fma(M[i + (int64_t)s * n], lam[i], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sh[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
      partial[(int64_t)blockIdx.x * S + s] = t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    double t = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(partial + (int64_t)b * S + s);
    mu_out[s * mu_stride] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
}

__global__ void __launch_bounds__(256) misfit_kernel(int64_t count, const double* probes,
                                                     const double* v, double* J) {
  __shared__ double sh[33];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {
    const double d = probes[i] - v[i];
    acc = fma(d, d, acc);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) sh[w] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    *J = t;
  }
}

__global__ void dsrc_kernel(int S, int64_t T, const double* mu, double* out) {
  // mu is S x (T+2) with mu[., 0] = mu[., T+1] = 0
  const int64_t tot = (int64_t)S * (T + 1);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx / (T + 1), j = idx % (T + 1);
    out[idx] = mu[s * (T + 2) + j + 1] - mu[s * (T + 2) + j];
  }
}

}  // namespace

void adj_rhs(cudaStream_t s, int64_t n, int P, double dt, const Csr& R, const double* lam_next,
             double* rhs, const double* probes_row, const double* v_row, const double* Ct) {
  int64_t g = (n + 255) / 256;
  if (g > num_sms() * 8) g = num_sms() * 8;
  adj_rhs_kernel<<<(unsigned)g, 256, 0, ::ec::counted(s)>>>(n, P, dt, R, lam_next, rhs,
                                                             probes_row, v_row, Ct);
}

void adj_accum(cudaStream_t s, int64_t n, int S, double dt, double theta, const double* lam,
               const double* Ik, const double* Ikm1, double* gR, const double* M, double* partial,
               unsigned* counter, double* mu_out, int64_t mu_stride, int grid) {
  adj_accum_kernel<<<grid, 256, 0, ::ec::counted(s)>>>(n, S, dt, theta, lam, Ik, Ikm1, gR, M,
                                                        partial, counter, mu_out, mu_stride);
}

void misfit(cudaStream_t s, int64_t count, const double* probes, const double* v, double* J) {
  misfit_kernel<<<1, 256, 0, ::ec::counted(s)>>>(count, probes, v, J);
}

void dsrc(cudaStream_t s, int S, int64_t T, const double* mu, double* out) {
  const int64_t tot = (int64_t)S * (T + 1);
  int64_t g = (tot + 255) / 256;
  if (g > 1024) g = 1024;
  if (g < 1) g = 1;
  dsrc_kernel<<<(unsigned)g, 256, 0, ::ec::counted(s)>>>(S, T, mu, out);
}

}  // namespace ec
