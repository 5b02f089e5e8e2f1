// Phasor extraction from sampled responses (the time-domain post-processing of
// Sec. 4.6: Fourier transform of each probe signal, read at the excitation tones).
//
//   X(f_j)_p = (2/T) sum_{k=0}^{T-1} y_k,p exp(-i 2 pi f_j (t0 + k dt))
//
// One CTA per (tone, probe); 256 threads stride over the samples, the angle is
// reduced to [0, 2) half-turns in FP64 before sincospi, and the partial sums are
// combined in a fixed order (deterministic).

#include "ec_internal.h"

namespace ec {

namespace {

__global__ void __launch_bounds__(256) phasor_kernel(int64_t T, int64_t P, const double* y,
                                                     double t0, double dt, const double* freqs,
                                                     double* out) {
  const int64_t j = blockIdx.x, p = blockIdx.y;
  const double f = freqs[j];
  double re = 0.0, im = 0.0;
  for (int64_t k = threadIdx.x; k < T; k += blockDim.x) {
    double turns = 2.0 * f * (t0 + (double)k * dt);     // angle / pi
    turns -= 2.0 * floor(0.5 * turns);
    double sn, cs;
    sincospi(turns, &sn, &cs);
    const double v = y[k * P + p];
    re = fma(v, cs, re);
    im = fma(-v, sn, im);
  }
  __shared__ double sr[8], si[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    sr[w] = re;
    si[w] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      a += sr[q];
      b += si[q];
    }
    const double sc = 2.0 / (double)T;
    out[(j * P + p) * 2] = sc * a;
    out[(j * P + p) * 2 + 1] = sc * b;
  }
}

}  // namespace

}  // namespace ec

extern "C" ec_status ec_phasors(int64_t T, int64_t P, const double* y, double t0, double dt,
                                int64_t nf, const double* freqs, double* out, int mem) {
  using namespace ec;
  if (T < 1 || P < 1 || nf < 1 || !y || !freqs || !out || !(dt > 0.0)) return EC_ERR_ARG;
  if (mem != EC_MEM_HOST && mem != EC_MEM_DEVICE) return EC_ERR_ARG;
  if (nf > 65535 || P > 65535) return EC_ERR_UNSUPPORTED;
  double *dy = nullptr, *df = nullptr, *dout = nullptr;
  const double* py = y;
  const double* pf = freqs;
  double* po = out;
  if (mem == EC_MEM_HOST) {
    if (cudaMalloc((void**)&dy, sizeof(double) * T * P) != cudaSuccess ||
        cudaMalloc((void**)&df, sizeof(double) * nf) != cudaSuccess ||
        cudaMalloc((void**)&dout, sizeof(double) * nf * P * 2) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(dy);
      cudaFree(df);
      return EC_ERR_OOM;
    }
    cudaMemcpy(dy, y, sizeof(double) * T * P, cudaMemcpyHostToDevice);
    cudaMemcpy(df, freqs, sizeof(double) * nf, cudaMemcpyHostToDevice);
    py = dy;
    pf = df;
    po = dout;
  }
  cudaStream_t s = 0;
  phasor_kernel<<<dim3((unsigned)nf, (unsigned)P), 256, 0, ::ec::counted(s)>>>(T, P, py, t0, dt,
                                                                               pf, po);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && mem == EC_MEM_HOST)
    e = cudaMemcpy(out, dout, sizeof(double) * nf * P * 2, cudaMemcpyDeviceToHost);
  cudaFree(dy);
  cudaFree(df);
  cudaFree(dout);
  return e == cudaSuccess ? EC_OK : EC_ERR_CUDA;
}
