// FP32 and FP32-pair products of the mode matrix U with a few columns: the snapshot
// reconstruction I = U x (Sec. 3.2, Eq. modal_decomposition_discrete) and the
// projections U^T [R_D | L_D | M_0], U^T (C K)^T of the modal form's reduced-precision
// variants (EC_PREC_FP32, EC_PREC_FP32X2).
//
// With a handful of right-hand columns the product streams U once from HBM and does a
// few multiply-adds per entry: in FP64 it is bound by GB300's FP64 pipe (about 0.25
// flop per byte already exceeds its balance point), while FP32 operands halve the bytes
// and move the arithmetic to the FP32 pipe, ~60x faster.  The pair variant keeps U as
// hi + lo FP32 parts (about 48 significant bits in 8 bytes) and runs compensated FP32
// arithmetic: every hi*hi product exact by FMA, the two cross terms added, float-float
// sums, FP64 sums every 64 products.
//
// Both operands carry power-of-two scales (one for U, one per right-hand column) so
// that FP32's exponent range never clips: the rounded entries lie in [-1, 1].

#include <cmath>
#include <cstring>

#include "ec_skinny32.h"

namespace ec {

namespace {

constexpr int NC_MAX = 8;      // right-hand columns per launch
constexpr int WARPS = 8;       // warps per CTA
constexpr int FLUSH = 64;      // pair products per float-float partial sum

__device__ __forceinline__ bool failed(const DevStatus* st) {
  return st != nullptr && *(volatile const int*)&st->code != 0;
}

// acc_h + acc_l += (uh + ul)(yh + yl), dropping ul*yl (2^-48 relative).  Rounded
// intrinsics keep the compiler from contracting the TwoSum's operations into FMAs.
__device__ __forceinline__ void ff_madd(float& sh, float& sl, float uh, float ul, float yh,
                                        float yl) {
  const float p = __fmul_rn(uh, yh);
  float e = fmaf(uh, yh, -p);                  // exact rounding error of p
  e = fmaf(uh, yl, e);
  e = fmaf(ul, yh, e);
  const float t = __fadd_rn(sh, p);
  const float bp = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  sl = __fadd_rn(sl, __fadd_rn(err, e));
  sh = t;
}

// Largest |entry| of a matrix as the bits of a non-negative double (ordered like the
// values), combined with atomicMax.
__global__ void absmax_kernel(int64_t M, int64_t N, const double* A, int64_t lda,
                              unsigned long long* out) {
  unsigned long long best = 0;
  const int64_t tot = M * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i % M, c = i / M;
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(A[r + c * lda]));
    best = b > best ? b : best;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
    best = v > best ? v : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

// Column c's power of two: e with max |Y[:, c]| * 2^-e in [0.5, 1) (0 for a zero or
// non-finite column).  One CTA per column.
__global__ void __launch_bounds__(256) col_exp_kernel(int64_t K, const double* Y, int64_t ldy,
                                                      int* yexp) {
  const int64_t c = blockIdx.x;
  double m = 0.0;
  for (int64_t k = threadIdx.x; k < K; k += blockDim.x) m = fmax(m, fabs(Y[k + c * ldy]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double sh[8];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, sh[w]);
    int e = 0;
    if (t > 0.0 && isfinite(t)) frexp(t, &e);
    yexp[c] = e;
  }
}

// dst (rows 0 .. ldd-1 of N columns) = src * 2^-e(c), rounded to FP32 or to an FP32
// hi/lo pair; rows >= M are zero.  e(c) = eexp[c] when given, else e0.
template <int PAIR>
__global__ void round_kernel(int64_t M, int64_t N, const double* src, int64_t lds, float* dst,
                             int64_t ldd, const int* eexp, int e0) {
  const int64_t tot = ldd * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i % ldd, c = i / ldd;
    const int e = eexp ? eexp[c] : e0;
    const double v = r < M ? ldexp(src[r + c * lds], -e) : 0.0;
    const float hi = __double2float_rn(v);
    if (PAIR) {
      dst[2 * i] = hi;
      dst[2 * i + 1] = __double2float_rn(v - (double)hi);
    } else {
      dst[i] = hi;
    }
  }
}

// Partial products of C = U Y over one K segment (blockIdx.y): a warp covers 32 x RPT
// consecutive rows with one 16-byte load per lane and K index, the 8 warps of a CTA
// interleave over K and are added in warp order.  part[(y * nc + c) * ldp + r].
template <int PAIR, int NC>
__global__ void __launch_bounds__(256, 2) nn_kernel(int64_t M, int64_t K, int64_t kseg, int nc,
                                                 const float* __restrict__ U, int64_t ldu,
                                                 const float* __restrict__ Y, int64_t ldy,
                                                 double* __restrict__ part, int64_t ldp,
                                                 const DevStatus* st) {
  if (failed(st)) return;
  constexpr int RPT = PAIR ? 2 : 4;
  constexpr int W = PAIR ? 2 : 1;                 // floats per element
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t r0 = ((int64_t)blockIdx.x * 32 + lane) * RPT;
  const bool live = r0 < M;
  const int64_t kb = (int64_t)blockIdx.y * kseg;
  const int64_t ke = (kb + kseg) < K ? (kb + kseg) : K;
  double out[RPT][NC];
  if (!PAIR) {
    float acc[RPT][NC];
#pragma unroll
    for (int j = 0; j < RPT; ++j)
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[j][c] = 0.f;
#pragma unroll 4
    for (int64_t k = kb + w; k < ke; k += WARPS) {
      const float4 u4 = live ? __ldcs(reinterpret_cast<const float4*>(U + r0 + k * ldu))
                             : make_float4(0.f, 0.f, 0.f, 0.f);
      const float u[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float y = c < nc ? __ldg(Y + k + c * ldy) : 0.f;
#pragma unroll
        for (int j = 0; j < RPT; ++j) acc[j][c] = fmaf(u[j], y, acc[j][c]);
      }
    }
#pragma unroll
    for (int j = 0; j < RPT; ++j)
#pragma unroll
      for (int c = 0; c < NC; ++c) out[j][c] = (double)acc[j][c];
  } else {
    float sh[RPT][NC], sl[RPT][NC];
#pragma unroll
    for (int j = 0; j < RPT; ++j)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        out[j][c] = 0.0;
        sh[j][c] = 0.f;
        sl[j][c] = 0.f;
      }
    for (int64_t k0 = kb + w; k0 < ke; k0 += (int64_t)WARPS * FLUSH) {
      const int64_t k1 = (k0 + (int64_t)WARPS * FLUSH) < ke ? (k0 + (int64_t)WARPS * FLUSH) : ke;
#pragma unroll 4
      for (int64_t k = k0; k < k1; k += WARPS) {
        const float4 u4 = live ? __ldcs(reinterpret_cast<const float4*>(U + W * (r0 + k * ldu)))
                               : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float2 y = c < nc ? __ldg(reinterpret_cast<const float2*>(Y + W * (k + c * ldy)))
                                  : make_float2(0.f, 0.f);
          ff_madd(sh[0][c], sl[0][c], u4.x, u4.y, y.x, y.y);
          ff_madd(sh[1][c], sl[1][c], u4.z, u4.w, y.x, y.y);
        }
      }
#pragma unroll
      for (int j = 0; j < RPT; ++j)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          out[j][c] += (double)sh[j][c] + (double)sl[j][c];
          sh[j][c] = 0.f;
          sl[j][c] = 0.f;
        }
    }
  }
  __shared__ double red[WARPS][32 * RPT];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (c >= nc) break;
#pragma unroll
    for (int j = 0; j < RPT; ++j) red[w][lane * RPT + j] = out[j][c];
    __syncthreads();
    if (threadIdx.x < 32 * RPT) {
      const int64_t r = (int64_t)blockIdx.x * 32 * RPT + threadIdx.x;
      if (r < M) {
        double v = red[0][threadIdx.x];
#pragma unroll
        for (int q = 1; q < WARPS; ++q) v += red[q][threadIdx.x];
        part[((int64_t)blockIdx.y * nc + c) * ldp + r] = v;
      }
    }
    __syncthreads();
  }
}

// C[r, c] = 2^(eU + yexp[c]) * sum over segments of part (segment order).
__global__ void nn_reduce_kernel(int64_t M, int nc, int ksplit, const double* part, int64_t ldp,
                                 const int* yexp, int eU, double* C, int64_t ldc,
                                 const DevStatus* st) {
  if (failed(st)) return;
  const int64_t tot = M * nc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i % M, c = i / M;
    double v = 0.0;
    for (int y = 0; y < ksplit; ++y) v += part[((int64_t)y * nc + c) * ldp + r];
    C[r + c * ldc] = ldexp(v, eU + yexp[c]);
  }
}

// C[r, c] = 2^(eU + yexp[c]) sum_k U[k, r] Y[k, c]: one warp per output row r (column r
// of U, contiguous), lanes over K with 16-byte loads, a shuffle tree per column.
template <int PAIR, int NC>
__global__ void __launch_bounds__(256) tn_kernel(int64_t M, int64_t Kp, int nc,
                                                 const float* __restrict__ U,
                                                 int64_t ldu, const float* __restrict__ Y,
                                                 int64_t ldy, const int* yexp, int eU,
                                                 double* C, int64_t ldc, const DevStatus* st) {
  if (failed(st)) return;
  constexpr int RPT = PAIR ? 2 : 4;
  constexpr int W = PAIR ? 2 : 1;
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
  if (r >= M) return;
  const float* col = U + W * r * ldu;
  double out[NC];
  if (!PAIR) {
    float acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.f;
    for (int64_t k = (int64_t)lane * RPT; k < Kp; k += 32 * RPT) {
      const float4 u = __ldcs(reinterpret_cast<const float4*>(col + k));
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float4 y = c < nc ? __ldg(reinterpret_cast<const float4*>(Y + k + c * ldy))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        acc[c] = fmaf(u.x, y.x, fmaf(u.y, y.y, fmaf(u.z, y.z, fmaf(u.w, y.w, acc[c]))));
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) out[c] = (double)acc[c];
  } else {
    float sh[NC], sl[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      out[c] = 0.0;
      sh[c] = 0.f;
      sl[c] = 0.f;
    }
    const int64_t span = (int64_t)32 * RPT * (FLUSH / RPT);
    for (int64_t k0 = (int64_t)lane * RPT; k0 < Kp; k0 += span) {
      const int64_t k1 = (k0 + span) < Kp ? (k0 + span) : Kp;
      for (int64_t k = k0; k < k1; k += 32 * RPT) {
        const float4 u = __ldcs(reinterpret_cast<const float4*>(col + W * k));
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float4 y = c < nc ? __ldg(reinterpret_cast<const float4*>(Y + W * (k + c * ldy)))
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
          ff_madd(sh[c], sl[c], u.x, u.y, y.x, y.y);
          ff_madd(sh[c], sl[c], u.z, u.w, y.z, y.w);
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        out[c] += (double)sh[c] + (double)sl[c];
        sh[c] = 0.f;
        sl[c] = 0.f;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double v = out[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && c < nc) C[r + c * ldc] = ldexp(v, eU + yexp[c]);
  }
}

int64_t round4(int64_t x) { return (x + 3) / 4 * 4; }

unsigned grid_for(int64_t work, int64_t per_block) {
  int64_t g = (work + per_block - 1) / per_block;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (g > cap) g = cap;
  return (unsigned)(g < 1 ? 1 : g);
}

template <typename T>
ec_status grow(T** p, size_t& cap, size_t count) {
  if (*p && count <= cap) return EC_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  cap = 0;
  if (device_alloc((void**)p, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return EC_ERR_OOM;
  }
  cap = count;
  return EC_OK;
}

template <int PAIR, int NC>
void launch_nn(cudaStream_t s, int nc, int64_t M, int64_t K, int64_t kseg, int ksplit,
               const float* U, int64_t ldu, const float* Y, int64_t ldy, double* part,
               int64_t ldp, const DevStatus* st) {
  constexpr int RPT = PAIR ? 2 : 4;
  const unsigned gx = (unsigned)((M + 32 * RPT - 1) / (32 * RPT));
  nn_kernel<PAIR, NC><<<dim3(gx, (unsigned)ksplit), 256, 0, ::ec::counted(s)>>>(
      M, K, kseg, nc, U, ldu, Y, ldy, part, ldp, st);
}

template <int PAIR, int NC>
void launch_tn(cudaStream_t s, int nc, int64_t M, int64_t Kp, const float* U, int64_t ldu,
               const float* Y, int64_t ldy, const int* yexp, int eU, double* C, int64_t ldc,
               const DevStatus* st) {
  tn_kernel<PAIR, NC><<<(unsigned)((M + WARPS - 1) / WARPS), 256, 0, ::ec::counted(s)>>>(
      M, Kp, nc, U, ldu, Y, ldy, yexp, eU, C, ldc, st);
}

// column counts 1, 2, 3-4 and 5-8 share kernels of width 1, 2, 4 and 8
template <int PAIR>
void nn_any(cudaStream_t s, int nc, int64_t M, int64_t K, int64_t kseg, int ksplit,
            const float* U, int64_t ldu, const float* Y, int64_t ldy, double* part, int64_t ldp,
            const DevStatus* st) {
  if (nc == 1) launch_nn<PAIR, 1>(s, nc, M, K, kseg, ksplit, U, ldu, Y, ldy, part, ldp, st);
  else if (nc == 2) launch_nn<PAIR, 2>(s, nc, M, K, kseg, ksplit, U, ldu, Y, ldy, part, ldp, st);
  else if (nc <= 4) launch_nn<PAIR, 4>(s, nc, M, K, kseg, ksplit, U, ldu, Y, ldy, part, ldp, st);
  else launch_nn<PAIR, 8>(s, nc, M, K, kseg, ksplit, U, ldu, Y, ldy, part, ldp, st);
}

template <int PAIR>
void tn_any(cudaStream_t s, int nc, int64_t M, int64_t Kp, const float* U, int64_t ldu,
            const float* Y, int64_t ldy, const int* yexp, int eU, double* C, int64_t ldc,
            const DevStatus* st) {
  if (nc == 1) launch_tn<PAIR, 1>(s, nc, M, Kp, U, ldu, Y, ldy, yexp, eU, C, ldc, st);
  else if (nc == 2) launch_tn<PAIR, 2>(s, nc, M, Kp, U, ldu, Y, ldy, yexp, eU, C, ldc, st);
  else if (nc <= 4) launch_tn<PAIR, 4>(s, nc, M, Kp, U, ldu, Y, ldy, yexp, eU, C, ldc, st);
  else launch_tn<PAIR, 8>(s, nc, M, Kp, U, ldu, Y, ldy, yexp, eU, C, ldc, st);
}

}  // namespace

ec_status u32_build(cudaStream_t s, int64_t n0, const double* U, int64_t ldu, int pair, U32* u) {
  u32_free(u);
  const int64_t ld = round4(n0);
  const size_t bytes = sizeof(float) * (pair ? 2 : 1) * (size_t)ld * (size_t)n0;
  unsigned long long* mx = nullptr;
  if (device_alloc(&u->data, bytes) != cudaSuccess ||
      device_alloc((void**)&mx, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    if (u->data) cudaFree(u->data);
    u->data = nullptr;
    return EC_ERR_OOM;
  }
  cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s);
  absmax_kernel<<<grid_for(n0 * n0, 256), 256, 0, ::ec::counted(s)>>>(n0, n0, U, ldu, mx);
  unsigned long long hb = 0;
  cudaMemcpyAsync(&hb, mx, sizeof(hb), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  cudaFree(mx);
  double amax = 0.0;
  static_assert(sizeof(double) == sizeof(unsigned long long), "");
  memcpy(&amax, &hb, sizeof(amax));
  int e = 0;
  if (amax > 0.0 && std::isfinite(amax)) std::frexp(amax, &e);
  u->ld = ld;
  u->pair = pair;
  u->eU = e;
  if (pair)
    round_kernel<1><<<grid_for(ld * n0, 256), 256, 0, ::ec::counted(s)>>>(
        n0, n0, U, ldu, (float*)u->data, ld, nullptr, e);
  else
    round_kernel<0><<<grid_for(ld * n0, 256), 256, 0, ::ec::counted(s)>>>(
        n0, n0, U, ldu, (float*)u->data, ld, nullptr, e);
  return EC_OK;
}

void u32_free(U32* u) {
  if (u->data) cudaFree(u->data);
  *u = U32{};
}

void skinny32_free(Skinny32Work* w) {
  if (w->y) cudaFree(w->y);
  if (w->yexp) cudaFree(w->yexp);
  if (w->part) cudaFree(w->part);
  *w = Skinny32Work{};
}

ec_status skinny32_product(cudaStream_t s, const U32& u, int64_t n0, int trans, int64_t N,
                           int64_t K, const double* Y, int64_t ldy, double* C, int64_t ldc,
                           Skinny32Work* w, const DevStatus* st) {
  if (N <= 0 || n0 <= 0) return EC_OK;
  if (!u.data) return EC_ERR_STATE;
  if (trans) K = n0;
  if (K <= 0 || K > n0) return EC_ERR_ARG;
  const int W = u.pair ? 2 : 1;
  const int64_t ldyc = round4(K);
  // the rounded right operand, all N columns at once, and its per-column exponents
  {
    char* yb = static_cast<char*>(w->y);
    size_t cap = w->ycap;
    const ec_status g = grow(&yb, cap, sizeof(float) * W * (size_t)ldyc * (size_t)N);
    w->y = yb;
    w->ycap = cap;
    if (g != EC_OK) return g;
  }
  if (grow(&w->yexp, w->ecap, (size_t)N) != EC_OK) return EC_ERR_OOM;
  col_exp_kernel<<<(unsigned)N, 256, 0, ::ec::counted(s)>>>(K, Y, ldy, w->yexp);
  float* yf = static_cast<float*>(w->y);
  if (u.pair)
    round_kernel<1><<<grid_for(ldyc * N, 256), 256, 0, ::ec::counted(s)>>>(K, N, Y, ldy, yf, ldyc,
                                                                          w->yexp, 0);
  else
    round_kernel<0><<<grid_for(ldyc * N, 256), 256, 0, ::ec::counted(s)>>>(K, N, Y, ldy, yf, ldyc,
                                                                          w->yexp, 0);
  const float* U = static_cast<const float*>(u.data);
  if (trans) {
    for (int64_t c0 = 0; c0 < N; c0 += NC_MAX) {
      const int nc = (int)((N - c0) < NC_MAX ? (N - c0) : NC_MAX);
      const float* Yc = yf + (size_t)W * ldyc * c0;
      if (u.pair)
        tn_any<1>(s, nc, n0, ldyc, U, u.ld, Yc, ldyc, w->yexp + c0, u.eU, C + c0 * ldc, ldc, st);
      else
        tn_any<0>(s, nc, n0, ldyc, U, u.ld, Yc, ldyc, w->yexp + c0, u.eU, C + c0 * ldc, ldc, st);
    }
    return EC_OK;
  }
  // K segments so that the grid covers the GPU about twice
  const int rpt = u.pair ? 2 : 4;
  const int64_t gx = (n0 + 32 * rpt - 1) / (32 * rpt);
  const int64_t want = 2 * 4 * (int64_t)num_sms();
  int64_t ksplit = (want + gx - 1) / gx;
  const int64_t kmax = (K + 511) / 512;                 // segments of at least 512
  if (ksplit > kmax) ksplit = kmax;
  if (ksplit < 1) ksplit = 1;
  const int64_t kseg = (K + ksplit - 1) / ksplit;
  ksplit = (K + kseg - 1) / kseg;
  const int64_t ldp = n0;
  if (grow(&w->part, w->pcap, (size_t)ksplit * NC_MAX * (size_t)ldp) != EC_OK) return EC_ERR_OOM;
  for (int64_t c0 = 0; c0 < N; c0 += NC_MAX) {
    const int nc = (int)((N - c0) < NC_MAX ? (N - c0) : NC_MAX);
    const float* Yc = yf + (size_t)W * ldyc * c0;
    if (u.pair)
      nn_any<1>(s, nc, n0, K, kseg, (int)ksplit, U, u.ld, Yc, ldyc, w->part, ldp, st);
    else
      nn_any<0>(s, nc, n0, K, kseg, (int)ksplit, U, u.ld, Yc, ldyc, w->part, ldp, st);
    nn_reduce_kernel<<<grid_for(n0 * nc, 256), 256, 0, ::ec::counted(s)>>>(
        n0, nc, (int)ksplit, w->part, ldp, w->yexp + c0, u.eU, C + c0 * ldc, ldc, st);
  }
  return EC_OK;
}

}  // namespace ec
