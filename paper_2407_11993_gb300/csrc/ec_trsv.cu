// Persistent blocked forward / backward substitution with a Cholesky factor
// (the per-step work of the plain form, Sec. 3.3.1: "forward substitution"
// C y = b, then "backward substitution" C^T x = y).
//
// The factor is column-major lower triangular, cut into 64 x 64 tiles.  Row
// block I of the forward solve needs y_J for every J < I; a CTA takes row
// blocks in increasing order from an atomic ticket, accumulates the tiles of
// its row as the y_J are published, applies the precomputed inverse of the
// diagonal block and publishes y_I by writing the solve's epoch into flag I.
// A CTA only ever waits on blocks whose tickets were drawn before its own, by
// CTAs that are already running, so the scheme needs no co-residency.  The
// backward solve runs the same way from the last block upwards on the
// transposed tiles.  b, y and x may all be the same buffer (in-place solve).
//
// Every wait polls a flag a bounded number of times; when the bound runs out
// the CTA records EC_ERR_TIMEOUT in the status block and returns, and every
// other CTA returns as soon as it sees the status.
//
// Bound on GB300: N^2 DFMA per solve pair at ~2 DFMA/clk/SM (FP64 pipe),
// against 8 N^2 bytes of factor traffic per pair from HBM.

#include "ec_internal.h"

namespace ec {

namespace {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ bool status_set(const DevStatus* st) {
  return *(volatile const int*)&st->code != 0;
}

// Thread 0 waits until flags[J] == epoch; returns false on timeout / failure.
__device__ bool wait_flag(const int* flags, int J, int epoch, long long limit, DevStatus* st,
                          int where) {
  long long it = 0;
  while (ld_acquire(flags + J) != epoch) {
    if (status_set(st)) return false;
    if (++it > limit) {
      if (atomicCAS(&st->code, 0, (int)EC_ERR_TIMEOUT) == 0) {
        st->info = J;
        st->where = where;
      }
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

__global__ void __launch_bounds__(256) trsv_fwd_kernel(int64_t n, const double* L, int64_t ldl,
                                                       const double* Dinv, const double* b,
                                                       double* y, int* flags, unsigned* ticket,
                                                       const int* epoch_ptr, long long limit,
                                                       DevStatus* st) {
  const int nblk = (int)((n + NB - 1) / NB);
  const int epoch = *epoch_ptr;
  __shared__ int sI, sReady, sOk;
  __shared__ double red[4][NB];
  __shared__ double rv[NB];
  const int tid = threadIdx.x;
  const int r = tid & 63, cg = tid >> 6;
  int ready = 0;
  for (;;) {
    if (tid == 0) sI = status_set(st) ? nblk : (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int I = sI;
    if (I >= nblk) return;
    const int64_t r0 = (int64_t)I * NB;
    const int kb = (int)((n - r0) < NB ? (n - r0) : NB);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int J = 0; J < I; ++J) {
      if (J >= ready) {
        if (tid == 0) {
          int ok = wait_flag(flags, J, epoch, limit, st, 1);
          int rd = J + 1;
          if (ok)
            while (rd < I && ld_acquire(flags + rd) == epoch) ++rd;
          sReady = rd;
          sOk = ok;
        }
        __syncthreads();
        if (!sOk) return;
        ready = sReady;
      }
      if (r < kb) {
        const double* Lp = L + (r0 + r) + (int64_t)(J * NB + cg * 16) * ldl;
        const double* yp = y + (int64_t)J * NB + cg * 16;
        double l[16], v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) l[c] = Lp[c * ldl];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = __ldcg(yp + c);
#pragma unroll
        for (int c = 0; c < 16; c += 4) {
          a0 = fma(l[c], v[c], a0);
          a1 = fma(l[c + 1], v[c + 1], a1);
          a2 = fma(l[c + 2], v[c + 2], a2);
          a3 = fma(l[c + 3], v[c + 3], a3);
        }
      }
    }
    red[cg][r] = (a0 + a1) + (a2 + a3);
    __syncthreads();
    if (tid < NB)
      rv[tid] = (tid < kb) ? __ldcg(b + r0 + tid) - ((red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]))
                           : 0.0;
    __syncthreads();
    {
      const double* Dp = Dinv + (int64_t)I * NB * NB + r + (cg * 16) * NB;
      double s0 = 0.0, s1 = 0.0;
#pragma unroll
      for (int c = 0; c < 16; c += 2) {
        s0 = fma(Dp[c * NB], rv[cg * 16 + c], s0);
        s1 = fma(Dp[(c + 1) * NB], rv[cg * 16 + c + 1], s1);
      }
      red[cg][r] = s0 + s1;
    }
    __syncthreads();
    if (tid < kb) {
      y[r0 + tid] = (red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]);
      __threadfence();
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(flags + I, epoch);
    }
  }
}

__global__ void __launch_bounds__(256) trsv_bwd_kernel(int64_t n, const double* L, int64_t ldl,
                                                       const double* Dinv, const double* y,
                                                       double* x, int* flags, unsigned* ticket,
                                                       const int* epoch_ptr, long long limit,
                                                       DevStatus* st) {
  const int nblk = (int)((n + NB - 1) / NB);
  const int epoch = *epoch_ptr;
  __shared__ int sI, sReady, sOk;
  __shared__ double red[NB];
  __shared__ double zv[NB];
  const int tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5;   // warp w owns columns w*8 .. w*8+7 of the tile
  int ready = nblk;                           // blocks >= ready are known published
  for (;;) {
    if (tid == 0) sI = status_set(st) ? nblk : (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int t = sI;
    if (t >= nblk) return;
    const int I = nblk - 1 - t;
    const int64_t c0 = (int64_t)I * NB;
    const int kb = (int)((n - c0) < NB ? (n - c0) : NB);
    double acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = 0.0;
    for (int J = nblk - 1; J > I; --J) {
      if (J < ready) {
        if (tid == 0) {
          int ok = wait_flag(flags, J, epoch, limit, st, 2);
          int rd = J;
          if (ok)
            while (rd - 1 > I && ld_acquire(flags + rd - 1) == epoch) --rd;
          sReady = rd;
          sOk = ok;
        }
        __syncthreads();
        if (!sOk) return;
        ready = sReady;
      }
      const int64_t rJ = (int64_t)J * NB;
      const int kbJ = (int)((n - rJ) < NB ? (n - rJ) : NB);
      const double x0 = (lane < kbJ) ? __ldcg(x + rJ + lane) : 0.0;
      const double x1 = (lane + 32 < kbJ) ? __ldcg(x + rJ + lane + 32) : 0.0;
      const double* Lp = L + rJ + lane + (c0 + w * 8) * ldl;
      double l0[8], l1[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        l0[c] = (lane < kbJ) ? Lp[c * ldl] : 0.0;
        l1[c] = (lane + 32 < kbJ) ? Lp[c * ldl + 32] : 0.0;
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[c] = fma(l1[c], x1, fma(l0[c], x0, acc[c]));
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      double v = acc[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[w * 8 + c] = v;
    }
    __syncthreads();
    if (tid < NB) zv[tid] = (tid < kb) ? __ldcg(y + c0 + tid) - red[tid] : 0.0;
    __syncthreads();
    {
      // x_I = Dinv_I^T z: column c of Dinv dotted with z
      const double* Dp = Dinv + (int64_t)I * NB * NB;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int col = w * 8 + c;
        double v = fma(Dp[lane + col * NB], zv[lane], Dp[lane + 32 + col * NB] * zv[lane + 32]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[col] = v;
      }
    }
    __syncthreads();
    if (tid < kb) {
      x[c0 + tid] = red[tid];
      __threadfence();
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(flags + I, epoch);
    }
  }
}

__global__ void trsv_begin_kernel(unsigned* tickets, int* epoch) {
  tickets[0] = 0u;
  tickets[1] = 0u;
  *epoch = *epoch + 1;
}

__global__ void wait_probe_kernel(int* flag, long long limit, DevStatus* st) {
  if (threadIdx.x == 0) wait_flag(flag, 0, 1, limit, st, 9);
}

}  // namespace

void trsv_begin(cudaStream_t s, const TrsvSync& sync) {
  trsv_begin_kernel<<<1, 1, 0, ::ec::counted(s)>>>(sync.tickets, sync.epoch);
}

void trsv_pair(cudaStream_t s, int64_t n, const double* Lf, int64_t ldl, const double* Dinv,
               const double* b, double* y, double* x, const TrsvSync& sync, int grid,
               long long limit, DevStatus* st, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], s);
  trsv_fwd_kernel<<<grid, 256, 0, ::ec::counted(s)>>>(n, Lf, ldl, Dinv, b, y, sync.flags_fwd,
                                                      sync.tickets, sync.epoch, limit, st);
  if (ev) cudaEventRecord(ev[1], s);
  trsv_bwd_kernel<<<grid, 256, 0, ::ec::counted(s)>>>(n, Lf, ldl, Dinv, y, x, sync.flags_bwd,
                                                      sync.tickets + 1, sync.epoch, limit, st);
  if (ev) cudaEventRecord(ev[2], s);
}

void wait_timeout_probe(cudaStream_t s, int* flag, long long limit, DevStatus* st) {
  wait_probe_kernel<<<1, 32, 0, ::ec::counted(s)>>>(flag, limit, st);
}

}  // namespace ec
