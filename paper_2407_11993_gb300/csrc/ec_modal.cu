// Modal form (Sec. 3.2, Eq. generalized_eigenvalues_discrete and
// modal_decomposition_discrete; Sec. 3.3.2).
//
// Setup, all FP64 on the GPU:
//   R_i = C_R C_R^T                       (blocked Cholesky)
//   A   = C_R^{-1} L_i C_R^{-T}           (two blocked triangular solves)
//   A   = Q T Q^T                         (Householder tridiagonalisation)
//   T   = S diag(lambda) S^T              (divide and conquer; timed on its own)
//   U   = C_R^{-T} Q S,  tau = lambda     (columns reordered by decreasing tau)
// so that U^T R_i U = 1 and U^T L_i U = diag(tau): R_n = 1, L_n = tau_n.
//
// Projections (Delta t independent, Sec. 5):  B = U^T [R_D | L_D | M_0],
// G^T = U^T (C K)^T.  With I_i = U x the theta-step of Eq. time_integration
// becomes, mode by mode,
//   x_n^{k+1} = a_n x_n^k + c_n beta_n^k,
//   a_n = (tau_n - (1 - theta) dt) / (tau_n + theta dt),  c_n = 1 / (tau_n + theta dt),
//   beta^k  = B_R (-dt i_D^k - theta dt d i_D) + B_L (-d i_D) + B_M (-d i_0),
// and the probes are y^k = G x^k + C E^T (E E^T)^{-1} i_D^k.
//
// Run: one thread per mode walks the time steps of a chunk with x in a
// register; the probe contraction G x^k is reduced per warp with shuffles,
// buffered in shared memory for 32 steps, and summed across warps; per-CTA
// partial sums are then added in CTA order by a second kernel (deterministic).
// Snapshot amplitudes are stored and turned into currents by one GEMM.

#include <algorithm>
#include <cmath>

#include "ec_modal.h"
#include "ec_oz.h"
#include "ec_skinny32.h"
#include "ec_sytrd.h"
#include "ec_tc.h"

namespace ec {

struct ModalState {
  int64_t n = 0, n0 = 0;
  int m = 0, S = 0, P = 0, ncoef = 0;
  double theta = 0.5, dt = 0.0;
  double* U = nullptr;
  double* tau = nullptr;
  double* ac = nullptr;       // a_n, q0_n, q1_n (3 x n0)
  int integ = EC_INTEG_THETA;
  int64_t nkeep = 0;          // modes integrated (the nkeep largest tau); the rest stay zero
  int rhs_mode = EC_RHS_SUM;  // EC_RHS_*: independent trajectories for INDEPENDENT / PAIRED
  int ntraj = 1;
  double* B = nullptr;        // n0 x ncoef
  double* Gt = nullptr;       // n0 x P
  double* x = nullptr;        // n0
  double* work = nullptr;     // n0
  double* Xsnap = nullptr;
  size_t xsnapCap = 0;
  double* partial = nullptr;
  size_t partialCap = 0;
  double* chunkbuf = nullptr;    // xend, apow, xstart (3 x nchunk x n0)
  size_t chunkCap = 0;
  double* small = nullptr;    // m x nsnap scratch (x2)
  size_t smallCap = 0;
  // reduced-precision copies (EC_PREC_BF16)
  int precision = EC_PREC_FP64;
  __nv_bfloat16* Ubf_rm = nullptr;   // U, K-major for U x           (n0 x ld)
  __nv_bfloat16* Ubf_cm = nullptr;   // U^T, K-major for U^T y        (n0 x ld)
  __nv_bfloat16* Ubf_rm_lo = nullptr;   // rounding remainders (EC_PREC_BF16X3)
  __nv_bfloat16* Ubf_cm_lo = nullptr;
  __nv_bfloat16* Ybf = nullptr;      // right operand (N x ld), hi and lo halves
  size_t ybfCap = 0;
  // FP32 / FP32-pair copy of U and the scratch of its products (EC_PREC_FP32, _FP32X2)
  U32 u32;
  Skinny32Work sk;
  // FP64-accurate tensor-core products (EC_GEMM_TENSOR): workspace, kept for the run's
  // snapshot reconstruction
  int gemm = EC_GEMM_TENSOR;
  OzWork oz;
  // U's slices, cut on the first FP64 reconstruction and kept (16 bytes per entry): each
  // later U x then streams them once instead of running U x on the FP64 pipe
  OzSplit usplit;
  bool usplit_tried = false;
  // setup scratch
  double* DinvR = nullptr;
  const double* CR = nullptr;
  int64_t ldCR = 0;
};

namespace {

constexpr int MT = 256;            // modes per CTA
constexpr int TS = 16;             // steps per shared-memory block of the probe contraction
constexpr int64_t SUPER = 32768;   // steps per launch group (bounds the partial-sum buffer)
constexpr int64_t CH_MIN = 256;    // shortest time chunk
constexpr int64_t ORM_GROUP = 1024;  // reflectors per compact-WY group of the tensor-core back-transform
// from this size on, FP64 snapshot reconstructions use U's kept slices (below it the
// FP64 cores finish U x in about the time of the tensor path's launches)
constexpr int64_t PRESPLIT_MIN = 4096;

cudaError_t dalloc(void** p, size_t b) { return device_alloc(p, b); }

template <typename T>
ec_status alloc_n(T** p, size_t count) {
  if (*p) return EC_OK;
  if (dalloc((void**)p, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return EC_ERR_OOM;
  }
  return EC_OK;
}

template <typename T>
ec_status grow_n(T** p, size_t& cap, size_t count) {
  if (*p && count <= cap) return EC_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  cap = 0;
  ec_status s = alloc_n(p, count);
  if (s == EC_OK) cap = count;
  return s;
}

struct Timer {
  cudaEvent_t a, b;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
  double ms() {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    cudaEventRecord(a, s);
    return t;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// Reverse the column order (ascending -> descending eigenvalues).
__global__ void reverse_kernel(int64_t n, const double* lam, const double* Q, double* tau,
                               double* U) {
  const int64_t c = blockIdx.y;
  for (int64_t cc = c; cc < n; cc += gridDim.y) {
    const int64_t src = n - 1 - cc;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
      U[r + cc * n] = Q[r + src * n];
    if (blockIdx.x == 0 && threadIdx.x == 0) tau[cc] = lam[src];
  }
}

// Per-mode step coefficients (a, q0, q1) of x^{k+1} = a x^k + q0 (B w0^k) + q1 (B w1^k).
//   theta-method (Sec. 3.3.2):  a = (tau - (1-theta) dt)/(tau + theta dt), q0 = 1/(tau + theta dt), q1 = 0
//   exact for piecewise-linear sources (h = dt/tau): a = e^{-h}, q0 = 1 - e^{-h},
//   q1 = 1 - (1 - e^{-h})/h, summed from its Taylor series for h < 1 (it cancels to h/2).
__global__ void coef_kernel(int64_t n0, const double* tau, double theta, double dt, int integ,
                            double* ac) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n0;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double t = tau[i];
    if (integ == EC_INTEG_EXACT) {
      const double h = dt / t;
      const double c0 = -expm1(-h);
      double c1;
      if (h < 1.0) {
        double term = 0.5 * h, ser = term;
        for (int j = 2; j <= 20; ++j) {
          term = -term * h / (double)(j + 1);
          ser += term;
        }
        c1 = ser;
      } else {
        c1 = 1.0 - c0 / h;
      }
      ac[i] = exp(-h);
      ac[n0 + i] = c0;
      ac[2 * n0 + i] = c1;
    } else {
      const double den = t + theta * dt;
      ac[i] = (t - (1.0 - theta) * dt) / den;
      ac[n0 + i] = 1.0 / den;
      ac[2 * n0 + i] = 0.0;
    }
  }
}

__device__ __forceinline__ double srcv(const double* a, int64_t T, int row, int64_t k) {
  return a[(int64_t)row * (T + 1) + k];
}

struct ScanArgs {
  int64_t n0, T;              // T: steps of the whole run (source arrays hold T+1 samples)
  int64_t nkeep;              // modes integrated: 0 .. nkeep-1
  int64_t k0, kn;             // this launch group: steps k0 .. k0+kn-1
  int64_t ch;                 // chunk length; chunk g covers [k0 + g ch, k0 + (g+1) ch)
  int nchunk;
  int m, S, P, ncoef;
  int integ;                  // EC_INTEG_*
  double theta, dt;
  const double* ac;           // a, q0, q1 (3 x n0)
  const double* B;
  const double* Gt;
  const double* src;
  const double* iD;
  const double* x;            // state at k0
  double* xout;               // state at k0 + kn
  double* xend;               // nchunk x n0: chunk end state from a zero start (pass 1)
  double* apow;               // nchunk x n0: a_n^(chunk length)
  double* xstart;             // nchunk x n0: true chunk start states (carry pass)
  double* partial;            // ntraj x nblk x kn x Pout
  double* Xsnap;              // n0 x (nsnap * ntraj), column j * ntraj + r
  int64_t stride;
  // independent trajectories (blockIdx.z = trajectory r): coil r drives trajectory r
  int ntraj;                  // 1 unless indep
  int indep;                  // trajectory r uses projected column r and source row r only
  int paired;                 // trajectory r is read by probe row r only
  int Pout;                   // probes per trajectory (paired: 1)
};

// Weights of projected source column c at step k.  which = 0: w0, which = 1: w1.
//   theta-method, Cholesky-form right-hand side (Sec. 3.3.1 projected, Sec. 3.3.2):
//     w0 = [-dt i_D^k - theta dt d i_D | -d i_D | -d i_0],  w1 = 0
//   exact integration of sources linear between samples: the forcing over the step is
//   e0 + e1 s with e0 = B w0, e1 = B w1,
//     w0 = [-i_D^k | -d i_D / dt | -d i_0 / dt],  w1 = [-d i_D | 0 | 0]
__device__ __forceinline__ double beta_coef(const ScanArgs& a, int c, int64_t k, int which) {
  const int m = a.m;
  if (a.integ == EC_INTEG_EXACT) {
    if (c < m) {
      const double d0 = srcv(a.iD, a.T, c, k), d1 = srcv(a.iD, a.T, c, k + 1);
      return which ? -(d1 - d0) : -d0;
    }
    if (which) return 0.0;
    if (c < 2 * m) return -(srcv(a.iD, a.T, c - m, k + 1) - srcv(a.iD, a.T, c - m, k)) / a.dt;
    return -(srcv(a.src, a.T, c - 2 * m, k + 1) - srcv(a.src, a.T, c - 2 * m, k)) / a.dt;
  }
  if (which) return 0.0;
  if (c < m) {
    const double d0 = srcv(a.iD, a.T, c, k), d1 = srcv(a.iD, a.T, c, k + 1);
    return -a.dt * d0 - a.theta * a.dt * (d1 - d0);
  }
  if (c < 2 * m) return -(srcv(a.iD, a.T, c - m, k + 1) - srcv(a.iD, a.T, c - m, k));
  return -(srcv(a.src, a.T, c - 2 * m, k + 1) - srcv(a.src, a.T, c - 2 * m, k));
}

// Column c of trajectory r: the source weights of the column of B it uses.
__device__ __forceinline__ int bcol(const ScanArgs& a, int c, int r) { return a.indep ? r : c; }
__device__ __forceinline__ double coef_for(const ScanArgs& a, int c, int r, int64_t k, int which) {
  return beta_coef(a, a.indep ? 2 * a.m + r : c, k, which);
}

__device__ __forceinline__ void chunk_range(const ScanArgs& a, int g, int64_t& c0, int64_t& c1) {
  c0 = a.k0 + (int64_t)g * a.ch;
  c1 = c0 + a.ch;
  if (c1 > a.k0 + a.kn) c1 = a.k0 + a.kn;
}

// Pass 1: every chunk from a zero start -> end state and a^len (no outputs).
__global__ void __launch_bounds__(MT) modal_chunk_end_kernel(ScanArgs a) {
  extern __shared__ double smem[];
  const int nc = a.ncoef, ncs = nc > 0 ? nc : 1;
  double* coef = smem;   // [2][TS][ncs]
  const int g = blockIdx.y, r = blockIdx.z;
  int64_t c0, c1;
  chunk_range(a, g, c0, c1);
  const int64_t nmode = blockIdx.x * (int64_t)MT + threadIdx.x;
  const bool live = nmode < a.nkeep;
  const bool two = a.integ == EC_INTEG_EXACT;
  double an = 0.0, q0 = 0.0, q1 = 0.0, b[2 * MAXM + 64];
  if (live) {
    an = a.ac[nmode];
    q0 = a.ac[a.n0 + nmode];
    q1 = a.ac[2 * a.n0 + nmode];
    for (int c = 0; c < nc; ++c) b[c] = a.B[nmode + (int64_t)bcol(a, c, r) * a.n0];
    if (!two)
      for (int c = 0; c < nc; ++c) b[c] *= q0;   // theta step: x <- a x + sum_c (q0 b_c) w_c
  }
  double x = 0.0, ap = 1.0;
  for (int64_t t0 = c0; t0 < c1; t0 += TS) {
    const int nt = (int)((c1 - t0) < TS ? (c1 - t0) : TS);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nt * nc; idx += MT) {
      coef[(idx / nc) * ncs + idx % nc] = coef_for(a, idx % nc, r, t0 + idx / nc, 0);
      if (two) coef[TS * ncs + (idx / nc) * ncs + idx % nc] = coef_for(a, idx % nc, r, t0 + idx / nc, 1);
    }
    __syncthreads();
    if (live) {
      if (two) {
        for (int tt = 0; tt < nt; ++tt) {
          double e0 = 0.0, e1 = 0.0;
          for (int c = 0; c < nc; ++c) e0 = fma(b[c], coef[tt * ncs + c], e0);
          for (int c = 0; c < nc; ++c) e1 = fma(b[c], coef[TS * ncs + tt * ncs + c], e1);
          x = fma(an, x, fma(q0, e0, q1 * e1));
        }
      } else {
        for (int tt = 0; tt < nt; ++tt) {
          double e0 = 0.0;
          for (int c = 0; c < nc; ++c) e0 = fma(b[c], coef[tt * ncs + c], e0);
          x = fma(an, x, e0);
        }
      }
    }
  }
  if (live) {
    // a^len by repeated squaring
    double base = an;
    for (int64_t e = c1 - c0; e > 0; e >>= 1) {
      if (e & 1) ap *= base;
      base *= base;
    }
    a.xend[((int64_t)g * a.ntraj + r) * a.n0 + nmode] = x;
    a.apow[((int64_t)g * a.ntraj + r) * a.n0 + nmode] = ap;
  }
}

// Carry: true start state of every chunk (chunk 0 starts from the state itself).
__global__ void modal_carry_kernel(ScanArgs a) {
  const int r = blockIdx.y;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < a.nkeep;
       n += (int64_t)gridDim.x * blockDim.x) {
    double xs = a.x[(int64_t)r * a.n0 + n];
    for (int g = 0; g < a.nchunk; ++g) {
      const int64_t o = ((int64_t)g * a.ntraj + r) * a.n0 + n;
      a.xstart[o] = xs;
      xs = fma(a.apow[o], xs, a.xend[o]);
    }
  }
}

// Pass 2: every chunk replayed from its true start with the outputs: snapshots and
// per-CTA probe partials (G x over the CTA's modes, as a shared-memory block product
// of TS steps at a time).
__global__ void __launch_bounds__(MT) modal_scan_kernel(ScanArgs a) {
  extern __shared__ double smem[];
  const int nc = a.ncoef, ncs = nc > 0 ? nc : 1;
  const int P = a.Pout;
  double* coef = smem;                  // [2][TS][ncs]
  double* X = coef + 2 * TS * ncs;      // [MT][TS + 1]
  double* Gs = X + MT * (TS + 1);       // [P][MT]
  double* gred = Gs + P * MT;           // [MT]: group sums of the probe product
  const int g = blockIdx.y, r = blockIdx.z;
  int64_t c0, c1;
  chunk_range(a, g, c0, c1);
  const int tid = threadIdx.x;
  const int64_t nmode = blockIdx.x * (int64_t)MT + tid;
  const bool live = nmode < a.nkeep;
  const bool two = a.integ == EC_INTEG_EXACT;
  double an = 0.0, q0 = 0.0, q1 = 0.0, x = 0.0, b[2 * MAXM + 64];
  if (live) {
    an = a.ac[nmode];
    q0 = a.ac[a.n0 + nmode];
    q1 = a.ac[2 * a.n0 + nmode];
    x = (g == 0) ? a.x[(int64_t)r * a.n0 + nmode]
                 : a.xstart[((int64_t)g * a.ntraj + r) * a.n0 + nmode];
    for (int c = 0; c < nc; ++c) b[c] = a.B[nmode + (int64_t)bcol(a, c, r) * a.n0];
    if (!two)
      for (int c = 0; c < nc; ++c) b[c] *= q0;   // as in modal_chunk_end_kernel
  }
  for (int p = 0; p < P; ++p)
    Gs[p * MT + tid] = live ? a.Gt[nmode + (int64_t)(a.paired ? r : p) * a.n0] : 0.0;
  for (int64_t t0 = c0; t0 < c1; t0 += TS) {
    const int nt = (int)((c1 - t0) < TS ? (c1 - t0) : TS);
    __syncthreads();
    for (int idx = tid; idx < nt * nc; idx += MT) {
      coef[(idx / nc) * ncs + idx % nc] = coef_for(a, idx % nc, r, t0 + idx / nc, 0);
      if (two) coef[TS * ncs + (idx / nc) * ncs + idx % nc] = coef_for(a, idx % nc, r, t0 + idx / nc, 1);
    }
    __syncthreads();
    for (int tt = 0; tt < nt; ++tt) {
      double e0 = 0.0;
      for (int c = 0; c < nc; ++c) e0 = fma(b[c], coef[tt * ncs + c], e0);
      if (two) {
        double e1 = 0.0;
        for (int c = 0; c < nc; ++c) e1 = fma(b[c], coef[TS * ncs + tt * ncs + c], e1);
        x = fma(an, x, fma(q0, e0, q1 * e1));
      } else {
        x = fma(an, x, e0);
      }
      X[tid * (TS + 1) + tt] = live ? x : 0.0;
      const int64_t k1 = t0 + tt + 1;   // state index after this step
      if (live && a.stride > 0 && a.Xsnap && k1 % a.stride == 0)
        a.Xsnap[nmode + ((k1 / a.stride - 1) * a.ntraj + r) * a.n0] = x;
    }
    __syncthreads();
    // probe block product: P x nt outputs, each a sum over the CTA's MT modes; with few
    // outputs the modes are cut into G groups so that every thread works, and the G group
    // sums are added in group order.  G depends on P only (not on nt), so every step's
    // sum has the same shape wherever the step falls in a block: runs split at any step
    // and resumed give the same bits.
    const int npf = P * TS;
    int G = 1;
    while (G * 2 * npf <= MT) G *= 2;
    if (G == 1) {
      for (int o = tid; o < P * nt; o += MT) {
        const int p = o / nt, tt = o % nt;
        const double* gp = Gs + p * MT;
        double s0 = 0.0, s1 = 0.0;
        for (int n = 0; n < MT; n += 2) {
          s0 = fma(gp[n], X[n * (TS + 1) + tt], s0);
          s1 = fma(gp[n + 1], X[(n + 1) * (TS + 1) + tt], s1);
        }
        a.partial[(((int64_t)r * gridDim.x + blockIdx.x) * a.kn + (t0 - a.k0) + tt) * P + p] = s0 + s1;
      }
    } else {
      const int o = tid % npf, g = tid / npf, nb = MT / G;
      const int p = o / TS, tt = o % TS;
      if (g < G && tt < nt) {
        const double* gp = Gs + p * MT;
        double s0 = 0.0, s1 = 0.0;
        for (int n = g * nb; n < (g + 1) * nb; n += 2) {
          s0 = fma(gp[n], X[n * (TS + 1) + tt], s0);
          s1 = fma(gp[n + 1], X[(n + 1) * (TS + 1) + tt], s1);
        }
        gred[g * npf + o] = s0 + s1;
      }
      __syncthreads();
      if (tid < npf && tt < nt) {
        double v = gred[tid];
        for (int gg = 1; gg < G; ++gg) v += gred[gg * npf + tid];
        a.partial[(((int64_t)r * gridDim.x + blockIdx.x) * a.kn + (t0 - a.k0) + tt) * P + p] = v;
      }
    }
  }
  if (live && g == a.nchunk - 1) a.xout[(int64_t)r * a.n0 + nmode] = x;
}

__global__ void probe_reduce_kernel(ScanArgs a, int nblk, const double* CPE, double* probes) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int Po = a.Pout;
  if (idx >= a.kn * a.ntraj * Po) return;
  const int64_t tt = idx / ((int64_t)a.ntraj * Po);
  const int r = (int)((idx / Po) % a.ntraj);
  const int p = (int)(idx % Po);
  double v = 0.0;
  for (int b = 0; b < nblk; ++b) v += a.partial[(((int64_t)r * nblk + b) * a.kn + tt) * Po + p];
  const int64_t k1 = a.k0 + tt + 1;
  if (!a.indep)
    for (int j = 0; j < a.m; ++j) v = fma(CPE[p + (int64_t)j * a.P], srcv(a.iD, a.T, j, k1), v);
  probes[((a.k0 + tt) * a.ntraj + r) * Po + p] = v;
}

// snaps (n x nsnap, ld n): add PE i_D at the snapshot times.
__global__ void snap_particular_kernel(int64_t n, int m, int64_t nsnap, int64_t stride, int64_t T,
                                       const double* PE, const double* iD, double* snaps) {
  const int64_t j = blockIdx.y;
  for (int64_t jj = j; jj < nsnap; jj += gridDim.y) {
    const int64_t k = (jj + 1) * stride;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
      double v = snaps[i + jj * n];
      for (int c = 0; c < m; ++c) v = fma(PE[i + (int64_t)c * n], srcv(iD, T, c, k), v);
      snaps[i + jj * n] = v;
    }
  }
}

}  // namespace

#define MS_TRY(x)               \
  do {                          \
    ec_status _s = (x);         \
    if (_s != EC_OK) return _s; \
  } while (0)

// C (n0 x N, column-major, ldc) = op(U) Y with Y n0 x N column-major (lds); op(U) = U^T
// (trans_u = 1) or U (trans_u = 0); arithmetic per ms->precision.
ec_status modal_product(cudaStream_t s, ModalState* ms, int trans_u, int64_t N, const double* Y,
                        int64_t lds, double* C, int64_t ldc, DevStatus* st, int64_t K = -1) {
  const int64_t n0 = ms->n0;
  if (N <= 0) return EC_OK;
  if (K < 0) K = n0;
  if (ms->precision == EC_PREC_FP32 || ms->precision == EC_PREC_FP32X2)
    return skinny32_product(s, ms->u32, n0, trans_u, N, K, Y, lds, C, ldc, &ms->sk, st);
  if (ms->precision == EC_PREC_FP64) {
    if (ms->gemm != EC_GEMM_FP64 && !trans_u && n0 >= PRESPLIT_MIN) {
      if (!ms->usplit.blocks && !ms->usplit_tried) {
        ms->usplit_tried = true;
        if (oz_presplit(s, N_, n0, n0, ms->U, n0, &ms->usplit) != EC_OK)
          oz_split_free(&ms->usplit);               // no room: the per-call paths below
      }
      if (ms->usplit.blocks) {
        const ec_status rc = oz_gemm_presplit(s, ms->usplit, K, N_, N, Y, lds, C, ldc, &ms->oz,
                                              st);
        if (rc != EC_ERR_OOM) return rc;
      }
    }
    gemm_auto(s, ms->gemm != EC_GEMM_FP64 ? &ms->oz : nullptr, trans_u ? T_ : N_, N_, n0, N, K,
              1.0, ms->U, n0, Y, lds, 0.0, C, ldc, 0, st);
    return EC_OK;
  }
  const int64_t ld = bf16_ld(n0);
  const bool x3 = ms->precision == EC_PREC_BF16X3;
  MS_TRY(grow_n(&ms->Ybf, ms->ybfCap, (size_t)(x3 ? 2 : 1) * N * ld));
  __nv_bfloat16* yh = ms->Ybf;
  __nv_bfloat16* yl = x3 ? ms->Ybf + (size_t)N * ld : nullptr;
  to_bf16(s, N, K, Y, lds, 1, yh, ld, yl);
  const __nv_bfloat16* ah = trans_u ? ms->Ubf_cm : ms->Ubf_rm;
  const __nv_bfloat16* al = trans_u ? ms->Ubf_cm_lo : ms->Ubf_rm_lo;
  if (x3) return tc_gemm_bf16x3(s, n0, N, K, 1.0, ah, al, ld, yh, yl, ld, C, ldc, st);
  return tc_gemm_bf16(s, n0, N, K, 1.0, ah, ld, yh, ld, 0.0, C, ldc, st);
}

ModalState* modal_create() { return new ModalState(); }

void modal_free(ModalState* ms) {
  if (!ms) return;
  double* ps[] = {ms->U, ms->tau, ms->ac, ms->B, ms->Gt, ms->x, ms->work, ms->Xsnap, ms->partial,
                  ms->small, ms->DinvR, ms->chunkbuf};
  for (double* p : ps)
    if (p) cudaFree(p);
  __nv_bfloat16* bs[] = {ms->Ubf_rm, ms->Ubf_cm, ms->Ubf_rm_lo, ms->Ubf_cm_lo, ms->Ybf};
  for (__nv_bfloat16* p : bs)
    if (p) cudaFree(p);
  oz_free(&ms->oz);
  oz_split_free(&ms->usplit);
  u32_free(&ms->u32);
  skinny32_free(&ms->sk);
  delete ms;
}

double* modal_state(ModalState* ms) { return ms->x; }

ec_status modal_set_mode_count(cudaStream_t s, ModalState* ms, int64_t nkeep) {
  if (nkeep < 1 || nkeep > ms->n0) return EC_ERR_ARG;
  ms->nkeep = nkeep;
  if (nkeep < ms->n0)
    for (int r = 0; r < ms->ntraj; ++r)
      cudaMemsetAsync(ms->x + (int64_t)r * ms->n0 + nkeep, 0, sizeof(double) * (ms->n0 - nkeep), s);
  return EC_OK;
}

int64_t modal_state_size(const ModalState* ms) { return ms->n0 * ms->ntraj; }
const double* modal_tau(ModalState* ms) { return ms->tau; }
const double* modal_U(ModalState* ms) { return ms->U; }


// Reduced-precision copy of U for the chosen arithmetic (dropping any other), then the
// projections B = U^T [R_D | L_D | M_0] and G^T = U^T (C K)^T with that arithmetic.
ec_status modal_products_prepare(cudaStream_t s, ModalState* ms, int precision, const double* RD,
                                 const double* LD, const double* Msrc, int64_t ldM,
                                 const double* CK, int64_t ldC, DevStatus* st) {
  const int64_t n0 = ms->n0;
  ms->precision = precision;
  u32_free(&ms->u32);
  for (__nv_bfloat16** p : {&ms->Ubf_rm, &ms->Ubf_cm, &ms->Ubf_rm_lo, &ms->Ubf_cm_lo}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  if (precision == EC_PREC_FP32 || precision == EC_PREC_FP32X2)
    MS_TRY(u32_build(s, n0, ms->U, n0, precision == EC_PREC_FP32X2 ? 1 : 0, &ms->u32));
  if (precision == EC_PREC_BF16 || precision == EC_PREC_BF16X3) {
    const int64_t ld = bf16_ld(n0);
    const bool x3 = precision == EC_PREC_BF16X3;
    MS_TRY(alloc_n(&ms->Ubf_rm, (size_t)n0 * ld));
    MS_TRY(alloc_n(&ms->Ubf_cm, (size_t)n0 * ld));
    if (x3) {
      MS_TRY(alloc_n(&ms->Ubf_rm_lo, (size_t)n0 * ld));
      MS_TRY(alloc_n(&ms->Ubf_cm_lo, (size_t)n0 * ld));
    }
    to_bf16(s, n0, n0, ms->U, n0, 0, ms->Ubf_rm, ld, x3 ? ms->Ubf_rm_lo : nullptr);
    to_bf16(s, n0, n0, ms->U, n0, 1, ms->Ubf_cm, ld, x3 ? ms->Ubf_cm_lo : nullptr);
  }
  if (ms->ncoef > 0) {
    double* Gm = nullptr;
    if (alloc_n(&Gm, (size_t)n0 * ms->ncoef)) return EC_ERR_OOM;
    if (ms->m > 0) {
      copy_matrix(s, n0, ms->m, RD, n0, Gm, n0);
      copy_matrix(s, n0, ms->m, LD, n0, Gm + n0 * ms->m, n0);
    }
    if (ms->S > 0) copy_matrix(s, n0, ms->S, Msrc, ldM, Gm + n0 * 2 * ms->m, n0);
    ec_status rc2 = modal_product(s, ms, 1, ms->ncoef, Gm, n0, ms->B, n0, st);
    cudaStreamSynchronize(s);
    cudaFree(Gm);
    if (rc2 != EC_OK) return rc2;
  }
  if (ms->P > 0) MS_TRY(modal_product(s, ms, 1, ms->P, CK, ldC, ms->Gt, n0, st));
  return EC_OK;
}

ec_status modal_set_precision(cudaStream_t s, ModalState* ms, int precision, const double* RD,
                              const double* LD, const double* Msrc, int64_t ldM,
                              const double* CK, int64_t ldC, DevStatus* st) {
  return modal_products_prepare(s, ms, precision, RD, LD, Msrc, ldM, CK, ldC, st);
}

ec_status modal_setup(cudaStream_t s, ModalState* ms, const ModalSetupArgs& a, ec_timing* tim) {
  const int64_t n0 = a.n0, ld = a.ld;
  ms->n = a.n; ms->n0 = n0; ms->m = a.m; ms->S = a.S; ms->P = a.P;
  ms->ncoef = 2 * a.m + a.S;
  ms->rhs_mode = a.rhs_mode;
  ms->ntraj = (a.rhs_mode == EC_RHS_SUM) ? 1 : a.S;
  ms->theta = a.theta; ms->dt = a.dt;
  const size_t nn = (size_t)n0 * n0;
  const int64_t nblk = (n0 + NB - 1) / NB;
  MS_TRY(alloc_n(&ms->DinvR, (size_t)nblk * NB * NB));
  MS_TRY(alloc_n(&ms->U, nn));
  MS_TRY(alloc_n(&ms->tau, (size_t)n0));
  MS_TRY(alloc_n(&ms->ac, (size_t)3 * n0));
  MS_TRY(alloc_n(&ms->B, (size_t)n0 * (ms->ncoef > 0 ? ms->ncoef : 1)));
  MS_TRY(alloc_n(&ms->Gt, (size_t)n0 * (a.P > 0 ? a.P : 1)));
  MS_TRY(alloc_n(&ms->x, (size_t)n0 * ms->ntraj));
  MS_TRY(alloc_n(&ms->work, (size_t)n0 * ms->ntraj));
  cudaMemsetAsync(ms->x, 0, sizeof(double) * n0 * ms->ntraj, s);
  ms->CR = a.Ri;
  ms->ldCR = ld;
  ms->gemm = a.gemm;
  OzWork* oz = a.gemm != EC_GEMM_FP64 ? &ms->oz : nullptr;

  Timer t(s);
  // a4: R_i = C_R C_R^T
  potrf(s, n0, a.Ri, ld, ms->DinvR, a.st, oz);
  tim->factor_ms = t.ms();
  {
    DevStatus h{};
    cudaMemcpy(&h, a.st, sizeof(h), cudaMemcpyDeviceToHost);
    if (h.code != 0) return EC_OK;   // reported by the caller's status collection
  }
  // a5: A = C_R^{-1} L_i C_R^{-T}
  trsm_left_lower(s, n0, n0, a.Ri, ld, ms->DinvR, a.Li, ld, a.st, oz);
  trsm_right_lower_t_sym(s, n0, a.Ri, ld, ms->DinvR, a.Li, ld, a.st, oz);
  symmetrize_lower(s, n0, a.Li, ld);
  tim->reduce_ms = t.ms();
  // a6: tridiagonalisation
  double *d = nullptr, *e = nullptr, *th = nullptr, *v = nullptr, *w = nullptr, *part = nullptr;
  double *lam = nullptr, *Q1 = nullptr, *Q2 = nullptr, *Wm = nullptr;
  double *Vb = nullptr, *Gb = nullptr, *Tb = nullptr, *W1 = nullptr, *W2 = nullptr;
  const int64_t pcap = (int64_t)(4 * num_sms() + 8) * n0;
  ec_status rc = EC_OK;
  auto cleanup = [&]() {
    double* ps[] = {d, e, th, v, w, part, lam, Q1, Q2, Wm, Vb, Gb, Tb, W1, W2};
    for (double* p : ps)
      if (p) cudaFree(p);
  };
  if (alloc_n(&d, n0) || alloc_n(&e, n0) || alloc_n(&th, n0) || alloc_n(&v, n0) ||
      alloc_n(&w, n0) || alloc_n(&part, (size_t)pcap) || alloc_n(&lam, n0) ||
      alloc_n(&Q1, nn) || alloc_n(&Q2, nn) || alloc_n(&Wm, nn) ||
      alloc_n(&Vb, (size_t)n0 * NB) || alloc_n(&Gb, (size_t)NB * NB) ||
      alloc_n(&Tb, (size_t)NB * NB) || alloc_n(&W1, (size_t)NB * n0) ||
      alloc_n(&W2, (size_t)NB * n0)) {
    cleanup();
    return EC_ERR_OOM;
  }
  if (oz) {
    // panels of 64 columns, their rank-128 trailing updates on the tensor cores
    double *Vp = nullptr, *Wp = nullptr, *yp = nullptr, *pp = nullptr;
    if (alloc_n(&Vp, (size_t)n0 * NB) || alloc_n(&Wp, (size_t)n0 * NB) || alloc_n(&yp, 128) ||
        alloc_n(&pp, (size_t)sytrd_blocked_scratch(n0))) {
      for (double* p : {Vp, Wp, yp, pp})
        if (p) cudaFree(p);
      cleanup();
      return EC_ERR_OOM;
    }
    sytrd_lower_blocked(s, n0, a.Li, ld, d, e, th, Vp, Wp, yp, pp, oz, a.st,
                        a.gemm == EC_GEMM_TENSOR_PAIRSYMV ? 1 : 0);
    cudaStreamSynchronize(s);
    for (double* p : {Vp, Wp, yp, pp}) cudaFree(p);
  } else {
    sytrd_lower(s, n0, a.Li, ld, d, e, th, v, w, part, pcap, a.st);
  }
  tim->tridiag_ms = t.ms();
  DcWork* dcw = dc_alloc(n0, dalloc);
  if (!dcw) {
    cleanup();
    return EC_ERR_OOM;
  }
  rc = dc_solve(s, n0, d, e, lam, Q1, Q2, Wm, dcw, a.st, oz);
  tim->eig_ms = t.ms();
  dc_free(dcw);
  if (rc != EC_OK) {
    cleanup();
    return rc;
  }
  // descending order, then U = C_R^{-T} Q S
  {
    dim3 g((unsigned)((n0 + 255) / 256 < 16 ? (n0 + 255) / 256 : 16),
           (unsigned)(n0 < 65535 ? n0 : 65535));
    reverse_kernel<<<g, 256, 0, ::ec::counted(s)>>>(n0, lam, Q1, ms->tau, ms->U);
  }
  if (oz) {
    // compact-WY groups of up to ORM_GROUP reflectors, products on the tensor cores
    const int64_t gsz = std::min<int64_t>(ORM_GROUP, (std::max<int64_t>(n0 - 2, 1) + NB - 1) / NB * NB);
    double *Vg = nullptr, *Gg = nullptr, *Tg = nullptr, *Xg = nullptr, *Wg = nullptr, *W2g = nullptr;
    auto gfree = [&]() {
      for (double* p : {Vg, Gg, Tg, Xg, Wg, W2g})
        if (p) cudaFree(p);
    };
    if (alloc_n(&Vg, (size_t)n0 * gsz) || alloc_n(&Gg, (size_t)gsz * gsz) ||
        alloc_n(&Tg, (size_t)gsz * gsz) || alloc_n(&Xg, (size_t)gsz * NB) ||
        alloc_n(&Wg, (size_t)gsz * n0) || alloc_n(&W2g, (size_t)gsz * n0)) {
      gfree();
      cleanup();
      return EC_ERR_OOM;
    }
    ormtr_lower_grouped(s, n0, a.Li, ld, th, ms->U, n0, n0, gsz, Vg, Gg, Tg, Xg, Wg, W2g, oz,
                        a.st);
    cudaStreamSynchronize(s);
    gfree();
  } else {
    const int64_t ws_cap = std::max<int64_t>((int64_t)dgemm_tn_splits(NB, n0, n0) * NB * n0,
                                             (int64_t)dgemm_tn_splits(NB, NB, n0) * NB * NB);
    double* ws = nullptr;
    if (alloc_n(&ws, (size_t)ws_cap)) ws = nullptr;   // without it the products run unsplit
    ormtr_lower(s, n0, a.Li, ld, th, ms->U, n0, n0, Vb, Gb, Tb, W1, W2, ws, ws ? ws_cap : 0, a.st);
    if (ws) {
      cudaStreamSynchronize(s);
      cudaFree(ws);
    }
  }
  trsm_left_lower_t(s, n0, n0, a.Ri, ld, ms->DinvR, ms->U, n0, a.st, oz);
  tim->backtransform_ms = t.ms();
  cleanup();
  // a7: projections and per-mode coefficients
  MS_TRY(modal_products_prepare(s, ms, a.precision, a.RD, a.LD, a.Msrc, a.ldM, a.CK, a.ldC,
                                a.st));
  ms->integ = a.integ;
  ms->nkeep = n0;
  coef_kernel<<<(unsigned)((n0 + 255) / 256 < 1024 ? (n0 + 255) / 256 : 1024), 256, 0, ::ec::counted(s)>>>(
      n0, ms->tau, ms->theta, ms->dt, ms->integ, ms->ac);
  tim->project_ms = t.ms();
  return EC_OK;
}

ec_status modal_set_step(cudaStream_t s, ModalState* ms, double theta, double dt) {
  ms->theta = theta;
  ms->dt = dt;
  const int64_t n0 = ms->n0;
  coef_kernel<<<(unsigned)((n0 + 255) / 256 < 1024 ? (n0 + 255) / 256 : 1024), 256, 0, ::ec::counted(s)>>>(
      n0, ms->tau, theta, dt, ms->integ, ms->ac);
  return EC_OK;
}

ec_status modal_run(cudaStream_t s, ModalState* ms, const StepArgs& sa,
                    std::vector<cudaEvent_t>* ev) {
  const int64_t n0 = ms->n0, T = sa.T;
  const int64_t nkeep = ms->nkeep;
  const int nt = ms->ntraj;
  const bool indep = ms->rhs_mode != EC_RHS_SUM;
  const int Pout = (ms->rhs_mode == EC_RHS_PAIRED) ? 1 : ms->P;
  const int nblk = (int)((nkeep + MT - 1) / MT);
  const int64_t nsnap = (sa.snap_stride > 0 && sa.snaps) ? T / sa.snap_stride : 0;
  if (nsnap > 0) MS_TRY(grow_n(&ms->Xsnap, ms->xsnapCap, (size_t)n0 * nsnap * nt));
  const int64_t kmax = T < SUPER ? T : SUPER;
  MS_TRY(grow_n(&ms->partial, ms->partialCap,
                (size_t)nblk * kmax * (Pout > 0 ? Pout : 1) * nt));
  // time chunks: the scan is bound by the FP64 pipe, so the chunk count minimises the
  // busiest SM's work, ceil(CTAs / SMs) x steps per chunk, with the chunk-end pass
  // (about half a replay) added when there is more than one chunk
  int64_t gcap = 1;
  {
    const int64_t sms = num_sms(), per = (int64_t)nblk * nt;
    const int64_t gmax = std::max<int64_t>(1, std::min<int64_t>(256, kmax / CH_MIN));
    double best = 1e300;
    for (int64_t g = 1; g <= gmax; ++g) {
      const double rounds = (double)((per * g + sms - 1) / sms);
      const double cost = rounds * ((double)kmax / (double)g) * (g > 1 ? 1.5 : 1.0);
      if (cost < 0.97 * best) {       // fewer chunks on near ties
        best = cost;
        gcap = g;
      }
    }
  }
  MS_TRY(grow_n(&ms->chunkbuf, ms->chunkCap, (size_t)3 * (gcap > 0 ? gcap : 1) * n0 * nt));
  ScanArgs a{};
  a.n0 = n0; a.T = T; a.m = ms->m; a.S = ms->S; a.P = ms->P;
  a.ncoef = indep ? 1 : ms->ncoef;
  a.nkeep = nkeep;
  a.ntraj = nt; a.indep = indep; a.paired = ms->rhs_mode == EC_RHS_PAIRED; a.Pout = Pout;
  a.theta = ms->theta; a.dt = ms->dt; a.ac = ms->ac; a.B = ms->B; a.Gt = ms->Gt;
  a.integ = ms->integ;
  a.src = sa.src; a.iD = sa.iD; a.partial = ms->partial;
  a.Xsnap = nsnap > 0 ? ms->Xsnap : nullptr; a.stride = nsnap > 0 ? sa.snap_stride : 0;
  const int ncs = a.ncoef > 0 ? a.ncoef : 1;
  const size_t smem1 = sizeof(double) * (size_t)(2 * TS * ncs);
  const size_t smem2 = sizeof(double) * (size_t)(2 * TS * ncs + MT * (TS + 1) + Pout * MT + MT);
  static std::atomic<unsigned long long> attr_set{0};
  if (first_on_device(attr_set))
    cudaFuncSetAttribute(modal_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  for (int64_t k0 = 0; k0 < T; k0 += SUPER) {
    a.k0 = k0;
    a.kn = (T - k0) < SUPER ? (T - k0) : SUPER;
    int64_t ch = (a.kn + gcap - 1) / (gcap > 0 ? gcap : 1);
    if (ch < CH_MIN) ch = CH_MIN;
    ch = (ch + TS - 1) / TS * TS;
    a.ch = ch;
    a.nchunk = (int)((a.kn + ch - 1) / ch);
    a.x = ms->x;
    a.xout = ms->work;
    a.xend = ms->chunkbuf;
    a.apow = ms->chunkbuf + (size_t)a.nchunk * n0 * nt;
    a.xstart = ms->chunkbuf + (size_t)2 * a.nchunk * n0 * nt;
    if (ev) {
      ev->resize(ev->size() + 2);
      cudaEventCreate(&(*ev)[ev->size() - 2]);
      cudaEventCreate(&(*ev)[ev->size() - 1]);
      cudaEventRecord((*ev)[ev->size() - 2], s);
    }
    if (a.nchunk > 1) {
      modal_chunk_end_kernel<<<dim3(nblk, a.nchunk, nt), MT, smem1, ::ec::counted(s)>>>(a);
      modal_carry_kernel<<<dim3((unsigned)((n0 + 255) / 256), nt), 256, 0, ::ec::counted(s)>>>(a);
    }
    modal_scan_kernel<<<dim3(nblk, a.nchunk, nt), MT, smem2, ::ec::counted(s)>>>(a);
    if (ev) cudaEventRecord(ev->back(), s);
    copy_matrix(s, nkeep, nt, ms->work, n0, ms->x, n0);
    if (Pout > 0 && sa.probes) {
      const int64_t tot = a.kn * Pout * nt;
      probe_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, ::ec::counted(s)>>>(
          a, nblk, sa.CPE, sa.probes);
    }
  }
  if (nsnap > 0) {
    const int64_t n = ms->n;
    const int m = ms->m;
    // rows m.. of each snapshot: U x; rows 0..m-1: 0; then apply Q and add the particular field
    if (m > 0) cudaMemsetAsync(sa.snaps, 0, sizeof(double) * (size_t)n * nsnap, s);
    MS_TRY(modal_product(s, ms, 0, nsnap * nt, ms->Xsnap, n0, sa.snaps + m, n, sa.st, nkeep));
    if (m > 0) {
      MS_TRY(grow_n(&ms->small, ms->smallCap, (size_t)2 * m * nsnap));
      one_sided_q(s, n, m, sa.snaps, nsnap, sa.V, sa.Tm, ms->small, ms->small + m * nsnap, sa.st);
      dim3 g((unsigned)((n + 255) / 256 < 16 ? (n + 255) / 256 : 16),
             (unsigned)(nsnap < 65535 ? nsnap : 65535));
      snap_particular_kernel<<<g, 256, 0, ::ec::counted(s)>>>(n, m, nsnap, sa.snap_stride, T, sa.PE, sa.iD,
                                               sa.snaps);
    }
  }
  return EC_OK;
}

void modal_set_internal_current(cudaStream_t s, ModalState* ms, const double* RiIi) {
  // x = U^T (R_i I_i): the caller passes R_i I_i; every trajectory starts from it.
  dgemm(s, T_, N_, ms->n0, 1, ms->n0, 1.0, ms->U, ms->n0, RiIi, ms->n0, 0.0, ms->x, ms->n0, 0,
        nullptr);
  for (int r = 1; r < ms->ntraj; ++r)
    copy_matrix(s, ms->n0, 1, ms->x, ms->n0, ms->x + (int64_t)r * ms->n0, ms->n0);
}

}  // namespace ec
