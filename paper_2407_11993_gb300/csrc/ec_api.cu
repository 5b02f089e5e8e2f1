// C ABI of the theta-method library (include/eddy_theta.h): context, setup
// and run orchestration for the plain and modal forms.

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ec_kernels.h"
#include "ec_modal.h"
#include "ec_oz.h"
#include "ec_tiles.h"

using namespace ec;

namespace ec {
static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace ec

struct ec_ctx {
  ec_config cfg{};
  cudaStream_t stream = nullptr;
  DevStatus* st = nullptr;
  long long spin_limit = 1ll << 24;
  int64_t n = 0, n0 = 0;
  int m = 0, S = 0, P = 0, D = 0;
  bool ready = false;
  // transformed matrices Q^T L Q, Q^T R Q (full, n x n)
  double* dL = nullptr;
  double* dR = nullptr;
  // plain
  double* dZ = nullptr;      // n0 x n0 Cholesky factor of L_i + theta dt R_i
  double* dDinv = nullptr;   // inverses of its 64 x 64 diagonal blocks
  double* dW = nullptr;      // n0 x n0 inverse factor C^{-1}, square column-major (kept
                             // only for independent right-hand sides; freed otherwise)
  TilePlan tiles;            // packed-tile layout of C^{-1} (EC_SOLVE_INVERSE)
  double* dWp = nullptr;     // C^{-1} as packed lower 64 x 64 tiles
  float* dWp32 = nullptr;    // EC_PREC_FP32: C^{-1} as packed FP32 tiles
  double* dLh = nullptr;     // EC_PREC_FP32: lower half of L (diagonal halved), packed tiles
  double* dDelta = nullptr;  // EC_PREC_FP32: refined solution (npad, zero tail)
  double* dRes = nullptr;    // EC_PREC_FP32: residual (npad, zero tail)
  double* dT1 = nullptr;     // EC_PREC_FP32: halves of L x
  double* dT2 = nullptr;
  float* dV32 = nullptr;     // EC_PREC_FP32: FP32 copy of the product input (npad, zero tail)
  float2* dWpx2 = nullptr;   // EC_PREC_FP32X2: C^{-1} as packed FP32 hi/lo pair tiles
  float2* dVx2 = nullptr;    // EC_PREC_FP32X2: pair copy of the product input (npad, zero tail)
  double* dPart1 = nullptr;  // unit partials of C^{-1} b
  double* dPart2 = nullptr;  // unit partials of C^{-T} y
  double* dYsol = nullptr;   // C^{-1} b (npad, zero tail)
  int ntraj = 1;             // trajectories (independent right-hand sides)
  double* dRhsM = nullptr;   // n0 x ntraj work (independent right-hand sides)
  double* dYM = nullptr;
  double* dXM = nullptr;
  // elimination
  double* dE = nullptr;
  double* dV = nullptr;
  double* dWR = nullptr;
  double* dT = nullptr;
  double* dVtWR = nullptr;
  double* dRrinvT = nullptr;
  double* dPE = nullptr;
  double* dCPE = nullptr;
  double* dRD = nullptr;     // n0 x m
  double* dLD = nullptr;     // n0 x m
  double* dM = nullptr;      // n x S   (Q^T M)
  double* dMD = nullptr;     // n x m   (Q^T M^D)
  double* dC = nullptr;      // n x P   (Q^T C^T)
  double* dY = nullptr;      // n x m scratch
  double* dX = nullptr;      // n x m scratch
  double* dSm = nullptr;     // small scratch
  double* dZm = nullptr;
  double* dGsrc = nullptr;
  double* dDmat = nullptr;
  double* dIi = nullptr;
  double* dWork = nullptr;
  double* dDots = nullptr;
  double* dPartial = nullptr;
  double* dTmpN = nullptr;
  unsigned* dCounter = nullptr;
  int64_t* dK = nullptr;
  Csr csr;
  int* dFlags = nullptr;      // 2 x nblk
  unsigned* dTickets = nullptr;
  int* dEpoch = nullptr;
  // run buffers
  double* dSrc = nullptr;
  size_t srcCap = 0;
  double* dIDs = nullptr;
  size_t idsCap = 0;
  double* dProbes = nullptr;
  size_t probesCap = 0;
  double* dSnaps = nullptr;
  size_t snapsCap = 0;
  int update_grid = 1;
  int trsv_grid = 1;
  ec_timing tim{};
  int64_t last_info = -1;
  ModalState* modal = nullptr;
  OzWork oz;               // tensor-core product workspace of the plain setup (EC_GEMM_TENSOR)
};

namespace ec {
// Test hook of ec_selftest_fail_alloc: < 0 disarmed; otherwise the number of
// allocations that still succeed before every later one reports failure.
std::atomic<long long> g_fail_alloc_after{-1};

cudaError_t device_alloc(void** p, size_t bytes) {
  long long left = g_fail_alloc_after.load();
  while (left >= 0) {
    if (left == 0) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
    if (g_fail_alloc_after.compare_exchange_weak(left, left - 1)) break;
  }
  return cudaMalloc(p, bytes ? bytes : 8);
}
}  // namespace ec
namespace {

cudaError_t dev_alloc(void** p, size_t bytes) { return device_alloc(p, bytes); }

// Non-finite entries in the copied inputs: the status records EC_ERR_ARG and the
// input's index (0 L, 1 R, 2 E, 3 M, 4 MD, 5 C) as the info value.
__global__ void finite_check_kernel(const double* a, int64_t count, int which, DevStatus* st) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!isfinite(a[i])) {
      if (atomicCAS(&st->code, 0, (int)EC_ERR_ARG) == 0) st->info = which;
      return;
    }
  }
}

void finite_check(cudaStream_t s, const double* a, int64_t count, int which, DevStatus* st) {
  if (count <= 0) return;
  int64_t g = (count + 255) / 256;
  if (g > (int64_t)num_sms() * 8) g = num_sms() * 8;
  finite_check_kernel<<<(unsigned)g, 256, 0, ::ec::counted(s)>>>(a, count, which, st);
}

template <typename T>
ec_status alloc(T** p, size_t count) {
  if (*p) return EC_OK;
  if (dev_alloc((void**)p, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return EC_ERR_OOM;
  }
  return EC_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <typename T>
ec_status grow(T** p, size_t& cap, size_t count) {
  if (count <= cap && *p) return EC_OK;
  dfree(*p);
  cap = 0;
  ec_status s = alloc(p, count);
  if (s == EC_OK) cap = count;
  return s;
}

void free_setup(ec_ctx* c) {
  dfree(c->dL); dfree(c->dR); dfree(c->dZ); dfree(c->dDinv); dfree(c->dE); dfree(c->dV);
  dfree(c->dW); dfree(c->dWp); tile_plan_free(&c->tiles); dfree(c->dPart1);
  dfree(c->dWp32); dfree(c->dLh); dfree(c->dDelta); dfree(c->dRes); dfree(c->dT1); dfree(c->dT2); dfree(c->dV32); dfree(c->dPart2); dfree(c->dYsol);
  dfree(c->dWpx2); dfree(c->dVx2);
  dfree(c->dRhsM); dfree(c->dYM); dfree(c->dXM);
  dfree(c->dWR); dfree(c->dT); dfree(c->dVtWR); dfree(c->dRrinvT); dfree(c->dPE);
  dfree(c->dCPE); dfree(c->dRD); dfree(c->dLD); dfree(c->dM); dfree(c->dMD); dfree(c->dC);
  dfree(c->dY); dfree(c->dX); dfree(c->dSm); dfree(c->dZm); dfree(c->dGsrc); dfree(c->dDmat);
  dfree(c->dIi); dfree(c->dWork); dfree(c->dDots); dfree(c->dPartial); dfree(c->dTmpN);
  dfree(c->dCounter); dfree(c->dK); dfree(c->csr.ptr); dfree(c->csr.col); dfree(c->csr.val);
  c->csr.nnz = 0;
  dfree(c->dFlags); dfree(c->dTickets); dfree(c->dEpoch);
  if (c->modal) { modal_free(c->modal); c->modal = nullptr; }
  oz_free(&c->oz);
  c->ready = false;
}

ec_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return EC_OK;
  if (e == cudaErrorMemoryAllocation) return EC_ERR_OOM;
  return EC_ERR_CUDA;
}

// Synchronise and collect the first error (CUDA or kernel-side status).
ec_status collect(ec_ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  DevStatus h{};
  e = cudaMemcpy(&h, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  if (h.code != 0) {
    c->last_info = h.info;
    return (ec_status)h.code;
  }
  return EC_OK;
}

ec_status copy_in(ec_ctx* c, double* dst, const double* src, size_t count, int mem) {
  if (count == 0) return EC_OK;
  cudaError_t e = cudaMemcpyAsync(dst, src, count * sizeof(double),
                                  mem == EC_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyHostToDevice,
                                  c->stream);
  return cuda_status(e);
}

ec_status copy_out(ec_ctx* c, double* dst, const double* src, size_t count, int mem) {
  if (count == 0) return EC_OK;
  cudaError_t e = cudaMemcpyAsync(dst, src, count * sizeof(double),
                                  mem == EC_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyDeviceToHost,
                                  c->stream);
  return cuda_status(e);
}

struct EventTimer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s;
  explicit EventTimer(cudaStream_t st) : s(st) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
  double stop_ms() {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
  ~EventTimer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

#define EC_TRY(x)                      \
  do {                                 \
    ec_status _s = (x);                \
    if (_s != EC_OK) return _s;        \
  } while (0)

StepArgs step_args(ec_ctx* c, int64_t T, double* probes, double* snaps, int64_t stride) {
  StepArgs a{};
  a.n = c->n; a.n0 = c->n0; a.m = c->m; a.S = c->S; a.P = c->P; a.D = c->D;
  a.theta = c->cfg.theta; a.dt = c->cfg.dt;
  a.src = c->dSrc; a.iD = c->dIDs; a.T = T; a.kstep = c->dK;
  a.V = c->dV; a.WR = c->dWR; a.Tm = c->dT; a.VtWR = c->dVtWR; a.PE = c->dPE; a.CPE = c->dCPE;
  a.R = c->csr; a.Gsrc = c->dGsrc; a.Dmat = c->dDmat; a.Ii = c->dIi; a.work = c->dWork;
  a.dots = c->dDots; a.partial = c->dPartial; a.counter = c->dCounter; a.ugrid = c->update_grid;
  a.probes = probes; a.snaps = snaps; a.snap_stride = stride;
  a.tickets = c->dTickets; a.epoch = c->dEpoch; a.st = c->st;
  return a;
}

}  // namespace

namespace {

ec_status form_sources(ec_ctx* c) {
  const int64_t n0 = c->n0;
  const int m = c->m;
  if (m > 0) {
    copy_matrix(c->stream, n0, m, c->dRD, n0, c->dGsrc, n0);
    copy_matrix(c->stream, n0, m, c->dLD, n0, c->dGsrc + n0 * m, n0);
    axpy_matrix(c->stream, n0, m, c->cfg.theta * c->cfg.dt, c->dRD, n0, c->dGsrc + n0 * m, n0);
  }
  if (c->S > 0) copy_matrix(c->stream, n0, c->S, c->dM + m, c->n, c->dGsrc + n0 * 2 * m, n0);
  return EC_OK;
}

ec_status plain_factor(ec_ctx* c) {
  const int64_t n = c->n, n0 = c->n0;
  const int m = c->m;
  EC_TRY(alloc(&c->dZ, (size_t)n0 * n0));
  EC_TRY(alloc(&c->dDinv, (size_t)((n0 + NB - 1) / NB) * NB * NB));
  EventTimer t(c->stream);
  copy_matrix(c->stream, n0, n0, c->dL + m + m * n, n, c->dZ, n0);
  add_lower(c->stream, n0, c->dZ, n0, c->dR + m + m * n, n, c->cfg.theta * c->cfg.dt);
  OzWork* oz = c->cfg.setup_gemm != EC_GEMM_FP64 ? &c->oz : nullptr;
  potrf(c->stream, n0, c->dZ, n0, c->dDinv, c->st, oz);
  if (c->cfg.plain_solver == EC_SOLVE_INVERSE) {
    EC_TRY(alloc(&c->dW, (size_t)n0 * n0));
    EC_TRY(tile_plan_create(n0, &c->tiles));
    const size_t prow = (size_t)tile_partial_rows(c->tiles), npad = (size_t)c->tiles.npad;
    EC_TRY(alloc(&c->dPart1, prow * npad));
    EC_TRY(alloc(&c->dPart2, prow * npad));
    EC_TRY(alloc(&c->dYsol, npad));
    cudaMemsetAsync(c->dYsol, 0, sizeof(double) * npad, c->stream);
    trtri_lower(c->stream, n0, c->dZ, n0, c->dDinv, c->dW, n0, c->st, oz);
    if (c->cfg.precision == EC_PREC_FP32) {
      // FP32 copy of C^{-1} for the solves; the lower half of L (= L_i, no electrodes)
      // in FP64 for the refinement residual.
      EC_TRY(alloc(&c->dWp32, tile_packed_doubles(c->tiles)));
      EC_TRY(alloc(&c->dLh, tile_packed_doubles(c->tiles)));
      for (double** v : {&c->dDelta, &c->dRes, &c->dT1, &c->dT2}) {
        EC_TRY(alloc(v, npad));
        cudaMemsetAsync(*v, 0, sizeof(double) * npad, c->stream);
      }
      EC_TRY(alloc(&c->dV32, npad));
      cudaMemsetAsync(c->dV32, 0, sizeof(float) * npad, c->stream);
      tile_pack_lower_f32(c->stream, c->tiles, c->dW, n0, c->dWp32);
      tile_pack_lower(c->stream, c->tiles, c->dL, c->n, c->dLh, 0.5);
      EC_TRY(tile_autotune_f32(c->stream, &c->tiles, c->dWp32, c->dWork, c->dV32, c->dPart1,
                               c->dYsol, c->dPart2, c->st, c->cfg.tile_variant));
    } else if (c->cfg.precision == EC_PREC_FP32X2) {
      // FP32 hi/lo pairs: as many bytes as FP64, arithmetic on the FP32 pipe
      EC_TRY(alloc(&c->dWpx2, tile_packed_doubles(c->tiles)));
      EC_TRY(alloc(&c->dVx2, npad));
      cudaMemsetAsync(c->dVx2, 0, sizeof(float2) * npad, c->stream);
      tile_pack_lower_x2(c->stream, c->tiles, c->dW, n0, c->dWpx2);
      EC_TRY(tile_autotune_x2(c->stream, &c->tiles, c->dWpx2, c->dWork, c->dVx2, c->dPart1,
                              c->dYsol, c->dPart2, c->st, c->cfg.tile_variant));
    } else {
      EC_TRY(alloc(&c->dWp, tile_packed_doubles(c->tiles)));
      tile_pack_lower(c->stream, c->tiles, c->dW, n0, c->dWp);
      EC_TRY(tile_autotune(c->stream, &c->tiles, c->dWp, c->dWork, c->dPart1, c->dYsol, c->dPart2,
                           c->st, c->cfg.tile_variant));
    }
    c->tim.tile_variant = c->tiles.variant + 1;
    for (int v = 0; v < TILE_VARIANTS && v < 4; ++v) c->tim.tile_tune_ms[v] = c->tiles.tune_ms[v];
  }
  c->tim.factor_ms = t.stop_ms();
  ec_status rc = collect(c);
  oz_free(&c->oz);   // the tensor-core workspace is needed during the factorisation only
  // The per-step products read the packed tiles; the square inverse is kept only
  // for the GEMMs of independent right-hand sides.
  if (rc == EC_OK && c->dW && c->cfg.rhs_mode == EC_RHS_SUM) dfree(c->dW);
  return rc;
}

// x = Z^{-1} b for the plain step, in the context's arithmetic; returns where x is.
//   FP64 inverse factor:  x overwrites b.
//   FP32 inverse factor:  x0 = C^{-T} C^{-1} b in FP32, then refine_steps sweeps
//                         x += C^{-T} C^{-1} (b - Z x) with the residual in FP64;
//                         x is in dDelta, b is kept.
//   substitution:         x overwrites b.
double* plain_solve(ec_ctx* c, const StepArgs& a, double* b, cudaEvent_t* e3) {
  if (c->cfg.plain_solver != EC_SOLVE_INVERSE) {
    TrsvSync sy{c->dFlags, c->dFlags + (c->n0 + NB - 1) / NB, c->dTickets, c->dEpoch};
    trsv_pair(c->stream, c->n0, c->dZ, c->n0, c->dDinv, b, b, b, sy, c->trsv_grid, c->spin_limit,
              c->st, e3);
    return b;
  }
  if (c->cfg.precision == EC_PREC_FP32X2) {
    tile_trmv_pair_x2(c->stream, c->tiles, c->dWpx2, b, c->dVx2, c->dPart1, c->dYsol, c->dPart2,
                      b, c->st, e3);
    return b;
  }
  if (c->cfg.precision != EC_PREC_FP32) {
    tile_trmv_pair(c->stream, c->tiles, c->dWp, b, c->dPart1, c->dYsol, c->dPart2, b, c->st, e3);
    return b;
  }
  tile_trmv_pair_f32(c->stream, c->tiles, c->dWp32, b, c->dV32, c->dPart1, c->dYsol, c->dPart2,
                     c->dDelta, 0, c->st, e3);
  for (int r = 0; r < c->cfg.refine_steps; ++r) {
    tile_sym_product(c->stream, c->tiles, c->dLh, c->dDelta, c->dPart1, c->dPart2, c->dT1, c->dT2,
                     c->st);
    plain_residual(c->stream, a, b, c->dDelta, c->dT1, c->dT2, c->dRes);
    tile_trmv_pair_f32(c->stream, c->tiles, c->dWp32, c->dRes, c->dV32, c->dPart1, c->dYsol,
                       c->dPart2, c->dDelta, 1, c->st);
  }
  return c->dDelta;
}

}  // namespace

extern "C" {

const char* ec_error_string(ec_status s) {
  switch (s) {
    case EC_OK: return "ok";
    case EC_ERR_ARG: return "invalid argument";
    case EC_ERR_SHAPE: return "inconsistent sizes";
    case EC_ERR_NOT_SPD: return "matrix is not symmetric positive definite";
    case EC_ERR_RANK: return "electrode operator E is rank deficient";
    case EC_ERR_OOM: return "device out of memory";
    case EC_ERR_CUDA: return "CUDA runtime error";
    case EC_ERR_TIMEOUT: return "bounded kernel-side wait timed out";
    case EC_ERR_STATE: return "call out of order";
    case EC_ERR_NOT_CONVERGED: return "eigen iteration did not converge";
    case EC_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

ec_status ec_create(ec_ctx** out, const ec_config* cfg) {
  if (!out || !cfg) return EC_ERR_ARG;
  *out = nullptr;
  if (cfg->form != EC_FORM_PLAIN && cfg->form != EC_FORM_MODAL) return EC_ERR_ARG;
  if (cfg->plain_solver != EC_SOLVE_INVERSE && cfg->plain_solver != EC_SOLVE_SUBSTITUTION)
    return EC_ERR_ARG;
  if (cfg->precision != EC_PREC_FP64 && cfg->precision != EC_PREC_BF16 &&
      cfg->precision != EC_PREC_BF16X3 && cfg->precision != EC_PREC_FP32 &&
      cfg->precision != EC_PREC_FP32X2)
    return EC_ERR_ARG;
  if ((cfg->precision == EC_PREC_BF16 || cfg->precision == EC_PREC_BF16X3) &&
      cfg->form != EC_FORM_MODAL)
    return EC_ERR_UNSUPPORTED;
  // plain form: the reduced-precision inverse factor serves the inverse solver of one
  // summed right-hand side; modal form: the products with U, any right-hand-side mode
  if ((cfg->precision == EC_PREC_FP32 || cfg->precision == EC_PREC_FP32X2) &&
      cfg->form == EC_FORM_PLAIN &&
      (cfg->plain_solver != EC_SOLVE_INVERSE || cfg->rhs_mode != EC_RHS_SUM))
    return EC_ERR_UNSUPPORTED;
  if (cfg->refine_steps < 0 || cfg->refine_steps > 8) return EC_ERR_ARG;
  if (cfg->integrator != EC_INTEG_THETA && cfg->integrator != EC_INTEG_EXACT) return EC_ERR_ARG;
  if (cfg->rhs_mode != EC_RHS_SUM && cfg->rhs_mode != EC_RHS_INDEPENDENT &&
      cfg->rhs_mode != EC_RHS_PAIRED)
    return EC_ERR_ARG;
  if (cfg->rhs_mode != EC_RHS_SUM && cfg->form == EC_FORM_PLAIN &&
      cfg->plain_solver != EC_SOLVE_INVERSE)
    return EC_ERR_UNSUPPORTED;
  if (cfg->integrator == EC_INTEG_EXACT && cfg->form != EC_FORM_MODAL) return EC_ERR_UNSUPPORTED;
  if (cfg->tile_variant < 0 || cfg->tile_variant > TILE_VARIANTS) return EC_ERR_ARG;
  if (cfg->setup_gemm != EC_GEMM_TENSOR && cfg->setup_gemm != EC_GEMM_FP64 &&
      cfg->setup_gemm != EC_GEMM_TENSOR_PAIRSYMV)
    return EC_ERR_ARG;
  if (!(cfg->theta >= 0.0 && cfg->theta <= 1.0) || !(cfg->dt > 0.0)) return EC_ERR_ARG;
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    cudaGetLastError();
    return EC_ERR_CUDA;
  }
  ec_ctx* c = new (std::nothrow) ec_ctx();
  if (!c) return EC_ERR_OOM;
  c->cfg = *cfg;
  c->stream = (cudaStream_t)cfg->stream;
  if (cfg->spin_limit > 0) c->spin_limit = cfg->spin_limit;
  if (alloc(&c->st, 1) != EC_OK) {
    delete c;
    return EC_ERR_OOM;
  }
  cudaMemset(c->st, 0, sizeof(DevStatus));
  *out = c;
  return EC_OK;
}

void ec_destroy(ec_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->cfg.device);
  cudaStreamSynchronize(c->stream);
  free_setup(c);
  dfree(c->dSrc); dfree(c->dIDs); dfree(c->dProbes); dfree(c->dSnaps);
  dfree(c->st);
  delete c;
}

int64_t ec_last_info(const ec_ctx* c) { return c ? c->last_info : -1; }

int64_t ec_state_size(const ec_ctx* c) {
  if (!c || !c->ready) return 0;
  return c->cfg.form == EC_FORM_MODAL ? modal_state_size(c->modal) : c->n0 * c->ntraj;
}

ec_status ec_sync(ec_ctx* c) {
  if (!c) return EC_ERR_ARG;
  return collect(c);
}

ec_status ec_timings(ec_ctx* c, ec_timing* out) {
  if (!c || !out) return EC_ERR_ARG;
  *out = c->tim;
  return EC_OK;
}

ec_status ec_setup(ec_ctx* c, int64_t n, const double* L, const double* R, int64_t m,
                   const double* E, int64_t s, const double* M, const double* MD, int64_t p,
                   const double* C, int mem) {
  if (!c || n < 1 || !L || !R || m < 0 || s < 0 || p < 0) return EC_ERR_ARG;
  if ((m > 0 && !E) || (s > 0 && !M) || (p > 0 && !C)) return EC_ERR_ARG;
  if (mem != EC_MEM_HOST && mem != EC_MEM_DEVICE) return EC_ERR_ARG;
  if (m >= n) return EC_ERR_SHAPE;
  if (c->cfg.form == EC_FORM_PLAIN && c->cfg.precision == EC_PREC_FP32 && m > 0)
    return EC_ERR_UNSUPPORTED;
  const bool indep = c->cfg.rhs_mode != EC_RHS_SUM;
  const bool paired = c->cfg.rhs_mode == EC_RHS_PAIRED;
  // (paired read-out computes each trajectory's own probe directly: no per-step dot
  // products, so no limit on the number of coils / probe rows)
  if (m > MAXM || (!indep && s > 64) || (!paired && p + 2 * m > MAXD)) return EC_ERR_UNSUPPORTED;
  if (indep && (m != 0 || s < 1 || s > 65535)) return EC_ERR_UNSUPPORTED;
  if (c->cfg.rhs_mode == EC_RHS_PAIRED && p != s) return EC_ERR_SHAPE;
  cudaSetDevice(c->cfg.device);
  free_setup(c);
  cudaMemsetAsync(c->st, 0, sizeof(DevStatus), c->stream);
  c->last_info = -1;
  c->tim = ec_timing{};
  c->n = n; c->m = (int)m; c->S = (int)s; c->P = (int)p; c->n0 = n - m;
  c->D = paired ? 0 : c->P + 2 * c->m;
  const int64_t n0 = c->n0;
  const size_t nn = (size_t)n * n;
  EventTimer whole(c->stream);

  EC_TRY(alloc(&c->dL, nn));
  EC_TRY(alloc(&c->dR, nn));
  EC_TRY(copy_in(c, c->dL, L, nn, mem));
  EC_TRY(copy_in(c, c->dR, R, nn, mem));
  // row-major lower triangle == column-major upper triangle
  sym_from_upper(c->stream, n, c->dL, n);
  sym_from_upper(c->stream, n, c->dR, n);
  EC_TRY(alloc(&c->dM, (size_t)n * (s > 0 ? s : 1)));
  EC_TRY(alloc(&c->dMD, (size_t)n * (m > 0 ? m : 1)));
  EC_TRY(alloc(&c->dC, (size_t)n * (p > 0 ? p : 1)));
  EC_TRY(copy_in(c, c->dM, M, (size_t)n * s, mem));
  if (m > 0) {
    if (MD) EC_TRY(copy_in(c, c->dMD, MD, (size_t)n * m, mem));
    else cudaMemsetAsync(c->dMD, 0, sizeof(double) * n * m, c->stream);
  }
  EC_TRY(copy_in(c, c->dC, C, (size_t)n * p, mem));
  // NaN or infinite inputs are refused before any factorisation sees them
  finite_check(c->stream, c->dL, (int64_t)nn, 0, c->st);
  finite_check(c->stream, c->dR, (int64_t)nn, 1, c->st);
  finite_check(c->stream, c->dM, (int64_t)n * s, 3, c->st);
  if (m > 0 && MD) finite_check(c->stream, c->dMD, (int64_t)n * m, 4, c->st);
  finite_check(c->stream, c->dC, (int64_t)n * p, 5, c->st);
  EC_TRY(collect(c));

  // CSR of the original R, for the O(nnz) R_i products of the plain step
  {
    ec_status st = build_csr(c->stream, n, c->dR, c->csr, dev_alloc);
    if (st != EC_OK) return st;
  }

  EventTimer te(c->stream);
  const int mm = c->m > 0 ? c->m : 1;
  EC_TRY(alloc(&c->dV, (size_t)n * mm));
  EC_TRY(alloc(&c->dWR, (size_t)n * mm));
  EC_TRY(alloc(&c->dT, (size_t)mm * mm));
  EC_TRY(alloc(&c->dVtWR, (size_t)mm * mm));
  EC_TRY(alloc(&c->dRrinvT, (size_t)mm * mm));
  EC_TRY(alloc(&c->dPE, (size_t)n * mm));
  EC_TRY(alloc(&c->dCPE, (size_t)(p > 0 ? p : 1) * mm));
  EC_TRY(alloc(&c->dRD, (size_t)n0 * mm));
  EC_TRY(alloc(&c->dLD, (size_t)n0 * mm));
  if (m > 0) {
    const int mi = c->m;
    const int64_t wcols = (s > mi ? s : mi) > p ? (s > mi ? s : mi) : p;
    EC_TRY(alloc(&c->dE, (size_t)n * mi));
    EC_TRY(alloc(&c->dY, (size_t)n * mi));
    EC_TRY(alloc(&c->dX, (size_t)n * mi));
    EC_TRY(alloc(&c->dSm, (size_t)mi * (wcols > mi ? wcols : mi)));
    EC_TRY(alloc(&c->dZm, (size_t)mi * (wcols > mi ? wcols : mi)));
    EC_TRY(copy_in(c, c->dE, E, (size_t)n * mi, mem));
    finite_check(c->stream, c->dE, (int64_t)n * mi, 2, c->st);
    EC_TRY(collect(c));
    house_qr(c->stream, n, mi, c->dE, c->dV, c->dT, c->dRrinvT, c->st);
    // WR = R V with the original R, and V^T WR
    dgemm(c->stream, N_, N_, n, mi, n, 1.0, c->dR, n, c->dV, n, 0.0, c->dWR, n, 0, c->st);
    dgemm(c->stream, T_, N_, mi, mi, n, 1.0, c->dV, n, c->dWR, n, 0.0, c->dVtWR, mi, 0, c->st);
    two_sided_update(c->stream, n, mi, c->dL, c->dV, c->dT, c->dY, c->dX, c->dSm, c->dZm, c->st);
    two_sided_update(c->stream, n, mi, c->dR, c->dV, c->dT, c->dY, c->dX, c->dSm, c->dZm, c->st);
    one_sided_qt(c->stream, n, mi, c->dM, s, c->dV, c->dT, c->dSm, c->dZm, c->st);
    one_sided_qt(c->stream, n, mi, c->dMD, mi, c->dV, c->dT, c->dSm, c->dZm, c->st);
    one_sided_qt(c->stream, n, mi, c->dC, p, c->dV, c->dT, c->dSm, c->dZm, c->st);
    // particular field PE = Q [Rr^{-T}; 0]
    cudaMemsetAsync(c->dPE, 0, sizeof(double) * n * mi, c->stream);
    copy_matrix(c->stream, mi, mi, c->dRrinvT, mi, c->dPE, n);
    one_sided_q(c->stream, n, mi, c->dPE, mi, c->dV, c->dT, c->dSm, c->dZm, c->st);
    // C PE = (C'[0:m, :])^T Rr^{-T}  (P x m)
    if (p > 0)
      dgemm(c->stream, T_, N_, p, mi, mi, 1.0, c->dC, n, c->dRrinvT, mi, 0.0, c->dCPE, p, 0, c->st);
    // R_D = R'[m:, 0:m] Rr^{-T},  L_D = L'[m:, 0:m] Rr^{-T} + MD'[m:, :]
    dgemm(c->stream, N_, N_, n0, mi, mi, 1.0, c->dR + mi, n, c->dRrinvT, mi, 0.0, c->dRD, n0, 0, c->st);
    copy_matrix(c->stream, n0, mi, c->dMD + mi, n, c->dLD, n0);
    dgemm(c->stream, N_, N_, n0, mi, mi, 1.0, c->dL + mi, n, c->dRrinvT, mi, 1.0, c->dLD, n0, 0, c->st);
  }
  c->tim.elim_ms = te.stop_ms();
  EC_TRY(collect(c));

  // source columns and dot-product rows
  EC_TRY(alloc(&c->dGsrc, (size_t)n0 * (2 * c->m + c->S > 0 ? 2 * c->m + c->S : 1)));
  EC_TRY(alloc(&c->dDmat, (size_t)n0 * (c->D > 0 ? c->D : 1)));
  form_sources(c);
  if (p > 0 && c->D > 0) copy_matrix(c->stream, n0, p, c->dC + c->m, n, c->dDmat, n0);
  if (m > 0) {
    copy_matrix(c->stream, n0, c->m, c->dV + c->m, n, c->dDmat + n0 * p, n0);
    copy_matrix(c->stream, n0, c->m, c->dWR + c->m, n, c->dDmat + n0 * (p + c->m), n0);
  }
  // state
  c->update_grid = (int)((n0 + 255) / 256);
  if (c->update_grid > num_sms() * 2) c->update_grid = num_sms() * 2;
  if (c->update_grid < 1) c->update_grid = 1;
  c->trsv_grid = num_sms() * 2;
  c->ntraj = indep ? c->S : 1;
  EC_TRY(alloc(&c->dIi, (size_t)n0 * c->ntraj));
  if (indep && c->cfg.form == EC_FORM_PLAIN) {
    EC_TRY(alloc(&c->dRhsM, (size_t)n0 * c->ntraj));
    EC_TRY(alloc(&c->dYM, (size_t)n0 * c->ntraj));
    EC_TRY(alloc(&c->dXM, (size_t)n0 * c->ntraj));
  }
  // padded to whole 64-row tiles with a zero tail (the packed-tile products read
  // their input vector in 64-entry segments)
  const size_t nwork = (size_t)((n0 + NB - 1) / NB) * NB;
  EC_TRY(alloc(&c->dWork, nwork));
  cudaMemsetAsync(c->dWork, 0, sizeof(double) * nwork, c->stream);
  EC_TRY(alloc(&c->dTmpN, (size_t)n));
  EC_TRY(alloc(&c->dDots, (size_t)MAXD));
  EC_TRY(alloc(&c->dPartial, (size_t)c->update_grid * (c->D > 0 ? c->D : 1)));
  EC_TRY(alloc(&c->dCounter, 1));
  EC_TRY(alloc(&c->dK, 1));
  const int64_t nblk = (n0 + NB - 1) / NB;
  EC_TRY(alloc(&c->dFlags, (size_t)2 * nblk));
  EC_TRY(alloc(&c->dTickets, 2));
  EC_TRY(alloc(&c->dEpoch, 1));
  cudaMemsetAsync(c->dIi, 0, sizeof(double) * n0 * c->ntraj, c->stream);
  cudaMemsetAsync(c->dDots, 0, sizeof(double) * MAXD, c->stream);
  cudaMemsetAsync(c->dCounter, 0, sizeof(unsigned), c->stream);
  cudaMemsetAsync(c->dK, 0, sizeof(int64_t), c->stream);
  cudaMemsetAsync(c->dFlags, 0, sizeof(int) * 2 * nblk, c->stream);
  cudaMemsetAsync(c->dTickets, 0, sizeof(unsigned) * 2, c->stream);
  cudaMemsetAsync(c->dEpoch, 0, sizeof(int), c->stream);
  EC_TRY(collect(c));

  if (c->cfg.form == EC_FORM_PLAIN) {
    EC_TRY(plain_factor(c));
  } else {
    c->modal = modal_create();
    if (!c->modal) return EC_ERR_OOM;
    ModalSetupArgs ma{};
    ma.n = n; ma.n0 = n0; ma.m = c->m; ma.S = c->S; ma.P = c->P;
    ma.Li = c->dL + c->m + c->m * n; ma.Ri = c->dR + c->m + c->m * n; ma.ld = n;
    ma.Gsrc = c->dGsrc; ma.RD = c->dRD; ma.LD = c->dLD; ma.Msrc = c->dM + c->m; ma.ldM = n;
    ma.CK = c->dC + c->m; ma.ldC = n;
    ma.theta = c->cfg.theta; ma.dt = c->cfg.dt;
    ma.precision = c->cfg.precision;
    ma.integ = c->cfg.integrator;
    ma.rhs_mode = c->cfg.rhs_mode;
    ma.gemm = c->cfg.setup_gemm;
    ma.st = c->st;
    EC_TRY(modal_setup(c->stream, c->modal, ma, &c->tim));
    EC_TRY(collect(c));
  }
  c->tim.setup_ms = whole.stop_ms();
  c->ready = true;
  if (c->cfg.release_inputs) {
    // stepping reads the factors / modes and the sparse R only
    dfree(c->dL);
    dfree(c->dR);
    if (c->cfg.form == EC_FORM_PLAIN && c->cfg.plain_solver == EC_SOLVE_INVERSE) dfree(c->dZ);
  }
  return EC_OK;
}

ec_status ec_set_step(ec_ctx* c, double theta, double dt) {
  if (!c) return EC_ERR_ARG;
  if (!(theta >= 0.0 && theta <= 1.0) || !(dt > 0.0)) return EC_ERR_ARG;
  if (!c->ready) return EC_ERR_STATE;
  if (c->cfg.form == EC_FORM_PLAIN && (!c->dL || !c->dR)) return EC_ERR_STATE;  // released
  c->cfg.theta = theta;
  c->cfg.dt = dt;
  form_sources(c);
  if (c->cfg.form == EC_FORM_PLAIN) return plain_factor(c);
  EC_TRY(modal_set_step(c->stream, c->modal, theta, dt));
  return collect(c);
}

ec_status ec_set_precision(ec_ctx* c, int precision) {
  if (!c) return EC_ERR_ARG;
  if (precision != EC_PREC_FP64 && precision != EC_PREC_BF16 && precision != EC_PREC_BF16X3 &&
      precision != EC_PREC_FP32 && precision != EC_PREC_FP32X2)
    return EC_ERR_ARG;
  if (!c->ready) return EC_ERR_STATE;
  if (c->cfg.form != EC_FORM_MODAL) return EC_ERR_UNSUPPORTED;
  cudaSetDevice(c->cfg.device);
  const int64_t n = c->n;
  ec_status rc = modal_set_precision(c->stream, c->modal, precision, c->dRD, c->dLD, c->dM + c->m,
                                     n, c->dC + c->m, n, c->st);
  if (rc == EC_OK) rc = collect(c);
  if (rc != EC_OK) {
    // keep a usable context: FP64 products from the same modes
    c->cfg.precision = EC_PREC_FP64;
    modal_set_precision(c->stream, c->modal, EC_PREC_FP64, c->dRD, c->dLD, c->dM + c->m, n,
                        c->dC + c->m, n, c->st);
    cudaStreamSynchronize(c->stream);
    return rc;
  }
  c->cfg.precision = precision;
  return EC_OK;
}

ec_status ec_run(ec_ctx* c, int64_t T, const double* src, const double* iD, double* probes,
                 int64_t stride, double* snaps, int mem) {
  if (!c) return EC_ERR_ARG;
  if (!c->ready) return EC_ERR_STATE;
  if (T < 0 || stride < 0) return EC_ERR_ARG;
  if ((c->S > 0 && !src) || (c->m > 0 && !iD)) return EC_ERR_ARG;
  if (mem != EC_MEM_HOST && mem != EC_MEM_DEVICE) return EC_ERR_ARG;
  cudaSetDevice(c->cfg.device);
  if (T == 0) return EC_OK;
  const int64_t n = c->n;
  const int64_t nsnap = (stride > 0 && snaps) ? T / stride : 0;
  const int64_t nt = c->ntraj;
  const int64_t pout = (c->cfg.rhs_mode == EC_RHS_PAIRED) ? 1 : c->P;
  EC_TRY(grow(&c->dSrc, c->srcCap, (size_t)(c->S > 0 ? c->S : 1) * (T + 1)));
  EC_TRY(grow(&c->dIDs, c->idsCap, (size_t)(c->m > 0 ? c->m : 1) * (T + 1)));
  EC_TRY(copy_in(c, c->dSrc, src, (size_t)c->S * (T + 1), mem));
  EC_TRY(copy_in(c, c->dIDs, iD, (size_t)c->m * (T + 1), mem));
  double* outP = nullptr;
  double* outS = nullptr;
  if (probes && c->P > 0) {
    if (mem == EC_MEM_DEVICE) outP = probes;
    else {
      EC_TRY(grow(&c->dProbes, c->probesCap, (size_t)T * nt * pout));
      outP = c->dProbes;
    }
  }
  if (nsnap > 0) {
    if (mem == EC_MEM_DEVICE) outS = snaps;
    else {
      EC_TRY(grow(&c->dSnaps, c->snapsCap, (size_t)nsnap * nt * n));
      outS = c->dSnaps;
    }
  }
  cudaMemsetAsync(c->dK, 0, sizeof(int64_t), c->stream);
  StepArgs a = step_args(c, T, outP, outS, nsnap > 0 ? stride : 0);
  c->tim.fwd_ms = c->tim.bwd_ms = c->tim.scan_ms = 0.0;
  c->tim.fwd_launches = c->tim.bwd_launches = c->tim.scan_launches = 0;
  std::vector<cudaEvent_t> ev;
  const bool prof = c->cfg.profile != 0;
  EventTimer t(c->stream);
  if (c->cfg.form == EC_FORM_PLAIN && nt > 1 || (c->cfg.form == EC_FORM_PLAIN && c->cfg.rhs_mode != EC_RHS_SUM)) {
    // independent right-hand sides: two GEMMs with the inverse factor per step
    const int64_t n0 = c->n0;
    const int S = (int)nt;
    for (int64_t k = 0; k < T; ++k) {
      plain_rhs_multi(c->stream, a, k, c->dIi, c->dRhsM);
      cudaEvent_t* e3 = nullptr;
      const int64_t every = T > 512 ? (T + 511) / 512 : 1;
      if (prof && k % every == 0) {
        ev.resize(ev.size() + 3);
        e3 = &ev[ev.size() - 3];
        for (int q = 0; q < 3; ++q) cudaEventCreate(&e3[q]);
      }
      if (e3) cudaEventRecord(e3[0], c->stream);
      dgemm(c->stream, N_, N_, n0, S, n0, 1.0, c->dW, n0, c->dRhsM, n0, 0.0, c->dYM, n0, 0, c->st);
      if (e3) cudaEventRecord(e3[1], c->stream);
      dgemm(c->stream, T_, N_, n0, S, n0, 1.0, c->dW, n0, c->dYM, n0, 0.0, c->dXM, n0, 0, c->st);
      if (e3) cudaEventRecord(e3[2], c->stream);
      axpy_matrix(c->stream, n0, S, 1.0, c->dXM, n0, c->dIi, n0);
      if (outP) {
        if (c->cfg.rhs_mode == EC_RHS_PAIRED)
          paired_probes(c->stream, n0, S, c->dC, n, c->dIi, outP + k * S);
        else
          dgemm(c->stream, T_, N_, c->P, S, n0, 1.0, c->dC, n, c->dIi, n0, 0.0,
                outP + k * S * c->P, c->P, 0, c->st);
      }
      if (outS && (k + 1) % stride == 0)
        copy_matrix(c->stream, n0, S, c->dIi, n0, outS + ((k + 1) / stride - 1) * S * n, n);
    }
  } else if (c->cfg.form == EC_FORM_PLAIN) {
    const int64_t every = T > 512 ? (T + 511) / 512 : 1;
    for (int64_t k = 0; k < T; ++k) {
      plain_rhs(c->stream, a);
      cudaEvent_t* e3 = nullptr;
      if (prof && k % every == 0) {
        ev.resize(ev.size() + 3);
        e3 = &ev[ev.size() - 3];
        for (int q = 0; q < 3; ++q) cudaEventCreate(&e3[q]);
      }
      StepArgs au = a;
      au.work = plain_solve(c, a, c->dWork, e3);
      plain_update(c->stream, au, c->update_grid, 0);
      if (outS) plain_snapshot(c->stream, a);
    }
  } else {
    EC_TRY(modal_run(c->stream, c->modal, a, prof ? &ev : nullptr));
  }
  c->tim.run_ms = t.stop_ms();
  c->tim.run_steps = T;
  if (!ev.empty()) {
    cudaStreamSynchronize(c->stream);
    if (c->cfg.form == EC_FORM_PLAIN) {
      for (size_t q = 0; q + 2 < ev.size(); q += 3) {
        float f = 0.f, b = 0.f;
        cudaEventElapsedTime(&f, ev[q], ev[q + 1]);
        cudaEventElapsedTime(&b, ev[q + 1], ev[q + 2]);
        c->tim.fwd_ms += f;
        c->tim.bwd_ms += b;
        ++c->tim.fwd_launches;
        ++c->tim.bwd_launches;
      }
    } else {
      for (size_t q = 0; q + 1 < ev.size(); q += 2) {
        float f = 0.f;
        cudaEventElapsedTime(&f, ev[q], ev[q + 1]);
        c->tim.scan_ms += f;
        ++c->tim.scan_launches;
      }
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  EC_TRY(collect(c));
  if (outP && outP != probes) EC_TRY(copy_out(c, probes, outP, (size_t)T * nt * pout, mem));
  if (outS && outS != snaps) EC_TRY(copy_out(c, snaps, outS, (size_t)nsnap * nt * n, mem));
  return collect(c);
}

ec_status ec_batch_run(ec_ctx* const* ctxs, int count, int64_t T, const double* const* src,
                       const double* const* iD, double* const* probes, int64_t stride,
                       double* const* snaps, int mem) {
  if (!ctxs || count < 1 || count > EC_BATCH_MAX || T < 0 || stride < 0) return EC_ERR_ARG;
  if (mem != EC_MEM_HOST && mem != EC_MEM_DEVICE) return EC_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    const ec_ctx* c = ctxs[i];
    if (!c) return EC_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return EC_ERR_ARG;
    if (!c->ready) return EC_ERR_STATE;
    if (c->cfg.form != EC_FORM_PLAIN || c->cfg.plain_solver != EC_SOLVE_INVERSE ||
        c->cfg.rhs_mode != EC_RHS_SUM || c->cfg.precision != EC_PREC_FP64)
      return EC_ERR_UNSUPPORTED;
    if (c->cfg.device != ctxs[0]->cfg.device) return EC_ERR_ARG;
    if ((c->S > 0 && (!src || !src[i])) || (c->m > 0 && (!iD || !iD[i]))) return EC_ERR_ARG;
  }
  if (T == 0) return EC_OK;
  cudaSetDevice(ctxs[0]->cfg.device);
  // Earlier work of every instance completes before the batch starts.
  for (int i = 0; i < count; ++i)
    if (cudaStreamSynchronize(ctxs[i]->stream) != cudaSuccess) return EC_ERR_CUDA;

  std::vector<StepArgs> args(count);
  std::vector<TileInst> inst(count);
  std::vector<double*> outP(count, nullptr), outS(count, nullptr);
  int64_t max_n0 = 0, max_n = 0;
  int max_ugrid = 1;
  bool any_snaps = false;
  for (int i = 0; i < count; ++i) {
    ec_ctx* c = ctxs[i];
    const int64_t nsnap = (stride > 0 && snaps && snaps[i]) ? T / stride : 0;
    EC_TRY(grow(&c->dSrc, c->srcCap, (size_t)(c->S > 0 ? c->S : 1) * (T + 1)));
    EC_TRY(grow(&c->dIDs, c->idsCap, (size_t)(c->m > 0 ? c->m : 1) * (T + 1)));
    EC_TRY(copy_in(c, c->dSrc, c->S > 0 ? src[i] : nullptr, (size_t)c->S * (T + 1), mem));
    EC_TRY(copy_in(c, c->dIDs, c->m > 0 ? iD[i] : nullptr, (size_t)c->m * (T + 1), mem));
    if (probes && probes[i] && c->P > 0) {
      if (mem == EC_MEM_DEVICE) outP[i] = probes[i];
      else {
        EC_TRY(grow(&c->dProbes, c->probesCap, (size_t)T * c->P));
        outP[i] = c->dProbes;
      }
    }
    if (nsnap > 0) {
      if (mem == EC_MEM_DEVICE) outS[i] = snaps[i];
      else {
        EC_TRY(grow(&c->dSnaps, c->snapsCap, (size_t)nsnap * c->n));
        outS[i] = c->dSnaps;
      }
      any_snaps = true;
    }
    cudaMemsetAsync(c->dK, 0, sizeof(int64_t), c->stream);
    args[i] = step_args(c, T, outP[i], outS[i], nsnap > 0 ? stride : 0);
    inst[i] = TileInst{&c->tiles, c->dWp, c->dWork, c->dPart1, c->dYsol, c->dPart2, c->dWork};
    max_n0 = std::max(max_n0, c->n0);
    max_n = std::max(max_n, c->n);
    max_ugrid = std::max(max_ugrid, c->update_grid);
  }
  for (int i = 0; i < count; ++i)
    if (cudaStreamSynchronize(ctxs[i]->stream) != cudaSuccess) return EC_ERR_CUDA;

  cudaStream_t st = nullptr;
  StepArgs* dA = nullptr;
  DevStatus* bst = nullptr;
  TileBatch B;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ec_status rc = EC_OK;
  auto release = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    tile_batch_free(&B);
    dfree(dA);
    dfree(bst);
    if (st) cudaStreamDestroy(st);
  };
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return EC_ERR_CUDA;
  if ((rc = alloc(&dA, (size_t)count)) || (rc = alloc(&bst, 1))) {
    release();
    return rc;
  }
  if (cudaMemcpy(dA, args.data(), sizeof(StepArgs) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(bst, 0, sizeof(DevStatus)) != cudaSuccess) {
    release();
    return EC_ERR_CUDA;
  }
  // One work list over every instance's tile units; launch shape tuned on the batch.
  if ((rc = tile_batch_create(inst.data(), count, &B)) ||
      (rc = tile_batch_autotune(st, &B, inst.data(), bst))) {
    release();
    return rc;
  }
  // One step of all instances, captured once and replayed T times.
  const int64_t launches0 = ec::g_launches.load(std::memory_order_relaxed);
  tile_prepare_launches();
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    release();
    return EC_ERR_CUDA;
  }
  plain_rhs_batch(st, dA, count, max_n0);
  tile_batch_pair(st, B, inst.data(), bst);
  plain_update_batch(st, dA, count, max_ugrid);
  if (any_snaps) plain_snapshot_batch(st, dA, count, max_n);
  const cudaError_t ce = cudaStreamEndCapture(st, &graph);
  const int64_t per_step = ec::g_launches.load(std::memory_order_relaxed) - launches0;
  if (ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    release();
    return EC_ERR_CUDA;
  }
  EventTimer t(st);
  for (int64_t k = 0; k < T; ++k)
    if (cudaGraphLaunch(exec, st) != cudaSuccess) {
      rc = EC_ERR_CUDA;
      break;
    }
  const double ms = t.stop_ms();
  // the capture counted one step's launches; the replays ran T steps
  ec::g_launches.fetch_add(per_step * (T - 1), std::memory_order_relaxed);
  if (cudaStreamSynchronize(st) != cudaSuccess) rc = EC_ERR_CUDA;
  DevStatus h{};
  if (rc == EC_OK && cudaMemcpy(&h, bst, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = EC_ERR_CUDA;
  if (rc == EC_OK && h.code != 0) {
    ctxs[0]->last_info = h.info;
    rc = (ec_status)h.code;
  }
  for (int i = 0; i < count && rc == EC_OK; ++i) {
    ec_ctx* c = ctxs[i];
    c->tim.run_ms = ms;
    c->tim.run_steps = T;
    rc = collect(c);
    const int64_t nsnap = outS[i] ? T / stride : 0;
    if (rc == EC_OK && outP[i] && outP[i] != probes[i])
      rc = copy_out(c, probes[i], outP[i], (size_t)T * c->P, mem);
    if (rc == EC_OK && outS[i] && outS[i] != snaps[i])
      rc = copy_out(c, snaps[i], outS[i], (size_t)nsnap * c->n, mem);
    if (rc == EC_OK) rc = collect(c);
  }
  release();
  return rc;
}

ec_status ec_get_state(ec_ctx* c, double* state, int mem) {
  if (!c || !state) return EC_ERR_ARG;
  if (!c->ready) return EC_ERR_STATE;
  const double* src = c->cfg.form == EC_FORM_PLAIN ? c->dIi : modal_state(c->modal);
  EC_TRY(copy_out(c, state, src, (size_t)ec_state_size(c), mem));
  return collect(c);
}

ec_status ec_set_state(ec_ctx* c, const double* state, int mem) {
  if (!c || !state) return EC_ERR_ARG;
  if (!c->ready) return EC_ERR_STATE;
  if (c->cfg.form == EC_FORM_PLAIN) {
    EC_TRY(copy_in(c, c->dIi, state, (size_t)ec_state_size(c), mem));
    if (c->ntraj == 1) {
      StepArgs a = step_args(c, 0, nullptr, nullptr, 0);
      plain_update(c->stream, a, c->update_grid, 1);
    }
  } else {
    EC_TRY(copy_in(c, modal_state(c->modal), state, (size_t)ec_state_size(c), mem));
  }
  return collect(c);
}

ec_status ec_set_current(ec_ctx* c, const double* I, int mem) {
  if (!c || !I) return EC_ERR_ARG;
  if (!c->ready) return EC_ERR_STATE;
  EC_TRY(copy_in(c, c->dTmpN, I, (size_t)c->n, mem));
  if (c->m > 0)
    one_sided_qt(c->stream, c->n, c->m, c->dTmpN, 1, c->dV, c->dT, c->dSm, c->dZm, c->st);
  if (c->cfg.form == EC_FORM_PLAIN) {
    for (int64_t r = 0; r < c->ntraj; ++r)
      copy_matrix(c->stream, c->n0, 1, c->dTmpN + c->m, c->n, c->dIi + r * c->n0, c->n0);
    StepArgs a = step_args(c, 0, nullptr, nullptr, 0);
    if (c->ntraj == 1) plain_update(c->stream, a, c->update_grid, 1);
  } else {
    copy_matrix(c->stream, c->n0, 1, c->dTmpN + c->m, c->n, c->dIi, c->n0);
    StepArgs a = step_args(c, 0, nullptr, nullptr, 0);
    plain_update(c->stream, a, c->update_grid, 1);
    ri_apply(c->stream, a, c->dWork);
    modal_set_internal_current(c->stream, c->modal, c->dWork);
  }
  return collect(c);
}

ec_status ec_get_modes(ec_ctx* c, double* tau, double* U, int mem) {
  if (!c) return EC_ERR_ARG;
  if (!c->ready || c->cfg.form != EC_FORM_MODAL) return EC_ERR_STATE;
  if (tau) EC_TRY(copy_out(c, tau, modal_tau(c->modal), (size_t)c->n0, mem));
  if (U) EC_TRY(copy_out(c, U, modal_U(c->modal), (size_t)c->n0 * c->n0, mem));
  return collect(c);
}

ec_status ec_solve_z(ec_ctx* c, const double* b, double* x, int mem) {
  if (!c || !b || !x) return EC_ERR_ARG;
  if (!c->ready || c->cfg.form != EC_FORM_PLAIN) return EC_ERR_STATE;
  if (mem != EC_MEM_HOST && mem != EC_MEM_DEVICE) return EC_ERR_ARG;
  cudaSetDevice(c->cfg.device);
  const int64_t n0 = c->n0;
  EC_TRY(copy_in(c, c->dWork, b, (size_t)n0, mem));
  if (c->cfg.plain_solver != EC_SOLVE_INVERSE) {
    TrsvSync sy{c->dFlags, c->dFlags + (n0 + NB - 1) / NB, c->dTickets, c->dEpoch};
    trsv_begin(c->stream, sy);
  }
  const double* out = plain_solve(c, step_args(c, 0, nullptr, nullptr, 0), c->dWork, nullptr);
  EC_TRY(copy_out(c, x, out, (size_t)n0, mem));
  return collect(c);
}

ec_status ec_get_inverse_factor(ec_ctx* c, double* W, int mem) {
  if (!c || !W) return EC_ERR_ARG;
  if (!c->ready || c->cfg.form != EC_FORM_PLAIN || c->cfg.plain_solver != EC_SOLVE_INVERSE)
    return EC_ERR_STATE;
  if (c->cfg.precision != EC_PREC_FP64) return EC_ERR_UNSUPPORTED;
  if (c->dW) {
    EC_TRY(copy_out(c, W, c->dW, (size_t)c->n0 * c->n0, mem));
    return collect(c);
  }
  // Square form from the packed tiles.
  if (mem == EC_MEM_DEVICE) {
    tile_unpack_lower(c->stream, c->tiles, c->dWp, W, c->n0);
    return collect(c);
  }
  double* tmp = nullptr;
  EC_TRY(alloc(&tmp, (size_t)c->n0 * c->n0));
  tile_unpack_lower(c->stream, c->tiles, c->dWp, tmp, c->n0);
  ec_status rc = copy_out(c, W, tmp, (size_t)c->n0 * c->n0, mem);
  if (rc == EC_OK) rc = collect(c);
  cudaStreamSynchronize(c->stream);
  dfree(tmp);
  return rc;
}

ec_status ec_grad(ec_ctx* c, int64_t T, const double* src, const double* v, int64_t ckpt,
                   double* J, double* dJ_dRdiag, double* dJ_dsrc, int mem) {
  if (!c || T < 1 || !v || ckpt < 1) return EC_ERR_ARG;
  if (mem != EC_MEM_HOST && mem != EC_MEM_DEVICE) return EC_ERR_ARG;
  if (!c->ready || c->cfg.form != EC_FORM_PLAIN) return EC_ERR_STATE;
  if (c->m != 0 || c->P < 1 || c->cfg.plain_solver != EC_SOLVE_INVERSE ||
      c->cfg.precision != EC_PREC_FP64)
    return EC_ERR_UNSUPPORTED;
  if (c->S > 0 && !src) return EC_ERR_ARG;
  cudaSetDevice(c->cfg.device);
  const int64_t n = c->n0;
  const int S = c->S, P = c->P;
  const double dt = c->cfg.dt, theta = c->cfg.theta;
  if (ckpt > T) ckpt = T;
  const int64_t nseg = (T + ckpt - 1) / ckpt;
  double *probes = nullptr, *vd = nullptr, *ck = nullptr, *seg = nullptr, *mu = nullptr;
  double *gR = nullptr, *lamA = nullptr, *lamB = nullptr, *rhs = nullptr, *fin = nullptr;
  double *Jd = nullptr, *gs = nullptr, *part = nullptr;
  const int grid = c->update_grid;
  auto release = [&]() {
    dfree(probes); dfree(vd); dfree(ck); dfree(seg); dfree(mu); dfree(gR); dfree(lamA);
    dfree(lamB); dfree(rhs); dfree(fin); dfree(Jd); dfree(gs); dfree(part);
  };
  ec_status rc = EC_OK;
  if ((rc = alloc(&probes, (size_t)T * P)) || (rc = alloc(&vd, (size_t)T * P)) ||
      (rc = alloc(&ck, (size_t)n * (nseg + 1))) || (rc = alloc(&seg, (size_t)n * (ckpt + 1))) ||
      (rc = alloc(&mu, (size_t)(S > 0 ? S : 1) * (T + 2))) || (rc = alloc(&gR, (size_t)n)) ||
      (rc = alloc(&lamA, (size_t)n)) || (rc = alloc(&lamB, (size_t)n)) ||
      (rc = alloc(&rhs, (size_t)c->tiles.npad)) || (rc = alloc(&fin, (size_t)n)) || (rc = alloc(&Jd, 1)) ||
      (rc = alloc(&gs, (size_t)(S > 0 ? S : 1) * (T + 1))) ||
      (rc = alloc(&part, (size_t)grid * (S > 0 ? S : 1)))) {
    release();
    return rc;
  }
  cudaStream_t st = c->stream;
  if ((rc = grow(&c->dSrc, c->srcCap, (size_t)(S > 0 ? S : 1) * (T + 1))) ||
      (rc = grow(&c->dIDs, c->idsCap, (size_t)(T + 1))) ||
      (rc = copy_in(c, c->dSrc, src, (size_t)S * (T + 1), mem)) ||
      (rc = copy_in(c, vd, v, (size_t)T * P, mem))) {
    release();
    return rc;
  }
  cudaMemsetAsync(mu, 0, sizeof(double) * (S > 0 ? S : 1) * (T + 2), st);
  cudaMemsetAsync(gR, 0, sizeof(double) * n, st);
  cudaMemsetAsync(lamA, 0, sizeof(double) * n, st);
  cudaMemsetAsync(lamB, 0, sizeof(double) * n, st);
  cudaMemsetAsync(rhs, 0, sizeof(double) * c->tiles.npad, st);
  // forward pass with checkpoints every ckpt steps
  cudaMemsetAsync(c->dK, 0, sizeof(int64_t), st);
  copy_matrix(st, n, 1, c->dIi, n, ck, n);
  StepArgs a = step_args(c, T, probes, nullptr, 0);
  for (int64_t k = 0; k < T; ++k) {
    plain_rhs(st, a);
    tile_trmv_pair(st, c->tiles, c->dWp, c->dWork, c->dPart1, c->dYsol, c->dPart2, c->dWork,
                   c->st);
    plain_update(st, a, c->update_grid, 0);
    if ((k + 1) % ckpt == 0) copy_matrix(st, n, 1, c->dIi, n, ck + ((k + 1) / ckpt) * n, n);
  }
  copy_matrix(st, n, 1, c->dIi, n, fin, n);
  misfit(st, T * P, probes, vd, Jd);
  // backward pass, segment by segment, recomputing the segment's states
  StepArgs ar = step_args(c, T, nullptr, nullptr, 0);
  double* lam_next = lamA;
  double* lam = lamB;
  for (int64_t sg = nseg - 1; sg >= 0; --sg) {
    const int64_t k0 = sg * ckpt, k1 = (k0 + ckpt < T) ? k0 + ckpt : T;
    copy_matrix(st, n, 1, ck + sg * n, n, c->dIi, n);
    copy_matrix(st, n, 1, ck + sg * n, n, seg, n);
    plain_update(st, ar, c->update_grid, 1);
    cudaMemcpyAsync(c->dK, &k0, sizeof(int64_t), cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);   // k0 lives on the host stack
    for (int64_t k = k0; k < k1; ++k) {
      plain_rhs(st, ar);
      tile_trmv_pair(st, c->tiles, c->dWp, c->dWork, c->dPart1, c->dYsol, c->dPart2, c->dWork,
                   c->st);
      plain_update(st, ar, c->update_grid, 0);
      copy_matrix(st, n, 1, c->dIi, n, seg + (k - k0 + 1) * n, n);
    }
    for (int64_t k = k1; k > k0; --k) {
      adj_rhs(st, n, P, dt, c->csr, lam_next, rhs, probes + (k - 1) * P, vd + (k - 1) * P, c->dC);
      tile_trmv_pair(st, c->tiles, c->dWp, rhs, c->dPart1, c->dYsol, c->dPart2, lam, c->st);
      adj_accum(st, n, S, dt, theta, lam, seg + (k - k0) * n, seg + (k - k0 - 1) * n, gR, c->dM,
                part, c->dCounter, mu + k, T + 2, grid);
      double* t = lam_next;
      lam_next = lam;
      lam = t;
    }
  }
  (void)lam;
  // dJ/ds^j = mu^{j+1} - mu^j (mu is S x (T+2), zero at both ends)
  if (S > 0) dsrc(st, S, T, mu, gs);
  // restore the end-of-forward state
  copy_matrix(st, n, 1, fin, n, c->dIi, n);
  plain_update(st, ar, c->update_grid, 1);
  rc = collect(c);
  if (rc == EC_OK && J) rc = copy_out(c, J, Jd, 1, mem);
  if (rc == EC_OK && dJ_dRdiag) rc = copy_out(c, dJ_dRdiag, gR, (size_t)n, mem);
  if (rc == EC_OK && dJ_dsrc && S > 0) rc = copy_out(c, dJ_dsrc, gs, (size_t)S * (T + 1), mem);
  if (rc == EC_OK) rc = collect(c);
  release();
  return rc;
}

ec_status ec_set_mode_count(ec_ctx* c, int64_t n_keep) {
  if (!c) return EC_ERR_ARG;
  if (!c->ready || c->cfg.form != EC_FORM_MODAL) return EC_ERR_STATE;
  EC_TRY(modal_set_mode_count(c->stream, c->modal, n_keep));
  return collect(c);
}

int64_t ec_launch_count(void) { return ec::g_launches.load(std::memory_order_relaxed); }

ec_status ec_selftest_wait_timeout(long long spin_limit, int* code_out) {
  if (!code_out || spin_limit < 1) return EC_ERR_ARG;
  DevStatus* st = nullptr;
  int* flag = nullptr;
  if (dev_alloc((void**)&st, sizeof(DevStatus)) != cudaSuccess) return EC_ERR_OOM;
  if (dev_alloc((void**)&flag, sizeof(int)) != cudaSuccess) {
    cudaFree(st);
    return EC_ERR_OOM;
  }
  cudaMemset(st, 0, sizeof(DevStatus));
  cudaMemset(flag, 0, sizeof(int));
  wait_timeout_probe(0, flag, spin_limit, st);
  cudaError_t e = cudaDeviceSynchronize();
  DevStatus h{};
  if (e == cudaSuccess) e = cudaMemcpy(&h, st, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(st);
  cudaFree(flag);
  if (e != cudaSuccess) return cuda_status(e);
  *code_out = h.code;
  return EC_OK;
}

ec_status ec_selftest_fail_alloc(int64_t after) {
  ec::g_fail_alloc_after.store(after < 0 ? -1 : (long long)after);
  return EC_OK;
}

}  // extern "C"
