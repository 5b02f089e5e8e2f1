// Forward and backward solve with an explicitly inverted Cholesky factor.
//
// The plain form solves C y = b and C^T x = y every step (Sec. 3.3.1) with the
// same factor C for all steps.  A substitution is a chain of NB dependent
// block solves; on GB300 each link costs a few microseconds of latency while
// the arithmetic of a whole solve at N = 8192 is ~50 us, so the chain, not the
// FP64 pipe, sets the pace.  Inverting C once at setup (W = C^{-1}, N^3/3
// extra flops, amortised over every step) turns both solves into triangular
// matrix-vector products y = W b and x = W^T y: the same N^2/2 multiply-adds
// per solve, but every 64 x 64 tile is independent.
//
// Each product is split over (row block, column chunk) CTAs; the chunk
// partial sums are written out and summed in a fixed order by the consumer
// (the next product, or the update kernel), so results are deterministic.

#include <mutex>

#include "ec_internal.h"

namespace ec {

namespace {

__global__ void set_identity_blocks_kernel(int64_t n, double* W, int64_t ldw) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    W[i + i * ldw] = 1.0;
}

// partial[c * n + i] = sum over tiles J in chunk c (J <= I) of W[I, J] b[J]
__global__ void __launch_bounds__(256) trmv_lower_kernel(int64_t n, const double* W, int64_t ldw,
                                                         const double* b, double* partial,
                                                         int chunk, const DevStatus* st) {
  if (*(volatile const int*)&st->code) return;
  const int64_t I = blockIdx.x;
  const int64_t J0 = (int64_t)blockIdx.y * chunk;   // chunks past the diagonal write zeros
  int64_t J1 = J0 + chunk;
  if (J1 > I + 1) J1 = I + 1;
  const int tid = threadIdx.x;
  const int r = tid & 63, cg = tid >> 6;
  const int64_t row = I * NB + r;
  __shared__ double red[4][NB];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  if (row < n) {
    for (int64_t J = J0; J < J1; ++J) {
      const int64_t c0 = J * NB + cg * 16;
      const double* Wp = W + row + c0 * ldw;
      double w[16], v[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const bool ok = (c0 + c) < n;
        w[c] = ok ? Wp[c * ldw] : 0.0;
        v[c] = ok ? b[c0 + c] : 0.0;
      }
#pragma unroll
      for (int c = 0; c < 16; c += 4) {
        a0 = fma(w[c], v[c], a0);
        a1 = fma(w[c + 1], v[c + 1], a1);
        a2 = fma(w[c + 2], v[c + 2], a2);
        a3 = fma(w[c + 3], v[c + 3], a3);
      }
    }
  }
  red[cg][r] = (a0 + a1) + (a2 + a3);
  __syncthreads();
  if (tid < NB && I * NB + tid < n)
    partial[blockIdx.y * n + I * NB + tid] =
        (red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]);
}

// x = W^T y with y given as nin partial vectors (summed here):
// partial_out[c * n + j] = sum over tiles I in chunk c (I >= J) of W[I, J]^T y[I]
__global__ void sum_partials_kernel(int64_t n, int nin, const double* part, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int q = 0; q < nin; ++q) v += part[q * n + i];
    out[i] = v;
  }
}

__global__ void __launch_bounds__(256) trmv_lower_t_kernel(int64_t n, const double* W, int64_t ldw,
                                                           const double* y, double* partial,
                                                           int chunk, const DevStatus* st) {
  if (*(volatile const int*)&st->code) return;
  const int64_t J = blockIdx.x;
  const int64_t nblk = (n + NB - 1) / NB;
  const int64_t I0 = J + (int64_t)blockIdx.y * chunk;   // chunks past the end write zeros
  int64_t I1 = I0 + chunk;
  if (I1 > nblk) I1 = nblk;
  const int tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5;   // warp w: columns w*8 .. w*8+7 of the tile
  __shared__ double red[NB];
  double acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = 0.0;
  const int64_t col0 = J * NB + w * 8;
  for (int64_t I = I0; I < I1; ++I) {
    const int64_t r0 = I * NB + lane, r1 = r0 + 32;
    const double y0 = (r0 < n) ? y[r0] : 0.0;
    const double y1 = (r1 < n) ? y[r1] : 0.0;
    double w0[8], w1[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const bool okc = (col0 + c) < n;
      w0[c] = (okc && r0 < n) ? W[r0 + (col0 + c) * ldw] : 0.0;
      w1[c] = (okc && r1 < n) ? W[r1 + (col0 + c) * ldw] : 0.0;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = fma(w1[c], y1, fma(w0[c], y0, acc[c]));
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    double v = acc[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[w * 8 + c] = v;
  }
  __syncthreads();
  if (tid < NB && J * NB + tid < n) partial[blockIdx.y * n + J * NB + tid] = red[tid];
}

}  // namespace

void trtri_lower(cudaStream_t s, int64_t n, const double* C, int64_t ldc, const double* Dinv,
                 double* W, int64_t ldw, const DevStatus* st, OzWork* oz) {
  // W = C^{-1}: forward block substitution on the identity, touching only the
  // columns that can be non-zero (W is lower triangular).
  cudaMemsetAsync(W, 0, sizeof(double) * (size_t)ldw * n, s);
  set_identity_blocks_kernel<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256,
                               0, ::ec::counted(s)>>>(n, W, ldw);
  // two-level blocking as in the triangular solves: rank-64 steps inside each 192-row
  // panel, one rank-192 update of the rows below it
  constexpr int64_t PW = 192;
  for (int64_t k0 = 0; k0 < n; k0 += PW) {
    const int64_t pe = (k0 + PW) < n ? (k0 + PW) : n;
    for (int64_t k = k0; k < pe; k += NB) {
      const int kb = (int)((n - k) < NB ? (n - k) : NB);
      const int64_t ncols = k + kb;
      const double* Dk = Dinv + (k / NB) * NB * NB;
      double* Wk = W + k;
      gemm_auto(s, oz, N_, N_, kb, ncols, kb, 1.0, Dk, NB, Wk, ldw, 0.0, Wk, ldw, 0, st);
      const int64_t inner = pe - k - kb;
      if (inner > 0)
        gemm_auto(s, oz, N_, N_, inner, ncols, kb, -1.0, C + (k + kb) + k * ldc, ldc, Wk, ldw,
                  1.0, W + k + kb, ldw, 0, st);
    }
    const int64_t rest = n - pe;
    if (rest > 0)   // W[pe:, 0:pe] -= C[pe:, k0:pe] W[k0:pe, 0:pe]
      gemm_auto(s, oz, N_, N_, rest, pe, pe - k0, -1.0, C + pe + k0 * ldc, ldc, W + k0, ldw, 1.0,
                W + pe, ldw, 0, st);
  }
}

int trmv_chunks(int64_t n, int chunk) {
  const int64_t nblk = (n + NB - 1) / NB;
  return (int)((nblk + chunk - 1) / chunk);
}

void sum_partials(cudaStream_t s, int64_t n, int nin, const double* part, double* out) {
  sum_partials_kernel<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0,
                        ::ec::counted(s)>>>(n, nin, part, out);
}

void trmv_pair(cudaStream_t s, int64_t n, const double* W, int64_t ldw, const double* b,
               double* part1, double* y, double* part2, int chunk, const DevStatus* st,
               cudaEvent_t* ev) {
  const int64_t nblk = (n + NB - 1) / NB;
  const int nc = trmv_chunks(n, chunk);
  if (ev) cudaEventRecord(ev[0], s);
  trmv_lower_kernel<<<dim3((unsigned)nblk, (unsigned)nc), 256, 0, ::ec::counted(s)>>>(
      n, W, ldw, b, part1, chunk, st);
  sum_partials_kernel<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0,
                        ::ec::counted(s)>>>(n, nc, part1, y);
  if (ev) cudaEventRecord(ev[1], s);
  trmv_lower_t_kernel<<<dim3((unsigned)nblk, (unsigned)nc), 256, 0, ::ec::counted(s)>>>(
      n, W, ldw, y, part2, chunk, st);
  if (ev) cudaEventRecord(ev[2], s);
}

}  // namespace ec

// ---------------------------------------------------------------------------
// Allocation-free variant of the inverse-factor solve (ec_solve_inverse_noalloc).
//
// Its scratch (status block, chunk partial sums of both products and the
// intermediate vector) lives in one file-scope device array sized for
// n <= EC_NOALLOC_MAX_N.  Every GPU that loads this library holds the array
// (about 1.1 MB) until the process exits.
namespace ec {
namespace {

constexpr int NOALLOC_CHUNK = 16;
constexpr int64_t NOALLOC_MAX_CHUNKS = ((EC_NOALLOC_MAX_N + NB - 1) / NB + NOALLOC_CHUNK - 1) / NOALLOC_CHUNK;
constexpr int64_t NOALLOC_HEAD = 32;   // doubles reserved for the status block (256 B)
constexpr int64_t NOALLOC_DOUBLES =
    NOALLOC_HEAD + 2 * NOALLOC_MAX_CHUNKS * EC_NOALLOC_MAX_N + EC_NOALLOC_MAX_N;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
unsigned long long g_noalloc_ctx[NOALLOC_MAX_DEVICES] = {};

// Unique id of the current CUDA context (cuCtxGetId, resolved through the runtime's
// driver entry-point query so the library needs no link against libcuda).  A
// cudaDeviceReset replaces the device's primary context, and the new one has a new
// id.  Returns 0 when the id is unavailable.
unsigned long long current_context_id() {
  typedef int (*GetCurrentFn)(void**);
  typedef int (*GetIdFn)(void*, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrentFn)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = (GetIdFn)p;
    cudaGetLastError();
  });
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array on the current device, with that device
// current (host code cannot use the symbol itself).  Set up once per device and
// context: the address is looked up on the first call on a device and again after
// the device's context has been replaced (cudaDeviceReset), since the array may then
// sit at another address.  Without a context id the lookup is repeated every call.
ec_status noalloc_scratch(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    cudaGetLastError();
    return EC_ERR_CUDA;
  }
  // before the first runtime call that needs the device, no context may be current
  // yet (id 0): the lookup below creates it, and the id is read again afterwards
  unsigned long long ctx_id = current_context_id();
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev] || ctx_id == 0 || g_noalloc_ctx[dev] != ctx_id) {
    double* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      g_noalloc_ptr[dev] = nullptr;
      return EC_ERR_CUDA;
    }
    if (ctx_id == 0) ctx_id = current_context_id();
    g_noalloc_ptr[dev] = p;
    g_noalloc_ctx[dev] = ctx_id;
  }
  *out = g_noalloc_ptr[dev];
  return EC_OK;
}

}  // namespace
}  // namespace ec

extern "C" ec_status ec_solve_inverse_noalloc(int64_t n, const double* Winv, int64_t ldw,
                                              const double* b, double* x, void* stream) {
  using namespace ec;
  if (!Winv || !b || !x || n < 1 || ldw < n) return EC_ERR_ARG;
  if (n > EC_NOALLOC_MAX_N) return EC_ERR_SHAPE;
  double* base = nullptr;
  ec_status st = noalloc_scratch(&base);
  if (st != EC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  DevStatus* dst = reinterpret_cast<DevStatus*>(base);
  const int nc = trmv_chunks(n, NOALLOC_CHUNK);
  double* part1 = base + NOALLOC_HEAD;
  double* y = part1 + (int64_t)nc * n;
  double* part2 = y + n;
  if (cudaMemsetAsync(dst, 0, sizeof(DevStatus), s) != cudaSuccess) {
    cudaGetLastError();
    return EC_ERR_CUDA;
  }
  trmv_pair(s, n, Winv, ldw, b, part1, y, part2, NOALLOC_CHUNK, dst);
  sum_partials(s, n, nc, part2, x);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? EC_OK : EC_ERR_CUDA;
}

