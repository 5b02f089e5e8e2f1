// Inverse-factor products y = W b and x = W^T y on packed lower-triangular tiles.
//
// The plain form solves with the same factor every step (Sec. 3.3.1); with
// W = C^{-1} both solves are triangular matrix-vector products.  On GB300 an SM
// retires two FP64 FMAs per clock, so a 64 x 64 tile costs 2048 SM-cycles of
// FP64 work and ~5 TB/s of HBM traffic keeps every FP64 pipe busy: the products
// are FP64-bound, and the kernel's job is to keep the FP64 pipe fed.
//
// Design:
//   * W lives as packed 64 x 64 tiles (lower triangle only: half the bytes of
//     the square array), each tile 32 KB contiguous, XOR-swizzled inside so
//     that both the row-wise and the column-wise product read shared memory
//     without bank conflicts;
//   * one CTA per SM, persistent: a producer lane streams tiles (and the 64
//     matching vector entries) into a shared-memory ring with bulk asynchronous
//     copies completing on mbarriers; eight consumer warps work on the tiles;
//   * work is split into units (a run of `chunk` tiles of one tile row, or one
//     tile column), ordered largest first and dealt round-robin to the CTAs, so
//     every SM gets the same FP64 work to within one unit;
//   * each warp owns 8 output rows (forward) or 8 output columns (transposed) of
//     a unit; lanes split the other index, partial sums are reduced with
//     shuffles and written per unit, then summed in a fixed order: results are
//     bitwise deterministic and independent of the grid size.
// Every mbarrier wait is bounded; a wait that runs out records EC_ERR_TIMEOUT.

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "ec_async.cuh"
#include "ec_tiles.h"

namespace ec {

namespace {

constexpr int TB = 64;
constexpr int TILE_DBL = TB * TB;   // entries of a tile
constexpr long long WAIT_LIMIT = 1ll << 26;
constexpr int CW = 8;   // consumer warps: 2 output halves x 4 quarters of the inner index
constexpr int F_FIRST = 1, F_LAST = 2, F_END = 4;

// What the consumers need of a stage: where the unit's partial rows go.
struct Meta {
  double* out;       // partial row 4c of the unit, offset to the unit's 64 outputs
  int64_t npad;      // stride between partial rows
  int flags;
};

template <int ST, typename WT>
struct Smem {
  WT W[ST][TILE_DBL];
  WT v[ST][TB];        // the 64 vector entries the tile multiplies (same type as the factor)
  uint64_t full[ST], empty[ST];
  Meta meta[ST];
};
template <int ST, typename WT>
constexpr size_t smem_bytes() {
  return sizeof(Smem<ST, WT>) + 128;   // + alignment slack
}

// One instance of the products (NI of them per launch, passed by value).
struct TileDesc {
  const void* Wp;      // packed tiles (double or float entries)
  const void* x;       // input vector (npad, zero tail), same entry type as the factor
  double* part;        // partial rows x npad
  int64_t nblk, npad;
  int chunk;
};

template <int NI>
struct TileArgs {
  TileDesc d[NI];
  const int4* units;   // (instance, tile row / column, unit index within it, 0)
  int64_t nunits;
  DevStatus* st;
};

__device__ __forceinline__ int64_t tile_index(int64_t I, int64_t J) { return I * (I + 1) / 2 + J; }

// Warp-uniform bounded wait: every lane polls, the warp leaves together.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, DevStatus* st,
                                          int where) {
  const int lane = threadIdx.x & 31;
  for (long long it = 0;; ++it) {
    const bool ok = dev::mbar_try_wait(bar, parity);
    if (__all_sync(0xffffffffu, ok)) return true;
    if (it > WAIT_LIMIT) {
      if (lane == 0 && atomicCAS(&st->code, 0, (int)EC_ERR_TIMEOUT) == 0) st->where = where;
      return false;
    }
    if ((it & (dev::STATUS_POLL - 1)) == 0) {
      int bad = 0;
      if (lane == 0) bad = *(volatile int*)&st->code != 0;
      if (__shfl_sync(0xffffffffu, bad, 0)) return false;
    }
  }
}

// 8 consumer warps, ST ring stages, MINB CTAs per SM.  Every variant sums each
// output entry in the same order, so all variants give bitwise identical results.
template <bool TRANS, int ST, int MINB, int NI, typename WT>
__global__ void __launch_bounds__(CW * 32 + 32, MINB) tile_trmv_kernel(const __grid_constant__ TileArgs<NI> a) {
  constexpr uint32_t TILE_BYTES = TILE_DBL * sizeof(WT);
  constexpr uint32_t SEG_BYTES = TB * sizeof(WT);
  if (*(volatile const int*)&a.st->code) return;
  extern __shared__ uint8_t smem_raw[];
  Smem<ST, WT>& sm = *reinterpret_cast<Smem<ST, WT>*>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      dev::mbar_init(&sm.full[s], 1);
      dev::mbar_init(&sm.empty[s], CW);
    }
    dev::fence_mbar_init();
  }
  __syncthreads();

  if (warp == CW) {
    // ---- producer: one lane streams the tiles of this CTA's units ----------
    if (lane != 0) return;
    const uint64_t pol = dev::policy_evict_first();
    int64_t it = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; u < a.nunits && ok; u += gridDim.x) {
      const int4 un = a.units[u];
      const TileDesc& d = a.d[NI == 1 ? 0 : un.x];
      const int64_t K = un.y;                       // tile row (forward) / column (transposed)
      int64_t t0, t1;
      if (!TRANS) {
        t0 = (int64_t)un.z * d.chunk;
        t1 = min(t0 + d.chunk, K + 1);
      } else {
        t0 = K + (int64_t)un.z * d.chunk;
        t1 = min(t0 + d.chunk, d.nblk);
      }
      double* out = d.part + (int64_t)un.z * 4 * d.npad + K * TB;
      for (int64_t t = t0; t < t1; ++t) {
        const int s = (int)(it % ST);
        const uint32_t ph = (uint32_t)((it / ST) & 1);
        if (!dev::mbar_wait(&sm.empty[s], ph ^ 1u, a.st, 40, WAIT_LIMIT)) {
          ok = false;
          break;
        }
        const int64_t I = TRANS ? t : K, J = TRANS ? K : t;
        sm.meta[s] = Meta{out, d.npad, (t == t0 ? F_FIRST : 0) | (t == t1 - 1 ? F_LAST : 0)};
        dev::mbar_expect_tx(&sm.full[s], TILE_BYTES + SEG_BYTES);
        dev::bulk_g2s_hint(sm.W[s], static_cast<const WT*>(d.Wp) + tile_index(I, J) * TILE_DBL,
                           TILE_BYTES, &sm.full[s], pol);
        dev::bulk_g2s(sm.v[s], static_cast<const WT*>(d.x) + t * TB, SEG_BYTES, &sm.full[s]);
        ++it;
      }
    }
    bool ended = false;
    if (ok) {
      const int s = (int)(it % ST);
      const uint32_t ph = (uint32_t)((it / ST) & 1);
      if (dev::mbar_wait(&sm.empty[s], ph ^ 1u, a.st, 41, WAIT_LIMIT)) {
        sm.meta[s].flags = F_END;
        dev::mbar_arrive(&sm.full[s]);
        ended = true;
      }
    }
    // Drain: every issued copy must land before the CTA's shared memory is released.
    for (int64_t j = max((int64_t)0, it - ST + (ended ? 1 : 0)); j < it; ++j) {
      const int s = (int)(j % ST);
      const uint32_t ph = (uint32_t)((j / ST) & 1);
      for (long long q = 0; q < WAIT_LIMIT && !dev::mbar_try_wait(&sm.full[s], ph); ++q) {
      }
    }
    return;
  }

  // ---- consumers ------------------------------------------------------------
  // Warp w = (h, q): lane l owns output row (forward) / column (transposed)
  // h * 32 + l of the tile and sums over the 16 inner indices q * 16 .. q * 16 + 15
  // with 2 independent accumulators.  Each (unit, q) writes its own partial row,
  // so no sum crosses lanes or warps inside the kernel (on GB300 an FP64 add costs
  // as much as an FMA: a shuffle reduction per unit would double the FP64 work).
  const int h = warp & 1, q = warp >> 1;
  const int o = h * 32 + lane;     // output index within the tile
  // (FP64 factor: FP64 arithmetic; FP32 factor: FP32 products and sums within a unit)
  // Two accumulators: the unit's closing add is then one DADD per lane (each DADD costs
  // the FP64 pipe a DFMA slot); two chains per lane and two warps per SMSP already
  // cover the DFMA latency at GB300's FP64 issue rate.
  if constexpr (std::is_same<WT, float2>::value) {
    // FP32 hi/lo pair factor: each product w v = (w_hi + w_lo)(v_hi + v_lo) as an
    // exact w_hi v_hi (TwoProd by FMA) plus the two cross terms, accumulated in an
    // unnormalised float-float sum (TwoSum of the high parts, low parts added); the
    // unit's sum is formed in FP64 once at its end.  About 2^-46 relative per entry.
    float sh[2] = {0.f, 0.f}, sl[2] = {0.f, 0.f};
    for (int64_t it = 0;; ++it) {
      const int s = (int)(it % ST);
      const uint32_t ph = (uint32_t)((it / ST) & 1);
      if (!warp_wait(&sm.full[s], ph, a.st, 42)) break;
      const Meta m = sm.meta[s];
      if (m.flags & F_END) break;
      if (m.flags & F_FIRST) {
        sh[0] = sh[1] = sl[0] = sl[1] = 0.f;
      }
      const float2* Wt = reinterpret_cast<const float2*>(sm.W[s]);
      const float2* vv = reinterpret_cast<const float2*>(sm.v[s]) + q * 16;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int i0 = q * 16 + k;
        const float2 w = !TRANS ? Wt[i0 * TB + (o ^ i0)] : Wt[o * TB + (i0 ^ o)];
        const float2 v = vv[k];                 // broadcast
        const int c = k & 1;
        // rounded intrinsics: no contraction of the TwoSum's operations into FMAs
        const float p = __fmul_rn(w.x, v.x);
        float e = fmaf(w.x, v.x, -p);
        e = fmaf(w.x, v.y, e);
        e = fmaf(w.y, v.x, e);
        const float t = __fadd_rn(sh[c], p);
        const float bp = __fsub_rn(t, sh[c]);
        const float err = __fadd_rn(__fsub_rn(sh[c], __fsub_rn(t, bp)), __fsub_rn(p, bp));
        sl[c] = __fadd_rn(sl[c], __fadd_rn(err, e));
        sh[c] = t;
      }
      __syncwarp();
      if (lane == 0) dev::mbar_arrive(&sm.empty[s]);
      if (m.flags & F_LAST) {
        m.out[q * m.npad + o] =
            ((double)sh[0] + (double)sh[1]) + ((double)sl[0] + (double)sl[1]);
      }
    }
    return;
  } else {
  WT acc[2] = {WT(0), WT(0)};
  for (int64_t it = 0;; ++it) {
    const int s = (int)(it % ST);
    const uint32_t ph = (uint32_t)((it / ST) & 1);
    if (!warp_wait(&sm.full[s], ph, a.st, 42)) break;
    const Meta m = sm.meta[s];
    if (m.flags & F_END) break;
    if (m.flags & F_FIRST) {
      acc[0] = acc[1] = WT(0);
    }
    const WT* Wt = sm.W[s];
    using WT2 = typename std::conditional<sizeof(WT) == 8, double2, float2>::type;
    const WT2* vv = reinterpret_cast<const WT2*>(sm.v[s] + q * 16);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
      const WT2 v = vv[k2];                    // inner indices i0, i0 + 1 (broadcast)
      const int i0 = q * 16 + 2 * k2, i1 = i0 + 1;
      WT w0, w1;
      if (!TRANS) {                            // W[o, i]: column i, row o
        w0 = Wt[i0 * TB + (o ^ i0)];
        w1 = Wt[i1 * TB + (o ^ i1)];
      } else {                                 // W[i, o]: column o, row i
        w0 = Wt[o * TB + (i0 ^ o)];
        w1 = Wt[o * TB + (i1 ^ o)];
      }
      acc[0] = fma(w0, v.x, acc[0]);
      acc[1] = fma(w1, v.y, acc[1]);
    }
    __syncwarp();
    if (lane == 0) dev::mbar_arrive(&sm.empty[s]);
    if (m.flags & F_LAST) {
      m.out[q * m.npad + o] = double(acc[0] + acc[1]);
    }
  }
  }
}

__device__ __forceinline__ int64_t tile_row_of(int64_t t) {
  int64_t I = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (I * (I + 1) / 2 > t) --I;
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  return I;
}

// Packed tiles of the lower triangle of W (column-major, ld ldw), entries converted to
// WT; the diagonal is multiplied by diag_scale (0.5 stores the half of a symmetric
// matrix whose product with its transpose-sum gives the full product).
template <typename WT>
__device__ __forceinline__ WT to_entry(double v) {
  return WT(v);
}
// FP32 pair: hi = fp32(v), lo = fp32(v - hi) (about 48 significant bits together)
template <>
__device__ __forceinline__ float2 to_entry<float2>(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

template <typename WT>
__global__ void pack_kernel(int64_t n, int64_t ntiles, const double* W, int64_t ldw, WT* Wp,
                            double diag_scale) {
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t I = tile_row_of(t), J = t - I * (I + 1) / 2;
    for (int e = threadIdx.x; e < TILE_DBL; e += blockDim.x) {
      const int c = e >> 6, r = (e & 63) ^ c;
      const int64_t row = I * TB + r, col = J * TB + c;
      const bool in = row < n && col < n && (I != J || r >= c);
      double v = in ? W[row + col * ldw] : 0.0;
      if (row == col) v *= diag_scale;
      Wp[t * TILE_DBL + e] = to_entry<WT>(v);
    }
  }
}

__global__ void unpack_kernel(int64_t n, int64_t ntiles, const double* Wp, double* W, int64_t ldw) {
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t I = tile_row_of(t), J = t - I * (I + 1) / 2;
    for (int e = threadIdx.x; e < TILE_DBL; e += blockDim.x) {
      const int c = e >> 6, r = (e & 63) ^ c;
      const int64_t row = I * TB + r, col = J * TB + c;
      if (row < n && col < n && (I != J || r >= c)) W[row + col * ldw] = Wp[t * TILE_DBL + e];
    }
  }
}

// out[i] = sum of the partial rows holding data for entry i.  A block covers 64
// consecutive entries with SUM_G thread rows; thread row g sums partial rows
// g, g + SUM_G, ... with two independent accumulators (so loads stay in flight),
// then the thread rows are combined in a fixed order.  The partials were just
// written and sit in L2; the kernel is latency-bound, hence the wide blocks.
// blockIdx.y selects the instance of a batched launch.
constexpr int SUM_G = 16;

struct SumDesc {
  const double* part;
  double* out;
  int64_t n, nblk, npad;
  int chunk;
  float* out32;        // optional FP32 copy of out (input of an FP32-factor product)
  float2* outx2;       // optional FP32 pair copy of out (input of a pair-factor product)
};

template <int NI>
struct SumArgs {
  SumDesc d[NI];
  int trans;
  int accumulate;      // 1: out[i] += sum (refinement corrections)
};

template <int NI>
__global__ void __launch_bounds__(TB * SUM_G) tile_sum_kernel(const __grid_constant__ SumArgs<NI> a) {
  __shared__ double red[SUM_G][TB];
  const SumDesc& d = a.d[NI == 1 ? 0 : blockIdx.y];
  if ((int64_t)blockIdx.x >= d.nblk) return;
  const int tx = threadIdx.x & 63, g = threadIdx.x >> 6;
  const int64_t i = (int64_t)blockIdx.x * TB + tx;
  double s0 = 0.0, s1 = 0.0;
  if (i < d.n) {
    const int64_t nc = a.trans ? tile_valid_rows_t(i, d.nblk, d.chunk) : tile_valid_rows(i, d.chunk);
    const double* p = d.part + i;
    int64_t r = g;
    for (; r + SUM_G < nc; r += 2 * SUM_G) {
      s0 += p[r * d.npad];
      s1 += p[(r + SUM_G) * d.npad];
    }
    if (r < nc) s0 += p[r * d.npad];
  }
  red[g][tx] = s0 + s1;
  __syncthreads();
#pragma unroll
  for (int h = SUM_G / 2; h > 0; h >>= 1) {
    if (g < h) red[g][tx] += red[g + h][tx];
    __syncthreads();
  }
  if (g == 0 && i < d.n) {
    const double v = a.accumulate ? d.out[i] + red[0][tx] : red[0][tx];
    d.out[i] = v;
    if (d.out32) d.out32[i] = (float)v;
    if (d.outx2) {
      const float hi = (float)v;
      d.outx2[i] = make_float2(hi, (float)(v - (double)hi));
    }
  }
}

__global__ void to_x2_kernel(int64_t n, const double* x, float2* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float hi = (float)x[i];
    y[i] = make_float2(hi, (float)(x[i] - (double)hi));
  }
}

__global__ void to_f32_kernel(int64_t n, const double* x, float* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

template <int NI>
struct Variant {
  void (*fwd)(TileArgs<NI>);
  void (*bwd)(TileArgs<NI>);
  int threads;
  size_t smem;
};

// Launch shapes the autotuner chooses from: (ring stages, CTAs per SM), for factors
// with WT entries.
template <int NI, typename WT = double>
const Variant<NI>* variants() {
  static const Variant<NI> v[TILE_VARIANTS] = {
      {tile_trmv_kernel<false, 4, 1, NI, WT>, tile_trmv_kernel<true, 4, 1, NI, WT>, CW * 32 + 32,
       smem_bytes<4, WT>()},
      {tile_trmv_kernel<false, 3, 2, NI, WT>, tile_trmv_kernel<true, 3, 2, NI, WT>, CW * 32 + 32,
       smem_bytes<3, WT>()},
      {tile_trmv_kernel<false, 6, 1, NI, WT>, tile_trmv_kernel<true, 6, 1, NI, WT>, CW * 32 + 32,
       smem_bytes<6, WT>()},
  };
  return v;
}

std::mutex g_attr_mu;
bool g_attr_done[64] = {};

template <int NI, typename WT = double>
void set_attributes() {
  for (int i = 0; i < TILE_VARIANTS; ++i) {
    const Variant<NI>& v = variants<NI, WT>()[i];
    cudaFuncSetAttribute(v.fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
    cudaFuncSetAttribute(v.bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
  }
}

}  // namespace

void tile_prepare_launches() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (dev < 0 || dev >= 64 || g_attr_done[dev]) return;
  set_attributes<1>();
  set_attributes<1, float>();
  set_attributes<1, float2>();
  set_attributes<TILE_BATCH_MAX>();
  g_attr_done[dev] = true;
}

namespace {

// Units of one instance: forward (row K, run c) and transposed (column K, run c).
void instance_units(int inst, int64_t nblk, int64_t chunk, std::vector<int4>& fwd,
                    std::vector<int4>& bwd) {
  for (int64_t K = 0; K < nblk; ++K) {
    for (int64_t c = 0; c < K / chunk + 1; ++c) fwd.push_back(make_int4(inst, (int)K, (int)c, 0));
    for (int64_t c = 0; c < (nblk - 1 - K) / chunk + 1; ++c)
      bwd.push_back(make_int4(inst, (int)K, (int)c, 0));
  }
}

// Largest unit first (ties: instance, row, run), so round-robin dealing balances.
void order_units(std::vector<int4>& u, const std::vector<int64_t>& nblk,
                 const std::vector<int64_t>& chunk, bool trans) {
  auto size = [&](const int4& x) {
    const int64_t ch = chunk[x.x];
    if (!trans) return std::min<int64_t>((int64_t)x.z * ch + ch, (int64_t)x.y + 1) - (int64_t)x.z * ch;
    const int64_t t0 = (int64_t)x.y + (int64_t)x.z * ch;
    return std::min<int64_t>(t0 + ch, nblk[x.x]) - t0;
  };
  std::stable_sort(u.begin(), u.end(), [&](const int4& a, const int4& b) {
    const int64_t sa = size(a), sb = size(b);
    if (sa != sb) return sa > sb;
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    return a.z < b.z;
  });
}

ec_status upload_units(const std::vector<int4>& fwd, const std::vector<int4>& bwd, int4** dfwd,
                       int4** dbwd) {
  if (device_alloc((void**)dfwd, sizeof(int4) * fwd.size()) != cudaSuccess ||
      device_alloc((void**)dbwd, sizeof(int4) * bwd.size()) != cudaSuccess) {
    cudaGetLastError();
    return EC_ERR_OOM;
  }
  if (cudaMemcpy(*dfwd, fwd.data(), sizeof(int4) * fwd.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(*dbwd, bwd.data(), sizeof(int4) * bwd.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return EC_ERR_CUDA;
  return EC_OK;
}

template <int NI>
void grids_for(int64_t nunits, int* grids) {
  const int64_t sms = num_sms();
  for (int v = 0; v < TILE_VARIANTS; ++v) {
    int per_sm = 0;
    const Variant<NI>& var = variants<NI>()[v];
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, var.fwd, var.threads, var.smem);
    if (per_sm < 1) per_sm = 1;
    grids[v] = (int)std::max<int64_t>(1, std::min<int64_t>(sms * per_sm, nunits));
  }
}

}  // namespace

ec_status tile_plan_create(int64_t n, TilePlan* p) {
  tile_plan_free(p);
  p->n = n;
  p->nblk = (n + TB - 1) / TB;
  p->npad = p->nblk * TB;
  p->ntiles = p->nblk * (p->nblk + 1) / 2;
  const int64_t sms = num_sms();
  p->chunk = (int)std::max<int64_t>(1, std::min<int64_t>(64, p->ntiles / (sms * 16)));
  std::vector<int4> fwd, bwd;
  instance_units(0, p->nblk, p->chunk, fwd, bwd);
  order_units(fwd, {p->nblk}, {(int64_t)p->chunk}, false);
  order_units(bwd, {p->nblk}, {(int64_t)p->chunk}, true);
  p->nunits = (int64_t)fwd.size();
  ec_status rc = upload_units(fwd, bwd, &p->units_fwd, &p->units_bwd);
  if (rc != EC_OK) {
    tile_plan_free(p);
    return rc;
  }
  tile_prepare_launches();
  grids_for<1>(p->nunits, p->grids);
  p->variant = 0;
  return EC_OK;
}

void tile_plan_free(TilePlan* p) {
  if (p->units_fwd) cudaFree(p->units_fwd);
  if (p->units_bwd) cudaFree(p->units_bwd);
  *p = TilePlan{};
}

void tile_pack_lower(cudaStream_t s, const TilePlan& p, const double* W, int64_t ldw,
                     double* Wp, double diag_scale) {
  const int64_t g = std::min<int64_t>(p.ntiles, (int64_t)num_sms() * 16);
  pack_kernel<double><<<(unsigned)g, 256, 0, ::ec::counted(s)>>>(p.n, p.ntiles, W, ldw, Wp,
                                                                  diag_scale);
}

void tile_pack_lower_f32(cudaStream_t s, const TilePlan& p, const double* W, int64_t ldw,
                         float* Wp) {
  const int64_t g = std::min<int64_t>(p.ntiles, (int64_t)num_sms() * 16);
  pack_kernel<float><<<(unsigned)g, 256, 0, ::ec::counted(s)>>>(p.n, p.ntiles, W, ldw, Wp, 1.0);
}

void tile_unpack_lower(cudaStream_t s, const TilePlan& p, const double* Wp, double* W,
                       int64_t ldw) {
  cudaMemset2DAsync(W, sizeof(double) * ldw, 0, sizeof(double) * p.n, p.n, s);
  const int64_t g = std::min<int64_t>(p.ntiles, (int64_t)num_sms() * 16);
  unpack_kernel<<<(unsigned)g, 256, 0, ::ec::counted(s)>>>(p.n, p.ntiles, Wp, W, ldw);
}

namespace {

void sum_launch(cudaStream_t s, const TilePlan& p, int trans, const double* part, double* out,
                int accumulate, float* out32 = nullptr, float2* outx2 = nullptr) {
  SumArgs<1> a{};
  a.d[0] = SumDesc{part, out, p.n, p.nblk, p.npad, p.chunk, out32, outx2};
  a.trans = trans;
  a.accumulate = accumulate;
  tile_sum_kernel<1><<<(unsigned)p.nblk, TB * SUM_G, 0, ::ec::counted(s)>>>(a);
}

// b_in / y_in: the vectors the two products read (b and y themselves for an FP64
// factor; their FP32 copies b32 / y32 for an FP32 factor).
template <typename WT>
void pair_launch(cudaStream_t s, const TilePlan& p, const WT* Wp, const void* b_in,
                 double* part1, double* y, float* y32, double* part2, double* x, int accumulate,
                 DevStatus* st, cudaEvent_t* ev, float2* yx2 = nullptr) {
  tile_prepare_launches();
  const Variant<1>& v = variants<1, WT>()[p.variant];
  const int grid = p.grids[p.variant];
  TileArgs<1> a{};
  a.d[0] = TileDesc{Wp, b_in, part1, p.nblk, p.npad, p.chunk};
  a.units = p.units_fwd;
  a.nunits = p.nunits;
  a.st = st;
  if (ev) cudaEventRecord(ev[0], s);
  v.fwd<<<grid, v.threads, v.smem, ::ec::counted(s)>>>(a);
  if (ev) cudaEventRecord(ev[1], s);
  sum_launch(s, p, 0, part1, y, 0, y32, yx2);
  const void* y_in = y32 ? (const void*)y32 : yx2 ? (const void*)yx2 : (const void*)y;
  a.d[0] = TileDesc{Wp, y_in, part2, p.nblk, p.npad, p.chunk};
  a.units = p.units_bwd;
  v.bwd<<<grid, v.threads, v.smem, ::ec::counted(s)>>>(a);
  if (ev) cudaEventRecord(ev[2], s);
  sum_launch(s, p, 1, part2, x, accumulate);
}

}  // namespace

void tile_sum(cudaStream_t s, const TilePlan& p, int trans, const double* part, double* out) {
  sum_launch(s, p, trans, part, out, 0);
}

void tile_trmv_pair(cudaStream_t s, const TilePlan& p, const double* Wp, const double* b,
                    double* part1, double* y, double* part2, double* x, DevStatus* st,
                    cudaEvent_t* ev) {
  pair_launch<double>(s, p, Wp, b, part1, y, nullptr, part2, x, 0, st, ev);
}

void tile_trmv_pair_f32(cudaStream_t s, const TilePlan& p, const float* Wp, const double* b,
                        float* v32, double* part1, double* y, double* part2, double* x,
                        int accumulate, DevStatus* st, cudaEvent_t* ev) {
  const int64_t g = std::min<int64_t>((p.n + 255) / 256, 1024);
  to_f32_kernel<<<(unsigned)(g < 1 ? 1 : g), 256, 0, ::ec::counted(s)>>>(p.n, b, v32);
  pair_launch<float>(s, p, Wp, v32, part1, y, v32, part2, x, accumulate, st, ev);
}

void tile_pack_lower_x2(cudaStream_t s, const TilePlan& p, const double* W, int64_t ldw,
                        float2* Wp) {
  const int64_t g = std::min<int64_t>(p.ntiles, (int64_t)num_sms() * 16);
  pack_kernel<float2><<<(unsigned)g, 256, 0, ::ec::counted(s)>>>(p.n, p.ntiles, W, ldw, Wp, 1.0);
}

void tile_trmv_pair_x2(cudaStream_t s, const TilePlan& p, const float2* Wp, const double* b,
                       float2* vx2, double* part1, double* y, double* part2, double* x,
                       DevStatus* st, cudaEvent_t* ev) {
  const int64_t g = std::min<int64_t>((p.n + 255) / 256, 1024);
  to_x2_kernel<<<(unsigned)(g < 1 ? 1 : g), 256, 0, ::ec::counted(s)>>>(p.n, b, vx2);
  pair_launch<float2>(s, p, Wp, vx2, part1, y, nullptr, part2, x, 0, st, ev, vx2);
}

void tile_sym_product(cudaStream_t s, const TilePlan& p, const double* Hp, const double* x,
                      double* part1, double* part2, double* out1, double* out2, DevStatus* st) {
  tile_prepare_launches();
  const Variant<1>& v = variants<1>()[p.variant];
  const int grid = p.grids[p.variant];
  TileArgs<1> a{};
  a.d[0] = TileDesc{Hp, x, part1, p.nblk, p.npad, p.chunk};
  a.units = p.units_fwd;
  a.nunits = p.nunits;
  a.st = st;
  v.fwd<<<grid, v.threads, v.smem, ::ec::counted(s)>>>(a);
  sum_launch(s, p, 0, part1, out1, 0);
  a.d[0] = TileDesc{Hp, x, part2, p.nblk, p.npad, p.chunk};
  a.units = p.units_bwd;
  v.bwd<<<grid, v.threads, v.smem, ::ec::counted(s)>>>(a);
  sum_launch(s, p, 1, part2, out2, 0);
}

namespace {

// Times every launch shape (one warm-up and three timed runs of `run` each) and
// returns the fastest; `run(v)` enqueues one product pair with shape v.
template <typename F>
ec_status autotune_shapes(cudaStream_t s, F run, int* best_out, float* tune_ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return EC_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return EC_ERR_CUDA;
  }
  float best = 1e30f;
  int best_v = 0;
  for (int v = 0; v < TILE_VARIANTS; ++v) {
    run(v);
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3; ++r) run(v);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      break;
    tune_ms[v] = ms / 3.f;
    if (ms < best) {
      best = ms;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best_out = best_v;
  return cudaGetLastError() == cudaSuccess ? EC_OK : EC_ERR_CUDA;
}

}  // namespace

ec_status tile_autotune(cudaStream_t s, TilePlan* p, const double* Wp, const double* b,
                        double* part1, double* y, double* part2, DevStatus* st, int forced) {
  if (forced >= 1 && forced <= TILE_VARIANTS) {
    p->variant = forced - 1;
    return EC_OK;
  }
  int best = 0;
  ec_status rc = autotune_shapes(
      s,
      [&](int v) {
        p->variant = v;
        tile_trmv_pair(s, *p, Wp, b, part1, y, part2, y, st);
      },
      &best, p->tune_ms);
  p->variant = best;
  return rc;
}

ec_status tile_autotune_f32(cudaStream_t s, TilePlan* p, const float* Wp, const double* b,
                            float* v32, double* part1, double* y, double* part2, DevStatus* st,
                            int forced) {
  if (forced >= 1 && forced <= TILE_VARIANTS) {
    p->variant = forced - 1;
    return EC_OK;
  }
  int best = 0;
  ec_status rc = autotune_shapes(
      s,
      [&](int v) {
        p->variant = v;
        tile_trmv_pair_f32(s, *p, Wp, b, v32, part1, y, part2, y, 0, st);
      },
      &best, p->tune_ms);
  p->variant = best;
  return rc;
}

ec_status tile_autotune_x2(cudaStream_t s, TilePlan* p, const float2* Wp, const double* b,
                           float2* vx2, double* part1, double* y, double* part2, DevStatus* st,
                           int forced) {
  if (forced >= 1 && forced <= TILE_VARIANTS) {
    p->variant = forced - 1;
    return EC_OK;
  }
  int best = 0;
  ec_status rc = autotune_shapes(
      s,
      [&](int v) {
        p->variant = v;
        tile_trmv_pair_x2(s, *p, Wp, b, vx2, part1, y, part2, y, st);
      },
      &best, p->tune_ms);
  p->variant = best;
  return rc;
}

// ---- batches of instances ---------------------------------------------------

ec_status tile_batch_create(const TileInst* inst, int count, TileBatch* B) {
  tile_batch_free(B);
  if (count < 1 || count > TILE_BATCH_MAX) return EC_ERR_ARG;
  std::vector<int4> fwd, bwd;
  std::vector<int64_t> nblk(count), chunk(count);
  for (int i = 0; i < count; ++i) {
    nblk[i] = inst[i].plan->nblk;
    chunk[i] = inst[i].plan->chunk;
    instance_units(i, nblk[i], chunk[i], fwd, bwd);
    B->max_nblk = std::max(B->max_nblk, nblk[i]);
  }
  order_units(fwd, nblk, chunk, false);
  order_units(bwd, nblk, chunk, true);
  B->count = count;
  B->nunits_fwd = (int64_t)fwd.size();
  B->nunits_bwd = (int64_t)bwd.size();
  ec_status rc = upload_units(fwd, bwd, &B->units_fwd, &B->units_bwd);
  if (rc != EC_OK) {
    tile_batch_free(B);
    return rc;
  }
  tile_prepare_launches();
  grids_for<TILE_BATCH_MAX>(std::min(B->nunits_fwd, B->nunits_bwd), B->grids);
  B->variant = 0;
  return EC_OK;
}

void tile_batch_free(TileBatch* B) {
  if (B->units_fwd) cudaFree(B->units_fwd);
  if (B->units_bwd) cudaFree(B->units_bwd);
  *B = TileBatch{};
}

void tile_batch_pair(cudaStream_t s, const TileBatch& B, const TileInst* inst, DevStatus* st) {
  const Variant<TILE_BATCH_MAX>& v = variants<TILE_BATCH_MAX>()[B.variant];
  const int grid = B.grids[B.variant];
  TileArgs<TILE_BATCH_MAX> a{};
  SumArgs<TILE_BATCH_MAX> sa{};
  for (int i = 0; i < B.count; ++i) {
    const TilePlan& p = *inst[i].plan;
    a.d[i] = TileDesc{inst[i].Wp, inst[i].b, inst[i].part1, p.nblk, p.npad, p.chunk};
    sa.d[i] = SumDesc{inst[i].part1, inst[i].y, p.n, p.nblk, p.npad, p.chunk, nullptr, nullptr};
  }
  a.units = B.units_fwd;
  a.nunits = B.nunits_fwd;
  a.st = st;
  v.fwd<<<grid, v.threads, v.smem, ::ec::counted(s)>>>(a);
  sa.trans = 0;
  tile_sum_kernel<TILE_BATCH_MAX><<<dim3((unsigned)B.max_nblk, (unsigned)B.count), TB * SUM_G, 0,
                                    ::ec::counted(s)>>>(sa);
  for (int i = 0; i < B.count; ++i) {
    const TilePlan& p = *inst[i].plan;
    a.d[i] = TileDesc{inst[i].Wp, inst[i].y, inst[i].part2, p.nblk, p.npad, p.chunk};
    sa.d[i] = SumDesc{inst[i].part2, inst[i].x, p.n, p.nblk, p.npad, p.chunk, nullptr, nullptr};
  }
  a.units = B.units_bwd;
  a.nunits = B.nunits_bwd;
  v.bwd<<<grid, v.threads, v.smem, ::ec::counted(s)>>>(a);
  sa.trans = 1;
  tile_sum_kernel<TILE_BATCH_MAX><<<dim3((unsigned)B.max_nblk, (unsigned)B.count), TB * SUM_G, 0,
                                    ::ec::counted(s)>>>(sa);
}

ec_status tile_batch_autotune(cudaStream_t s, TileBatch* B, const TileInst* inst, DevStatus* st) {
  int best = 0;
  ec_status rc = autotune_shapes(
      s,
      [&](int v) {
        B->variant = v;
        tile_batch_pair(s, *B, inst, st);
      },
      &best, B->tune_ms);
  B->variant = best;
  return rc;
}

}  // namespace ec
