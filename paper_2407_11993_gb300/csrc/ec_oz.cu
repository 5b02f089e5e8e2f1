// FP64-accurate dense products on the tensor cores (tcgen05), for the dense
// contractions of the modal setup (Sec. 3.2: Cholesky of R_i, the two-sided
// reduction to standard form, the eigenvector merges and back-transformation) and
// of the plain setup (Sec. 3.3.1: Cholesky of Z and its inverse).
//
// GB300 retires about two FP64 FMAs per SM per clock (1.2 TFLOP/s), but about
// 3,500 BF16 multiply-adds.  The product is therefore computed exactly on integer
// slices (the error-free splitting of Ozaki et al., 2012), restated here:
//
//   * every row i of op(A) is scaled by 2^-e_i with max_k |a_ik| < 2^(e_i - 1) and
//     rounded to a 64-bit fixed-point integer F_ik (|F| < 2^63; an entry loses only
//     the bits below 2^(e_i - 64), i.e. 2^-62 of its row's largest entry);
//   * F is cut into eight balanced base-256 digits, F = sum_s d_s 256^(7-s),
//     |d_s| <= 128, and slice s holds d_s 2^-8s in BF16 (exact: 8 significant bits);
//   * columns of op(B) likewise (exponents f_j, slices t);
//   * a_ik b_kj = 2^(e_i + f_j - 16) sum_{s,t} A_s B_t, and the 36 pairs with
//     s + t <= 7 are kept (the dropped ones lie below 2^-61 of the row / column scales,
//     so the product keeps FP64 accuracy even where a row's entries span many decades).
//
// One CTA per SM (persistent) computes 128 x 64 tiles of C over a K range of at most 192:
//   * warp 0 / lane 0 streams, per 32-wide K block, all eight A slices (one 3-D TMA
//     box of 128 x 32 x 8) and all eight B slices (64 x 32 x 8) into a two-stage
//     shared-memory ring (64-byte swizzle), guarded by mbarriers;
//   * warp 1 / lane 0 issues one tcgen05.mma (kind::f16, BF16 in, FP32 accumulate,
//     M = 128, N = 64, K = 16) per slice pair and 16-wide K step into six FP32
//     accumulators in tensor memory: one per diagonal s + t = d for d <= 4, whose
//     sums are exact (integers times 2^-8d below 2^24 in magnitude, because
//     (d + 1) 2^14 K < 2^24 for K <= 192), and one shared by d = 5, 6, 7, whose FP32
//     rounding lies below 2^-60 of the leading diagonal;
//   * eight epilogue warps read the accumulators (warp w reads TMEM lanes
//     32 (w % 4) .. + 31, the tile's rows, for half of the columns), rebuild each
//     entry as an exact 64-bit integer (staged in tensor memory, which releases the
//     accumulators to the next tile's MMAs) at granularity
//     2^-40, convert it to binary64 with integer instructions (one rounding), apply
//     2^(e_i + f_j - 56) and alpha, and add beta C.
// Longer K is done as consecutive launches that accumulate into C in FP64.
// Every mbarrier wait is bounded; a wait that runs out records EC_ERR_TIMEOUT in the
// status block and the kernel skips its remaining work and frees its TMEM.

#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "ec_async.cuh"
#include "ec_internal.h"
#include "ec_oz.h"
#include "ec_oz_int.h"
#include "ec_tc.h"

namespace ec {

namespace {

constexpr int OZ_S = 8;                 // slices per operand
constexpr int OZ_DMAX = 7;              // slice pairs with s + t <= OZ_DMAX
constexpr int OZ_EXACT = 5;             // diagonals 0 .. 4 have their own accumulator
constexpr int NACC = OZ_EXACT + 1;      // + one shared by the diagonals 5 .. 7
constexpr int TM = 128, TN = 64, TK = 32;
constexpr int STAGES = 2;
constexpr int A_SLICE = TM * TK * 2;    // 8 KB
constexpr int B_SLICE = TN * TK * 2;    // 4 KB
constexpr int A_BYTES = OZ_S * A_SLICE;
constexpr int B_BYTES = OZ_S * B_SLICE;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;   // 96 KB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr int TMEM_COLS = 512;
constexpr int GROUP_M = 16;             // tile rows per raster group (L2 reuse of A)
constexpr long long WAIT_LIMIT = 1ll << 26;

static_assert(NACC * TN <= TMEM_COLS, "accumulators exceed tensor memory");
static_assert(5 * 128 * 128 * OZ_KCHUNK < (1 << 24), "diagonal 4 would not be exact");

using dev::mbar_expect_tx;
using dev::mbar_init;
using dev::smem_u32;

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, DevStatus* st,
                                          int where) {
  return dev::mbar_wait(bar, parity, st, where, WAIT_LIMIT);
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile, rows of 64 bytes, 64-byte swizzle,
// 8-row groups 512 bytes apart, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return ((uint64_t)(addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(512 >> 4) << 32) |
         (1ull << 46) | (4ull << 61);
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = TM, N = nmma
// (TN, or 16 / 32 for products whose B block has that few columns).
__host__ __device__ constexpr uint32_t idesc_for(int nmma) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nmma >> 3) << 17) |
         ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

struct OzArgs {
  int M, N;                // C block (rows, columns)
  int k0, klen;            // K range of this launch
  int tiles_m, tiles_n;
  int tri;                 // keep only rows >= columns (of the C block)
  int amode, bmode;        // alpha: 0 = 1, 1 = -1, 2 = other; beta: 0 = 0, 1 = 1, 2 = other
  double alpha, beta;
  double* C;
  int64_t ldc;
  const int* ea;           // row exponents of op(A)
  const int* eb;           // column exponents of op(B)
  int nmma;                // MMA width and B rows per stage: TN, or 16 / 32 when N is that small
};

// Tile of a launch: row groups of GROUP_M tile rows, columns innermost within a group
// (the group's A slices stay in L2 while B streams).
__device__ __forceinline__ void tile_of(int t, int tiles_m, int tiles_n, int& bm, int& bn) {
  const int per_group = GROUP_M * tiles_n;
  const int g = t / per_group;
  const int r = t - g * per_group;
  const int gm = min(GROUP_M, tiles_m - g * GROUP_M);
  bn = r / gm;
  bm = g * GROUP_M + (r - bn * gm);
}

constexpr int EPI_WARPS = 8;                       // two per TMEM lane quarter
constexpr int OZ_THREADS = (2 + EPI_WARPS) * 32;   // producer, MMA issuer, epilogue
constexpr int STAGE_COL = NACC * TN;               // TMEM columns 384..511: the exact integers

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
      "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
}

// Tiles of this launch handled by a CTA: t = blockIdx.x, blockIdx.x + gridDim.x, ...;
// lower-triangle products skip the tiles entirely above the diagonal.  Every warp
// role walks the same sequence.
__device__ __forceinline__ bool next_tile(const OzArgs& a, int& t, int& m0, int& n0) {
  const int ntiles = a.tiles_m * a.tiles_n;
  for (; t < ntiles; t += gridDim.x) {
    int bm, bn;
    tile_of(t, a.tiles_m, a.tiles_n, bm, bn);
    m0 = bm * TM;
    n0 = bn * TN;
    if (!(a.tri && n0 > m0 + TM - 1)) return true;
  }
  return false;
}

// Persistent: one CTA per SM walks its tiles.  Warp 0 (one lane) streams the slices of
// every tile's K blocks through the shared-memory ring without stopping at tile
// boundaries; warp 1 (one lane) issues the MMAs of a tile once the epilogue has
// released the accumulators; warps 2..9 first fold the six accumulators of each entry
// into its exact 64-bit integer (kept in TMEM columns 384..511), release the
// accumulators -- the next tile's MMAs start -- and then convert and store while those
// run.
__global__ void __launch_bounds__(OZ_THREADS, 1) oz_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                                                         const __grid_constant__ CUtensorMap mapB,
                                                         const OzArgs a, DevStatus* st) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], acc_full, acc_empty,
      done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, issued, consumed, skip;
  if (threadIdx.x == 0) skip = *(volatile int*)&st->code;
  __syncthreads();
  if (skip) return;                                  // an earlier failure: leave together
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (a.klen + TK - 1) / TK;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&acc_full, 1);
    mbar_init(&acc_empty, EPI_WARPS);
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    issued = 0;
    consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // producer: all eight slices of A and of B for each 32-wide K block, tile after tile
      uint32_t it = 0;
      int t = blockIdx.x, m0 = 0, n0 = 0;
      for (; next_tile(a, t, m0, n0) && !*(volatile int*)&abort_flag; t += gridDim.x) {
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          const uint32_t use = it / STAGES;
          if (it >= STAGES && !mbar_wait(&empty_bar[s], (use - 1) & 1, st, 41)) {
            *(volatile int*)&abort_flag = 1;
            break;
          }
          uint8_t* sa = smem + s * STAGE_BYTES;
          uint8_t* sb = sa + A_BYTES;
          mbar_expect_tx(&full_bar[s], A_BYTES + OZ_S * a.nmma * TK * 2);
          tma_load_3d(sa, &mapA, &full_bar[s], a.k0 + kb * TK, m0, 0);
          tma_load_3d(sb, &mapB, &full_bar[s], a.k0 + kb * TK, n0, 0);
          *(volatile int*)&issued = (int)(it + 1);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: one MMA per slice pair and 16-wide K step
      uint32_t it = 0, tc = 0;
      const uint32_t idesc = idesc_for(a.nmma);
      const uint32_t b_slice = (uint32_t)(a.nmma * TK * 2);   // B slices lie densely packed
      int t = blockIdx.x, m0 = 0, n0 = 0;
      bool ok = true;
      for (; ok && next_tile(a, t, m0, n0) && !*(volatile int*)&abort_flag; t += gridDim.x, ++tc) {
        // the epilogue must have taken the previous tile's accumulators
        if (tc > 0 && !mbar_wait(&acc_empty, (tc - 1) & 1, st, 46)) {
          *(volatile int*)&abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          if (!mbar_wait(&full_bar[s], (it / STAGES) & 1, st, 42)) {
            *(volatile int*)&abort_flag = 1;
            ok = false;
            break;
          }
          *(volatile int*)&consumed = (int)(it + 1);
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
          const uint64_t dA0 = smem_desc(sa), dB0 = smem_desc(sa + A_BYTES);
#pragma unroll
          for (int d = 0; d <= OZ_DMAX; ++d) {
            const int acc = d < OZ_EXACT ? d : OZ_EXACT;
            const uint32_t tacc = tmem + (uint32_t)(acc * TN);
#pragma unroll
            for (int si = 0; si <= d; ++si) {
              const int ti = d - si;
              if (si >= OZ_S || ti >= OZ_S) continue;
              const uint64_t da = dA0 + (uint64_t)((si * A_SLICE) >> 4);
              const uint64_t db = dB0 + (uint64_t)((ti * b_slice) >> 4);
#pragma unroll
              for (int kk = 0; kk < TK / 16; ++kk) {
                // the first product into each accumulator overwrites it
                const bool first = kb == 0 && kk == 0 && si == 0 && d <= OZ_EXACT;
                mma_bf16(tacc, da + 2 * kk, db + 2 * kk, idesc, first ? 0u : 1u);
              }
            }
          }
          mma_commit(&empty_bar[s]);
        }
        // arrives once this tile's MMAs have completed (also after a failure, so the
        // epilogue's wait ends)
        mma_commit(&acc_full);
      }
      // arrives once every MMA this thread issued has completed
      mma_commit(&done_bar);
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of the tile) and half of
    // the columns, [32 h, 32 h + 32) with h = (w - 2) / 4
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    uint32_t tc = 0;
    int t = blockIdx.x, m0 = 0, n0 = 0;
    for (; next_tile(a, t, m0, n0); t += gridDim.x, ++tc) {
      if (!mbar_wait(&acc_full, tc & 1, st, 47)) {
        *(volatile int*)&abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (*(volatile int*)&abort_flag) break;
      const int row = m0 + quarter * 32 + lane;
      const bool row_ok = row < a.M;
      // phase 1: the exact integer of each entry at granularity 2^-40 (diagonal d holds
      // integers times 2^-8d): the top two diagonals in 32 bits, the rest by wide
      // multiply-adds, then the shared group of the small diagonals rounded at 2^-40
#pragma unroll 1
      for (int c0 = half * (TN / 2); c0 < (half + 1) * (TN / 2); c0 += 16) {
        if (n0 + c0 >= a.N) break;                   // columns past C (and past nmma)
        uint32_t r[NACC][16];
#pragma unroll
        for (int q = 0; q < NACC; ++q) tmem_ld16(lane_base + (uint32_t)(q * TN + c0), r[q]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        uint32_t xs[32];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int i0 = __float2int_rn(__uint_as_float(r[0][j]));
          const int i1 = __float2int_rn(__uint_as_float(r[1][j]) * 256.0f);
          const int i2 = __float2int_rn(__uint_as_float(r[2][j]) * 65536.0f);
          const int i3 = __float2int_rn(__uint_as_float(r[3][j]) * 16777216.0f);
          const int i4 = __float2int_rn(__uint_as_float(r[4][j]) * 4294967296.0f);
          const int ig = __float2int_rn(__uint_as_float(r[OZ_EXACT][j]) * 1099511627776.0f);
          int64_t X = (int64_t)(i0 * 256 + i1) * 4294967296ll;
          X += (int64_t)i2 * (1 << 24);
          X += (int64_t)i3 * (1 << 16);
          X += (int64_t)i4 * (1 << 8);
          X += ig;
          xs[2 * j] = (uint32_t)(uint64_t)X;
          xs[2 * j + 1] = (uint32_t)((uint64_t)X >> 32);
        }
        tmem_st32(lane_base + (uint32_t)(STAGE_COL + 2 * c0), xs);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) dev::mbar_arrive(&acc_empty);
      // phase 2 (overlaps the next tile's MMAs): binary64 conversion, scaling, C update
      const int erow = row_ok ? a.ea[row] - 56 : 0;
#pragma unroll 1
      for (int c0 = half * (TN / 2); c0 < (half + 1) * (TN / 2); c0 += 16) {
        if (n0 + c0 >= a.N) break;
        uint32_t xs[32];
        tmem_ld32(lane_base + (uint32_t)(STAGE_COL + 2 * c0), xs);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!row_ok) continue;
        // columns of this chunk all inside C (and, for lower-triangle products, all at
        // or left of this row): no per-entry checks
        const bool whole = (n0 + c0 + 16 <= a.N) && (!a.tri || n0 + c0 + 15 <= row);
        int ebc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) ebc[j] = (n0 + c0 + j < a.N) ? a.eb[n0 + c0 + j] : 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c0 + j;
          if (!whole && (col >= a.N || (a.tri && col > row))) continue;
          const int64_t X = (int64_t)(((uint64_t)xs[2 * j + 1] << 32) | xs[2 * j]);
          const int sc = erow + ebc[j];
          uint64_t bits;
          if (!oz::i64_scaled_to_f64_bits_fast(X, sc, &bits)) {
            const double slow = X == 0 ? 0.0 : ldexp((double)X, sc);
            bits = (uint64_t)__double_as_longlong(slow);
          }
          // alpha and beta arrive classified, so no FP64 compare runs per entry
          if (a.amode == 1) bits ^= (1ull << 63);
          double v = __longlong_as_double((long long)bits);
          if (a.amode == 2) v *= a.alpha;
          double* cp = a.C + (int64_t)row + (int64_t)col * a.ldc;
          if (a.bmode == 0) *cp = v;
          else if (a.bmode == 1) *cp += v;
          else *cp = fma(a.beta, *cp, v);
        }
      }
    }
  }
  __syncwarp();
  __syncthreads();
  if (threadIdx.x == 0) {
    // no MMA may still write tensor memory when it is freed
    if (!mbar_wait(&done_bar, 0, st, 43)) abort_flag = 1;
    // a failed pipeline: let the copies already issued land before shared memory is released
    if (abort_flag)
      for (int it = consumed; it < issued; ++it)
        mbar_wait(&full_bar[it % STAGES], (it / STAGES) & 1, st, 44);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

// ---- few-column products from kept slices (stream-K) ------------------------
// C (M x N, N <= 32) = A B with A's slices cut once (OzSplit) and K long: the work is
// the list of (row tile, 192-long K chunk) items in tile-major order, cut into equal
// contiguous ranges, one per CTA, so every SM streams the same share of A's slices in a
// single launch.  Per A slice s and 16-long K step one MMA multiplies it by B's slices
// t = 0 .. 7 - s at once: B's slices lie in shared memory in reverse order (slot p holds
// slice 7 - p), so the window of slots s .. 7 is N = (8 - s) nmma wide and its column
// block j always holds diagonal s + t = 7 - j.  Eight MMAs per K step (N = 8 nmma down to
// nmma) do the 36 slice pairs' work; a chunk's eight diagonal accumulators go to one of
// two TMEM sets (the MMAs of the next chunk run while the epilogue folds this one).  The
// first MMA of a chunk (s = 0) spans every block and overwrites it.  The epilogue turns every chunk
// into binary64 (exact integer, one rounding) and sums the chunks of a tile in FP64
// registers.  A tile whose chunks all lie in one range is stored; a tile cut between two
// ranges is added by both CTAs into the zeroed C with atomicAdd -- two addends onto zero,
// so the result does not depend on their order.
constexpr int NW_EPI_WARPS = 4;                         // one per TMEM lane quarter
constexpr int NW_THREADS = (2 + NW_EPI_WARPS) * 32;
constexpr int NW_NMAX = 32;
constexpr int NW_DIAGS = OZ_DMAX + 1;                   // diagonals s + t = 0 .. 7
constexpr int NW_SET_COLS = NW_DIAGS * NW_NMAX;         // 256 columns per accumulator set
constexpr int NW_TMEM_COLS = 512;
constexpr int NW_MAX_STAGES = 3;
constexpr int NW_COPIES = 8;                            // bulk copies per A stage (8 KB each)
static_assert(NW_COPIES == OZ_S, "one copy lane per B slice");
// stages of A_BYTES + 8 nmma 64 bytes: three of 72 KB for nmma = 16, two of 80 KB for 32
__host__ __device__ constexpr int nw_stage_bytes(int nmma) { return A_BYTES + OZ_S * nmma * TK * 2; }
__host__ __device__ constexpr int nw_stages(int nmma) { return nmma <= 16 ? 3 : 2; }
constexpr int NW_SMEM = 3 * nw_stage_bytes(16) + 1024;
static_assert(NW_SMEM >= 2 * nw_stage_bytes(32) + 1024, "ring sized for the widest stage");
static_assert(2 * NW_SET_COLS <= NW_TMEM_COLS, "two accumulator sets exceed tensor memory");

struct NarrowArgs {
  int M, N, nmma;          // rows, columns (<= nmma), MMA width (16 or 32)
  int K, nkc;              // K and its 192-long chunks
  int64_t items, per_cta;  // (tile, chunk) items and the items of one CTA's range
  int stages, stage_bytes; // ring depth and stride (nw_stages / nw_stage_bytes of nmma)
  const uint8_t* Ablk;     // A's kept slices, 64 KB per (row tile, K block)
  int64_t nkb;             // K blocks of A
  double* C;
  int64_t ldc;
  const int* ea;
  const int* eb;
};

template <int NMMA>
__global__ void __launch_bounds__(NW_THREADS, 1) oz_narrow_kernel(
    const __grid_constant__ CUtensorMap mapB, const NarrowArgs a, DevStatus* st) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[NW_MAX_STAGES], empty_bar[NW_MAX_STAGES], acc_full[2],
      acc_empty[2], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, issued, consumed, skip;
  if (threadIdx.x == 0) skip = *(volatile int*)&st->code;
  __syncthreads();
  if (skip) return;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i0 = (int64_t)blockIdx.x * a.per_cta;
  const int64_t i1 = (i0 + a.per_cta) < a.items ? (i0 + a.per_cta) : a.items;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(NW_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < a.stages; ++q) {
      mbar_init(&full_bar[q], 1);
      mbar_init(&empty_bar[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&acc_full[q], 1);
      mbar_init(&acc_empty[q], NW_EPI_WARPS);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    issued = 0;
    consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t b_bytes = (uint32_t)(OZ_S * a.nmma * TK * 2);

  if (warp == 0) {
    // producer warp: lane 0 waits for a free stage and posts the byte count; the A block
    // then goes as NW_COPIES bulk copies issued by as many lanes (one copy per lane keeps
    // several requests in flight), B as one tensor copy
    uint32_t it = 0;
    bool stop = false;
    for (int64_t i = i0; i < i1 && !stop; ++i) {
      const int tile = (int)(i / a.nkc), kc = (int)(i % a.nkc);
      const int kbeg = kc * OZ_KCHUNK;
      const int klen = (a.K - kbeg) < OZ_KCHUNK ? (a.K - kbeg) : OZ_KCHUNK;
      const int nkb = (klen + TK - 1) / TK;
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int q = (int)(it % (uint32_t)a.stages);
        const uint32_t use = it / (uint32_t)a.stages;
        int ok = 1;
        if (lane == 0) {
          if (*(volatile int*)&abort_flag ||
              (it >= (uint32_t)a.stages && !mbar_wait(&empty_bar[q], (use - 1) & 1, st, 51))) {
            *(volatile int*)&abort_flag = 1;
            ok = 0;
          } else {
            mbar_expect_tx(&full_bar[q], A_BYTES + b_bytes);
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          stop = true;
          break;
        }
        uint8_t* sa = smem + q * a.stage_bytes;
        uint8_t* sb = sa + A_BYTES;
        // A: one 64 KB block, already in the swizzled shared-memory image
        const uint8_t* src = a.Ablk + ((int64_t)tile * a.nkb + kbeg / TK + kb) * (int64_t)A_BYTES;
        if (lane < NW_COPIES) {
          dev::bulk_g2s(sa + lane * (A_BYTES / NW_COPIES), src + lane * (A_BYTES / NW_COPIES),
                        A_BYTES / NW_COPIES, &full_bar[q]);
          // B slice t = lane into slot 7 - t
          tma_load_3d(sb + (OZ_S - 1 - lane) * (b_bytes / OZ_S), &mapB, &full_bar[q],
                      kbeg + kb * TK, 0, lane);
        }
        if (lane == 0) *(volatile int*)&issued = (int)(it + 1);
        __syncwarp();
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t b_slice = (uint32_t)(NMMA * TK * 2);
      uint32_t it = 0;
      bool ok = true;
      for (int64_t i = i0; ok && i < i1 && !*(volatile int*)&abort_flag; ++i) {
        const int64_t li = i - i0;
        const int set = (int)(li & 1);
        const int kc = (int)(i % a.nkc);
        const int kbeg = kc * OZ_KCHUNK;
        const int klen = (a.K - kbeg) < OZ_KCHUNK ? (a.K - kbeg) : OZ_KCHUNK;
        const int nkb = (klen + TK - 1) / TK;
        // the epilogue must have taken this set's previous chunk
        if (li >= 2 && !mbar_wait(&acc_empty[set], (uint32_t)(((li >> 1) - 1) & 1), st, 56)) {
          *(volatile int*)&abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t tset = tmem + (uint32_t)(set * NW_SET_COLS);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int q = (int)(it % (uint32_t)a.stages);
          if (!mbar_wait(&full_bar[q], (it / (uint32_t)a.stages) & 1, st, 52)) {
            *(volatile int*)&abort_flag = 1;
            ok = false;
            break;
          }
          *(volatile int*)&consumed = (int)(it + 1);
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(smem + q * a.stage_bytes);
          // descriptors of the stage, offsets in 16-byte units added per slice and K step
          // (the address field cannot overflow below 256 KB of shared memory)
          const uint64_t dA0 = smem_desc(sa), dB0 = smem_desc(sa + A_BYTES);
          const uint32_t kb0 = kb == 0 ? 0u : 1u;
#pragma unroll
          for (int si = 0; si < OZ_S; ++si) {
            // slots si .. 7 hold B slices 7 - si .. 0: diagonal 7 - j in column block j
            const uint64_t da = dA0 + (uint64_t)((si * A_SLICE) >> 4);
            const uint64_t db = dB0 + (uint64_t)((si * b_slice) >> 4);
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk) {
              // the chunk's first MMA (slice 0 spans all eight blocks) overwrites the set
              const uint32_t accum = (kk == 0 && si == 0) ? kb0 : 1u;
              mma_bf16(tset, da + 2 * kk, db + 2 * kk, idesc_for((OZ_S - si) * NMMA), accum);
            }
          }
          mma_commit(&empty_bar[q]);
        }
        mma_commit(&acc_full[set]);
      }
      mma_commit(&done_bar);
    }
  } else {
    // epilogue: a warp may read only TMEM lanes 32 (warp % 4) .. + 31: warps 2..5 cover
    // the four lane quarters (rows of the tile)
    const int quarter = warp & 3;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    double acc[NMMA];
#pragma unroll
    for (int j = 0; j < NMMA; ++j) acc[j] = 0.0;
    for (int64_t i = i0; i < i1; ++i) {
      const int64_t li = i - i0;
      const int set = (int)(li & 1);
      const int tile = (int)(i / a.nkc), kc = (int)(i % a.nkc);
      if (!mbar_wait(&acc_full[set], (uint32_t)((li >> 1) & 1), st, 57)) {
        *(volatile int*)&abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (*(volatile int*)&abort_flag) break;
      const int row = tile * TM + quarter * 32 + lane;
      const bool row_ok = row < a.M;
      const int erow = row_ok ? a.ea[row] - 56 : 0;
#pragma unroll
      for (int g = 0; g < NMMA / 16; ++g) {
        // r[d]: diagonal d, in column block 7 - d of the set
        uint32_t r[NW_DIAGS][16];
#pragma unroll
        for (int d = 0; d < NW_DIAGS; ++d)
          tmem_ld16(lane_base + (uint32_t)(set * NW_SET_COLS + (OZ_DMAX - d) * NMMA + g * 16),
                    r[d]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = g * 16 + j;
          const int i0v = __float2int_rn(__uint_as_float(r[0][j]));
          const int i1v = __float2int_rn(__uint_as_float(r[1][j]) * 256.0f);
          const int i2v = __float2int_rn(__uint_as_float(r[2][j]) * 65536.0f);
          const int i3v = __float2int_rn(__uint_as_float(r[3][j]) * 16777216.0f);
          const int i4v = __float2int_rn(__uint_as_float(r[4][j]) * 4294967296.0f);
          // diagonals 5 .. 7 summed in FP32 first, as one shared accumulator would
          const float tail = __uint_as_float(r[5][j]) +
                             (__uint_as_float(r[6][j]) + __uint_as_float(r[7][j]));
          const int igv = __float2int_rn(tail * 1099511627776.0f);
          int64_t X = (int64_t)(i0v * 256 + i1v) * 4294967296ll;
          X += (int64_t)i2v * (1 << 24);
          X += (int64_t)i3v * (1 << 16);
          X += (int64_t)i4v * (1 << 8);
          X += igv;
          const int sc = erow + (col < a.N ? a.eb[col] : 0);
          uint64_t bits;
          if (!oz::i64_scaled_to_f64_bits_fast(X, sc, &bits)) {
            const double slow = X == 0 ? 0.0 : ldexp((double)X, sc);
            bits = (uint64_t)__double_as_longlong(slow);
          }
          acc[col] += __longlong_as_double((long long)bits);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) dev::mbar_arrive(&acc_empty[set]);
      // the tile's last chunk in this range: store, or add when another range has
      // (or will have) the rest of the tile
      const bool last_here = kc == a.nkc - 1 || i + 1 == i1;
      if (last_here) {
        const int64_t tile_first = (int64_t)tile * a.nkc;
        const bool whole = tile_first >= i0 && kc == a.nkc - 1;
        if (row_ok) {
#pragma unroll
          for (int j = 0; j < NMMA; ++j) {
            if (j >= a.N) break;
            double* cp = a.C + (int64_t)row + (int64_t)j * a.ldc;
            if (whole) *cp = acc[j];
            else atomicAdd(cp, acc[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < NMMA; ++j) acc[j] = 0.0;
      }
    }
  }
  __syncwarp();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!mbar_wait(&done_bar, 0, st, 53)) abort_flag = 1;
    if (abort_flag)
      for (int it = consumed; it < issued; ++it)
        mbar_wait(&full_bar[it % a.stages], (it / a.stages) & 1, st, 54);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(NW_TMEM_COLS)
                 : "memory");
}

// ---- operand split --------------------------------------------------------
// Logical operand X (R x K): element (r, k) at src[r * rs + k * ks] (one of rs, ks is 1).
constexpr int ST = 64;   // split tile: 64 rows x 64 K

// maxb[r] = max over k of the bits of |X(r, k)| (non-negative binary64 bits order as
// unsigned integers).
__global__ void __launch_bounds__(256) oz_absmax_kernel(int64_t R, int64_t K, const double* src,
                                                        int64_t rs, int64_t ks,
                                                        unsigned long long* maxb) {
  __shared__ unsigned long long tile[ST][ST + 1];
  const int64_t r0 = (int64_t)blockIdx.x * ST, k0 = (int64_t)blockIdx.y * ST;
  const int tid = threadIdx.x;
  for (int q = tid; q < ST * ST; q += 256) {
    int rr, kk;
    if (rs == 1) { rr = q % ST; kk = q / ST; } else { kk = q % ST; rr = q / ST; }
    const int64_t r = r0 + rr, k = k0 + kk;
    unsigned long long b = 0;
    if (r < R && k < K)
      b = (unsigned long long)__double_as_longlong(fabs(src[r * rs + k * ks]));
    tile[rr][kk] = b;
  }
  __syncthreads();
  if (tid < ST) {
    const int64_t r = r0 + tid;
    unsigned long long m = 0;
    for (int kk = 0; kk < ST; ++kk) m = tile[tid][kk] > m ? tile[tid][kk] : m;
    if (r < R && m) atomicMax(maxb + r, m);
  }
}

// Slices (K-major, leading dimension ldk, slice stride R * ldk):
//   out[s][r][k] = bf16(d_s(r, k) 2^-8s),  exps[r] = e_r.
__global__ void __launch_bounds__(256) oz_split_kernel(int64_t R, int64_t K, const double* src,
                                                       int64_t rs, int64_t ks,
                                                       const unsigned long long* maxb,
                                                       __nv_bfloat16* out, int64_t ldk,
                                                       int* exps) {
  __shared__ double tile[ST][ST + 1];
  __shared__ int ex[ST];
  const int64_t r0 = (int64_t)blockIdx.x * ST, k0 = (int64_t)blockIdx.y * ST;
  const int tid = threadIdx.x;
  for (int q = tid; q < ST * ST; q += 256) {
    int rr, kk;
    if (rs == 1) { rr = q % ST; kk = q / ST; } else { kk = q % ST; rr = q / ST; }
    const int64_t r = r0 + rr, k = k0 + kk;
    tile[rr][kk] = (r < R && k < K) ? src[r * rs + k * ks] : 0.0;
  }
  if (tid < ST) {
    const int64_t r = r0 + tid;
    const int e = r < R ? oz::row_exponent(maxb[r]) : 0;
    ex[tid] = e;
    if (r < R && blockIdx.y == 0) exps[r] = e;
  }
  __syncthreads();
  const int64_t slice = R * ldk;
  // thread -> (row, pair of K entries): 32 pairs per row, 8 rows per pass
  const int kp = (tid & 31) * 2, rsub = tid >> 5;
  for (int rr = rsub; rr < ST; rr += 8) {
    const int64_t r = r0 + rr;
    const int64_t k = k0 + kp;
    if (r >= R || k >= K) continue;
    int d0[OZ_S], d1[OZ_S];
    oz::digits8(oz::f64_to_fixed64((uint64_t)__double_as_longlong(tile[rr][kp]), ex[rr]), d0);
    const bool two = (k + 1 < K);
    oz::digits8(two ? oz::f64_to_fixed64((uint64_t)__double_as_longlong(tile[rr][kp + 1]), ex[rr])
                    : 0,
                d1);
    __nv_bfloat16* o = out + r * ldk + k;
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      const float sc = __int_as_float((127 - 8 * s) << 23);   // 2^-8s
      const __nv_bfloat16 h0 = __float2bfloat16_rn((float)d0[s] * sc);
      if (two && ((k & 1) == 0)) {
        __nv_bfloat162 pr;
        pr.x = h0;
        pr.y = __float2bfloat16_rn((float)d1[s] * sc);
        *reinterpret_cast<__nv_bfloat162*>(o + s * slice) = pr;
      } else {
        o[s * slice] = h0;
        if (two) o[s * slice + 1] = __float2bfloat16_rn((float)d1[s] * sc);
      }
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 3-D map over the slices of an R x K operand: (k, row, slice), box TK x box_rows x 8;
// consecutive slices lie Rs * ldk elements apart (Rs >= R).
bool make_slice_map_ld(CUtensorMap* map, const __nv_bfloat16* base, int64_t R, int64_t K,
                       int64_t ldk, int64_t Rs, int box_rows, int box_slices = OZ_S) {
  EncodeTiledFn fn = (EncodeTiledFn)tensor_map_encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)R, (cuuint64_t)OZ_S};
  cuuint64_t strides[2] = {(cuuint64_t)ldk * 2, (cuuint64_t)(Rs * ldk) * 2};
  cuuint32_t box[3] = {(cuuint32_t)TK, (cuuint32_t)box_rows, (cuuint32_t)box_slices};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_slice_map(CUtensorMap* map, const __nv_bfloat16* base, int64_t R, int64_t K,
                    int64_t ldk, int box_rows, int box_slices = OZ_S) {
  return make_slice_map_ld(map, base, R, K, ldk, R, box_rows, box_slices);
}

ec_status grow_ws(OzWork* w, int64_t slice_elems, int64_t rows) {
  if (slice_elems > w->slices_cap) {
    if (w->slices) cudaFree(w->slices);
    w->slices = nullptr;
    w->slices_cap = 0;
    if (device_alloc((void**)&w->slices, sizeof(__nv_bfloat16) * (size_t)slice_elems) !=
        cudaSuccess) {
      cudaGetLastError();
      w->slices = nullptr;
      return EC_ERR_OOM;
    }
    w->slices_cap = slice_elems;
  }
  if (rows > w->rows_cap) {
    if (w->exps) cudaFree(w->exps);
    if (w->maxb) cudaFree(w->maxb);
    w->exps = nullptr;
    w->maxb = nullptr;
    w->rows_cap = 0;
    if (device_alloc((void**)&w->exps, sizeof(int) * (size_t)rows) != cudaSuccess ||
        device_alloc((void**)&w->maxb, sizeof(unsigned long long) * (size_t)rows) != cudaSuccess) {
      cudaGetLastError();
      return EC_ERR_OOM;
    }
    w->rows_cap = rows;
  }
  return EC_OK;
}

// Split rows [r0, r0 + R) of the logical operand into slices at `out` (ld ldk) with
// exponents at `exps`; maxb is scratch of R entries.
// Kept slices in the narrow kernel's shared-memory image: CTA (row tile t, K block kb),
// thread r = row of the tile; block (t, kb) holds slice s at s * A_SLICE, row r at 64 r,
// and the 16-byte chunk c (K values 8c .. 8c + 7) at chunk position c ^ ((r >> 1) & 3),
// the 64-byte swizzle the tensor-core descriptors read.  Rows >= R and K >= K are zero.
__global__ void __launch_bounds__(TM) oz_split_blocked_kernel(int64_t R, int64_t K,
                                                              const double* src, int64_t rs,
                                                              int64_t ks,
                                                              const unsigned long long* maxb,
                                                              uint8_t* out, int64_t nkb,
                                                              int* exps) {
  const int64_t t = blockIdx.x, kb = blockIdx.y;
  const int r = threadIdx.x;
  const int64_t row = t * TM + r;
  const bool live = row < R;
  const int e = live ? oz::row_exponent(maxb[row]) : 0;
  if (live && kb == 0) exps[row] = e;
  uint8_t* blk = out + (t * nkb + kb) * (int64_t)A_BYTES + (int64_t)r * 64;
  const int swz = (r >> 1) & 3;
  for (int c = 0; c < 4; ++c) {
    int d[8][OZ_S];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t k = kb * TK + 8 * c + j;
      const double v = (live && k < K) ? src[row * rs + k * ks] : 0.0;
      oz::digits8(oz::f64_to_fixed64((uint64_t)__double_as_longlong(v), e), d[j]);
    }
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      const float sc = __int_as_float((127 - 8 * s) << 23);   // 2^-8s
      uint32_t w4[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 pr = __floats2bfloat162_rn((float)d[2 * q][s] * sc,
                                                        (float)d[2 * q + 1][s] * sc);
        w4[q] = *reinterpret_cast<const uint32_t*>(&pr);
      }
      *reinterpret_cast<uint4*>(blk + s * A_SLICE + ((c ^ swz) * 16)) =
          make_uint4(w4[0], w4[1], w4[2], w4[3]);
    }
  }
}

void split(cudaStream_t s, int64_t R, int64_t K, const double* src, int64_t rs, int64_t ks,
           unsigned long long* maxb, __nv_bfloat16* out, int64_t ldk, int* exps) {
  cudaMemsetAsync(maxb, 0, sizeof(unsigned long long) * (size_t)R, s);
  dim3 grid((unsigned)((R + ST - 1) / ST), (unsigned)((K + ST - 1) / ST));
  oz_absmax_kernel<<<grid, 256, 0, ::ec::counted(s)>>>(R, K, src, rs, ks, maxb);
  oz_split_kernel<<<grid, 256, 0, ::ec::counted(s)>>>(R, K, src, rs, ks, maxb, out, ldk, exps);
}

}  // namespace

int64_t oz_kchunk() { return OZ_KCHUNK; }

namespace {
__global__ void set_status_kernel(DevStatus* st, int code) {
  if (atomicCAS(&st->code, 0, code) == 0) st->where = 45;
}
}  // namespace

void gemm_auto(cudaStream_t s, OzWork* oz, Op ta, Op tb, int64_t M, int64_t N, int64_t K,
               double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
               double beta, double* C, int64_t ldc, int tri, const DevStatus* st) {
  // below these sizes the split and the integer epilogue outweigh the FP64 work saved
  if (oz && M >= 64 && N >= 32 && K >= 16 && M * N >= 32768 && (!tri || M == N)) {
    const ec_status rc = oz_gemm(s, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tri, oz,
                                 const_cast<DevStatus*>(st));
    if (rc == EC_OK) return;
    if (rc != EC_ERR_OOM) {   // launched work may be incomplete: fail the pipeline
      set_status_kernel<<<1, 1, 0, ::ec::counted(s)>>>(const_cast<DevStatus*>(st), (int)rc);
      return;
    }
    // no room for the slices (nothing was launched): the FP64 kernels do the product
  }
  dgemm(s, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tri, st);
}

void oz_free(OzWork* w) {
  if (!w) return;
  if (w->slices) cudaFree(w->slices);
  if (w->exps) cudaFree(w->exps);
  if (w->maxb) cudaFree(w->maxb);
  *w = OzWork{};
}

namespace {

// MMA width (and B rows per stage) for a B block of nj columns.
int nmma_for(int64_t nj) { return nj <= 16 ? 16 : (nj <= 32 ? 32 : TN); }

// One mi x nj panel of C = alpha A B + beta C from the slices behind maps ma, mb: K in
// chunks of OZ_KCHUNK, the first with beta, the rest accumulating.
ec_status launch_panel(cudaStream_t s, const CUtensorMap& ma, const CUtensorMap& mb, int64_t mi,
                       int64_t nj, int64_t K, double alpha, double beta, double* C, int64_t ldc,
                       const int* eA, const int* eB, int tri, DevStatus* st) {
  OzArgs args{};
  args.M = (int)mi;
  args.N = (int)nj;
  args.tiles_m = (int)((mi + TM - 1) / TM);
  args.tiles_n = (int)((nj + TN - 1) / TN);
  args.alpha = alpha;
  args.C = C;
  args.ldc = ldc;
  args.ea = eA;
  args.eb = eB;
  args.tri = tri;
  args.nmma = nmma_for(nj);
  const int64_t tiles = (int64_t)args.tiles_m * args.tiles_n;
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, (int64_t)num_sms());
  for (int64_t k0 = 0; k0 < K; k0 += OZ_KCHUNK) {
    args.k0 = (int)k0;
    args.klen = (int)std::min<int64_t>(OZ_KCHUNK, K - k0);
    args.beta = k0 == 0 ? beta : 1.0;
    args.amode = alpha == 1.0 ? 0 : alpha == -1.0 ? 1 : 2;
    args.bmode = args.beta == 0.0 ? 0 : args.beta == 1.0 ? 1 : 2;
    oz_gemm_kernel<<<grid, OZ_THREADS, SMEM_BYTES, ::ec::counted(s)>>>(ma, mb, args, st);
  }
  return cudaGetLastError() == cudaSuccess ? EC_OK : EC_ERR_CUDA;
}

void set_kernel_attributes() {
  static std::atomic<unsigned long long> attr_set{0};
  if (first_on_device(attr_set))
    cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

}  // namespace

ec_status oz_presplit(cudaStream_t s, Op ta, int64_t R, int64_t K, const double* A, int64_t lda,
                      OzSplit* out) {
  oz_split_free(out);
  if (R <= 0 || K <= 0) return EC_ERR_ARG;
  if (R > (1ll << 30)) return EC_ERR_UNSUPPORTED;
  const int64_t tiles = (R + TM - 1) / TM, nkb = (K + TK - 1) / TK;
  if (nkb > 65535) return EC_ERR_UNSUPPORTED;
  unsigned long long* maxb = nullptr;
  if (device_alloc((void**)&out->blocks, (size_t)A_BYTES * (size_t)tiles * (size_t)nkb) !=
          cudaSuccess ||
      device_alloc((void**)&out->exps, sizeof(int) * (size_t)R) != cudaSuccess ||
      device_alloc((void**)&maxb, sizeof(unsigned long long) * (size_t)R) != cudaSuccess) {
    cudaGetLastError();
    if (maxb) cudaFree(maxb);
    oz_split_free(out);
    return EC_ERR_OOM;
  }
  const int64_t ars = ta == N_ ? 1 : lda, aks = ta == N_ ? lda : 1;
  cudaMemsetAsync(maxb, 0, sizeof(unsigned long long) * (size_t)R, s);
  oz_absmax_kernel<<<dim3((unsigned)((R + ST - 1) / ST), (unsigned)((K + ST - 1) / ST)), 256, 0,
                     ::ec::counted(s)>>>(R, K, A, ars, aks, maxb);
  oz_split_blocked_kernel<<<dim3((unsigned)tiles, (unsigned)nkb), TM, 0, ::ec::counted(s)>>>(
      R, K, A, ars, aks, maxb, out->blocks, nkb, out->exps);
  cudaStreamSynchronize(s);
  cudaFree(maxb);
  out->R = R;
  out->K = K;
  out->nkb = nkb;
  return cudaGetLastError() == cudaSuccess ? EC_OK : EC_ERR_CUDA;
}

void oz_split_free(OzSplit* a) {
  if (a->blocks) cudaFree(a->blocks);
  if (a->exps) cudaFree(a->exps);
  *a = OzSplit{};
}

ec_status oz_gemm_presplit(cudaStream_t s, const OzSplit& a, int64_t kuse, Op tb, int64_t N,
                           const double* B, int64_t ldb, double* C, int64_t ldc, OzWork* w,
                           DevStatus* st) {
  if (N <= 0 || a.R <= 0) return EC_OK;
  if (!w || !a.blocks || kuse <= 0 || kuse > a.K) return EC_ERR_ARG;
  if (N > (1ll << 30)) return EC_ERR_UNSUPPORTED;
  if (!tensor_map_encode_fn()) return EC_ERR_UNSUPPORTED;
  static std::atomic<unsigned long long> nw_attr{0};
  if (first_on_device(nw_attr))
  {
    cudaFuncSetAttribute(oz_narrow_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, NW_SMEM);
    cudaFuncSetAttribute(oz_narrow_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, NW_SMEM);
  }
  const int64_t ldk = a.nkb * TK;            // B's slices padded like A's K blocks
  const int64_t per_row = (int64_t)OZ_S * ldk;
  {
    const ec_status g = grow_ws(w, per_row * NW_NMAX, NW_NMAX);
    if (g != EC_OK) return g;
  }
  const int64_t brs = tb == N_ ? ldb : 1, bks = tb == N_ ? 1 : ldb;
  const int64_t tiles = (a.R + TM - 1) / TM;
  const int nkc = (int)((kuse + OZ_KCHUNK - 1) / OZ_KCHUNK);
  // ranges of at least one tile's chunks, so a tile is cut between two ranges at most
  const int64_t items = tiles * nkc;
  int64_t grid = std::min<int64_t>((int64_t)num_sms(), items / nkc);
  if (grid < 1) grid = 1;
  const int64_t per_cta = (items + grid - 1) / grid;
  grid = (items + per_cta - 1) / per_cta;
  if (cudaMemset2DAsync(C, sizeof(double) * (size_t)ldc, 0, sizeof(double) * (size_t)a.R,
                        (size_t)N, s) != cudaSuccess)
    return EC_ERR_CUDA;
  for (int64_t j0 = 0; j0 < N; j0 += NW_NMAX) {
    const int64_t nj = std::min<int64_t>(NW_NMAX, N - j0);
    split(s, nj, kuse, B + j0 * brs, brs, bks, w->maxb, w->slices, ldk, w->exps);
    const int nm = nmma_for(nj);
    CUtensorMap mb;
    if (!make_slice_map(&mb, w->slices, nj, kuse, ldk, nm, 1)) return EC_ERR_CUDA;
    NarrowArgs na{};
    na.M = (int)a.R;
    na.N = (int)nj;
    na.nmma = nm;
    na.K = (int)kuse;
    na.nkc = nkc;
    na.stages = nw_stages(nm);
    na.stage_bytes = nw_stage_bytes(nm);
    na.items = items;
    na.per_cta = per_cta;
    na.C = C + j0 * ldc;
    na.ldc = ldc;
    na.ea = a.exps;
    na.eb = w->exps;
    na.Ablk = a.blocks;
    na.nkb = a.nkb;
    if (nm == 16)
      oz_narrow_kernel<16><<<(unsigned)grid, NW_THREADS, NW_SMEM, ::ec::counted(s)>>>(mb, na, st);
    else
      oz_narrow_kernel<32><<<(unsigned)grid, NW_THREADS, NW_SMEM, ::ec::counted(s)>>>(mb, na, st);
    if (cudaGetLastError() != cudaSuccess) return EC_ERR_CUDA;
  }
  return EC_OK;
}

ec_status oz_gemm(cudaStream_t s, Op ta, Op tb, int64_t M, int64_t N, int64_t K, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                  double* C, int64_t ldc, int tri, OzWork* w, DevStatus* st) {
  if (M <= 0 || N <= 0) return EC_OK;
  if (!w || K < 0) return EC_ERR_ARG;
  if (K == 0) {
    if (beta != 1.0) {
      // C = beta C: no product; done with the FP64 kernels' K = 0 path
      dgemm(s, N_, N_, M, N, 0, alpha, A, lda, B, ldb, beta, C, ldc, tri, st);
    }
    return EC_OK;
  }
  if (tri && M != N) return EC_ERR_ARG;
  if (M > (1ll << 30) || N > (1ll << 30)) return EC_ERR_UNSUPPORTED;
  if (!tensor_map_encode_fn()) return EC_ERR_UNSUPPORTED;
  set_kernel_attributes();
  const int64_t ldk = (K + 7) / 8 * 8;
  // panels so that the slices of one A panel and one B panel fit the workspace cap
  const int64_t per_row = (int64_t)OZ_S * ldk;
  int64_t cap_rows = w->cap_elems / per_row;
  if (cap_rows < 2 * TM) cap_rows = 2 * TM;
  int64_t pm = M, pn = N;
  if (pm + pn > cap_rows) {
    pm = std::min<int64_t>(M, std::max<int64_t>(TM, cap_rows / 2 / TM * TM));
    pn = std::min<int64_t>(N, std::max<int64_t>(TN, (cap_rows - pm) / TN * TN));
  }
  if (tri) {            // square lower-triangle update: panels of equal size along both
    pm = pn = std::min(pm, pn) / TM * TM;
    if (pm < TM) pm = pn = TM;
  }
  {
    const ec_status g = grow_ws(w, per_row * (pm + pn), pm + pn);
    if (g != EC_OK) return g;
  }
  __nv_bfloat16* sA = w->slices;
  __nv_bfloat16* sB = w->slices + per_row * pm;
  int* eA = w->exps;
  int* eB = w->exps + pm;
  // op(A) row r, k: A[r + k lda] (N) or A[k + r lda] (T); op(B) column c, k:
  // B[k + c ldb] (N) or B[c + k ldb] (T)
  const int64_t ars = ta == N_ ? 1 : lda, aks = ta == N_ ? lda : 1;
  const int64_t brs = tb == N_ ? ldb : 1, bks = tb == N_ ? 1 : ldb;
  for (int64_t i0 = 0; i0 < M; i0 += pm) {
    const int64_t mi = std::min(pm, M - i0);
    split(s, mi, K, A + i0 * ars, ars, aks, w->maxb, sA, ldk, eA);
    for (int64_t j0 = 0; j0 < N; j0 += pn) {
      const int64_t nj = std::min(pn, N - j0);
      if (tri && j0 > i0 + mi - 1) break;            // panel entirely above the diagonal
      split(s, nj, K, B + j0 * brs, brs, bks, w->maxb + pm, sB, ldk, eB);
      CUtensorMap ma, mb;
      if (!make_slice_map(&ma, sA, mi, K, ldk, TM) ||
          !make_slice_map(&mb, sB, nj, K, ldk, nmma_for(nj)))
        return EC_ERR_CUDA;
      // a tri panel on the diagonal (i0 == j0) keeps rows >= columns; a panel below it
      // is full
      const ec_status rc = launch_panel(s, ma, mb, mi, nj, K, alpha, beta, C + i0 + j0 * ldc,
                                        ldc, eA, eB, (tri && i0 == j0) ? 1 : 0, st);
      if (rc != EC_OK) return rc;
    }
  }
  return EC_OK;
}

}  // namespace ec

extern "C" ec_status ec_gemm_f64_emulated(int ta, int tb, int64_t M, int64_t N, int64_t K,
                                          double alpha, const double* A, int64_t lda,
                                          const double* B, int64_t ldb, double beta, double* C,
                                          int64_t ldc, int lower, void* stream) {
  using namespace ec;
  if ((ta != 0 && ta != 1) || (tb != 0 && tb != 1) || M < 0 || N < 0 || K < 0) return EC_ERR_ARG;
  if (M == 0 || N == 0) return EC_OK;
  if (!A || !B || !C) return EC_ERR_ARG;
  const int64_t arows = ta ? K : M, brows = tb ? N : K;
  if (lda < (arows > 1 ? arows : 1) || ldb < (brows > 1 ? brows : 1) || ldc < M) return EC_ERR_ARG;
  if ((lower & ~3) != 0) return EC_ERR_ARG;
  const bool presplit = (lower & 2) != 0 && K > 0;
  lower &= 1;
  if (presplit && (lower || alpha != 1.0 || beta != 0.0)) return EC_ERR_ARG;
  if (lower && M != N) return EC_ERR_SHAPE;
  cudaStream_t s = (cudaStream_t)stream;
  DevStatus* st = nullptr;
  if (device_alloc((void**)&st, sizeof(DevStatus)) != cudaSuccess) {
    cudaGetLastError();
    return EC_ERR_OOM;
  }
  cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
  OzWork w;
  ec_status rc = EC_OK;
  if (presplit) {
    OzSplit sa;
    rc = oz_presplit(s, ta ? T_ : N_, M, K, A, lda, &sa);
    if (rc == EC_OK)
      rc = oz_gemm_presplit(s, sa, K, tb ? T_ : N_, N, B, ldb, C, ldc, &w, st);
    cudaStreamSynchronize(s);
    oz_split_free(&sa);
  } else {
    rc = oz_gemm(s, ta ? T_ : N_, tb ? T_ : N_, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                 lower ? 1 : 0, &w, st);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  DevStatus h{};
  if (e == cudaSuccess) e = cudaMemcpy(&h, st, sizeof(h), cudaMemcpyDeviceToHost);
  oz_free(&w);
  cudaFree(st);
  if (rc != EC_OK) return rc;
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? EC_ERR_OOM : EC_ERR_CUDA;
  return h.code ? (ec_status)h.code : EC_OK;
}
