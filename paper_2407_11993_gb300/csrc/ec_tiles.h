// Inverse-factor products on packed lower-triangular tiles (ec_tiles.cu).
#pragma once

#include "ec_internal.h"

namespace ec {

// Work decomposition of the two products y = W b and x = W^T y for a lower
// triangular W of order n stored as packed 64 x 64 tiles.
//   * tile (I, J), J <= I, is tile number I (I + 1) / 2 + J, 4096 doubles;
//     element (r, c) of the tile sits at c * 64 + (r ^ c) (an XOR swizzle that
//     keeps both products free of shared-memory bank conflicts); rows / columns
//     past n and the upper half of diagonal tiles hold zeros;
//   * a unit is a run of at most `chunk` consecutive tiles of one tile row
//     (forward product) or one tile column (transposed product); unit (I, c)
//     writes the partial sums of outputs I*64 .. I*64+63 over inner-index
//     quarter q (inner index mod 64 in q*16 .. q*16+15) into partial row 4c + q;
//   * partial arrays are 4 ((nblk - 1) / chunk + 1) rows of npad doubles.
constexpr int TILE_VARIANTS = 3;   // launch shapes of the product kernels

struct TilePlan {
  int64_t n = 0, nblk = 0, npad = 0, ntiles = 0, nunits = 0;
  int chunk = 1;
  int variant = 0;              // launch shape in use (index into the variant table)
  int grids[TILE_VARIANTS] = {};   // CTAs per launch of each shape
  float tune_ms[TILE_VARIANTS] = {};   // autotuner: time of one product pair per shape
  int4* units_fwd = nullptr;    // device, nunits entries (0, I, c, 0), largest first
  int4* units_bwd = nullptr;    // device, nunits entries (0, J, c, 0)
};

ec_status tile_plan_create(int64_t n, TilePlan* p);
void tile_plan_free(TilePlan* p);
inline int64_t tile_partial_rows(const TilePlan& p) { return 4 * ((p.nblk - 1) / p.chunk + 1); }
inline size_t tile_packed_doubles(const TilePlan& p) { return (size_t)p.ntiles * 4096; }

// Packed tiles <- lower triangle of the column-major W (n x n, ld ldw), the
// diagonal multiplied by diag_scale.
void tile_pack_lower(cudaStream_t s, const TilePlan& p, const double* W, int64_t ldw,
                     double* Wp, double diag_scale = 1.0);
// The same, rounded to FP32 entries (same layout, half the bytes).
void tile_pack_lower_f32(cudaStream_t s, const TilePlan& p, const double* W, int64_t ldw,
                         float* Wp);
// Column-major W (n x n, ld ldw) <- packed tiles, zeros above the diagonal.
void tile_unpack_lower(cudaStream_t s, const TilePlan& p, const double* Wp, double* W,
                       int64_t ldw);

// x = W^T (W b): y = W b (partials part1, summed into y), then W^T y (partials
// part2, summed into x).  b and y hold npad doubles whose entries past n are zero
// (y's tail is never written); x may alias b.  part1 / part2 hold
// tile_partial_rows(p) x npad doubles.  ev (optional, 3 events) is recorded before
// the forward product, right after it, and right after the transposed product.
void tile_trmv_pair(cudaStream_t s, const TilePlan& p, const double* Wp, const double* b,
                    double* part1, double* y, double* part2, double* x, DevStatus* st,
                    cudaEvent_t* ev = nullptr);

// The same pair with an FP32 factor: the vectors are rounded to FP32 (b into v32, y
// again into v32 by the partial-sum kernel), products and sums within each unit are
// FP32, partial rows and y, x are FP64.  v32: npad floats with a zero tail.
// accumulate = 1 adds the result into x instead of overwriting it (x must then not
// alias b).
void tile_trmv_pair_f32(cudaStream_t s, const TilePlan& p, const float* Wp, const double* b,
                        float* v32, double* part1, double* y, double* part2, double* x,
                        int accumulate, DevStatus* st, cudaEvent_t* ev = nullptr);

// Symmetric product from a half: with Hp the packed lower triangle of H (diagonal
// included), out1 = H x and out2 = H^T-part: out1 + out2 = (H + H^T) x.  Packing a
// symmetric S with diag_scale 0.5 gives out1 + out2 = S x.
void tile_sym_product(cudaStream_t s, const TilePlan& p, const double* Hp, const double* x,
                      double* part1, double* part2, double* out1, double* out2, DevStatus* st);

// Self-tuning of the launch shape: times every shape on the actual factor (one
// warm-up and three timed product pairs each, synchronising the stream) and keeps
// the fastest.  forced in 1 .. TILE_VARIANTS selects shape forced - 1 instead.
// The shapes differ only in how work is mapped to warps and CTAs, not in the order
// of any sum, so the choice never changes a result bit.
ec_status tile_autotune(cudaStream_t s, TilePlan* p, const double* Wp, const double* b,
                        double* part1, double* y, double* part2, DevStatus* st, int forced);
// The same for an FP32 factor.
ec_status tile_autotune_f32(cudaStream_t s, TilePlan* p, const float* Wp, const double* b,
                            float* v32, double* part1, double* y, double* part2, DevStatus* st,
                            int forced);

// FP32 hi/lo pair factor (EC_PREC_FP32X2): packed tiles of {fp32(w), fp32(w - hi)} (8 bytes
// per entry, as FP64), products in compensated FP32 arithmetic with FP64 partial rows.
// vx2: pair copy of the product input (npad entries, zero tail).
void tile_pack_lower_x2(cudaStream_t s, const TilePlan& p, const double* W, int64_t ldw,
                        float2* Wp);
void tile_trmv_pair_x2(cudaStream_t s, const TilePlan& p, const float2* Wp, const double* b,
                       float2* vx2, double* part1, double* y, double* part2, double* x,
                       DevStatus* st, cudaEvent_t* ev = nullptr);
ec_status tile_autotune_x2(cudaStream_t s, TilePlan* p, const float2* Wp, const double* b,
                           float2* vx2, double* part1, double* y, double* part2, DevStatus* st,
                           int forced);

// out[i] = sum over the partial rows unit products wrote for row i, in row order
// (trans = 0: partials of W b; trans = 1: partials of W^T y).
void tile_sum(cudaStream_t s, const TilePlan& p, int trans, const double* part, double* out);

// ---- batches: the products of up to TILE_BATCH_MAX instances in one launch ----
// Every instance keeps its own plan (tiles, unit decomposition, partial rows), so
// a batched product computes bit for bit what the instance's own launch computes;
// the batch merges all instances' units into one largest-first list dealt to one
// persistent grid.
constexpr int TILE_BATCH_MAX = 64;

struct TileInst {
  const TilePlan* plan;
  const double* Wp;
  const double* b;     // input (npad, zero tail)
  double* part1;
  double* y;           // W b (npad, zero tail)
  double* part2;
  double* x;           // W^T y
};

struct TileBatch {
  int count = 0;
  int64_t max_nblk = 0, nunits_fwd = 0, nunits_bwd = 0;
  int4* units_fwd = nullptr;    // device, (instance, K, c, 0), largest first
  int4* units_bwd = nullptr;
  int variant = 0;
  int grids[TILE_VARIANTS] = {};
  float tune_ms[TILE_VARIANTS] = {};
};

ec_status tile_batch_create(const TileInst* inst, int count, TileBatch* B);
void tile_batch_free(TileBatch* B);
// x_i = W_i^T (W_i b_i) for every instance: 4 launches in all.
void tile_batch_pair(cudaStream_t s, const TileBatch& B, const TileInst* inst, DevStatus* st);
// Chooses B->variant by timing every launch shape on the batch (synchronises s).
ec_status tile_batch_autotune(cudaStream_t s, TileBatch* B, const TileInst* inst, DevStatus* st);

// Sets the shared-memory attributes of every product kernel on the current device
// (idempotent; call once before capturing launches into a graph).
void tile_prepare_launches();

// Number of partial rows holding data for output i of the forward / transposed
// product (they are the first rows of the partial array).
__host__ __device__ inline int64_t tile_valid_rows(int64_t i, int chunk) {
  return 4 * ((i >> 6) / chunk + 1);
}
__host__ __device__ inline int64_t tile_valid_rows_t(int64_t i, int64_t nblk, int chunk) {
  return 4 * ((nblk - 1 - (i >> 6)) / chunk + 1);
}

}  // namespace ec
