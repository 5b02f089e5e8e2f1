// Declarations of the setup and stepping kernels used by the C ABI layer.
#pragma once

#include "ec_internal.h"

namespace ec {

constexpr int MAXM = 16;   // most electrode rows (N_e - 1) supported
constexpr int MAXD = 64;   // most dot products per step (probes + 2 m)

struct Csr {
  long long* ptr = nullptr;
  int* col = nullptr;
  double* val = nullptr;
  long long nnz = 0;
};

// ---- ec_elim.cu ------------------------------------------------------------
void house_qr(cudaStream_t s, int64_t n, int m, const double* E, double* V, double* T,
              double* RrinvT, DevStatus* st);
void sym_from_upper(cudaStream_t s, int64_t n, double* A, int64_t lda);
void two_sided_update(cudaStream_t s, int64_t n, int m, double* A, const double* V,
                      const double* T, double* Y, double* X, double* Sm, double* Zm,
                      const DevStatus* st);
void one_sided_qt(cudaStream_t s, int64_t n, int m, double* B, int64_t ncol, const double* V,
                  const double* T, double* S1, double* S2, const DevStatus* st);
void one_sided_q(cudaStream_t s, int64_t n, int m, double* B, int64_t ncol, const double* V,
                 const double* T, double* S1, double* S2, const DevStatus* st);
ec_status build_csr(cudaStream_t s, int64_t n, const double* A, Csr& out,
                    cudaError_t (*alloc)(void**, size_t));

// ---- ec_step.cu: per-step kernels of both forms ----------------------------
// Everything a step kernel needs, by value (device pointers + sizes).
struct StepArgs {
  int64_t n, n0;
  int m, S, P, D;              // D = P + 2 m dot products per step
  double theta, dt;
  // sources (device): src S x (T+1), iD m x (T+1), row-major
  const double* src;
  const double* iD;
  int64_t T;
  int64_t* kstep;              // device step counter within the run
  // elimination pieces (m > 0)
  const double* V;             // n x m
  const double* WR;            // n x m  (R V)
  const double* Tm;            // m x m
  const double* VtWR;          // m x m  (V^T R V)
  const double* PE;            // n x m  particular field
  const double* CPE;           // P x m  column-major: C E^T (E E^T)^{-1}
  // plain form
  Csr R;                        // CSR of the original R
  const double* Gsrc;          // n0 x (2m + S): [R_D | L_D + theta dt R_D | M_0]
  const double* Dmat;          // n0 x D: [ (C K)^T | V[m:,:] | WR[m:,:] ]
  double* Ii;                  // n0 state (plain)
  double* work;                // n0 right-hand side / solution
  double* dots;                // D values for the current state
  double* partial;             // ugrid x D partial sums
  int ugrid;                   // CTAs of this instance's update (batched launches)
  unsigned* counter;           // last-block counter
  double* probes;              // T x P output (may be null)
  double* snaps;               // nsnap x n output (may be null)
  int64_t snap_stride;
  unsigned* tickets;
  int* epoch;
  DevStatus* st;
};

void plain_rhs(cudaStream_t s, const StepArgs& a);
void plain_update(cudaStream_t s, const StepArgs& a, int grid, int mode);  // mode 0: += work; 1: dots only
void plain_snapshot(cudaStream_t s, const StepArgs& a);
// r = b - (t1 + t2) - theta dt R x: residual of Z x = b with t1 + t2 = L x (m = 0).
void plain_residual(cudaStream_t s, const StepArgs& a, const double* b, const double* x,
                    const double* t1, const double* t2, double* r);
// Batched forms over `count` instances (dA: device array of their StepArgs): one
// launch each, blockIdx.y = instance; each instance computes exactly what its own
// launch computes (the update uses the instance's own ugrid).
void plain_rhs_batch(cudaStream_t s, const StepArgs* dA, int count, int64_t max_n0);
void plain_update_batch(cudaStream_t s, const StepArgs* dA, int count, int max_grid);
void plain_snapshot_batch(cudaStream_t s, const StepArgs* dA, int count, int64_t max_n);
// Independent right-hand sides (no electrodes): out (n0 x S) = -dt R I - M_0 diag(ds^k).
void plain_rhs_multi(cudaStream_t s, const StepArgs& a, int64_t k, const double* I, double* out);
// out[r] = C[:, r] . I[:, r]
void paired_probes(cudaStream_t s, int64_t n0, int S, const double* C, int64_t ldc,
                   const double* I, double* out);
// out = R_i I_i for the state in a.Ii (needs a.dots current for that state).
void ri_apply(cudaStream_t s, const StepArgs& a, double* out);

// ---- ec_adjoint.cu: misfit gradient of the plain form ---------------------
void adj_rhs(cudaStream_t s, int64_t n, int P, double dt, const Csr& R, const double* lam_next,
             double* rhs, const double* probes_row, const double* v_row, const double* Ct);
void adj_accum(cudaStream_t s, int64_t n, int S, double dt, double theta, const double* lam,
               const double* Ik, const double* Ikm1, double* gR, const double* M, double* partial,
               unsigned* counter, double* mu_out, int64_t mu_stride, int grid);
void misfit(cudaStream_t s, int64_t count, const double* probes, const double* v, double* J);
void dsrc(cudaStream_t s, int S, int64_t T, const double* mu, double* out);

}  // namespace ec
