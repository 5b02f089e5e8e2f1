// Modal form (Sec. 3.2 and Sec. 3.3.2): one-time generalised eigensolve and the
// per-mode theta-recurrence.
#pragma once

#include <vector>

#include "ec_kernels.h"

namespace ec {

struct ModalState;

struct ModalSetupArgs {
  int64_t n, n0;
  int m, S, P;
  double* Li;          // n0 x n0 block of Q^T L Q (ld), overwritten
  double* Ri;          // n0 x n0 block of Q^T R Q (ld), overwritten by its Cholesky factor
  int64_t ld;
  const double* Gsrc;  // n0 x (2m + S) source columns (for the projections)
  const double* RD;    // n0 x m
  const double* LD;    // n0 x m
  const double* Msrc;  // n0 x S  (ld ldM)
  int64_t ldM;
  const double* CK;    // n0 x P  ((C K)^T, ld ldC)
  int64_t ldC;
  double theta, dt;
  int precision;       // EC_PREC_*
  int integ;           // EC_INTEG_*
  int rhs_mode;        // EC_RHS_*
  int gemm;            // EC_GEMM_*: the setup's dense products on the tensor cores or FP64 cores
  DevStatus* st;
};

ModalState* modal_create();
void modal_free(ModalState* ms);
ec_status modal_setup(cudaStream_t s, ModalState* ms, const ModalSetupArgs& a, ec_timing* tim);
ec_status modal_set_step(cudaStream_t s, ModalState* ms, double theta, double dt);
// Switch the arithmetic of the products with U (EC_PREC_*): rebuilds the reduced copy
// of U and the projections from the same modes; the modal state is kept.
ec_status modal_set_precision(cudaStream_t s, ModalState* ms, int precision, const double* RD,
                              const double* LD, const double* Msrc, int64_t ldM,
                              const double* CK, int64_t ldC, DevStatus* st);
// ev (optional): receives an event pair around every scan launch.
ec_status modal_run(cudaStream_t s, ModalState* ms, const StepArgs& a,
                    std::vector<cudaEvent_t>* ev = nullptr);
double* modal_state(ModalState* ms);
int64_t modal_state_size(const ModalState* ms);
// Integrate only the nkeep modes of largest tau; the others are held at zero.
ec_status modal_set_mode_count(cudaStream_t s, ModalState* ms, int64_t nkeep);
const double* modal_tau(ModalState* ms);
const double* modal_U(ModalState* ms);
// x = U^T R_i I_i for an internal current I_i (device, length n0)
void modal_set_internal_current(cudaStream_t s, ModalState* ms, const double* Ii);

}  // namespace ec
