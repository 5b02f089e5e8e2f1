// Modal form: placeholder until the eigen pipeline lands.
#include "ec_modal.h"

namespace ec {

struct ModalState {
  double* x = nullptr;
};

ModalState* modal_create() { return new ModalState(); }
void modal_free(ModalState* ms) { delete ms; }
ec_status modal_setup(cudaStream_t, ModalState*, const ModalSetupArgs&, ec_timing*) {
  return EC_ERR_UNSUPPORTED;
}
ec_status modal_set_step(cudaStream_t, ModalState*, double, double) { return EC_ERR_UNSUPPORTED; }
ec_status modal_run(cudaStream_t, ModalState*, const StepArgs&) { return EC_ERR_UNSUPPORTED; }
double* modal_state(ModalState* ms) { return ms->x; }
const double* modal_tau(ModalState*) { return nullptr; }
const double* modal_U(ModalState*) { return nullptr; }
void modal_set_internal_current(cudaStream_t, ModalState*, const double*) {}

}  // namespace ec
