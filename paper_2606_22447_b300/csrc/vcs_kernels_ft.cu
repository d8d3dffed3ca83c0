// Step kernel instantiations for batches with the whole TIA (player 1, the
// missiles, the ball and the collision latches; vcs_tia.cuh), which also
// take every cartridge format; compiled apart from the other two so the
// three build in parallel.
#include <cuda_runtime.h>

#include "vcs_step.cuh"

namespace vcs {

int launch_step_ft(const StepParams& p, int n_blocks, int E, void* stream) {
  return launch_run<false, true, true>(p, n_blocks, E, stream);
}

int launch_soft_forward_ft(const StepParams& p, int n_blocks, int E, void* stream) {
  return launch_run<true, true, true>(p, n_blocks, E, stream);
}

}  // namespace vcs
