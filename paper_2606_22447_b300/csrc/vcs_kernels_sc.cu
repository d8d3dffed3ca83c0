// Step kernel instantiations for batches that hold Superchip carts (their
// 128 bytes of cartridge RAM live in RAM words 32..63 and the bus decodes
// its ports); compiled apart from vcs_kernels.cu so the two build in
// parallel.
#include <cuda_runtime.h>

#include "vcs_step.cuh"

namespace vcs {

int launch_step_sc(const StepParams& p, int n_blocks, int E, void* stream) {
  return launch_run<false, true>(p, n_blocks, E, stream);
}

int launch_soft_forward_sc(const StepParams& p, int n_blocks, int E, void* stream) {
  return launch_run<true, true>(p, n_blocks, E, stream);
}

}  // namespace vcs
