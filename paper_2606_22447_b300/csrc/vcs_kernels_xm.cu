// Step kernel instantiations for batches that hold Superchip or E0 carts
// (extended mappers: the Superchip's 128 bytes of cartridge RAM live in RAM
// words 32..63 and the bus decodes its ports; E0 maps 1 KB slices into the
// four segments of the cartridge window); compiled apart from
// vcs_kernels.cu so the two build in parallel.
#include <cuda_runtime.h>

#include "vcs_step.cuh"

namespace vcs {

int launch_step_xm(const StepParams& p, int n_blocks, int E, void* stream) {
  return launch_run<false, true, false>(p, n_blocks, E, stream);
}

int launch_soft_forward_xm(const StepParams& p, int n_blocks, int E, void* stream) {
  return launch_run<true, true, false>(p, n_blocks, E, stream);
}

}  // namespace vcs
