// step_fp32.cu -- FP32-mixed explicit step (placeholder until the FP32 tile
// kernel lands: the FP64 path is the parity reference).
#include <cuda_runtime.h>

#include "cem_internal.h"

namespace cem {

cudaError_t launch_step_fp32(const DevState &, int, bool, bool, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace cem
