// step_tiled.cu -- FP32 shared-memory tiled kernel with K steps per launch
// (temporal blocking).  Placeholder until the tiled kernel lands.
#include "device_common.cuh"

namespace flood {

size_t tiled_smem_bytes(int, int, int) { return 0; }

cudaError_t launch_step_tiled(const StepArgs<float> &, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace flood
