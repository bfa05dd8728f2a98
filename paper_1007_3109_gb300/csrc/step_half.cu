// Reduced-storage step (float rho* plus 16-bit deviations): not built yet.
#include "lbrd_kernels.h"

namespace lbrd {

StepShape step_shape_half(int64_t, int64_t) { return {dim3(max_persistent_blocks()), dim3(128)}; }

cudaError_t launch_step_half(int, int, int, const StepArgs &, cudaStream_t) { return cudaErrorNotSupported; }

cudaError_t launch_init_half(int, int, int, const InitArgs &, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace lbrd
