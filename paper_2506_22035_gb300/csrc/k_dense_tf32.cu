// Instantiates the DenseTF32 stencil kernels (one translation unit per mode so
// the build compiles them in parallel).
#include "launch_impl.cuh"

namespace spider {
cudaError_t launch_dense_tf32(int cls, int r, const LaunchCtx& ctx) { return launch_mode<Mode::DenseTF32>(cls, r, ctx); }
}  // namespace spider
