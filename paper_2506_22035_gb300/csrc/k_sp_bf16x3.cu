// Instantiates the SpBF16x3 stencil kernels (one translation unit per mode so
// the build compiles them in parallel).
#include "launch_impl.cuh"

namespace spider {
cudaError_t launch_sp_bf16x3(int cls, int r, const LaunchCtx& ctx) { return launch_mode<Mode::SpBF16x3>(cls, r, ctx); }
}  // namespace spider
