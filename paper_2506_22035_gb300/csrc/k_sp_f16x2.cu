// Instantiates the SpF16x2 stencil kernels (one translation unit per mode so
// the build compiles them in parallel).
#include "launch_impl.cuh"

namespace spider {
cudaError_t launch_sp_f16x2(int cls, int r, const LaunchCtx& ctx) { return launch_mode<Mode::SpF16x2>(cls, r, ctx); }
}  // namespace spider
