// Instantiates the fused (T = 2..4 steps per pass) SpF16x2 kernels.
#include "launch_impl.cuh"

namespace spider {
cudaError_t launch_fused_sp_f16x2(int r, int T, const LaunchCtx& ctx) { return launch_fused_mode<Mode::SpF16x2>(r, T, ctx); }
}  // namespace spider
