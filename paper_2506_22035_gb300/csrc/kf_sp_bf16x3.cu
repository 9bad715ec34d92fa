// Instantiates the fused (T = 2..4 steps per pass) SpBF16x3 kernels.
#include "launch_impl.cuh"

namespace spider {
cudaError_t launch_fused_sp_bf16x3(int r, int T, const LaunchCtx& ctx) { return launch_fused_mode<Mode::SpBF16x3>(r, T, ctx); }
}  // namespace spider
