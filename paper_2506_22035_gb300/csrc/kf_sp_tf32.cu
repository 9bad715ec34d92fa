// Instantiates the fused (T = 2..4 steps per pass) SpTF32 kernels.
#include "launch_impl.cuh"

namespace spider {
cudaError_t launch_fused_sp_tf32(int r, int T, const LaunchCtx& ctx) { return launch_fused_mode<Mode::SpTF32>(r, T, ctx); }
}  // namespace spider
