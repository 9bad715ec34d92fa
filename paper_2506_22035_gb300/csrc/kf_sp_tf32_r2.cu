// Instantiates the fused TF32 sparse kernels for radius 2 (one translation
// unit per radius so the build compiles them in parallel).
#include "launch_impl.cuh"

namespace spider {
cudaError_t launch_fused_sp_tf32_r2(int T, const LaunchCtx& ctx) { return launch_fused_r<Mode::SpTF32, 2>(T, ctx); }
}  // namespace spider
