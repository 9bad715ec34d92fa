// Instantiates the fused TF32 sparse kernels for radius 1 (one translation
// unit per radius so the build compiles them in parallel), including the
// deep tiles of 5..10 steps per pass.
#include "launch_impl.cuh"

namespace spider {
cudaError_t launch_fused_sp_tf32_r1(int T, const LaunchCtx& ctx) {
  if (T > 4) return launch_fused_deep<Mode::SpTF32, 1>(T, ctx);  // 5..10 steps per pass
  return launch_fused_r<Mode::SpTF32, 1>(T, ctx);
}
}  // namespace spider
