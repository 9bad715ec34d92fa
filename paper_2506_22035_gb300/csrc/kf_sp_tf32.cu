// Fused TF32 sparse kernels: dispatch on the radius to the per-radius
// translation units.
#include "launch.h"

namespace spider {
cudaError_t launch_fused_sp_tf32_r1(int T, const LaunchCtx& ctx);
cudaError_t launch_fused_sp_tf32_r2(int T, const LaunchCtx& ctx);
cudaError_t launch_fused_sp_tf32_r3(int T, const LaunchCtx& ctx);

cudaError_t launch_fused_sp_tf32(int r, int T, const LaunchCtx& ctx) {
  switch (r) {
    case 1: return launch_fused_sp_tf32_r1(T, ctx);
    case 2: return launch_fused_sp_tf32_r2(T, ctx);
    case 3: return launch_fused_sp_tf32_r3(T, ctx);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace spider
