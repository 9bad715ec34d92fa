// Dispatch of 3-D fused passes, sparse TF32 (one translation unit).
#include "launch_impl.cuh"

namespace spider {
cudaError_t launch_fused3d_sp_tf32(int r, int T, const LaunchCtx& ctx) {
  return launch_fused3d_mode<Mode::SpTF32>(r, T, ctx);
}
}  // namespace spider
