// Dispatch of the wide layout (radius 4..7 in 1-D and 2-D, radius 1..3 in
// 1-D; sparse TF32).
#include "launch_impl.cuh"

namespace spider {
cudaError_t launch_wide_sp_tf32(int cls, int r, const LaunchCtx& ctx) {
  switch (r) {
    case 1: return launch_wide_r<1>(cls, ctx);
    case 2: return launch_wide_r<2>(cls, ctx);
    case 3: return launch_wide_r<3>(cls, ctx);
    case 4: return launch_wide_r<4>(cls, ctx);
    case 5: return launch_wide_r<5>(cls, ctx);
    case 6: return launch_wide_r<6>(cls, ctx);
    case 7: return launch_wide_r<7>(cls, ctx);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_wide1d_fused_sp_tf32(int r, int T, const LaunchCtx& ctx) {
  switch (r) {
    case 1: return launch_wide1d_fused_r<1>(T, ctx);
    case 2: return launch_wide1d_fused_r<2>(T, ctx);
    case 3: return launch_wide1d_fused_r<3>(T, ctx);
    case 4: return launch_wide1d_fused_r<4>(T, ctx);
    case 5: return launch_wide1d_fused_r<5>(T, ctx);
    case 6: return launch_wide1d_fused_r<6>(T, ctx);
    case 7: return launch_wide1d_fused_r<7>(T, ctx);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace spider
