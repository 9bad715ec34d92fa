// Instantiates the SpTF32Copy stencil kernel: SPIDER with the input row swap
// done by an explicit copy of the windows (2-D grids only).
#include "launch_impl.cuh"

namespace spider {
cudaError_t launch_sp_tf32_copy(int cls, int r, const LaunchCtx& ctx) {
  if (cls != 2) return cudaErrorNotSupported;
  return launch_mode<Mode::SpTF32Copy>(cls, r, ctx);
}
}  // namespace spider
