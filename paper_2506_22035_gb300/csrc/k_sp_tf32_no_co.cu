// Instantiates the SpTF32NoCO stencil kernel: SPIDER without the computing
// optimisations of Sec. 3.3 (kernel-matrix operands read from shared memory
// by every MMA instead of kept in registers; 2-D grids only, the one-step
// tile of launch_class).
#include "launch_impl.cuh"

namespace spider {
cudaError_t launch_sp_tf32_no_co(int cls, int r, const LaunchCtx& ctx) {
  if (cls != 2) return cudaErrorNotSupported;
  switch (r) {
    case 1: return launch_cfg<TileCfg<0, 1, 1, 1, 4, 2, 16>, Mode::SpTF32NoCO>(ctx);
    case 2: return launch_cfg<TileCfg<0, 2, 2, 1, 4, 2, 16>, Mode::SpTF32NoCO>(ctx);
    case 3: return launch_cfg<TileCfg<0, 3, 3, 1, 4, 2, 16>, Mode::SpTF32NoCO>(ctx);
    default: return cudaErrorNotSupported;
  }
}
}  // namespace spider
