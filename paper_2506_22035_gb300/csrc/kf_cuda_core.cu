// Instantiates the fused (T = 2..4 steps per pass) CudaCore kernels.
#include "launch_impl.cuh"

namespace spider {
cudaError_t launch_fused_cuda_core(int r, int T, const LaunchCtx& ctx) { return launch_fused_mode<Mode::CudaCore>(r, T, ctx); }
}  // namespace spider
