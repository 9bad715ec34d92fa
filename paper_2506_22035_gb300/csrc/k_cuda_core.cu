// Instantiates the CudaCore stencil kernels (one translation unit per mode so
// the build compiles them in parallel).
#include "launch_impl.cuh"

namespace spider {
cudaError_t launch_cuda_core(int cls, int r, const LaunchCtx& ctx) { return launch_mode<Mode::CudaCore>(cls, r, ctx); }
}  // namespace spider
