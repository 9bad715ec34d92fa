// Host-side launch of one stencil time step.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "spider_internal.h"

namespace spider {

struct LaunchCtx {
  const spider_plan_t* plan;
  const float* src;
  float* dst;
  cudaStream_t stream;
  int sms;
  // TF32 modes only: the source grid holds values already rounded to TF32
  // (written by the previous pass with out_tf32), and the destination grid
  // is read by a later pass, so it may be stored rounded.
  bool in_tf32 = false;
  bool out_tf32 = false;
  // Row pitches of src and dst in floats (0: nx, the packed layout).  A
  // padded source must be TMA-describable; planes are ny * pitch apart.
  int64_t src_pitch = 0;
  int64_t dst_pitch = 0;
};

// Launches one time step src -> dst for the plan's engine and precision.
// Returns cudaSuccess, or the launch/tensor-map error.
cudaError_t launch_step(const LaunchCtx& ctx);

// Per-mode dispatchers (one translation unit each, compiled in parallel).
// `cls` is 1, 2 or 3 (stencil dimensionality), r the radius.
// Each returns cudaErrorNotSupported when it has no kernel for (cls, r).
cudaError_t launch_sp_tf32(int cls, int r, const LaunchCtx& ctx);
cudaError_t launch_sp_f16x2(int cls, int r, const LaunchCtx& ctx);
cudaError_t launch_sp_bf16x3(int cls, int r, const LaunchCtx& ctx);
cudaError_t launch_dense_tf32(int cls, int r, const LaunchCtx& ctx);
cudaError_t launch_cuda_core(int cls, int r, const LaunchCtx& ctx);
// SPIDER_ENGINE_SPARSE_TC_COPY: the explicit row-swap copy (2-D only).
cudaError_t launch_sp_tf32_copy(int cls, int r, const LaunchCtx& ctx);
// SPIDER_ENGINE_SPARSE_TC_NO_CO: operands from shared memory per MMA (2-D only).
cudaError_t launch_sp_tf32_no_co(int cls, int r, const LaunchCtx& ctx);
// Radius 4..7 (1-D and 2-D), sparse TF32, wide layout.
cudaError_t launch_wide_sp_tf32(int cls, int r, const LaunchCtx& ctx);
// Fused passes of T = 2..4 steps for 1-D sparse TF32 plans (wide layout,
// lengths that are a multiple of 8).
cudaError_t launch_wide1d_fused_sp_tf32(int r, int T, const LaunchCtx& ctx);

// Fused passes of T = 2..4 time steps (2-D stencils, TMA-aligned grids).
// cudaErrorNotSupported when no fused kernel applies; the caller then runs
// single steps.
cudaError_t launch_pass(const LaunchCtx& ctx, int T);
cudaError_t launch_fused_sp_tf32(int r, int T, const LaunchCtx& ctx);
cudaError_t launch_fused_sp_f16x2(int r, int T, const LaunchCtx& ctx);
cudaError_t launch_fused_sp_bf16x3(int r, int T, const LaunchCtx& ctx);
cudaError_t launch_fused_dense_tf32(int r, int T, const LaunchCtx& ctx);
cudaError_t launch_fused_cuda_core(int r, int T, const LaunchCtx& ctx);
// Fused passes of T = 2..4 time steps for 3-D stencils of radius 1 (TF32
// modes, TMA-describable grids).
cudaError_t launch_fused3d_sp_tf32(int r, int T, const LaunchCtx& ctx);

// Deepest 2-D fusion built for the sparse TF32 mode: radius 1 up to 10 steps
// per pass (deep tiles of 5..10 for small grids), radius 2 and 3 up to 4.
// Deep tiles of 5..6 steps for radius 2 and 3 were built and measured: the
// autotuner never chose them on 512^2..2048^2 grids (the halo of 2r rows per
// level costs more than the passes saved).
constexpr int max_deep_steps(int r) { return r == 1 ? 10 : 4; }

// Builds a 3-D tiled tensor map over a float32 grid (nz, ny, nx) with the
// given box; out-of-range box elements read as zero.  Returns false if the
// grid cannot be described (row pitch or base not 16-byte aligned).
bool make_tensor_map(CUtensorMap* map, const float* base, int64_t nx, int64_t ny, int64_t nz, int box_x, int box_y,
                     int box_z);
// The same for a grid whose rows start `pitch` floats apart (pitch >= nx,
// pitch * 4 a multiple of 16; planes ny * pitch apart): box elements at
// x >= nx read as zero, so whatever the row padding holds is never loaded.
bool make_tensor_map_pitched(CUtensorMap* map, const float* base, int64_t nx, int64_t ny, int64_t nz, int64_t pitch,
                             int box_x, int box_y, int box_z);

int device_sm_count();

// Limit of the kernels' bounded waits in SM cycles (spider_set_wait_limit).
long long wait_limit_cycles();

}  // namespace spider
