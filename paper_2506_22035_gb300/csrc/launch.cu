// Dispatch of one stencil step to the kernel of the plan's engine/precision,
// and TMA tensor-map encoding through the driver entry point (no link-time
// dependency on libcuda).
#include <atomic>
#include <cstring>
#include <mutex>

#include "launch.h"

namespace spider {

namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}
}  // namespace

bool make_tensor_map(CUtensorMap* map, const float* base, int64_t nx, int64_t ny, int64_t nz, int box_x, int box_y,
                     int box_z) {
  return make_tensor_map_pitched(map, base, nx, ny, nz, nx, box_x, box_y, box_z);
}

bool make_tensor_map_pitched(CUtensorMap* map, const float* base, int64_t nx, int64_t ny, int64_t nz, int64_t pitch,
                             int box_x, int box_y, int box_z) {
  // TMA needs a 16-byte aligned base and row/plane pitches that are
  // multiples of 16 bytes.
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (pitch * 4) % 16 != 0 || pitch < nx) return false;
  if (pitch >= (1LL << 32) || ny >= (1LL << 32) || nz >= (1LL << 32)) return false;
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)(pitch * 4), (cuuint64_t)(pitch * ny * 4)};
  const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)box_z};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {
std::atomic<long long> g_wait_cycles{kDefaultWaitCycles};
}

long long wait_limit_cycles() { return g_wait_cycles.load(std::memory_order_relaxed); }

void set_wait_limit_cycles(long long cycles) { g_wait_cycles.store(cycles, std::memory_order_relaxed); }

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
  return sms;
}

cudaError_t launch_step(const LaunchCtx& ctx) {
  const spider_plan_t* p = ctx.plan;
  const int cls = p->ndim;
  if (p->wide()) return launch_wide_sp_tf32(cls, p->r, ctx);
  switch (p->engine) {
    case SPIDER_ENGINE_CUDA_CORE: return launch_cuda_core(cls, p->r, ctx);
    case SPIDER_ENGINE_DENSE_TC: return launch_dense_tf32(cls, p->r, ctx);
    case SPIDER_ENGINE_SPARSE_TC_COPY: return launch_sp_tf32_copy(cls, p->r, ctx);
    case SPIDER_ENGINE_SPARSE_TC_NO_CO: return launch_sp_tf32_no_co(cls, p->r, ctx);
    default: break;
  }
  switch (p->prec) {
    case SPIDER_F16X2: return launch_sp_f16x2(cls, p->r, ctx);
    case SPIDER_BF16X3: return launch_sp_bf16x3(cls, p->r, ctx);
    default: return launch_sp_tf32(cls, p->r, ctx);
  }
}

}  // namespace spider

namespace spider {

cudaError_t launch_pass(const LaunchCtx& ctx, int T) {
  if (T <= 1) return launch_step(ctx);
  const spider_plan_t* p = ctx.plan;
  if (p->engine == SPIDER_ENGINE_SPARSE_TC_COPY || p->engine == SPIDER_ENGINE_SPARSE_TC_NO_CO)
    return cudaErrorNotSupported;
  if (p->ndim == 1) return p->wide() ? launch_wide1d_fused_sp_tf32(p->r, T, ctx) : cudaErrorNotSupported;
  if (p->ndim == 3) {
    if (p->engine == SPIDER_ENGINE_SPARSE_TC && p->prec != SPIDER_F16X2 && p->prec != SPIDER_BF16X3)
      return launch_fused3d_sp_tf32(p->r, T, ctx);
    return cudaErrorNotSupported;
  }
  switch (p->engine) {
    case SPIDER_ENGINE_CUDA_CORE: return launch_fused_cuda_core(p->r, T, ctx);
    case SPIDER_ENGINE_DENSE_TC: return launch_fused_dense_tf32(p->r, T, ctx);
    default: break;
  }
  switch (p->prec) {
    case SPIDER_F16X2: return launch_fused_sp_f16x2(p->r, T, ctx);
    case SPIDER_BF16X3: return launch_fused_sp_bf16x3(p->r, T, ctx);
    default: return launch_fused_sp_tf32(p->r, T, ctx);
  }
}

}  // namespace spider
