// spider_run_static: spider_run without any device allocation.
//
// spider_run allocates, on first use, the plan's device copy of its packed
// operands and a scratch grid for ping-ponging between time steps.  This entry
// point keeps both in file-scope __device__ arrays instead, so it never calls
// cudaMalloc or cudaFree.  It runs the same passes as spider_run (fused time
// steps where the plan fuses) on grids TMA can read in their own layout.  The
// arrays have fixed sizes, are shared by every call in the process, and are
// held by every GPU that loads the library until the process exits.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "launch.h"
#include "spider_internal.h"

namespace spider {
namespace {

constexpr int64_t kStaticMaxPoints = int64_t(1) << 22;  // 4,194,304 grid points (16 MiB of float32)
constexpr size_t kStaticOperandWords = 16384;           // packed A fragments (64 KiB)
constexpr size_t kStaticMetaWords = 4096;               // metadata (16 KiB)
constexpr size_t kStaticCoeffs = 512;                   // coefficient cube (r <= 3, 3-D: 343)

static __device__ __align__(256) float g_scratch[kStaticMaxPoints];
static __device__ __align__(256) uint32_t g_operands[kStaticOperandWords];
static __device__ __align__(256) uint32_t g_meta[kStaticMetaWords];
static __device__ __align__(256) float g_coeffs[kStaticCoeffs];
static __device__ __align__(256) int g_status;

// Device addresses of the arrays, looked up once per device (with that device
// current).  In host code the array names are host-side stand-ins, never
// device addresses, so only these looked-up pointers are passed to kernels.
struct StaticAddrs {
  bool ready = false;
  float* scratch = nullptr;
  uint32_t* operands = nullptr;
  uint32_t* meta = nullptr;
  float* coeffs = nullptr;
  int* status = nullptr;
};
constexpr int kMaxDevices = 64;
std::mutex g_mu;
StaticAddrs g_addrs[kMaxDevices];

spider_status setup_device(int dev, StaticAddrs* out) {
  std::lock_guard<std::mutex> lock(g_mu);
  StaticAddrs& a = g_addrs[dev];
  if (!a.ready) {
    cudaError_t e = cudaGetSymbolAddress((void**)&a.scratch, g_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&a.operands, g_operands);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&a.meta, g_meta);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&a.coeffs, g_coeffs);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&a.status, g_status);
    if (e != cudaSuccess) {
      a = StaticAddrs();
      return fail(SPIDER_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    a.ready = true;
  }
  *out = a;
  return SPIDER_OK;
}

}  // namespace
}  // namespace spider

using namespace spider;

extern "C" spider_status spider_run_static(spider_plan p, const float* grid_in, float* grid_out, int64_t steps,
                                           cudaStream_t stream) {
  set_error("");
  if (!p) return fail(SPIDER_ERR_INVALID, "plan is NULL");
  if (!grid_in || !grid_out) return fail(SPIDER_ERR_INVALID, "grid pointer is NULL");
  if (steps < 0) return fail(SPIDER_ERR_INVALID, "steps must be >= 0");
  const size_t bytes = (size_t)p->points() * sizeof(float);
  {
    const char* x = reinterpret_cast<const char*>(grid_in);
    const char* y = reinterpret_cast<const char*>(grid_out);
    if (x < y + bytes && y < x + bytes) return fail(SPIDER_ERR_INVALID, "grid_out overlaps grid_in");
  }
  if (p->points() > kStaticMaxPoints)
    return fail(SPIDER_ERR_INVALID, "spider_run_static: grid has " + std::to_string(p->points()) +
                                        " points; its static scratch holds at most " +
                                        std::to_string(kStaticMaxPoints));
  if (p->a_words.size() > kStaticOperandWords || p->meta_words.size() > kStaticMetaWords ||
      p->w.size() > kStaticCoeffs)
    return fail(SPIDER_ERR_INVALID, "spider_run_static: plan operands exceed the static operand area");

  std::lock_guard<std::mutex> lock(p->mu);
  if (steps == 0) {
    cudaError_t e = cudaMemcpyAsync(grid_out, grid_in, bytes, cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) return fail(SPIDER_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    return SPIDER_OK;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SPIDER_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(SPIDER_ERR_UNSUPPORTED, "device index out of range");
  StaticAddrs a;
  spider_status s = setup_device(dev, &a);
  if (s != SPIDER_OK) return s;

  // The shared arrays keep the previous call's contents: load this plan's
  // operands and clear the status word that must start at zero.
  if (!p->a_words.empty())
    e = cudaMemcpyAsync(a.operands, p->a_words.data(), p->a_words.size() * 4, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess && !p->meta_words.empty())
    e = cudaMemcpyAsync(a.meta, p->meta_words.data(), p->meta_words.size() * 4, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(a.coeffs, p->w.data(), p->w.size() * 4, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.status, 0, sizeof(int), stream);
  if (e != cudaSuccess) return fail(SPIDER_ERR_CUDA, std::string("operand upload: ") + cudaGetErrorString(e));

  // A stack view of the plan whose device state points at the static arrays;
  // the launch code reads only its geometry, engine, precision, fusion depth,
  // tile variant and pointers.
  spider_plan_t view;
  view.ndim = p->ndim;
  view.nx = p->nx;
  view.ny = p->ny;
  view.nz = p->nz;
  view.r = p->r;
  view.rx = p->rx;
  view.ry = p->ry;
  view.rz = p->rz;
  view.shape = p->shape;
  view.prec = p->prec;
  view.engine = p->engine;
  view.steps_per_pass = p->steps_per_pass;
  view.tile_variant = p->tile_variant;
  view.dev.device = dev;
  view.dev.a_words = a.operands;
  view.dev.meta_words = a.meta;
  view.dev.w_dense = a.coeffs;
  view.dev.status = a.status;
  view.dev.scratch = a.scratch;

  // The same passes as spider_run takes on grids TMA can read in their own
  // layout: T fused steps per pass (the plan's setting), a single-step first
  // pass when the input cannot be read through TMA, grids between passes
  // stored rounded to TF32 in the TF32 engines.  Grids whose rows TMA cannot
  // describe have no padded grids here: they run one step per pass.
  auto aligned = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  const int m = p->ndim == 1 ? 8 : 4;
  const bool tma_out = p->nx % m == 0 && aligned(grid_out);
  const bool tma_in = p->nx % m == 0 && aligned(grid_in);
  const int T = tma_out ? std::min(p->steps_per_pass, max_steps_per_pass(p)) : 1;
  const int head = (T > 1 && !tma_in) ? 1 : 0;
  const int64_t body = steps - head;
  const int64_t full = body / T;
  const int rem = (int)(body % T);
  const int64_t npasses = head + full + (rem ? 1 : 0);
  const bool tf32 = tma_out && (p->engine == SPIDER_ENGINE_DENSE_TC || p->engine == SPIDER_ENGINE_SPARSE_TC_COPY ||
                                p->engine == SPIDER_ENGINE_SPARSE_TC_NO_CO ||
                                (p->engine == SPIDER_ENGINE_SPARSE_TC && p->prec != SPIDER_F16X2 &&
                                 p->prec != SPIDER_BF16X3));
  LaunchCtx ctx;
  ctx.plan = &view;
  ctx.stream = stream;
  ctx.sms = device_sm_count();
  float* bufs[2] = {grid_out, a.scratch};
  const int first = (npasses % 2 == 1) ? 0 : 1;  // the last pass lands in grid_out
  for (int64_t k = 0; k < npasses; ++k) {
    const bool last = k + 1 == npasses;
    const int n = k < head ? 1 : (k - head < full ? T : rem);
    ctx.dst = bufs[(first + k) % 2];
    ctx.src = (k == 0) ? grid_in : bufs[(first + k - 1) % 2];
    ctx.in_tf32 = tf32 && k > 0;
    ctx.out_tf32 = tf32 && !last;
    e = launch_pass(ctx, n);
    if (e == cudaErrorNotSupported) return fail(SPIDER_ERR_UNSUPPORTED, "no kernel for this stencil/engine");
    if (e != cudaSuccess) return fail(SPIDER_ERR_CUDA, std::string("stencil pass launch: ") + cudaGetErrorString(e));
  }
  return SPIDER_OK;
}
