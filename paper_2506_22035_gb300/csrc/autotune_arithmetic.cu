// Picks the arithmetic (precision split and engine) of a stencil for an error
// target by timing the candidates on the caller's grids: the split-depth part
// of the autotuner.  The paper states no precision; the candidates and their
// error bounds are the library's (error_model in api.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "launch.h"
#include "spider_internal.h"

namespace spider {
namespace {

// Largest |a[i]| as FP32 bits (NaN bits order above every finite value).
__global__ void max_abs_bits_kernel(const float* __restrict__ a, int64_t n, unsigned int* out) {
  unsigned int m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(a[i]) & 0x7FFFFFFFu);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

struct Candidate {
  spider_precision prec;
  spider_engine engine;
};

}  // namespace
}  // namespace spider

using namespace spider;

extern "C" spider_status spider_plan_autotune_arithmetic(spider_plan p, const float* grid_in, float* grid_out,
                                                        int64_t steps, double err_target, cudaStream_t stream,
                                                        spider_precision* prec, spider_engine* engine,
                                                        double* gstencil_s) {
  set_error("");
  if (!p || !grid_in || !grid_out) return fail(SPIDER_ERR_INVALID, "plan or grid is NULL");
  if (steps < 1) return fail(SPIDER_ERR_INVALID, "steps must be >= 1");
  if (!(err_target > 0.0) || !std::isfinite(err_target)) return fail(SPIDER_ERR_INVALID, "bad error target");
  const int64_t n = p->points();

  // the FP16 split holds grid values below 16384 in magnitude
  unsigned int* d_bits = nullptr;
  unsigned int bits = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&d_bits), sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bits, 0, sizeof(unsigned int), stream);
  if (e == cudaSuccess) {
    const int blocks = 2 * device_sm_count();
    max_abs_bits_kernel<<<blocks, 256, 0, stream>>>(grid_in, n, d_bits);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, d_bits, sizeof(bits), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (d_bits) cudaFree(d_bits);
  if (e != cudaSuccess) return fail(SPIDER_ERR_CUDA, std::string("largest |value|: ") + cudaGetErrorString(e));
  float amax;
  std::memcpy(&amax, &bits, sizeof(amax));

  const Candidate cands[] = {{SPIDER_TF32, SPIDER_ENGINE_SPARSE_TC},
                             {SPIDER_F16X2, SPIDER_ENGINE_SPARSE_TC},
                             {SPIDER_BF16X3, SPIDER_ENGINE_SPARSE_TC},
                             {SPIDER_TF32, SPIDER_ENGINE_CUDA_CORE}};
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e != cudaSuccess) {
    if (t0) cudaEventDestroy(t0);
    return fail(SPIDER_ERR_CUDA, "events");
  }
  double best_rate = -1.0;
  Candidate best = cands[0];
  spider_status err = SPIDER_OK;
  for (const Candidate& c : cands) {
    if (c.prec == SPIDER_F16X2 && !(amax < 16384.f)) continue;
    const ErrorModel m = error_model(p, c.prec, c.engine);
    if (!m.built || (double)steps * (m.wsum + m.drift) + m.floor > err_target) continue;
    spider_plan q = nullptr;
    err = spider_plan_create(p->ndim, p->extents, p->shape, p->r, p->w.data(), c.prec, &q);
    if (err == SPIDER_OK && c.engine != SPIDER_ENGINE_SPARSE_TC) err = spider_plan_set_engine(q, c.engine);
    if (err == SPIDER_OK) err = spider_plan_autotune(q, grid_in, grid_out, steps, stream, nullptr, nullptr);
    float best_ms = 0.f;
    for (int rep = 0; rep < 2 && err == SPIDER_OK; ++rep) {
      cudaEventRecord(t0, stream);
      err = spider_run(q, grid_in, grid_out, steps, stream);
      cudaEventRecord(t1, stream);
      if (err == SPIDER_OK) err = spider_plan_sync(q, stream);
      float ms = 0.f;
      if (err == SPIDER_OK && cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess)
        best_ms = rep == 0 ? ms : std::min(best_ms, ms);
    }
    if (q) spider_plan_destroy(q);
    if (err != SPIDER_OK) break;
    const double rate = (double)n * (double)steps / ((double)best_ms * 1e-3) / 1e9;
    if (rate > best_rate) {
      best_rate = rate;
      best = c;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (err != SPIDER_OK) return err;
  if (best_rate < 0) return fail(SPIDER_ERR_UNSUPPORTED, "no arithmetic's error bound meets the target");
  if (prec) *prec = best.prec;
  if (engine) *engine = best.engine;
  if (gstencil_s) *gstencil_s = best_rate;
  return SPIDER_OK;
}
