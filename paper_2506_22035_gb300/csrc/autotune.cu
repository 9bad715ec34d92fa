// Autotuner: picks time steps per pass and the fused tile variant by timing
// them on the caller's grids; results are cached per kind of stencil and
// grid-size bucket.
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "spider_internal.h"

namespace spider {
namespace {

using Key = std::tuple<int, int, int, int, int, int>;  // ndim, r, shape, prec, engine, log2(points) bucket
std::mutex g_cache_mu;
std::map<Key, std::pair<int, int>> g_cache;

Key key_of(const spider_plan_t* p) {
  const int bucket = (int)std::floor(std::log2((double)std::max<int64_t>(p->points(), 1)));
  return Key(p->ndim, p->r, (int)p->shape, (int)p->prec, (int)p->engine, bucket);
}

}  // namespace

bool autotune_lookup(const spider_plan_t* p, int* steps_per_pass, int* variant) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  auto it = g_cache.find(key_of(p));
  if (it == g_cache.end()) return false;
  *steps_per_pass = it->second.first;
  *variant = it->second.second;
  return true;
}

}  // namespace spider

using namespace spider;

extern "C" spider_status spider_plan_set_tile_variant(spider_plan p, int variant) {
  if (!p) return fail(SPIDER_ERR_INVALID, "plan is NULL");
  if (variant < 0 || variant > 5) return fail(SPIDER_ERR_INVALID, "tile variant must be 0..5");
  std::lock_guard<std::mutex> lock(p->mu);
  p->tile_variant = variant;
  return SPIDER_OK;
}

extern "C" spider_status spider_plan_autotune(spider_plan p, const float* grid_in, float* grid_out, int64_t steps,
                                              cudaStream_t stream, int* steps_per_pass, int* variant) {
  set_error("");
  if (!p) return fail(SPIDER_ERR_INVALID, "plan is NULL");
  if (!grid_in || !grid_out || steps < 1) return fail(SPIDER_ERR_INVALID, "bad grids or steps");
  const Key key = key_of(p);
  bool cached = false;
  std::pair<int, int> hit;
  {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) { cached = true; hit = it->second; }
  }
  if (cached) {
    std::lock_guard<std::mutex> plock(p->mu);
    p->steps_per_pass = hit.first;
    p->tile_variant = hit.second;
    if (steps_per_pass) *steps_per_pass = hit.first;
    if (variant) *variant = hit.second;
    return SPIDER_OK;
  }
  std::lock_guard<std::mutex> plock(p->mu);
  const int old_T = p->steps_per_pass, old_v = p->tile_variant;
  const int maxT = max_steps_per_pass(p);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(SPIDER_ERR_CUDA, "cudaEventCreate");
  float best_ms = 1e30f;
  int best_T = 1, best_v = 0;
  spider_status st = SPIDER_OK;
  // variant 4 (small 2-D tiles) only where the grid cannot fill the GPU
  // with the 64-row tiles; more than 4 steps per pass (deep radius-1 tiles)
  // only there too, and for at most the run's step count, with the small
  // tile for the remainder pass
  const bool small2d = p->ndim == 2 && p->points() <= (int64_t(1) << 22);
  for (int T = 1; T <= maxT && st == SPIDER_OK; ++T) {
    if (T > 4 && (!small2d || T > steps)) break;
    const int v0 = T > 4 ? 4 : 0;
    // variant 5 (16-byte final-level stores) measured slower than 2 and is
    // not a candidate
    const int nv = T == 1 ? 1 : small2d ? 5 : 4;
    for (int v = v0; v < nv && st == SPIDER_OK; ++v) {
      p->steps_per_pass = T;
      p->tile_variant = v;
      st = run_device(p, grid_in, grid_out, steps, stream);  // warm-up
      if (st != SPIDER_OK) break;
      cudaEventRecord(e0, stream);
      for (int k = 0; k < 2 && st == SPIDER_OK; ++k) st = run_device(p, grid_in, grid_out, steps, stream);
      cudaEventRecord(e1, stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { st = fail(SPIDER_ERR_CUDA, "autotune timing"); break; }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) { best_ms = ms; best_T = T; best_v = v; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SPIDER_OK) {
    p->steps_per_pass = old_T;
    p->tile_variant = old_v;
    return st;
  }
  p->steps_per_pass = best_T;
  p->tile_variant = best_v;
  {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    g_cache[key] = {best_T, best_v};
  }
  if (steps_per_pass) *steps_per_pass = best_T;
  if (variant) *variant = best_v;
  return SPIDER_OK;
}
