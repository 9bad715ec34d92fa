// spider_batch and the serving entry points.
#include "spider_internal.h"

namespace spider {

}
using namespace spider;

extern "C" {

spider_status spider_batch(int n, const spider_plan* plans, const float* const* ins, float* const* outs,
                           const int64_t* steps, cudaStream_t stream) {
  set_error("");
  if (n < 0 || n > 4096) return fail(SPIDER_ERR_INVALID, "n must be in [0, 4096]");
  if (n > 0 && (!plans || !ins || !outs || !steps)) return fail(SPIDER_ERR_INVALID, "NULL array");
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !ins[i] || !outs[i] || steps[i] < 0) return fail(SPIDER_ERR_INVALID, "bad job");
  }
  for (int i = 0; i < n; ++i) {
    std::lock_guard<std::mutex> lock(plans[i]->mu);
    spider_status s = run_device(plans[i], ins[i], outs[i], steps[i], stream);
    if (s != SPIDER_OK) return s;
  }
  return SPIDER_OK;
}

spider_status spider_server_create(size_t, spider_server* out) {
  if (out) *out = nullptr;
  return fail(SPIDER_ERR_UNSUPPORTED, "serving is not built yet");
}
spider_status spider_submit(spider_server, spider_plan, const float*, int64_t, double, uint64_t*) {
  return fail(SPIDER_ERR_UNSUPPORTED, "serving is not built yet");
}
spider_status spider_poll(spider_server, uint64_t, float*, int*, double*) {
  return fail(SPIDER_ERR_UNSUPPORTED, "serving is not built yet");
}
void spider_server_destroy(spider_server) {}

}  // extern "C"
