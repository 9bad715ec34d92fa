// The C ABI (include/spider.h): plan lifecycle, spider_run, spider_run_host.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>

#include "launch.h"
#include <algorithm>

#include "spider_internal.h"

namespace spider {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

spider_status fail(spider_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

static spider_status cuda_fail(cudaError_t e, const char* what) {
  return fail(SPIDER_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SPIDER_CUDA(call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
  } while (0)

static void drop_graphs(spider_plan_t* p) {
  for (auto& g : p->dev.graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  p->dev.graphs.clear();
}

// Device memory of a plan: cudaMalloc / cudaFree, or stream-ordered from the
// plan's pool (see DeviceState::pool).
static cudaError_t dev_alloc(spider_plan_t* p, void** ptr, size_t bytes) {
  if (p->dev.pool) return cudaMallocFromPoolAsync(ptr, bytes, p->dev.pool, p->dev.pool_stream);
  return cudaMalloc(ptr, bytes);
}
static void dev_free(spider_plan_t* p, void* ptr) {
  if (!ptr) return;
  if (p->dev.pool) cudaFreeAsync(ptr, p->dev.pool_stream);
  else cudaFree(ptr);
}
// Host -> device copy of plan data (pageable host memory: the call returns
// once the data is staged, so the host vectors may change afterwards).
static cudaError_t dev_upload(spider_plan_t* p, void* dst, const void* src, size_t bytes) {
  if (p->dev.pool) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, p->dev.pool_stream);
  return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
}

static void free_device(spider_plan_t* p) {
  DeviceState& d = p->dev;
  if (d.device >= 0) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != d.device) cudaSetDevice(d.device);
    // cudaFree waits for the device, so no replay of a cached graph is still
    // running when the graphs are destroyed (a pooled plan has no graphs:
    // its frees are ordered after its work on its stream)
    dev_free(p, d.a_words);
    dev_free(p, d.meta_words);
    dev_free(p, d.w_dense);
    dev_free(p, d.scratch);
    dev_free(p, d.pad);
    dev_free(p, d.host_stage_in);
    dev_free(p, d.host_stage_out);
    for (auto& h : d.host_slots) {
      dev_free(p, h.in);
      dev_free(p, h.out);
      if (h.copied_in) cudaEventDestroy(h.copied_in);
      if (h.stepped) cudaEventDestroy(h.stepped);
      if (h.copied_out) cudaEventDestroy(h.copied_out);
    }
    if (d.h2d_stream) cudaStreamDestroy(d.h2d_stream);
    if (d.d2h_stream) cudaStreamDestroy(d.d2h_stream);
    dev_free(p, d.status);
    drop_graphs(p);
    if (d.capture_stream) cudaStreamDestroy(d.capture_stream);
    if (cur >= 0 && cur != d.device) cudaSetDevice(cur);
  }
  const cudaMemPool_t pool = d.pool;
  const cudaStream_t pool_stream = d.pool_stream;
  d = DeviceState();
  d.pool = pool;
  d.pool_stream = pool_stream;
}

// Uploads the packed operands on first use (or after an engine change).
static spider_status ensure_device(spider_plan_t* p) {
  int dev = 0;
  SPIDER_CUDA(cudaGetDevice(&dev));
  DeviceState& d = p->dev;
  if (d.device >= 0 && d.device != dev)
    return fail(SPIDER_ERR_INVALID, "plan was first used on another device");
  if (d.device < 0) d.device = dev;
  if (!d.status) {
    SPIDER_CUDA(dev_alloc(p, (void**)&d.status, sizeof(int)));
    if (d.pool) SPIDER_CUDA(cudaMemsetAsync(d.status, 0, sizeof(int), d.pool_stream));
    else SPIDER_CUDA(cudaMemset(d.status, 0, sizeof(int)));
  }
  if (!d.a_words && !p->a_words.empty()) {
    SPIDER_CUDA(dev_alloc(p, (void**)&d.a_words, p->a_words.size() * 4));
    SPIDER_CUDA(dev_upload(p, d.a_words, p->a_words.data(), p->a_words.size() * 4));
  }
  if (!d.meta_words && !p->meta_words.empty()) {
    SPIDER_CUDA(dev_alloc(p, (void**)&d.meta_words, p->meta_words.size() * 4));
    SPIDER_CUDA(dev_upload(p, d.meta_words, p->meta_words.data(), p->meta_words.size() * 4));
  }
  if (!d.w_dense) {
    SPIDER_CUDA(dev_alloc(p, (void**)&d.w_dense, p->w.size() * 4));
    SPIDER_CUDA(dev_upload(p, d.w_dense, p->w.data(), p->w.size() * 4));
  }
  return SPIDER_OK;
}

static spider_status ensure_scratch(spider_plan_t* p) {
  const size_t bytes = (size_t)p->points() * sizeof(float);
  if (p->dev.scratch && p->dev.scratch_bytes >= bytes) return SPIDER_OK;
  dev_free(p, p->dev.scratch);
  p->dev.scratch = nullptr;
  cudaError_t e = dev_alloc(p, (void**)&p->dev.scratch, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p->dev.scratch = nullptr;
    return fail(SPIDER_ERR_OOM, std::string("scratch grid: ") + cudaGetErrorString(e));
  }
  p->dev.scratch_bytes = bytes;
  return SPIDER_OK;
}

spider_status ensure_plan_pad(spider_plan_t* p, size_t bytes) {
  if (p->dev.pad && p->dev.pad_bytes >= bytes) return SPIDER_OK;
  dev_free(p, p->dev.pad);  // cudaFree waits for the device: no earlier run still uses it
  if (p->dev.pad) drop_graphs(p);  // cached run graphs hold the old address
  p->dev.pad = nullptr;
  p->dev.pad_bytes = 0;
  cudaError_t e = dev_alloc(p, (void**)&p->dev.pad, bytes);
  // zero once: the kernels never store beyond nx, so the 1-D grids' tails
  // stay zero and read as the halo
  if (p->dev.pool) {
    // ordered before the plan's kernels on its own stream
    if (e == cudaSuccess) e = cudaMemsetAsync(p->dev.pad, 0, bytes, p->dev.pool_stream);
  } else {
    if (e == cudaSuccess) e = cudaMemset(p->dev.pad, 0, bytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();  // before any stream of the caller writes it
  }
  if (e != cudaSuccess) {
    dev_free(p, p->dev.pad);
    p->dev.pad = nullptr;
    cudaGetLastError();
    return fail(SPIDER_ERR_OOM, std::string("padded grids: ") + cudaGetErrorString(e));
  }
  p->dev.pad_bytes = bytes;
  return SPIDER_OK;
}

spider_status ensure_plan_device(spider_plan_t* p, bool scratch) {
  spider_status s = ensure_device(p);
  if (s != SPIDER_OK || !scratch) return s;
  return ensure_scratch(p);
}

static bool overlaps(const void* a, const void* b, size_t bytes) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + bytes && y < x + bytes;
}

// Enqueues `steps` steps from `in` to `out` (device pointers) on `stream`.
int max_steps_per_pass(const spider_plan_t* p) {
  if (p->engine == SPIDER_ENGINE_SPARSE_TC_COPY || p->engine == SPIDER_ENGINE_SPARSE_TC_NO_CO) return 1;
  if (p->wide()) return p->ndim == 1 ? 4 : 1;
  const bool sparse_tf32 = p->engine == SPIDER_ENGINE_SPARSE_TC && p->prec != SPIDER_F16X2 && p->prec != SPIDER_BF16X3;
  if (p->ndim == 2) return sparse_tf32 ? max_deep_steps(p->r) : 4;  // deep tiles beyond 4
  if (p->ndim == 3 && p->r == 1 && sparse_tf32) return 4;
  return 1;
}

// A priori error model of an arithmetic (spider_plan_error_bound).  The
// relative L2 error of n steps against exact arithmetic is bounded by
// n * (wsum + drift) + floor:
//  * wsum: the plan's weight-sum error in that arithmetic, |sum of the
//    weights the products use - sum of the FP32 weights| / sum |w|; it
//    scales the constant mode every step, so on fields of one sign the
//    error grows by about that much per step;
//  * drift: the rest of the per-step bias, measured on fields of one sign.
//    TF32: rounding the grid to 11 bits every step is biased where the field
//    is smooth (neighbouring values within one TF32 unit round the same way),
//    up to 5e-5 per step measured.  FP16 hi/lo: the tensor core aligns each
//    MMA's 22-bit products to the largest and drops their lowest bits, about
//    4e-8 per step.  BF16 hi/mid/lo: 16-bit products lose no bits, 6e-9.
//    FP32 on CUDA cores: round-to-nearest FMAs with exact weights, none.
//  * floor: the error that does not grow with the step count.
// The constants are twice the largest values measured on GB300 over radius
// 1..3 star and box stencils, 2-D and 3-D, 10..500 steps, fields uniform on
// [0, 1) and [-1, 1).
ErrorModel error_model(const spider_plan_t* p, spider_precision prec, spider_engine engine) {
  ErrorModel m;
  const bool wide = p->r > kMaxR || (p->ndim == 1 && engine == SPIDER_ENGINE_SPARSE_TC && prec == SPIDER_TF32);
  if (engine == SPIDER_ENGINE_CUDA_CORE) {
    m.built = p->r <= kMaxR;
    m.wsum = 0;  // FP32 weights, exact
    m.drift = 1e-10;
    m.floor = 3e-7;
    return m;
  }
  if (engine == SPIDER_ENGINE_DENSE_TC || engine == SPIDER_ENGINE_SPARSE_TC_COPY ||
      engine == SPIDER_ENGINE_SPARSE_TC_NO_CO) {
    m.built = p->r <= kMaxR && prec == SPIDER_TF32 && (engine == SPIDER_ENGINE_DENSE_TC || p->ndim == 2);
    m.wsum = p->wsum_rel[0];
    m.drift = 1e-4;
    m.floor = 7e-4;
    return m;
  }
  switch (prec) {
    case SPIDER_F16X2:
      m.built = p->r <= kMaxR && !wide;
      m.wsum = p->wsum_rel[1];
      m.drift = 8e-8;
      m.floor = 1e-6;
      break;
    case SPIDER_BF16X3:
      m.built = p->r <= kMaxR && !wide;
      m.wsum = p->wsum_rel[2];
      m.drift = 1.5e-8;
      m.floor = 3e-7;
      break;
    default:
      m.built = true;
      m.wsum = p->wsum_rel[0];
      m.drift = 1e-4;
      m.floor = 7e-4;
      break;
  }
  return m;
}

// A run steps through the plan's padded grids when `out` is not a grid TMA
// can read in its packed layout: 2-D and 3-D rows of a multiple of 4
// floats, 1-D arrays (read as rows of 8 floats) of a multiple of 8, and a
// 16-byte aligned base.
static int tma_multiple(const spider_plan_t* p) { return p->ndim == 1 ? 8 : 4; }
static bool run_is_padded(const spider_plan_t* p, const float* out, int64_t steps) {
  return steps > 1 && !(p->nx % tma_multiple(p) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0);
}
// Row pitch (1-D: length) of the padded grids.
static int64_t padded_pitch(const spider_plan_t* p) {
  const int m = tma_multiple(p);
  return (p->nx + m - 1) / m * m;
}

// Every buffer a run of `steps` steps into `out` needs (operands, scratch
// grid, padded grids), allocated before its launches are issued or captured.
static spider_status ensure_run_buffers(spider_plan_t* p, const float* out, int64_t steps) {
  spider_status s = ensure_device(p);
  if (s == SPIDER_OK && steps > 1) s = ensure_scratch(p);
  if (s == SPIDER_OK && run_is_padded(p, out, steps))
    s = ensure_plan_pad(p, 2 * (size_t)padded_pitch(p) * (size_t)p->ny * (size_t)p->nz * sizeof(float));
  return s;
}

spider_status run_device(spider_plan_t* p, const float* in, float* out, int64_t steps, cudaStream_t stream) {
  const size_t bytes = (size_t)p->points() * sizeof(float);
  if (steps == 0) {
    SPIDER_CUDA(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, stream));
    return SPIDER_OK;
  }
  spider_status s = ensure_run_buffers(p, out, steps);
  if (s != SPIDER_OK) return s;
  LaunchCtx ctx;
  ctx.plan = p;
  ctx.stream = stream;
  ctx.sms = device_sm_count();
  auto aligned = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  // TMA reads a grid whose rows are a multiple of 16 bytes (1-D: whose
  // length is a multiple of 8 floats) from a 16-byte aligned base.  When out
  // is not such a grid, the passes between
  // the first and the last run in the plan's two padded grids (rows rounded
  // up to 4 floats), so that every pass after the first reads through TMA
  // and may fuse time steps; the first pass reads `in` as it is and the last
  // writes `out` in the caller's packed layout.
  const bool padded = run_is_padded(p, out, steps);
  const bool in_tma = p->nx % tma_multiple(p) == 0 && aligned(in);
  // Passes of T fused time steps, then one pass with the remainder; a first
  // pass that cannot read `in` through TMA takes one step on its own.
  const int T = std::min(p->steps_per_pass, max_steps_per_pass(p));
  const int head = (T > 1 && !in_tma) ? 1 : 0;  // a single-step first pass
  const int64_t body = steps - head;
  const int64_t full = body / T;
  const int rem = (int)(body % T);
  const int64_t npasses = head + full + (rem ? 1 : 0);
  auto pass_steps = [&](int64_t k) { return k < head ? 1 : (k - head < full ? T : rem); };
  // TF32 engines: every grid between two passes is stored rounded to TF32 as
  // the next pass would round it, and that pass skips the rounding; the
  // caller's input is rounded on load and the final grid is stored unrounded.
  const bool tf32 = p->engine == SPIDER_ENGINE_DENSE_TC || p->engine == SPIDER_ENGINE_SPARSE_TC_COPY ||
                    p->engine == SPIDER_ENGINE_SPARSE_TC_NO_CO ||
                    (p->engine == SPIDER_ENGINE_SPARSE_TC && p->prec != SPIDER_F16X2 && p->prec != SPIDER_BF16X3);
  float* bufs[2] = {out, p->dev.scratch};
  int first = (npasses % 2 == 1) ? 0 : 1;  // packed: the last pass lands in out
  int64_t pitch = p->nx;
  if (padded) {
    pitch = padded_pitch(p);
    const size_t grid_bytes = (size_t)pitch * (size_t)p->ny * (size_t)p->nz * sizeof(float);
    bufs[0] = p->dev.pad;
    bufs[1] = p->dev.pad + grid_bytes / sizeof(float);
    first = 0;
  }
  for (int64_t k = 0; k < npasses; ++k) {
    const bool last = k + 1 == npasses;
    ctx.dst = (padded && last) ? out : bufs[(first + k) % 2];
    ctx.src = (k == 0) ? in : bufs[(first + k - 1) % 2];
    ctx.dst_pitch = (padded && !last) ? pitch : 0;
    ctx.src_pitch = (padded && k > 0) ? pitch : 0;
    ctx.in_tf32 = tf32 && k > 0;
    ctx.out_tf32 = tf32 && !last;
    cudaError_t e = launch_pass(ctx, pass_steps(k));
    if (e == cudaErrorNotSupported) return fail(SPIDER_ERR_UNSUPPORTED, "no kernel for this stencil/engine");
    if (e != cudaSuccess) return cuda_fail(e, "stencil pass launch");
  }
  return SPIDER_OK;
}

// Repeated runs replay a CUDA graph.  A time-stepping loop calls spider_run
// with the same grids and step count again and again; for small grids the
// host cost of its launches (tensor-map encoding, one launch per pass) is
// larger than the kernels.  The first call with a given (grids, steps,
// configuration) runs directly and is remembered; the second captures the
// same launches on a private stream (thread-local capture mode, after every
// allocation the run needs) and instantiates them; later calls launch that
// graph on the caller's stream.  Graphs hold the grids' addresses, which is
// all a run depends on besides the plan's own buffers, and are dropped when
// the plan's device state is.
constexpr size_t kMaxRunGraphs = 8;

spider_status run_cached(spider_plan_t* p, const float* in, float* out, int64_t steps, cudaStream_t stream) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (steps < 1 || cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return run_device(p, in, out, steps, stream);  // the caller is capturing: plain launches
  }
  DeviceState& d = p->dev;
  RunGraph* hit = nullptr;
  for (auto& g : d.graphs)
    if (g.in == in && g.out == out && g.steps == steps && g.steps_per_pass == p->steps_per_pass &&
        g.tile_variant == p->tile_variant && g.engine == (int)p->engine)
      hit = &g;
  if (hit && hit->exec) {
    hit->last_use = ++d.graph_clock;
    SPIDER_CUDA(cudaGraphLaunch(hit->exec, stream));
    return SPIDER_OK;
  }
  if (!hit) {
    if (d.graphs.size() >= kMaxRunGraphs) {
      auto lru = d.graphs.begin();
      for (auto it = d.graphs.begin(); it != d.graphs.end(); ++it)
        if (it->last_use < lru->last_use) lru = it;
      if (lru->exec) cudaGraphExecDestroy(lru->exec);
      d.graphs.erase(lru);
    }
    RunGraph g;
    g.in = in;
    g.out = out;
    g.steps = steps;
    g.steps_per_pass = p->steps_per_pass;
    g.tile_variant = p->tile_variant;
    g.engine = (int)p->engine;
    g.last_use = ++d.graph_clock;
    d.graphs.push_back(g);
    return run_device(p, in, out, steps, stream);  // first sight: run directly
  }
  // second sight: capture
  hit->last_use = ++d.graph_clock;
  spider_status s = ensure_run_buffers(p, out, steps);
  if (s != SPIDER_OK) return s;
  if (!d.capture_stream) SPIDER_CUDA(cudaStreamCreateWithFlags(&d.capture_stream, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ok = cudaStreamBeginCapture(d.capture_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    const spider_status rs = run_device(p, in, out, steps, d.capture_stream);
    ok = cudaStreamEndCapture(d.capture_stream, &graph) == cudaSuccess && rs == SPIDER_OK && graph;
  }
  ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    // capture is an optimisation only: run the launches directly
    cudaGetLastError();
    set_error("");
    return run_device(p, in, out, steps, stream);
  }
  hit->exec = exec;
  SPIDER_CUDA(cudaGraphLaunch(exec, stream));
  return SPIDER_OK;
}

}  // namespace spider

using namespace spider;

extern "C" {

const char* spider_last_error(void) { return spider::g_last_error.c_str(); }

spider_status spider_plan_create(int ndim, const int64_t* extents, spider_shape shape, int radius,
                                 const float* coeffs, spider_precision prec, spider_plan* out) {
  set_error("");
  if (!out) return fail(SPIDER_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (ndim < 1 || ndim > 3) return fail(SPIDER_ERR_INVALID, "ndim must be 1, 2 or 3");
  if (!extents || !coeffs) return fail(SPIDER_ERR_INVALID, "extents/coeffs is NULL");
  if (radius < 1) return fail(SPIDER_ERR_INVALID, "radius must be >= 1");
  if (radius > kMaxRWide) return fail(SPIDER_ERR_UNSUPPORTED, "radius > 7 is not built");
  if (radius > kMaxR && (ndim > 2 || (prec != SPIDER_TF32 && prec != SPIDER_AUTO)))
    return fail(SPIDER_ERR_UNSUPPORTED, "radius 4..7 is built for 1-D and 2-D stencils in TF32");
  if (shape != SPIDER_STAR && shape != SPIDER_BOX) return fail(SPIDER_ERR_INVALID, "bad shape");
  if (prec < SPIDER_TF32 || prec > SPIDER_AUTO) return fail(SPIDER_ERR_INVALID, "bad precision");
  long double total = 1;
  for (int i = 0; i < ndim; ++i) {
    if (extents[i] < 1) return fail(SPIDER_ERR_INVALID, "extents must be >= 1");
    total *= (long double)extents[i];
  }
  if (total >= (long double)(1LL << 40)) return fail(SPIDER_ERR_INVALID, "grid too large");
  const int side = 2 * radius + 1;
  size_t ncoef = 1;
  for (int i = 0; i < ndim; ++i) ncoef *= side;
  for (size_t i = 0; i < ncoef; ++i) {
    if (!std::isfinite(coeffs[i])) return fail(SPIDER_ERR_INVALID, "non-finite coefficient");
    if (shape == SPIDER_STAR && coeffs[i] != 0.0f) {
      // on-axis iff at most one offset differs from the centre
      size_t rem = i;
      int off_axis = 0;
      for (int d = 0; d < ndim; ++d) {
        if ((int)(rem % side) != radius) ++off_axis;
        rem /= side;
      }
      if (off_axis > 1) return fail(SPIDER_ERR_INVALID, "star stencil with a non-zero off-axis coefficient");
    }
  }
  spider_plan_t* p = new (std::nothrow) spider_plan_t();
  if (!p) return fail(SPIDER_ERR_OOM, "host allocation");
  p->ndim = ndim;
  for (int i = 0; i < ndim; ++i) p->extents[i] = extents[i];
  p->nx = extents[ndim - 1];
  p->ny = ndim >= 2 ? extents[ndim - 2] : 1;
  p->nz = ndim >= 3 ? extents[0] : 1;
  p->shape = shape;
  p->r = radius;
  p->rx = radius;
  p->ry = ndim >= 2 ? radius : 0;
  p->rz = ndim >= 3 ? radius : 0;
  p->prec = prec == SPIDER_AUTO ? SPIDER_TF32 : prec;
  p->w.assign(coeffs, coeffs + ncoef);
  spider_status s = build_operands(p);
  if (s != SPIDER_OK) {
    delete p;
    return s;
  }
  *out = p;
  return SPIDER_OK;
}

spider_status spider_plan_set_engine(spider_plan p, spider_engine engine) {
  if (!p) return fail(SPIDER_ERR_INVALID, "plan is NULL");
  if (engine < SPIDER_ENGINE_SPARSE_TC || engine > SPIDER_ENGINE_SPARSE_TC_NO_CO)
    return fail(SPIDER_ERR_INVALID, "bad engine");
  const bool tf32_only = engine == SPIDER_ENGINE_DENSE_TC || engine == SPIDER_ENGINE_SPARSE_TC_COPY ||
                         engine == SPIDER_ENGINE_SPARSE_TC_NO_CO;
  if (tf32_only && p->prec != SPIDER_TF32)
    return fail(SPIDER_ERR_UNSUPPORTED, "the dense, explicit-copy and no-CO comparators run TF32 only");
  if ((engine == SPIDER_ENGINE_SPARSE_TC_COPY || engine == SPIDER_ENGINE_SPARSE_TC_NO_CO) && p->ndim != 2)
    return fail(SPIDER_ERR_UNSUPPORTED, "the explicit-copy and no-CO comparators are built for 2-D grids");
  if (engine != SPIDER_ENGINE_SPARSE_TC && p->r > kMaxR)
    return fail(SPIDER_ERR_UNSUPPORTED, "radius 4..7 is built for the sparse tensor-core engine only");
  std::lock_guard<std::mutex> lock(p->mu);
  if (p->engine == engine) return SPIDER_OK;
  p->engine = engine;
  spider_status s = build_operands(p);
  if (s != SPIDER_OK) return s;
  // drop device copies of the old operands (uploaded again lazily) and the
  // run graphs that read them
  if (p->dev.device >= 0) {
    cudaFree(p->dev.a_words);  // waits for the device: no graph replay is running
    cudaFree(p->dev.meta_words);
    p->dev.a_words = nullptr;
    p->dev.meta_words = nullptr;
    drop_graphs(p);
  }
  return SPIDER_OK;
}

spider_status spider_plan_set_steps_per_pass(spider_plan p, int steps_per_pass) {
  if (!p) return fail(SPIDER_ERR_INVALID, "plan is NULL");
  if (steps_per_pass < 1) return fail(SPIDER_ERR_INVALID, "steps_per_pass must be >= 1");
  if (steps_per_pass > max_steps_per_pass(p))
    return fail(SPIDER_ERR_UNSUPPORTED,
                "temporal fusion is built for 2-D stencils (2..4 steps per pass; 2..10 for radius 1 in sparse TF32) "
                "and for 3-D radius-1 and 1-D sparse TF32 plans (2..4)");
  p->steps_per_pass = steps_per_pass;
  return SPIDER_OK;
}

spider_status spider_plan_operands(spider_plan p, uint32_t* operand_words, size_t operand_capacity,
                                   size_t* n_operand_words, uint32_t* meta_words, size_t meta_capacity,
                                   size_t* n_meta_words) {
  if (!p) return fail(SPIDER_ERR_INVALID, "plan is NULL");
  if (n_operand_words) *n_operand_words = p->a_words.size();
  if (n_meta_words) *n_meta_words = p->meta_words.size();
  if (operand_words) {
    if (operand_capacity < p->a_words.size()) return fail(SPIDER_ERR_INVALID, "operand buffer too small");
    std::memcpy(operand_words, p->a_words.data(), p->a_words.size() * 4);
  }
  if (meta_words) {
    if (meta_capacity < p->meta_words.size()) return fail(SPIDER_ERR_INVALID, "metadata buffer too small");
    std::memcpy(meta_words, p->meta_words.data(), p->meta_words.size() * 4);
  }
  return SPIDER_OK;
}

spider_status spider_run(spider_plan p, const float* grid_in, float* grid_out, int64_t steps, cudaStream_t stream) {
  set_error("");
  if (!p) return fail(SPIDER_ERR_INVALID, "plan is NULL");
  if (!grid_in || !grid_out) return fail(SPIDER_ERR_INVALID, "grid pointer is NULL");
  if (steps < 0) return fail(SPIDER_ERR_INVALID, "steps must be >= 0");
  if (overlaps(grid_in, grid_out, (size_t)p->points() * sizeof(float)))
    return fail(SPIDER_ERR_INVALID, "grid_out overlaps grid_in");
  std::lock_guard<std::mutex> lock(p->mu);
  return run_cached(p, grid_in, grid_out, steps, stream);
}

spider_status spider_run_host(spider_plan p, const float* host_in, float* host_out, int64_t steps,
                              cudaStream_t stream) {
  set_error("");
  if (!p) return fail(SPIDER_ERR_INVALID, "plan is NULL");
  if (!host_in || !host_out) return fail(SPIDER_ERR_INVALID, "host pointer is NULL");
  if (steps < 0) return fail(SPIDER_ERR_INVALID, "steps must be >= 0");
  std::lock_guard<std::mutex> lock(p->mu);
  spider_status s = ensure_device(p);
  if (s != SPIDER_OK) return s;
  const size_t bytes = (size_t)p->points() * sizeof(float);
  if (!p->dev.host_stage_in) {
    cudaError_t e = cudaMalloc(&p->dev.host_stage_in, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->dev.host_stage_out, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(SPIDER_ERR_OOM, "device grids for host run");
    }
  }
  SPIDER_CUDA(cudaMemcpyAsync(p->dev.host_stage_in, host_in, bytes, cudaMemcpyHostToDevice, stream));
  s = run_cached(p, p->dev.host_stage_in, p->dev.host_stage_out, steps, stream);
  if (s != SPIDER_OK) return s;
  SPIDER_CUDA(cudaMemcpyAsync(host_out, p->dev.host_stage_out, bytes, cudaMemcpyDeviceToHost, stream));
  SPIDER_CUDA(cudaStreamSynchronize(stream));
  int status = 0;
  SPIDER_CUDA(cudaMemcpy(&status, p->dev.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (status != 0) return fail(SPIDER_ERR_TIMEOUT, "a device-side wait ran out");
  return SPIDER_OK;
}

spider_status spider_run_host_async(spider_plan p, const float* host_in, float* host_out, int64_t steps,
                                    cudaStream_t stream) {
  set_error("");
  if (!p) return fail(SPIDER_ERR_INVALID, "plan is NULL");
  if (!host_in || !host_out) return fail(SPIDER_ERR_INVALID, "host pointer is NULL");
  if (steps < 0) return fail(SPIDER_ERR_INVALID, "steps must be >= 0");
  std::lock_guard<std::mutex> lock(p->mu);
  spider_status s = ensure_device(p);
  if (s != SPIDER_OK) return s;
  DeviceState& d = p->dev;
  const size_t bytes = (size_t)p->points() * sizeof(float);
  if (!d.h2d_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&d.h2d_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&d.d2h_stream, cudaStreamNonBlocking);
    for (auto& h : d.host_slots) {
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.copied_in, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.stepped, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.copied_out, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(e, "host pipeline streams and events");
  }
  DeviceState::HostSlot& h = d.host_slots[d.host_next];
  if (!h.in) {
    cudaError_t e = dev_alloc(p, reinterpret_cast<void**>(&h.in), bytes);
    if (e == cudaSuccess) e = dev_alloc(p, reinterpret_cast<void**>(&h.out), bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(SPIDER_ERR_OOM, "device grids for host run");
    }
  }
  d.host_next ^= 1;
  // the slot's input grid was last read by the steps of the call two back,
  // its output grid by that call's copy back
  if (h.used) SPIDER_CUDA(cudaStreamWaitEvent(d.h2d_stream, h.stepped, 0));
  SPIDER_CUDA(cudaMemcpyAsync(h.in, host_in, bytes, cudaMemcpyHostToDevice, d.h2d_stream));
  SPIDER_CUDA(cudaEventRecord(h.copied_in, d.h2d_stream));
  SPIDER_CUDA(cudaStreamWaitEvent(stream, h.copied_in, 0));
  if (h.used) SPIDER_CUDA(cudaStreamWaitEvent(stream, h.copied_out, 0));
  s = run_cached(p, h.in, h.out, steps, stream);
  if (s != SPIDER_OK) return s;
  SPIDER_CUDA(cudaEventRecord(h.stepped, stream));
  SPIDER_CUDA(cudaStreamWaitEvent(d.d2h_stream, h.stepped, 0));
  SPIDER_CUDA(cudaMemcpyAsync(host_out, h.out, bytes, cudaMemcpyDeviceToHost, d.d2h_stream));
  SPIDER_CUDA(cudaEventRecord(h.copied_out, d.d2h_stream));
  h.used = true;
  return SPIDER_OK;
}

spider_status spider_plan_sync(spider_plan p, cudaStream_t stream) {
  if (!p) return fail(SPIDER_ERR_INVALID, "plan is NULL");
  SPIDER_CUDA(cudaStreamSynchronize(stream));
  // the copies of spider_run_host_async calls (their steps ran on `stream`)
  if (p->dev.h2d_stream) SPIDER_CUDA(cudaStreamSynchronize(p->dev.h2d_stream));
  if (p->dev.d2h_stream) SPIDER_CUDA(cudaStreamSynchronize(p->dev.d2h_stream));
  if (p->dev.status) {
    int status = 0;
    SPIDER_CUDA(cudaMemcpy(&status, p->dev.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != 0) {
      cudaMemset(p->dev.status, 0, sizeof(int));
      return fail(SPIDER_ERR_TIMEOUT, "a device-side wait ran out");
    }
  }
  return SPIDER_OK;
}

spider_status spider_plan_error_bound(spider_plan p, spider_precision prec, spider_engine engine, int64_t steps,
                                      double* bound) {
  if (!p || !bound) return fail(SPIDER_ERR_INVALID, "plan or bound is NULL");
  if (steps < 0) return fail(SPIDER_ERR_INVALID, "steps must be >= 0");
  if (prec == SPIDER_AUTO) prec = SPIDER_TF32;
  if (prec < SPIDER_TF32 || prec > SPIDER_BF16X3) return fail(SPIDER_ERR_INVALID, "bad precision");
  if (engine < SPIDER_ENGINE_SPARSE_TC || engine > SPIDER_ENGINE_SPARSE_TC_NO_CO)
    return fail(SPIDER_ERR_INVALID, "bad engine");
  const ErrorModel m = error_model(p, prec, engine);
  if (!m.built) return fail(SPIDER_ERR_UNSUPPORTED, "no kernel for this stencil in that arithmetic");
  *bound = (double)steps * (m.wsum + m.drift) + m.floor;
  return SPIDER_OK;
}

spider_status spider_plan_device_bytes(spider_plan p, size_t* bytes) {
  if (!p || !bytes) return fail(SPIDER_ERR_INVALID, "plan or bytes is NULL");
  std::lock_guard<std::mutex> lock(p->mu);
  const DeviceState& d = p->dev;
  size_t b = 0;
  if (d.a_words) b += p->a_words.size() * 4;
  if (d.meta_words) b += p->meta_words.size() * 4;
  if (d.w_dense) b += p->w.size() * 4;
  if (d.status) b += sizeof(int);
  if (d.scratch) b += d.scratch_bytes;
  if (d.pad) b += d.pad_bytes;
  if (d.host_stage_in) b += 2 * (size_t)p->points() * sizeof(float);
  for (const auto& h : d.host_slots)
    if (h.in) b += 2 * (size_t)p->points() * sizeof(float);
  *bytes = b;
  return SPIDER_OK;
}

void spider_plan_destroy(spider_plan p) {
  if (!p) return;
  free_device(p);
  delete p;
}

}  // extern "C"
