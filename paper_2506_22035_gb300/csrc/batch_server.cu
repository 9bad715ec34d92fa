// Serving: continuous batching of stencil jobs on one GPU.
//
// spider_submit copies the job (plan parameters, host grid) into a FIFO queue.
// Three threads serve it, and none of them holds the server's lock while it
// calls CUDA:
//  * the worker owns kSlots CUDA streams and a stream-ordered memory pool
//    (cudaMemPool_t) that keeps up to the HBM budget reserved.  It admits
//    queued jobs in arrival order while a stream slot is free and the job's
//    device memory (three grids: current, next, and the plan's scratch) fits
//    the HBM budget next to the jobs already on the device; a job's grids
//    and its plan's buffers are allocated from the pool on the job's stream
//    and returned to it there (cudaMallocFromPoolAsync / cudaFreeAsync), so
//    admitting or finishing a job never waits for the device or for the
//    other jobs' work.  It advances every running job by one chunk of at most
//    kChunkSteps time steps once its previous chunk has finished, so a job
//    admitted while others run starts within one chunk and its kernels
//    interleave with theirs on the device;
//  * an upload thread copies admitted jobs' grids to the device, and a
//    download thread copies finished results back and records the
//    submit-to-completion latency.  Host copies (of pageable memory) thus
//    never stall the launches of the other jobs.
// A job's arithmetic does not depend on what else runs: the result is the
// same as a lone spider_run of the same plan in the arithmetic chosen for
// it.  The arithmetic is, among those whose a priori error bound
// (spider_plan_error_bound) meets the job's error target, the one measured
// fastest for the job's class of stencil (sparse TF32, the FP16 hi/lo split,
// FP32 on CUDA cores), run with fused time steps where they are built.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "spider_internal.h"

namespace spider {
namespace {

constexpr int kSlots = 16;
constexpr int64_t kChunkSteps = 16;
constexpr size_t kMaxQueued = 1 << 16;

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t ticket = 0;
  spider_plan plan = nullptr;
  double bound = 0;         // a priori error bound of the chosen arithmetic
  spider_precision prec = SPIDER_TF32;
  spider_engine engine = SPIDER_ENGINE_SPARSE_TC;
  int steps_per_pass = 1;
  int64_t steps = 0, done_steps = 0;
  std::unique_ptr<float[]> host;  // input at submit, result when done
  size_t npts = 0;
  float* cur = nullptr;
  float* nxt = nullptr;
  size_t reserve = 0;       // bytes charged against the budget
  int slot = -1;
  cudaEvent_t ev = nullptr;
  bool finished = false;
  spider_status status = SPIDER_OK;
  std::string error;
  Clock::time_point t_submit, t_done;
};

}  // namespace
}  // namespace spider

struct spider_server_t {
  size_t budget = 0, used = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;       // wakes the worker
  std::condition_variable copy_cv;  // wakes the copy threads
  std::condition_variable done_cv;  // wakes spider_server_wait
  std::deque<uint64_t> completed;   // finished tickets not yet handed out by spider_server_wait
  std::deque<spider::Job*> pending;    // submitted, waiting for admission
  std::deque<spider::Job*> uploads;    // admitted, grid to copy to the device
  std::deque<spider::Job*> ready;      // on the device, first chunk to launch
  std::deque<spider::Job*> downloads;  // computed (or failed), result to copy back
  int uploading = 0;                   // uploads taken by the upload thread, not yet ready
  std::map<uint64_t, std::unique_ptr<spider::Job>> jobs;
  uint64_t next_ticket = 1;
  bool stop = false;       // no more submissions: finish what is queued
  bool worker_done = false;
  cudaStream_t streams[spider::kSlots] = {};
  bool slot_busy[spider::kSlots] = {};
  cudaMemPool_t pool = nullptr;
  std::thread worker, uploader, downloader;
};

namespace spider {
namespace {

size_t job_bytes(const spider_plan_t* p) {
  // two grids of the job and the plan's scratch grid, plus its two padded
  // grids when its rows are not a multiple of 4 floats
  size_t b = 3 * (size_t)p->points() * sizeof(float) + 65536;
  if (p->ndim >= 2 && p->nx % 4 != 0) b += 2 * (size_t)((p->nx + 3) / 4 * 4) * p->ny * p->nz * sizeof(float);
  return b;
}

// Measured speed of the arithmetics per stencil class (GStencil/s on one
// GB300, autotuned, 2048^2 2-D and 160^3 3-D grids of U[0,1) values), used
// to rank the arithmetics whose error bound meets a job's target, and the
// steps per pass / tile variant the autotuner chose there.  2-D: FP32 on
// CUDA cores beats the FP16 split for radius 1, the split wins for larger
// stencils.  3-D (by shape: a star's off-centre planes hold one weight):
// CUDA cores beat the split for every star and the radius-1 and radius-2
// boxes, the split wins for the radius-3 box.
struct ClassRate {
  double tf32, f16x2, cuda_core;
  int t_tf32, v_tf32, t_f16, v_f16, t_cc, v_cc;
};
ClassRate class_rate(const spider_plan_t* p) {
  const int r = std::min(p->r, kMaxR);
  if (p->ndim == 3) {
    static const ClassRate star[3] = {{242, 139, 219, 1, 0, 1, 0, 1, 0},
                                      {192, 131, 230, 1, 0, 1, 0, 1, 0},
                                      {147, 88, 168, 1, 0, 1, 0, 1, 0}};
    static const ClassRate box[3] = {{229, 137, 171, 1, 0, 1, 0, 1, 0},
                                     {136, 83, 93, 1, 0, 1, 0, 1, 0},
                                     {85, 42, 37, 1, 0, 1, 0, 1, 0}};
    return p->shape == SPIDER_STAR ? star[r - 1] : box[r - 1];
  }
  static const ClassRate k2[3] = {{998, 636, 731, 3, 3, 2, 4, 2, 4},
                                  {809, 494, 477, 2, 3, 2, 3, 1, 0},
                                  {699, 400, 331, 2, 0, 3, 1, 1, 0}};
  return k2[r - 1];
}

// Copies n floats, a few threads for large grids (one host thread copies at
// about 12 GB/s on the GPU machine's host, a fraction of its memory bandwidth).
void parallel_copy(float* dst, const float* src, int64_t n) {
  const int64_t kPerThread = int64_t(1) << 22;
  const int nt = (int)std::min<int64_t>(8, std::max<int64_t>(1, n / kPerThread));
  const int64_t chunk = (n + nt - 1) / nt;
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) {
    const int64_t a = std::min(n, t * chunk), b = std::min(n, (t + 1) * chunk);
    th.emplace_back([=] { std::memcpy(dst + a, src + a, (size_t)(b - a) * sizeof(float)); });
  }
  std::memcpy(dst, src, (size_t)std::min(n, chunk) * sizeof(float));
  for (auto& x : th) x.join();
}

// Copies n floats and returns the largest |value| (NaN counts as larger than
// every finite value), in one pass: a few threads for large grids.  The
// largest |value| decides whether the FP16 split can hold the field.
float copy_and_max_abs(float* dst, const float* src, int64_t n) {
  auto part = [](float* d, const float* s, int64_t m) {
    uint32_t mx = 0;  // |x| as bits: integer order = magnitude order for non-negative floats
    for (int64_t i = 0; i < m; ++i) {
      uint32_t b;
      std::memcpy(&b, s + i, 4);
      d[i] = s[i];
      mx = std::max(mx, b & 0x7FFFFFFFu);
    }
    return mx;
  };
  const int64_t kPerThread = int64_t(1) << 22;
  const int nt = (int)std::min<int64_t>(8, std::max<int64_t>(1, n / kPerThread));
  std::vector<uint32_t> mx(nt, 0);
  std::vector<std::thread> th;
  const int64_t chunk = (n + nt - 1) / nt;
  for (int t = 1; t < nt; ++t) {
    const int64_t a = std::min(n, t * chunk), b = std::min(n, (t + 1) * chunk);
    th.emplace_back([&, t, a, b] { mx[t] = part(dst + a, src + a, b - a); });
  }
  mx[0] = part(dst, src, std::min(n, chunk));
  for (auto& x : th) x.join();
  const uint32_t m = *std::max_element(mx.begin(), mx.end());
  float f;
  std::memcpy(&f, &m, 4);
  return f;
}

// Device side of finishing a job (no lock held): stream-ordered frees after
// the job's own work, without waiting for it.
void release_device(spider_server_t* s, Job* j) {
  cudaStream_t js = j->slot >= 0 ? s->streams[j->slot] : nullptr;
  if (j->cur) cudaFreeAsync(j->cur, js);
  if (j->nxt) cudaFreeAsync(j->nxt, js);
  j->cur = j->nxt = nullptr;
  if (j->ev) cudaEventDestroy(j->ev);
  j->ev = nullptr;
  if (j->plan) spider_plan_destroy(j->plan);
  j->plan = nullptr;
}

// Bookkeeping of finishing a job (lock held): its slot and budget return.
void mark_done(spider_server_t* s, Job* j, spider_status st, const std::string& err) {
  if (j->slot >= 0) s->slot_busy[j->slot] = false;
  j->slot = -1;
  s->used -= j->reserve;
  j->reserve = 0;
  j->status = st;
  j->error = err;
  j->finished = true;
  j->t_done = Clock::now();
  s->completed.push_back(j->ticket);
  s->cv.notify_all();
  s->done_cv.notify_all();
}

// Enqueues the job's next chunk on its stream (worker thread, no lock held).
spider_status advance(spider_server_t* s, Job* j) {
  cudaStream_t st = s->streams[j->slot];
  const int64_t n = std::min<int64_t>(kChunkSteps, j->steps - j->done_steps);
  if (n > 0) {
    spider_status r;
    {
      std::lock_guard<std::mutex> lock(j->plan->mu);
      r = run_device(j->plan, j->cur, j->nxt, n, st);
    }
    if (r != SPIDER_OK) return r;
    std::swap(j->cur, j->nxt);
    j->done_steps += n;
  }
  const cudaError_t e = cudaEventRecord(j->ev, st);
  return e == cudaSuccess ? SPIDER_OK : SPIDER_ERR_CUDA;
}

void worker_loop(spider_server_t* s) {
  cudaSetDevice(s->device);
  std::vector<Job*> running;  // worker-owned: chunks in flight
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    // admission in arrival order: reserve a slot and the job's memory
    std::vector<Job*> admitted;
    while (!s->pending.empty()) {
      Job* j = s->pending.front();
      int slot = -1;
      for (int k = 0; k < kSlots; ++k)
        if (!s->slot_busy[k]) { slot = k; break; }
      if (slot < 0 || s->used + j->reserve > s->budget) break;
      s->slot_busy[slot] = true;
      j->slot = slot;
      s->used += j->reserve;
      s->pending.pop_front();
      admitted.push_back(j);
    }
    std::vector<Job*> starting(s->ready.begin(), s->ready.end());
    s->ready.clear();
    const bool quit = s->stop && s->pending.empty() && s->uploads.empty() && s->uploading == 0 &&
                      starting.empty() && running.empty() && admitted.empty();
    if (quit) break;
    lock.unlock();

    std::vector<std::pair<Job*, spider_status>> failed;
    std::vector<Job*> to_upload, computed;
    for (Job* j : admitted) {
      cudaStream_t st = s->streams[j->slot];
      const size_t bytes = j->npts * sizeof(float);
      cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&j->cur), bytes, s->pool, st);
      if (e == cudaSuccess) e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&j->nxt), bytes, s->pool, st);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming);
      if (e != cudaSuccess) {
        cudaGetLastError();
        j->error = std::string("job grids: ") + cudaGetErrorString(e);
        failed.push_back({j, SPIDER_ERR_OOM});
        continue;
      }
      // the plan's own buffers come from the pool too, on the job's stream
      j->plan->dev.pool = s->pool;
      j->plan->dev.pool_stream = st;
      to_upload.push_back(j);
    }
    for (Job* j : starting) {
      const spider_status r = advance(s, j);
      if (r != SPIDER_OK) {
        j->error = spider_last_error();
        failed.push_back({j, r});
      } else {
        running.push_back(j);
      }
    }
    bool progressed = !admitted.empty() || !starting.empty();
    for (size_t i = 0; i < running.size();) {
      Job* j = running[i];
      if (cudaEventQuery(j->ev) != cudaSuccess) {
        ++i;
        continue;
      }
      progressed = true;
      spider_status r = SPIDER_OK;
      if (j->done_steps < j->steps) r = advance(s, j);
      if (r != SPIDER_OK) {
        j->error = spider_last_error();
        failed.push_back({j, r});
      } else if (j->done_steps >= j->steps) {
        computed.push_back(j);
      } else {
        ++i;
        continue;
      }
      running.erase(running.begin() + i);
    }
    for (auto& f : failed) release_device(s, f.first);

    lock.lock();
    for (Job* j : to_upload) s->uploads.push_back(j);
    for (Job* j : computed) s->downloads.push_back(j);
    for (auto& f : failed) mark_done(s, f.first, f.second, f.first->error);
    if (!to_upload.empty() || !computed.empty()) s->copy_cv.notify_all();
    if (!progressed) {
      if (running.empty()) s->cv.wait_for(lock, std::chrono::milliseconds(2));
      else s->cv.wait_for(lock, std::chrono::microseconds(50));
    }
  }
  s->worker_done = true;
  s->copy_cv.notify_all();
}

// Host -> device copies of admitted jobs' grids.  The copy is stream-ordered
// before the job's first chunk, which the worker launches once the job is
// handed back as ready.
void upload_loop(spider_server_t* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    s->copy_cv.wait(lock, [&] { return !s->uploads.empty() || s->worker_done; });
    if (s->uploads.empty()) break;  // the worker has finished: nothing more comes
    Job* j = s->uploads.front();
    s->uploads.pop_front();
    ++s->uploading;
    lock.unlock();
    const cudaError_t e = cudaMemcpyAsync(j->cur, j->host.get(), j->npts * sizeof(float), cudaMemcpyHostToDevice,
                                          s->streams[j->slot]);
    if (e != cudaSuccess) {
      j->error = cudaGetErrorString(e);
      release_device(s, j);
    }
    lock.lock();
    --s->uploading;
    if (e != cudaSuccess) mark_done(s, j, SPIDER_ERR_CUDA, j->error);
    else s->ready.push_back(j);
    s->cv.notify_all();
  }
}

// Device -> host copies of computed results, then the job's memory returns
// to the pool and its latency is recorded.
void download_loop(spider_server_t* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    s->copy_cv.wait(lock, [&] { return !s->downloads.empty() || s->worker_done; });
    if (s->downloads.empty()) break;
    Job* j = s->downloads.front();
    s->downloads.pop_front();
    lock.unlock();
    cudaStream_t st = s->streams[j->slot];
    cudaError_t e = cudaMemcpyAsync(j->host.get(), j->cur, j->npts * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    const std::string err = e == cudaSuccess ? "" : cudaGetErrorString(e);
    release_device(s, j);
    lock.lock();
    mark_done(s, j, e == cudaSuccess ? SPIDER_OK : SPIDER_ERR_CUDA, err);
  }
}

}  // namespace
}  // namespace spider

using namespace spider;

extern "C" {

spider_status spider_server_create(size_t hbm_budget_bytes, spider_server* out) {
  set_error("");
  if (!out) return fail(SPIDER_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes == 0) return fail(SPIDER_ERR_INVALID, "budget must be > 0");
  auto* s = new (std::nothrow) spider_server_t();
  if (!s) return fail(SPIDER_ERR_OOM, "host allocation");
  s->budget = hbm_budget_bytes;
  if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return fail(SPIDER_ERR_CUDA, "cudaGetDevice"); }
  for (int k = 0; k < kSlots; ++k) {
    if (cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) != cudaSuccess) {
      for (int m = 0; m < k; ++m) cudaStreamDestroy(s->streams[m]);
      delete s;
      return fail(SPIDER_ERR_CUDA, "cudaStreamCreate");
    }
  }
  // a pool of device memory that keeps what it has grown to (up to the
  // budget) instead of returning it at every synchronisation
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = s->device;
  cudaError_t pe = cudaMemPoolCreate(&s->pool, &props);
  if (pe == cudaSuccess) {
    uint64_t keep = hbm_budget_bytes;
    pe = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (pe != cudaSuccess) {
    cudaGetLastError();
    if (s->pool) cudaMemPoolDestroy(s->pool);
    for (int k = 0; k < kSlots; ++k) cudaStreamDestroy(s->streams[k]);
    delete s;
    return fail(SPIDER_ERR_CUDA, std::string("memory pool: ") + cudaGetErrorString(pe));
  }
  s->worker = std::thread(worker_loop, s);
  s->uploader = std::thread(upload_loop, s);
  s->downloader = std::thread(download_loop, s);
  *out = s;
  return SPIDER_OK;
}

spider_status spider_submit(spider_server s, spider_plan plan, const float* host_in, int64_t steps,
                            double err_target, uint64_t* ticket) {
  set_error("");
  if (!s || !plan || !host_in || !ticket || steps < 0 || !(err_target > 0))
    return fail(SPIDER_ERR_INVALID, "bad arguments");
  // a private plan in the fastest arithmetic whose a priori error bound
  // meets the target: sparse TF32 (the plan's precision and engine as
  // given, when they meet it), the FP16 hi/lo split (|values| must stay below
  // the FP16 range: the input's largest magnitude, the field not growing),
  // then FP32 on CUDA cores
  const int64_t npts = plan->points();
  std::unique_ptr<float[]> host(new (std::nothrow) float[npts]);
  if (!host) return fail(SPIDER_ERR_OOM, "host copy of the job's grid");
  const float amax = copy_and_max_abs(host.get(), host_in, npts);
  // among the arithmetics whose a priori bound meets the target, the one
  // measured fastest for this class of stencil; the caller's own plan
  // settings when they meet it
  struct Choice { spider_precision prec; spider_engine engine; double rate; };
  const ClassRate cr = class_rate(plan);
  std::vector<Choice> choices = {{SPIDER_TF32, SPIDER_ENGINE_SPARSE_TC, cr.tf32},
                                 {SPIDER_TF32, SPIDER_ENGINE_CUDA_CORE, cr.cuda_core}};
  if (amax < 16384.f) choices.push_back({SPIDER_F16X2, SPIDER_ENGINE_SPARSE_TC, cr.f16x2});
  int pick = -1;
  double bound = 0;
  {
    const ErrorModel own = error_model(plan, plan->prec, plan->engine);
    const double b = (double)steps * (own.wsum + own.drift) + own.floor;
    if (own.built && b <= err_target) {
      choices.insert(choices.begin(), {plan->prec, plan->engine, 1e30});
      pick = 0;
      bound = b;
    }
  }
  if (pick < 0) {
    double best = -1;
    for (size_t k = 0; k < choices.size(); ++k) {
      const ErrorModel m = error_model(plan, choices[k].prec, choices[k].engine);
      if (!m.built) continue;
      const double b = (double)steps * (m.wsum + m.drift) + m.floor;
      if (b <= err_target && choices[k].rate > best) {
        best = choices[k].rate;
        pick = (int)k;
        bound = b;
      }
    }
  }
  if (pick < 0)
    return fail(SPIDER_ERR_UNSUPPORTED, "no arithmetic built for this stencil meets the error target");
  spider_plan copy = nullptr;
  spider_status st = spider_plan_create(plan->ndim, plan->extents, plan->shape, plan->r, plan->w.data(),
                                        choices[pick].prec, &copy);
  if (st != SPIDER_OK) return st;
  if (choices[pick].engine != SPIDER_ENGINE_SPARSE_TC) {
    st = spider_plan_set_engine(copy, choices[pick].engine);
    if (st != SPIDER_OK) {
      spider_plan_destroy(copy);
      return st;
    }
  }
  // fused passes: the caller's setting, else the autotuner's choice for
  // this kind of stencil if one was measured in this process, else the
  // class's measured choice
  int T = plan->steps_per_pass, v = plan->tile_variant;
  if (T <= 1 && !autotune_lookup(copy, &T, &v)) {
    const bool tf32 = copy->engine == SPIDER_ENGINE_SPARSE_TC && copy->prec == SPIDER_TF32;
    const bool f16 = copy->engine == SPIDER_ENGINE_SPARSE_TC && copy->prec == SPIDER_F16X2;
    T = tf32 ? cr.t_tf32 : f16 ? cr.t_f16 : copy->engine == SPIDER_ENGINE_CUDA_CORE ? cr.t_cc : 1;
    v = tf32 ? cr.v_tf32 : f16 ? cr.v_f16 : copy->engine == SPIDER_ENGINE_CUDA_CORE ? cr.v_cc : 0;
  }
  copy->steps_per_pass = std::max(1, std::min(T, max_steps_per_pass(copy)));
  copy->tile_variant = v;
  auto j = std::make_unique<Job>();
  j->plan = copy;
  j->bound = bound;
  j->prec = copy->prec;
  j->engine = copy->engine;
  j->steps_per_pass = copy->steps_per_pass;
  j->steps = steps;
  j->reserve = job_bytes(copy);
  if (j->reserve > s->budget) {
    spider_plan_destroy(copy);
    return fail(SPIDER_ERR_OOM, "job larger than the server's HBM budget");
  }
  j->host = std::move(host);
  j->npts = (size_t)npts;
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->pending.size() >= kMaxQueued) {
    spider_plan_destroy(copy);
    return fail(SPIDER_ERR_BUSY, "queue full");
  }
  j->ticket = s->next_ticket++;
  *ticket = j->ticket;
  s->pending.push_back(j.get());
  s->jobs.emplace(j->ticket, std::move(j));
  s->cv.notify_all();
  return SPIDER_OK;
}

spider_status spider_poll(spider_server s, uint64_t ticket, float* out, int* done, double* latency_s) {
  set_error("");
  if (!s || !done) return fail(SPIDER_ERR_INVALID, "bad arguments");
  std::unique_ptr<Job> owned;  // a released record, copied out without the lock
  Job* j = nullptr;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return fail(SPIDER_ERR_INVALID, "unknown ticket");
    j = it->second.get();
    *done = j->finished ? 1 : 0;
    if (!j->finished) return SPIDER_OK;
    if (latency_s) *latency_s = std::chrono::duration<double>(j->t_done - j->t_submit).count();
    if (out) {
      owned = std::move(it->second);
      s->jobs.erase(it);
    }
    if (j->status != SPIDER_OK) return fail(j->status, j->error);
  }
  if (owned && out) parallel_copy(out, owned->host.get(), (int64_t)owned->npts);
  return SPIDER_OK;
}

spider_status spider_server_job_arithmetic(spider_server s, uint64_t ticket, spider_precision* prec,
                                          spider_engine* engine, int* steps_per_pass, double* bound) {
  set_error("");
  if (!s) return fail(SPIDER_ERR_INVALID, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return fail(SPIDER_ERR_INVALID, "unknown ticket");
  const Job* j = it->second.get();
  if (prec) *prec = j->prec;
  if (engine) *engine = j->engine;
  if (steps_per_pass) *steps_per_pass = j->steps_per_pass;
  if (bound) *bound = j->bound;
  return SPIDER_OK;
}

spider_status spider_server_wait(spider_server s, double timeout_s, uint64_t* ticket, int* got) {
  set_error("");
  if (!s || !ticket || !got || !(timeout_s >= 0)) return fail(SPIDER_ERR_INVALID, "bad arguments");
  *got = 0;
  std::unique_lock<std::mutex> lock(s->mu);
  const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  s->done_cv.wait_until(lock, until, [&] { return !s->completed.empty(); });
  if (s->completed.empty()) return SPIDER_OK;
  *ticket = s->completed.front();
  s->completed.pop_front();
  *got = 1;
  return SPIDER_OK;
}

void spider_server_destroy(spider_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();  // every job computed; the copy threads then drain
  if (s->uploader.joinable()) s->uploader.join();
  if (s->downloader.joinable()) s->downloader.join();
  for (int k = 0; k < kSlots; ++k) {
    cudaStreamSynchronize(s->streams[k]);  // the stream-ordered frees have run
    cudaStreamDestroy(s->streams[k]);
  }
  if (s->pool) cudaMemPoolDestroy(s->pool);
  delete s;
}

}  // extern "C"
