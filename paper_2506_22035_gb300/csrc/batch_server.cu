// Serving: continuous batching of stencil jobs on one GPU.
//
// spider_submit copies the job (plan parameters, host grid) into a FIFO queue.
// A worker thread owns kSlots CUDA streams and a stream-ordered memory pool
// (cudaMemPool_t) that keeps up to the HBM budget reserved.  Each loop it
//  * admits queued jobs in arrival order while a stream slot is free and the
//    job's device memory (three grids: current, next, and the plan's scratch)
//    fits the HBM budget next to the jobs already on the device; a job's
//    grids and its plan's buffers are allocated from the pool on the job's
//    stream and returned to it there (cudaMallocFromPoolAsync /
//    cudaFreeAsync), so admitting or finishing a job never waits for the
//    device or for the other jobs' work;
//  * advances every running job by one chunk of at most kChunkSteps time
//    steps once its previous chunk has finished, so a job admitted while
//    others run starts within one chunk and its kernels interleave with
//    theirs on the device;
//  * copies finished results back, frees their memory and records the
//    submit-to-completion latency.
// A job's arithmetic does not depend on what else runs: the result is the
// same as a lone spider_run of the same plan in the arithmetic chosen for
// it.  The arithmetic is the fastest whose a priori error bound
// (spider_plan_error_bound) meets the job's error target: sparse TF32, then
// the FP16 hi/lo split, then FP32 on CUDA cores.
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

constexpr int kSlots = 8;
constexpr int64_t kChunkSteps = 16;
constexpr size_t kMaxQueued = 1 << 16;

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t ticket = 0;
  spider_plan plan = nullptr;
  double bound = 0;         // a priori error bound of the chosen arithmetic
  int64_t steps = 0, done_steps = 0;
  std::vector<float> host;  // input at submit, result when done
  float* cur = nullptr;
  float* nxt = nullptr;
  size_t reserve = 0;       // bytes charged against the budget
  int slot = -1;
  cudaEvent_t ev = nullptr;
  bool copying = false, finished = false;
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
  std::condition_variable cv;
  std::deque<spider::Job*> pending;
  std::vector<spider::Job*> running;
  std::map<uint64_t, std::unique_ptr<spider::Job>> jobs;
  uint64_t next_ticket = 1;
  bool stop = false;
  cudaStream_t streams[spider::kSlots] = {};
  bool slot_busy[spider::kSlots] = {};
  cudaMemPool_t pool = nullptr;
  std::thread worker;
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

void finish(spider_server_t* s, Job* j, spider_status st, const std::string& err) {
  // stream-ordered frees: after the job's own work, without waiting for it
  cudaStream_t js = j->slot >= 0 ? s->streams[j->slot] : nullptr;
  if (j->cur) cudaFreeAsync(j->cur, js);
  if (j->nxt) cudaFreeAsync(j->nxt, js);
  j->cur = j->nxt = nullptr;
  if (j->ev) cudaEventDestroy(j->ev);
  j->ev = nullptr;
  if (j->plan) spider_plan_destroy(j->plan);
  j->plan = nullptr;
  if (j->slot >= 0) s->slot_busy[j->slot] = false;
  j->slot = -1;
  s->used -= j->reserve;
  j->reserve = 0;
  j->status = st;
  j->error = err;
  j->finished = true;
  j->t_done = Clock::now();
}

// Enqueues the job's next chunk (or the copy-back) on its stream.
void advance(spider_server_t* s, Job* j) {
  cudaStream_t st = s->streams[j->slot];
  if (j->done_steps < j->steps) {
    const int64_t n = std::min<int64_t>(kChunkSteps, j->steps - j->done_steps);
    spider_status r;
    {
      std::lock_guard<std::mutex> lock(j->plan->mu);
      r = run_device(j->plan, j->cur, j->nxt, n, st);
    }
    if (r != SPIDER_OK) { finish(s, j, r, spider_last_error()); return; }
    std::swap(j->cur, j->nxt);
    j->done_steps += n;
  } else {
    cudaError_t e = cudaMemcpyAsync(j->host.data(), j->cur, j->host.size() * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) { finish(s, j, SPIDER_ERR_CUDA, cudaGetErrorString(e)); return; }
    j->copying = true;
  }
  cudaEventRecord(j->ev, st);
}

bool admit(spider_server_t* s, Job* j) {
  int slot = -1;
  for (int k = 0; k < kSlots; ++k)
    if (!s->slot_busy[k]) { slot = k; break; }
  if (slot < 0 || s->used + j->reserve > s->budget) return false;
  const size_t bytes = j->host.size() * sizeof(float);
  cudaStream_t st = s->streams[slot];
  cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&j->cur), bytes, s->pool, st);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&j->nxt), bytes, s->pool, st);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (j->cur) cudaFreeAsync(j->cur, st);
    if (j->nxt) cudaFreeAsync(j->nxt, st);
    j->cur = j->nxt = nullptr;
    return false;  // device memory is short right now: retry when a job finishes
  }
  s->slot_busy[slot] = true;
  j->slot = slot;
  s->used += j->reserve;
  // the plan's own buffers come from the pool too, on the job's stream
  j->plan->dev.pool = s->pool;
  j->plan->dev.pool_stream = st;
  e = cudaMemcpyAsync(j->cur, j->host.data(), bytes, cudaMemcpyHostToDevice, s->streams[slot]);
  if (e != cudaSuccess) { finish(s, j, SPIDER_ERR_CUDA, cudaGetErrorString(e)); return true; }
  s->running.push_back(j);
  advance(s, j);
  return true;
}

void worker_loop(spider_server_t* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    // admission in arrival order
    while (!s->pending.empty() && admit(s, s->pending.front())) s->pending.pop_front();
    // progress
    bool progressed = false;
    for (size_t i = 0; i < s->running.size();) {
      Job* j = s->running[i];
      if (!j->finished && cudaEventQuery(j->ev) == cudaSuccess) {
        progressed = true;
        if (j->copying) finish(s, j, SPIDER_OK, "");
        else advance(s, j);
      }
      if (j->finished) {
        s->running.erase(s->running.begin() + i);
        s->cv.notify_all();
      } else {
        ++i;
      }
    }
    if (s->stop && s->pending.empty() && s->running.empty()) break;
    if (!progressed) {
      if (s->running.empty() && s->pending.empty()) s->cv.wait(lock);
      else s->cv.wait_for(lock, std::chrono::microseconds(50));
    }
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
  float amax = 0.f;
  for (int64_t i = 0; i < npts; ++i) amax = std::max(amax, std::fabs(host_in[i]));
  struct Choice { spider_precision prec; spider_engine engine; };
  std::vector<Choice> choices = {{plan->prec, plan->engine}, {SPIDER_TF32, SPIDER_ENGINE_SPARSE_TC}};
  if (amax < 16384.f) choices.push_back({SPIDER_F16X2, SPIDER_ENGINE_SPARSE_TC});
  choices.push_back({SPIDER_TF32, SPIDER_ENGINE_CUDA_CORE});
  int pick = -1;
  double bound = 0;
  for (size_t k = 0; k < choices.size() && pick < 0; ++k) {
    const ErrorModel m = error_model(plan, choices[k].prec, choices[k].engine);
    if (!m.built) continue;
    bound = (double)steps * (m.wsum + m.drift) + m.floor;
    if (bound <= err_target) pick = (int)k;
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
  copy->steps_per_pass = std::min(plan->steps_per_pass, max_steps_per_pass(copy));
  copy->tile_variant = plan->tile_variant;
  auto j = std::make_unique<Job>();
  j->plan = copy;
  j->bound = bound;
  j->steps = steps;
  j->reserve = job_bytes(copy);
  if (j->reserve > s->budget) {
    spider_plan_destroy(copy);
    return fail(SPIDER_ERR_OOM, "job larger than the server's HBM budget");
  }
  j->host.assign(host_in, host_in + copy->points());
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
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return fail(SPIDER_ERR_INVALID, "unknown ticket");
  Job* j = it->second.get();
  *done = j->finished ? 1 : 0;
  if (!j->finished) return SPIDER_OK;
  if (latency_s) *latency_s = std::chrono::duration<double>(j->t_done - j->t_submit).count();
  const spider_status st = j->status;
  const std::string err = j->error;
  if (out) {
    if (st == SPIDER_OK) std::memcpy(out, j->host.data(), j->host.size() * sizeof(float));
    s->jobs.erase(it);
  }
  if (st != SPIDER_OK) return fail(st, err);
  return SPIDER_OK;
}

void spider_server_destroy(spider_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  for (int k = 0; k < kSlots; ++k) {
    cudaStreamSynchronize(s->streams[k]);  // the stream-ordered frees have run
    cudaStreamDestroy(s->streams[k]);
  }
  if (s->pool) cudaMemPoolDestroy(s->pool);
  delete s;
}

}  // extern "C"
