// spider_batch: many 2-D grids of different sizes, radii and step counts in
// one call.  Small grids (and single steps) share one persistent launch over
// a device work queue; larger grids run as fused multi-step passes of their
// own on side streams beside it (see kFuseMinPoints).
//
// Queue work items are (pass p, job, tile); CTAs claim them with one atomic
// counter, in pass-major order.  Every item runs the fused kernel's level
// scheme on a tile of (56 - 2r) x 120 outputs: a two-step pass computes
// level 1 (56 x 128) into shared memory and level 2 into the grid from one
// input box of (56 + 2r) x 136 points; a one-step pass (the first pass of a
// job whose step count is odd or whose input rows TMA cannot describe, the
// last when one step is left, every pass of a one-step job, or every pass
// when spider_batch_configure asks for one step per item) computes one level
// from a 56 x 128 box.  Item (p, j, tile) reads job j's grid after pass p-1
// over the tile plus a halo narrower than a tile, so it may start only after
// the tile and its eight neighbours have finished pass p-1 (those are also
// the last readers of the buffer it overwrites).  Each job keeps one
// completion counter per tile; the producer warp tests the neighbours'
// counters (acquire loads) and publishes a tile's counter with a release
// store once the consumer warps have stored the tile.  The deadlock-freedom
// argument is at batch_kernel.
//
// Each job brings its own tensor maps and packed operands (TF32 sparse MMA).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "fused_kernels.cuh"
#include "launch.h"
#include "stencil_kernels.cuh"

namespace spider {

// api.cu: run_device, with repeated (grids, steps, configuration) calls
// captured once and replayed as a CUDA graph (plan lock held by the caller).
spider_status run_cached(spider_plan_t* p, const float* in, float* out, int64_t steps, cudaStream_t stream);

namespace {

// Every queue item runs the fused kernel's level scheme on a tile of
// (56 - 2r) x 120 outputs, one or two time steps: level 1 of a two-step item
// is 56 x 128, i.e. 7 x 2 warp units of 8 rows x 64 columns, two for each of
// the seven consumer warps (level 2 and one-step items: 7 x 2 units as
// well).  Seven consumer warps and one producer warp make 256 threads, so
// three CTAs per SM keep 80 registers a thread, the stand-alone fused
// kernel's budget (with a ninth warp the cap of 72 made the tile code spill).
constexpr int kConsumerWarps = 7;
constexpr int kThreads = kConsumerWarps * 32;  // consumer threads
constexpr int kQueueThreads = kThreads + 32;    // and one producer warp
constexpr int kTileL1 = 56;                     // rows of level 1 (two-step) / of the box (one-step)
// The largest box: a two-step pass, (56 - 2r + 4r) x (120 + 16) points.
constexpr int kMaxStageFloats = (kTileL1 + 2 * kMaxR) * (120 + 4 * kHaloX);
constexpr int kStageStride = (kMaxStageFloats * 4 + 1023) / 1024 * 1024;
constexpr int kLevelFloats = kTileL1 * 128;  // level 1 of a two-step pass (pitch 128)
// Shared memory: one stage | level buffer | the current job's packed
// operands (A words, metadata) and record | barriers and slot | tables.
constexpr int kOpsABytes = (2 * kMaxR + 2) * 32 * 16;  // uint4 per lane per A index
constexpr int kOpsEBytes = (2 * kMaxR + 2) * 32 * 4;   // metadata word per lane per A index
constexpr int kJobBytes = 256;                         // >= sizeof(BatchJob), checked below
constexpr int kLevelOff = kStageStride;
constexpr int kOpsOff = kLevelOff + kLevelFloats * 4;
constexpr int kJobOff = kOpsOff + kOpsABytes + kOpsEBytes;
constexpr int kBarOff = kJobOff + kJobBytes;
constexpr int kTablesOff = kBarOff + 128;
constexpr int kSmemBase = kTablesOff + 1024;  // + alignment slack
// queue tables go to shared memory only while three CTAs still fit on an SM
constexpr int kMaxTableSmem = 3 * 1024;
static_assert(3 * (kSmemBase + kMaxTableSmem + 1024) <= 228 * 1024, "three CTAs per SM");
// Grids of at least this many points (with more than one step) run as fused
// passes of their own on side streams; smaller ones, and single steps, go
// through the persistent queue.  Measured on the mixed batch of 64 grids of
// 256^2..4096^2 (GStencil/s, replayed), with two fused steps per queue item:
// 2^16 (every grid of the mix fused): 1120, every grid in the queue: 957
// (an earlier queue kernel: 2^20: 1026, 2^18: 1066, 2^17: 1045).  A fused
// pass is statically scheduled, while a queue item pays a claim, a
// dependency test and a hand-over, and consecutive passes of one job on a
// side stream find its grids in L2.  Below it the queue wins: 256 grids of
// 32^2..255^2 points run at 278 GStencil/s through it and at 41 as fused
// passes on side streams (grids of a few tiles are all launch latency).
constexpr long long kFuseMinPoints = 1LL << 16;
constexpr int kQueueStepsPerItem = 2;
// Routing of spider_batch (spider_batch_configure): grids of at least
// g_fuse_min_points points (and more than one step) run as fused passes on
// side streams; queue items take g_queue_steps steps (1 or 2).
std::atomic<long long> g_fuse_min_points{kFuseMinPoints};
std::atomic<int> g_queue_steps{kQueueStepsPerItem};

// Queue item the next spider_batch call leaves out (spider_batch_drop_item), -1: none.
std::atomic<long long> g_drop_item{-1};

// The last persistent launch of each device, kept for replay: the queue's
// tables, tensor maps and counters stay in the device's work-queue buffer,
// and a later spider_batch call whose queued jobs are the same grids (same
// plans, buffers, step counts and routing) relaunches the instantiated graph
// (counter reset + kernel) without rebuilding or uploading anything.  Any
// other call rebuilds the buffer and replaces the entry.  Guarded by the
// device's batch lock.
struct QueueReplay {
  std::vector<uint64_t> key;
  cudaGraphExec_t exec = nullptr;
  const int* status = nullptr;
};
QueueReplay g_replay[64];
constexpr int kSideStreams = 8;                  // streams the fused grids run on, next to the queue

// Non-blocking streams for the grids that run as fused passes beside the
// persistent queue, kept per device for the process.  spider_batch calls on
// one device take batch_lock(dev) for their whole duration, so two calls
// (from different threads or caller streams) never share these streams at
// the same time: one call's join never waits on another call's work.
cudaStream_t side_stream(int dev, int k) {
  static std::mutex mu;
  static cudaStream_t pool[64][kSideStreams] = {};
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!pool[dev][k] && cudaStreamCreateWithFlags(&pool[dev][k], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    pool[dev][k] = nullptr;
  }
  return pool[dev][k];
}

std::mutex& batch_lock(int dev) {
  static std::mutex locks[64];
  return locks[dev < 0 || dev >= 64 ? 0 : dev];
}

// Orders `stream` after the work issued on the side streams (on every way
// out of spider_batch, so a caller's later work on `stream` sees the grids).
struct SideJoin {
  cudaStream_t stream = nullptr;
  cudaStream_t sides[kSideStreams] = {};
  bool used = false;
  void join() {
    if (!used) return;
    used = false;
    for (cudaStream_t s : sides) {
      if (!s) continue;
      cudaEvent_t ev;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamSynchronize(s);  // no event: wait on the host instead
        continue;
      }
      cudaEventRecord(ev, s);
      cudaStreamWaitEvent(stream, ev, 0);
      cudaEventDestroy(ev);
    }
  }
  ~SideJoin() { join(); }
};

// A job runs in passes.  Pass p reads `in` (p = 0) or bufs[(first + p - 1)
// % 2] and writes `out` (the last pass) or bufs[(first + p) % 2].  When in,
// out and the plan's scratch grid are all TMA-describable, bufs = {out,
// scratch} with the parity `first` chosen so that the last pass lands in out,
// and pitch = nx.  Otherwise (rows of nx floats are not a multiple of 16
// bytes, or a buffer is not 16-byte aligned) bufs are the plan's two padded
// grids with rows `pitch` (nx rounded up to 4) floats apart, first = 0: every
// pass but the first then loads through TMA, and only the first pass's halo
// boxes are loaded by the consumers (`tma0` = 0).
//
// Every job runs on tiles of (56 - 2r) x 120 outputs.  A job with `two` = 0
// takes one step per pass (a 56 x 128 box).  A job with `two` = 1 takes two
// steps per pass: level 1, grown by r rows and 4 columns on each side, goes
// to shared memory, level 2 to the grid, from one input box of (56 + 2r) x
// 136 points.  Its first pass takes a single step when the step count is odd
// or the consumers load it (`head1`), and its last a single step when what
// is left is odd (`tail1`), on the same tiles.
struct alignas(16) BatchJob {  // 16-byte multiple: records are bulk-copied
  int64_t nx, ny;
  int64_t pitch;       // row pitch of bufs (floats)
  int r;
  int tiles_x, tiles_y;
  int steps;           // time steps of the run
  int passes;          // passes of the run
  int two;             // 1: two steps per pass on fused tiles
  int head1, tail1;    // two: the first / last pass takes one step
  int by, bx;          // output tile
  int first;
  int map0;            // tensor maps: map0 + 0 = in, + 1 = bufs[0], + 2 = bufs[1] (box of a full pass);
                       // + 3 = in, + 4 = bufs[0], + 5 = bufs[1] (box of a one-step pass of a two-step job)
  const uint4* a;      // packed A operands (TF32, per A index)
  const uint32_t* meta;
  float* bufs[2];
  float* out;
  const float* in;
  int* done;           // per-tile count of completed passes
  int tma0;            // 1: `in` is TMA-describable; 0: consumers load the first pass's boxes
};

static_assert(sizeof(BatchJob) <= kJobBytes && sizeof(BatchJob) % 16 == 0, "job record copy");

// Steps of pass p of a job.
__host__ __device__ inline int pass_steps(const BatchJob& jb, int p) {
  if (!jb.two) return 1;
  if (jb.head1 && p == 0) return 1;
  if (jb.tail1 && p == jb.passes - 1) return 1;
  return 2;
}

// Two-step pass and one-step pass on the queue tile of radius R: the output
// tile is (56 - 2R) x 120; level 1 of the two-step pass is 56 x 128.
template <int R>
using BatchFused2 = FuseCfg<R, 2, kTileL1 - 2 * R, 120, 8, kConsumerWarps>;
template <int R>
using BatchFused1 = FuseCfg<R, 1, kTileL1 - 2 * R, 120, 8, kConsumerWarps>;
static_assert(BatchFused2<1>::kPStride == kLevelFloats * 4 && BatchFused2<3>::kPStride == kLevelFloats * 4,
              "level buffer");
static_assert(BatchFused2<kMaxR>::kInBytes <= kStageStride && BatchFused1<1>::kInBytes <= kStageStride, "stage");

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr int kNA = 2 * kMaxR + 2;  // packed A operands of the largest radius

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One pass of a job on the fused tile at (x0, y0): STEPS = 2 runs level 1
// from the staged box into the shared level buffer P and level 2 into the
// grid; STEPS = 1 runs one level from the box into the grid.  Every step but
// a job's last stores its outputs rounded to TF32 (`out_tf32`), so the steps
// after the first read operands that need no rounding (RIN = false); the MMA
// sees the same values either way.  A8 / E8 hold the job's packed operands
// (the first 2R + 2 entries).  The consumer warps synchronise among
// themselves (named barrier 1), not with the producer warp: once every
// consumer has read the box, thread 0 arrives on `boxfree` (the producer may
// load the next item's box into the stage), and once every consumer has
// stored its outputs, on `done` (the producer publishes the tile).
template <int R, int STEPS, bool RIN>
__device__ __forceinline__ void batch_fused(const BatchJob& jb, const uint4 (&A8)[kNA], const uint32_t (&E8)[kNA],
                                            const float* S, float* P, float* dst, int64_t pitch, int x0, int y0,
                                            bool out_tf32, int* status, uint64_t* boxfree, uint64_t* done) {
  using F = typename std::conditional<STEPS == 2, BatchFused2<R>, BatchFused1<R>>::type;
  uint4 A[F::NA];
  uint32_t E[F::NA];
#pragma unroll
  for (int a = 0; a < F::NA; ++a) {
    A[a] = A8[a];
    E[a] = E8[a];
  }
  uint4 Ad[F::NA][2];                        // unused in the sparse TF32 mode
  uint4 Am[F::RY + 1];
  uint32_t Em[F::RY + 1];
  float W[(2 * F::RY + 1) * (2 * F::RX + 1)];
  StepArgs args = {};
  args.dst = dst;
  args.nx = jb.nx;
  args.ny = jb.ny;
  args.nz = 1;
  args.pitch = pitch;
  args.status = status;
  args.out_tf32 = out_tf32 ? 1 : 0;
  FusedCtx c;
  c.args = &args;
  c.x0 = x0;
  c.y0 = y0;
  c.lane = threadIdx.x & 31;
  c.warp = threadIdx.x >> 5;
  c.g = c.lane >> 2;
  c.q = c.lane & 3;
  if constexpr (STEPS == 2) {
    fused_level<F, Mode::SpTF32, RIN, 1>(c, S, P, A, E, Ad, Am, Em, W);
    asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");  // level 1 complete in P, box read
    if (threadIdx.x == 0) mbar_arrive(boxfree);
    fused_level<F, Mode::SpTF32, RIN, 2>(c, P, nullptr, A, E, Ad, Am, Em, W);
    asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");  // stores issued, P free for the next item
    if (threadIdx.x == 0) mbar_arrive(done);
  } else {
    fused_level<F, Mode::SpTF32, RIN, 1>(c, S, nullptr, A, E, Ad, Am, Em, W);
    asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
    if (threadIdx.x == 0) {
      mbar_arrive(boxfree);
      mbar_arrive(done);
    }
  }
}

// Warp-parallel search: the largest index i in [0, n) with table[i] <= key
// (table ascending, table[0] <= key).  32 probes per round.
__device__ __forceinline__ int warp_search(const long long* __restrict__ table, int n, long long key, int lane) {
  int lo = 0, len = n;
  while (len > 1) {
    const int step = (len + 31) / 32;
    const int idx = lo + lane * step;
    const bool ok = idx < lo + len && idx < n && table[idx] <= key;
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    const int best = 31 - __clz(m);  // lane 0 always qualifies
    lo = lo + best * step;
    len = min(step, n - lo);
  }
  return lo;
}

struct ItemSlot {
  int job, s, tile, end;
  int skip;  // the item was left out (spider_batch_drop_item): no load, no compute, no publication
};

// Waits for phase `parity` of `bar` like mbar_wait_bounded, but sleeps
// `ns` nanoseconds between polls, so a warp that waits for a long time (a
// producer two items ahead of its consumers) leaves the issue slots to the
// warps that compute.
__device__ __forceinline__ bool mbar_wait_backoff(uint64_t* bar, uint32_t parity, int* status, unsigned ns,
                                                  long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) {
      atomicExch(status, kStatusTimeout);
      return false;
    }
    __nanosleep(ns);
  }
  return true;
}

// The producer warp's view of one claimed item.
struct Claim {
  int end, skip;  // past the last item / left out (spider_batch_drop_item)
  int job, s, tile, tx, ty;
};

// Claims the next queue item (one global atomic by lane 0) and decodes it
// into (job, pass, tile) with a warp-parallel search of the entry table.
__device__ __forceinline__ Claim claim_item(int* counter, long long total, const long long* __restrict__ ent_prefix,
                                            const int2* __restrict__ ent, int n_ent,
                                            const BatchJob* __restrict__ jobs, long long drop_item, int lane) {
  long long item = 0;
  if (lane == 0) item = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(counter), 1ULL);
  item = __shfl_sync(0xffffffffu, item, 0);
  Claim c = {};
  c.end = item >= total;
  if (c.end) return c;
  const int e = warp_search(ent_prefix, n_ent, item, lane);
  const int2 je = ent[e];
  c.job = je.x;
  c.s = je.y;
  c.tile = (int)(item - ent_prefix[e]);
  c.tx = c.tile % jobs[c.job].tiles_x;
  c.ty = c.tile / jobs[c.job].tiles_x;
  c.skip = item == drop_item;
  return c;
}

// Whether a wait of this launch has run out (the status word is set).
__device__ __forceinline__ bool failed(const int* status) {
  return *reinterpret_cast<const volatile int*>(status) != 0;
}

// All consumer threads' `v` and-ed (named barrier 1), so every consumer warp
// takes the same way out of the item loop.
__device__ __forceinline__ bool consumers_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kThreads)
      : "memory");
  return r != 0;
}

// Whether the 3 x 3 neighbourhood of the item's tile has finished pass s - 1
// (lanes 0..8 read one pass counter each, acquire).  With `block` it waits
// until they have (bounded: past the limit, or once another wait of the
// launch ran out, it records a timeout and returns true; the producer then
// ends its CTA's queue, see batch_kernel).
__device__ __forceinline__ bool deps_ready(const BatchJob& jb, const Claim& c, bool block, int lane, int* status,
                                           long long limit) {
  bool mine = true;
  if (c.s > 0 && lane < 9) {
    const int ntx = c.tx + lane % 3 - 1, nty = c.ty + lane / 3 - 1;
    if (ntx >= 0 && nty >= 0 && ntx < jb.tiles_x && nty < jb.tiles_y) {
      const int* flag = jb.done + nty * jb.tiles_x + ntx;
      if (ld_acquire(flag) < c.s) {
        if (!block) {
          mine = false;
        } else {
          const long long t0 = clock64();
          while (ld_acquire(flag) < c.s) {
            // past the limit, or another wait already ran out: give up
            if (clock64() - t0 > limit || failed(status)) { atomicExch(status, kStatusTimeout); break; }
            __nanosleep(128);
          }
        }
      }
    }
  }
  const bool all = __all_sync(0xffffffffu, mine);
  __syncwarp();  // the other lanes' acquires before lane 0's load below
  return all;
}

// Asynchronous global -> shared copy of `bytes` bytes (16-byte aligned, a
// multiple of 16), completing on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Where the producer puts an item's data for the consumers.
struct Stage {
  float* box;            // the item's input box
  uint4* ops_a;          // the job's packed A operands (2r + 2 per lane)
  uint32_t* ops_e;       // its metadata words
  BatchJob* job;         // its record
  ItemSlot* slot;
  uint64_t* full;        // completes when all of it has landed
};

// Lane 0 hands item `c` to the consumers: its slot, then (completing
// `full`) its box (TMA) and, when the job differs from the previous item's
// (`*prev_job`), the job's record and packed operands (bulk copies from
// `jobs_g`, the job table in global memory, and the plan's buffers); a plain
// arrival when there is nothing to load (the end, a left-out item).
// Returns whether a copy was issued.
__device__ __forceinline__ bool hand_over(const Claim& c, const BatchJob* __restrict__ jobs,
                                         const BatchJob* __restrict__ jobs_g, const CUtensorMap* __restrict__ maps,
                                         const Stage& sg, int* prev_job, int lane) {
  bool copies = false;
  if (lane == 0) {
    sg.slot->job = c.job;
    sg.slot->s = c.s;
    sg.slot->tile = c.tile;
    sg.slot->end = c.end;
    sg.slot->skip = c.skip;
    const BatchJob* jb = (c.end || c.skip) ? nullptr : &jobs[c.job];
    if (jb) {
      // the box, unless the consumers load this first pass themselves
      const bool box = c.s > 0 || jb->tma0;
      const bool fresh = c.job != *prev_job;
      const int np = pass_steps(*jb, c.s);
      const int bw = jb->bx + 2 * kHaloX * np, bh = jb->by + 2 * jb->r * np;
      const uint32_t na = 2 * jb->r + 2;
      const uint32_t bytes = (box ? (uint32_t)(bw * bh * 4) : 0u) +
                             (fresh ? na * 16 * 32 + na * 4 * 32 + (uint32_t)sizeof(BatchJob) : 0u);
      if (bytes > 0) {
        mbar_arrive_expect_tx(sg.full, bytes);
        if (box) {
          // the neighbours' generic-proxy stores must be visible to the TMA read
          asm volatile("fence.proxy.async.global;" ::: "memory");
          // the pass's input box: the tile grown by r rows and 4 columns per step
          const int src_map = jb->map0 + (np == 1 ? 3 : 0) + (c.s == 0 ? 0 : 1 + (jb->first + c.s - 1) % 2);
          tma_load_3d(sg.box, &maps[src_map], sg.full, c.tx * jb->bx - kHaloX * np, c.ty * jb->by - jb->r * np, 0);
        }
        if (fresh) {
          bulk_load(sg.ops_a, jb->a, na * 16 * 32, sg.full);
          bulk_load(sg.ops_e, jb->meta, na * 4 * 32, sg.full);
          bulk_load(sg.job, jobs_g + c.job, (uint32_t)sizeof(BatchJob), sg.full);
          *prev_job = c.job;
        }
        copies = true;
      } else {
        mbar_arrive(sg.full);
      }
    } else {
      mbar_arrive(sg.full);
    }
  }
  return __shfl_sync(0xffffffffu, (int)copies, 0) != 0;
}

// The persistent queue kernel: seven consumer warps compute the items'
// tiles; one producer warp claims the items, decodes them, tests their
// dependencies and loads their boxes, one item ahead of the consumers, so
// that work runs beside the tensor-core work.  One stage: the next item's
// box is loaded into it as soon as the consumers have read the current one
// (after level 1 of a two-step item), so the load overlaps level 2.  Three
// CTAs per SM, as for the stand-alone fused kernel.
//
// The producer never blocks on another CTA's progress while its CTA holds
// an unpublished item: the next item's dependencies are first only tested;
// if they are not met, the producer publishes the current item before it
// waits for them (and claims nothing further meanwhile).  Every awaited item
// is of an earlier pass, hence claimed earlier, and the earliest unfinished
// item always progresses: the queue cannot deadlock, whatever the residency.
// Once any wait of the launch has run out (status word set), every producer
// stops claiming and every dependency wait gives up at once, so a failure
// ends the launch promptly instead of draining the queue one expired wait at
// a time.
//
// The queue tables (job records, (job, pass) entries, tile prefix sums) are
// one contiguous block `tables` of `tables_bytes` bytes whose parts start at
// the given offsets; with `tables_in_smem` the CTA copies the block into
// shared memory first.
__global__ void __launch_bounds__(kQueueThreads, 3) batch_kernel(const unsigned char* __restrict__ tables,
                                                             int tables_bytes, int tables_in_smem, int o_ent,
                                                             int o_prefix, int n_ent,
                                                             const CUtensorMap* __restrict__ maps,
                                                             int* __restrict__ counter, int* __restrict__ status,
                                                             long long wait_cycles, long long drop_item,
                                                             int claim_ahead) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t base_u32 = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024 - (base_u32 & 1023)) & 1023);
  float* stage = reinterpret_cast<float*>(smem);
  float* level = reinterpret_cast<float*>(smem + kLevelOff);  // level 1 of two-step items
  // full: the item's box (or slot) is ready; boxfree: the consumers have
  // read the box; done[k & 1]: the consumers have stored item k.  `done`
  // alternates between two barriers because the consumers may finish item
  // k + 1 before the producer, busy claiming, has waited for item k: with
  // one barrier that wait would then see the wrong phase.  (`full` and
  // `boxfree` cannot run ahead: each completes only after the producer's
  // previous wait on it.)
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kBarOff);
  uint64_t* boxfree = full + 1;
  uint64_t* done = full + 2;  // two barriers
  ItemSlot* slot = reinterpret_cast<ItemSlot*>(full + 4);
  Stage sg;
  sg.box = stage;
  sg.ops_a = reinterpret_cast<uint4*>(smem + kOpsOff);
  sg.ops_e = reinterpret_cast<uint32_t*>(smem + kOpsOff + kOpsABytes);
  sg.job = reinterpret_cast<BatchJob*>(smem + kJobOff);
  sg.slot = slot;
  sg.full = full;
  const BatchJob* jobs_g = reinterpret_cast<const BatchJob*>(tables);  // the global copy (bulk-copy source)
  unsigned char* tsm = smem + kTablesOff;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tables_in_smem) {
    const uint4* src = reinterpret_cast<const uint4*>(tables);
    uint4* dstv = reinterpret_cast<uint4*>(tsm);
    for (int i = tid; i < tables_bytes / 16; i += blockDim.x) dstv[i] = src[i];
  }
  const unsigned char* tb = tables_in_smem ? tsm : tables;
  const BatchJob* __restrict__ jobs = reinterpret_cast<const BatchJob*>(tb);
  const int2* __restrict__ ent = reinterpret_cast<const int2*>(tb + o_ent);  // (job, pass)
  const long long* __restrict__ ent_prefix = reinterpret_cast<const long long*>(tb + o_prefix);
  if (tid == 0) {
    mbar_init(full, 1);
    mbar_init(boxfree, 1);
    mbar_init(&done[0], 1);
    mbar_init(&done[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const long long total = ent_prefix[n_ent];

  if (warp == kConsumerWarps) {
    // ---------------- producer warp ----------------
    // the first item: nothing is held yet, so its dependencies may be awaited
    int prev_job = -1;  // the job whose record and operands the consumers have (lane 0)
    Claim cur = claim_item(counter, total, ent_prefix, ent, n_ent, jobs, drop_item, lane);
    if (!cur.end && !cur.skip) (void)deps_ready(jobs[cur.job], cur, true, lane, status, wait_cycles);
    bool last_tma = hand_over(cur, jobs, jobs_g, maps, sg, &prev_job, lane);
    long long handed = 1;  // phases of `full` handed over
    bool ok = true;
    // The item after `cur` is claimed, decoded and its dependencies tested
    // while the consumers compute `cur` (pass counters only grow: a test
    // passed early still holds when the box is loaded).  With `claim_ahead`
    // (queues whose layers are much wider than the grid) the claim of the
    // item after that follows as soon as `nxt` is handed over, i.e. during
    // the last level of `cur`: the producer's claim, decode and test then
    // never delay a load.  On narrow queues, whose items wait for their
    // neighbours, claiming that early only reserves items a CTA cannot start
    // yet, so there the claim waits for the next item.  After a failed wait
    // anywhere in the launch (status word set) the producer claims nothing
    // more: the CTA's queue ends after the items it holds.
    auto claim_tested = [&](Claim& c) -> bool {
      if (failed(status)) {
        c = Claim{};
        c.end = 1;
        return true;
      }
      c = claim_item(counter, total, ent_prefix, ent, n_ent, jobs, drop_item, lane);
      return c.end || c.skip || deps_ready(jobs[c.job], c, false, lane, status, wait_cycles);
    };
    Claim nxt = {};
    bool have_nxt = false, ready = false;
    for (long long k = 0; !cur.end; ++k) {
      const uint32_t par = (uint32_t)(k & 1);
      if (!have_nxt) ready = claim_tested(nxt);
      if (lane == 0) ok = mbar_wait_backoff(boxfree, par, status, 32, wait_cycles);
      if (!__shfl_sync(0xffffffffu, (int)ok, 0)) break;
      // item k's box is read: load the next one now if it may start
      if (!ready) ready = deps_ready(jobs[nxt.job], nxt, false, lane, status, wait_cycles);
      Claim after = {};
      bool have_after = false, ready_after = false;
      if (ready) {
        last_tma = hand_over(nxt, jobs, jobs_g, maps, sg, &prev_job, lane);
        ++handed;
        if (claim_ahead && !nxt.end) {
          ready_after = claim_tested(after);
          have_after = true;
        }
      }
      // item k's outputs are stored: publish its tile's pass counter
      if (lane == 0) ok = mbar_wait_backoff(&done[k & 1], (uint32_t)((k >> 1) & 1), status, 32, wait_cycles);
      if (!__shfl_sync(0xffffffffu, (int)ok, 0)) break;
      if (lane == 0 && !cur.skip) st_release(jobs[cur.job].done + cur.tile, cur.s + 1);
      if (!ready) {
        // this CTA holds no unpublished item now: wait for the dependencies
        (void)deps_ready(jobs[nxt.job], nxt, true, lane, status, wait_cycles);
        last_tma = hand_over(nxt, jobs, jobs_g, maps, sg, &prev_job, lane);
        ++handed;
      }
      cur = nxt;
      nxt = after;
      have_nxt = have_after;
      ready = ready_after;
    }
    if (!ok && last_tma && lane == 0) {
      // giving up: the last load may still land in this CTA's shared
      // memory; wait for it once more (bounded) before the CTA exits
      (void)mbar_wait_bounded(full, (uint32_t)((handed - 1) & 1), status, wait_cycles);
    }
    return;
  }

  // ---------------- consumer warps ----------------
  // The packed operands of the current job stay in registers while its
  // tiles follow one another.
  uint4 A8[kNA];
  uint32_t E8[kNA];
  int cur_job = -1;
  for (uint32_t k = 0;; ++k) {
    const bool landed = mbar_wait_backoff(full, k & 1, status, 32, wait_cycles);
    if (!consumers_all(landed)) break;
    const ItemSlot it = *slot;
    if (it.end) break;
    if (it.skip) {
      asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");  // every consumer has read the slot
      if (tid == 0) {
        mbar_arrive(boxfree);
        mbar_arrive(&done[k & 1]);
      }
      continue;
    }
    // the job's record and operands are in shared memory (the producer
    // copied them there with the box whenever the job changed); the record
    // is read here, before the item's first barrier, after which the next
    // item's copy may overwrite it
    const BatchJob& jb = *sg.job;
    if (it.job != cur_job) {
      const int na = 2 * jb.r + 2;
#pragma unroll
      for (int a = 0; a < kNA; ++a)
        if (a < na) {
          A8[a] = sg.ops_a[a * 32 + lane];
          E8[a] = sg.ops_e[a * 32 + lane];
        }
      cur_job = it.job;
    }
    const int tx = it.tile % jb.tiles_x, ty = it.tile / jb.tiles_x;
    const int np = pass_steps(jb, it.s);
    if (it.s == 0 && !jb.tma0) {
      // a first pass of one step on a grid TMA cannot describe
      load_box_async(jb.in, jb.nx, jb.ny, 1, (int64_t)tx * jb.bx - kHaloX, (int64_t)ty * jb.by - jb.r, 0,
                     jb.bx + 2 * kHaloX, jb.by + 2 * jb.r, 1, stage, warp, kConsumerWarps, lane);
      asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
    }
    const bool last = it.s + 1 == jb.passes;
    float* dst = last ? jb.out : jb.bufs[(jb.first + it.s) % 2];
    const int64_t pitch = last ? jb.nx : jb.pitch;
    const bool out_tf32 = !last;
    const int x0 = tx * jb.bx, y0 = ty * jb.by;
    uint64_t* stored = &done[k & 1];
#define SPIDER_BATCH_FUSED(R)                                                                               \
  if (np == 2) {                                                                                            \
    if (it.s == 0)                                                                                          \
      batch_fused<R, 2, true>(jb, A8, E8, stage, level, dst, pitch, x0, y0, out_tf32, status, boxfree, stored);  \
    else                                                                                                    \
      batch_fused<R, 2, false>(jb, A8, E8, stage, level, dst, pitch, x0, y0, out_tf32, status, boxfree, stored); \
  } else {                                                                                                  \
    if (it.s == 0)                                                                                          \
      batch_fused<R, 1, true>(jb, A8, E8, stage, level, dst, pitch, x0, y0, out_tf32, status, boxfree, stored);  \
    else                                                                                                    \
      batch_fused<R, 1, false>(jb, A8, E8, stage, level, dst, pitch, x0, y0, out_tf32, status, boxfree, stored); \
  }
    switch (jb.r) {
      case 1: SPIDER_BATCH_FUSED(1) break;
      case 2: SPIDER_BATCH_FUSED(2) break;
      default: SPIDER_BATCH_FUSED(3) break;
    }
#undef SPIDER_BATCH_FUSED
  }
}

}  // namespace
}  // namespace spider

using namespace spider;

extern "C" spider_status spider_set_wait_limit(long long cycles) {
  set_error("");
  if (cycles < 1000) return fail(SPIDER_ERR_INVALID, "wait limit must be >= 1000 cycles");
  set_wait_limit_cycles(cycles);
  return SPIDER_OK;
}

extern "C" spider_status spider_batch_configure(long long fuse_min_points, int queue_steps_per_item) {
  set_error("");
  if (fuse_min_points < 0 || queue_steps_per_item < 0 || queue_steps_per_item > 2)
    return fail(SPIDER_ERR_INVALID, "fuse_min_points >= 0, queue_steps_per_item 0..2");
  g_fuse_min_points.store(fuse_min_points > 0 ? fuse_min_points : kFuseMinPoints);
  g_queue_steps.store(queue_steps_per_item > 0 ? queue_steps_per_item : kQueueStepsPerItem);
  return SPIDER_OK;
}

extern "C" spider_status spider_batch_drop_item(long long item) {
  set_error("");
  if (item < -1) return fail(SPIDER_ERR_INVALID, "item must be >= -1");
  g_drop_item.store(item);
  return SPIDER_OK;
}

extern "C" spider_status spider_batch(int n, const spider_plan* plans, const float* const* ins, float* const* outs,
                                      const int64_t* steps, cudaStream_t stream) {
  set_error("");
  const long long drop_item = g_drop_item.exchange(-1);  // the hook applies to this call only
  if (n < 0 || n > 4096) return fail(SPIDER_ERR_INVALID, "n must be in [0, 4096]");
  if (n == 0) return SPIDER_OK;
  if (!plans || !ins || !outs || !steps) return fail(SPIDER_ERR_INVALID, "NULL array");
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !ins[i] || !outs[i] || steps[i] < 0) return fail(SPIDER_ERR_INVALID, "bad job");
    const size_t bytes = (size_t)plans[i]->points() * 4;
    const char* a = reinterpret_cast<const char*>(ins[i]);
    const char* b = reinterpret_cast<const char*>(outs[i]);
    if (a < b + bytes && b < a + bytes) return fail(SPIDER_ERR_INVALID, "grid_out overlaps grid_in");
    for (int k = 0; k < i; ++k)
      if (plans[k] == plans[i]) return fail(SPIDER_ERR_INVALID, "a plan may appear once per batch (its scratch grid)");
  }
  int batch_dev = 0;
  if (cudaGetDevice(&batch_dev) != cudaSuccess) return fail(SPIDER_ERR_CUDA, "cudaGetDevice");
  std::lock_guard<std::mutex> whole_call(batch_lock(batch_dev));
  const long long fuse_min_points = g_fuse_min_points.load();
  const bool two_step_items = g_queue_steps.load() == 2;
  // Jobs the persistent queue handles: 2-D sparse TF32, radius <= 3, at
  // least one step, and fewer than kFuseMinPoints points.  Larger grids of
  // several steps run as fused multi-step passes of their own (the plan's
  // tuned depth and tile, else those of its kind, else 2 steps per pass on
  // tile variant 2), on side streams beside the queue: the queue takes one
  // step per HBM pass.  The rest run through their own plan after the
  // persistent launch.
  std::vector<int> queued, fused, direct;
  for (int i = 0; i < n; ++i) {
    spider_plan_t* p = plans[i];
    const bool ok = p->ndim == 2 && p->r <= kMaxR && p->engine == SPIDER_ENGINE_SPARSE_TC && p->prec == SPIDER_TF32 &&
                    steps[i] > 0;
    const bool big = ok && steps[i] > 1 && p->points() >= fuse_min_points;
    (big ? fused : ok ? queued : direct).push_back(i);
  }
  // The fused grids run on side streams (after the work already on
  // `stream`), concurrently with each other and with the queue: a pass over
  // one of these grids lasts microseconds, so one after another they would
  // be bound by launch latency.  Repeated calls with the
  // same grids replay each job's passes as a CUDA graph.
  SideJoin side;
  side.stream = stream;
  if (!fused.empty()) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaEvent_t start;
    if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess)
      return fail(SPIDER_ERR_CUDA, "batch event");
    cudaEventRecord(start, stream);
    for (int k = 0; k < kSideStreams; ++k) {
      side.sides[k] = side_stream(dev, k);
      if (side.sides[k]) cudaStreamWaitEvent(side.sides[k], start, 0);
    }
    cudaEventDestroy(start);
    side.used = true;
    for (size_t f = 0; f < fused.size(); ++f) {
      const int i = fused[f];
      cudaStream_t s_run = side.sides[f % kSideStreams] ? side.sides[f % kSideStreams] : stream;
      spider_plan_t* p = plans[i];
      std::lock_guard<std::mutex> lock(p->mu);
      const int old_T = p->steps_per_pass, old_v = p->tile_variant;
      int T = old_T, v = old_v;
      if (T < 2 && !autotune_lookup(p, &T, &v)) {
        T = 2;
        v = 2;  // measured best untuned choice on the mixed batch (v 0: 805, v 2: 847, v 4: 777 GStencil/s)
      }
      p->steps_per_pass = T;
      p->tile_variant = v;
      spider_status s = run_cached(p, ins[i], outs[i], steps[i], s_run);
      p->steps_per_pass = old_T;
      p->tile_variant = old_v;
      if (s != SPIDER_OK) return s;
    }
  }
  if (!queued.empty() && (batch_dev < 0 || batch_dev >= 64))
    return fail(SPIDER_ERR_UNSUPPORTED, "device index out of range");
  // what the queue's device image is built from: replaying the previous
  // launch is correct exactly when all of it is unchanged
  auto make_key = [&](std::vector<uint64_t>& key) -> spider_status {
    key = {(uint64_t)two_step_items, (uint64_t)wait_limit_cycles(), (uint64_t)queued.size()};
    for (int i : queued) {
      spider_plan_t* p = plans[i];
      std::lock_guard<std::mutex> lock(p->mu);
      spider_status st = ensure_plan_device(p, steps[i] > 1);
      if (st != SPIDER_OK) return st;
      const uint64_t part[] = {(uint64_t)(uintptr_t)p, (uint64_t)p->nx, (uint64_t)p->ny, (uint64_t)p->r,
                               (uint64_t)steps[i], (uint64_t)(uintptr_t)ins[i], (uint64_t)(uintptr_t)outs[i],
                               (uint64_t)(uintptr_t)p->dev.a_words, (uint64_t)(uintptr_t)p->dev.meta_words,
                               (uint64_t)(uintptr_t)p->dev.scratch, (uint64_t)(uintptr_t)p->dev.pad};
      key.insert(key.end(), std::begin(part), std::end(part));
    }
    return SPIDER_OK;
  };
  std::vector<uint64_t> key;
  if (!queued.empty()) {
    spider_status st = make_key(key);
    if (st != SPIDER_OK) return st;
  }
  QueueReplay* replay = queued.empty() ? nullptr : &g_replay[batch_dev];
  if (replay && drop_item < 0 && replay->exec && replay->key == key) {
    cudaError_t e = cudaGraphLaunch(replay->exec, stream);
    side.join();
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, replay->status, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(SPIDER_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    if (status != 0) return fail(SPIDER_ERR_TIMEOUT, "a dependency wait in the batch queue ran out");
  } else if (!queued.empty()) {
    // the buffer is about to be rewritten: the kept graph no longer matches it
    if (replay->exec) cudaGraphExecDestroy(replay->exec);
    replay->exec = nullptr;
    replay->key.clear();
    const int nq = (int)queued.size();
    std::vector<BatchJob> jobs(nq);
    std::vector<CUtensorMap> maps(6 * (size_t)nq);
    std::vector<long long> tiles(nq);
    long long total_tiles = 0;
    int max_steps = 0;  // the longest job's passes: queue items are (pass, job, tile)
    for (int k = 0; k < nq; ++k) {
      const int i = queued[k];
      spider_plan_t* p = plans[i];
      std::lock_guard<std::mutex> lock(p->mu);
      spider_status st = ensure_plan_device(p, steps[i] > 1);
      if (st != SPIDER_OK) return st;
      BatchJob& jb = jobs[k];
      jb.nx = p->nx;
      jb.ny = p->ny;
      jb.r = p->r;
      jb.steps = (int)steps[i];
      // two steps per pass on the fused tile for jobs of several steps
      jb.two = (steps[i] > 1 && two_step_items) ? 1 : 0;
      jb.by = kTileL1 - 2 * p->r;  // the queue tile, for one- and two-step passes
      jb.bx = 120;
      jb.tiles_x = (int)((p->nx + jb.bx - 1) / jb.bx);
      jb.tiles_y = (int)((p->ny + jb.by - 1) / jb.by);
      jb.map0 = 6 * k;
      jb.a = reinterpret_cast<const uint4*>(p->dev.a_words);
      jb.meta = p->dev.meta_words;
      jb.out = outs[i];
      jb.in = ins[i];
      jb.done = nullptr;
      // boxes: a pass of T steps reads (by + 2r T) x (bx + 8 T): a two-step
      // pass (56 + 2r) x 136 (maps 0..2), a one-step pass 56 x 128 (maps 3..5)
      const int box_x = 120 + 4 * kHaloX, box_y = kTileL1 + 2 * p->r;
      const int box1_x = 128, box1_y = kTileL1;
      CUtensorMap* mp = &maps[6 * k];
      std::memset(mp, 0, 6 * sizeof(CUtensorMap));
      jb.tma0 = make_tensor_map(&mp[0], ins[i], p->nx, p->ny, 1, box_x, box_y, 1) ? 1 : 0;
      if (jb.tma0) make_tensor_map(&mp[3], ins[i], p->nx, p->ny, 1, box1_x, box1_y, 1);
      if (jb.two) {
        jb.head1 = (jb.steps % 2 == 1 || !jb.tma0) ? 1 : 0;
        jb.tail1 = ((jb.steps - jb.head1) % 2 == 1) ? 1 : 0;
        jb.passes = jb.head1 + (jb.steps - jb.head1 - jb.tail1) / 2 + jb.tail1;
      } else {
        jb.head1 = jb.tail1 = 0;
        jb.passes = jb.steps;
      }
      const bool direct = jb.tma0 && make_tensor_map(&mp[1], outs[i], p->nx, p->ny, 1, box_x, box_y, 1) &&
                          (jb.passes == 1 ||
                           make_tensor_map(&mp[2], p->dev.scratch, p->nx, p->ny, 1, box_x, box_y, 1));
      if (direct) {
        jb.pitch = p->nx;
        jb.first = (jb.passes % 2 == 1) ? 0 : 1;
        jb.bufs[0] = outs[i];
        jb.bufs[1] = p->dev.scratch;
        if (jb.passes == 1) mp[2] = mp[0];
        make_tensor_map(&mp[4], outs[i], p->nx, p->ny, 1, box1_x, box1_y, 1);
        if (jb.passes > 1) make_tensor_map(&mp[5], p->dev.scratch, p->nx, p->ny, 1, box1_x, box1_y, 1);
      } else {
        jb.pitch = (p->nx + 3) / 4 * 4;
        jb.first = 0;
        jb.bufs[0] = jb.bufs[1] = nullptr;
        if (jb.passes > 1) {
          const size_t grid_bytes = (size_t)jb.pitch * (size_t)p->ny * 4;
          st = ensure_plan_pad(p, 2 * grid_bytes);
          if (st != SPIDER_OK) return st;
          jb.bufs[0] = p->dev.pad;
          jb.bufs[1] = p->dev.pad + grid_bytes / 4;
          for (int m = 0; m < 2; ++m) {
            if (!make_tensor_map_pitched(&mp[1 + m], jb.bufs[m], p->nx, p->ny, 1, jb.pitch, box_x, box_y, 1) ||
                !make_tensor_map_pitched(&mp[4 + m], jb.bufs[m], p->nx, p->ny, 1, jb.pitch, box1_x, box1_y, 1))
              return fail(SPIDER_ERR_CUDA, "tensor map of a padded grid");
          }
        }
        if (!jb.tma0) mp[0] = jb.passes > 1 ? mp[1] : mp[0];  // unused: the consumers load pass 0
      }
      tiles[k] = (long long)jb.tiles_x * jb.tiles_y;
      total_tiles += tiles[k];
      max_steps = std::max(max_steps, jb.passes);
    }
    // Queue order: entries (job, pass), each covering the job's tiles, in
    // pass-major order (pass 0 of every job, then pass 1, ...), jobs of more
    // passes first within a pass, so an item only waits for items earlier in
    // the queue.  (Measured alternatives with every grid of the 64-grid mix
    // in the queue: an order that advances every job in proportion to its
    // pass count -- pass p of P in layer p M / P -- 3 % faster there but 3-9 %
    // slower on 256 small grids; a window of jobs whose grids fit a byte
    // budget, so that a job's passes follow one another while its grids sit
    // in L2, no faster at 96 MB and 13 % slower at 48 MB.)
    std::vector<int> order(nq);
    for (int k = 0; k < nq; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return jobs[a].passes > jobs[b].passes; });
    std::vector<int> ent;  // job, pass, job, pass, ...
    std::vector<long long> ent_prefix(1, 0);
    long long widest_layer = 1;
    const long long layer_count = max_steps;
    for (int L = 0; L < max_steps; ++L) {
      long long layer_items = 0;
      for (int k = 0; k < nq && jobs[order[k]].passes > L; ++k) {
        const int j = order[k];
        ent.push_back(j);
        ent.push_back(L);
        ent_prefix.push_back(ent_prefix.back() + tiles[j]);
        layer_items += tiles[j];
      }
      widest_layer = std::max(widest_layer, layer_items);
    }
    const int n_ent = (int)(ent.size() / 2);
    // one device block: [tables: jobs | entries | entry prefix] | maps | done | counter | status
    auto align = [](size_t x) { return (x + 127) / 128 * 128; };
    const size_t o_jobs = 0;
    const size_t o_ent = align(o_jobs + sizeof(BatchJob) * nq);
    const size_t o_prefix = align(o_ent + sizeof(int) * ent.size());
    const size_t tables_bytes = align(o_prefix + sizeof(long long) * (n_ent + 1));
    const size_t o_maps = tables_bytes;
    const size_t o_done = align(o_maps + sizeof(CUtensorMap) * maps.size());
    const size_t o_ctr = align(o_done + sizeof(int) * total_tiles);
    const size_t o_status = o_ctr + 16;
    const size_t bytes = align(o_status + 16);
    const int tables_in_smem = tables_bytes <= (size_t)kMaxTableSmem ? 1 : 0;
    const int smem_bytes = kSmemBase + (tables_in_smem ? (int)tables_bytes : 0);
    // the queue buffer is kept between calls (per device) and grown on demand
    static std::mutex qmu;
    static unsigned char* qbuf[64] = {nullptr};
    static size_t qcap[64] = {0};
    std::lock_guard<std::mutex> qlock(qmu);
    int devid = 0;
    cudaGetDevice(&devid);
    if (devid < 0 || devid >= 64) return fail(SPIDER_ERR_UNSUPPORTED, "device index out of range");
    cudaError_t e = cudaSuccess;
    if (qcap[devid] < bytes) {
      e = cudaStreamSynchronize(stream);  // the old buffer may still be in use on this stream
      if (e == cudaSuccess && qbuf[devid]) cudaFree(qbuf[devid]);
      qbuf[devid] = nullptr;
      qcap[devid] = 0;
      if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&qbuf[devid]), bytes * 2);
      if (e != cudaSuccess) { cudaGetLastError(); return fail(SPIDER_ERR_OOM, "batch work queue"); }
      qcap[devid] = bytes * 2;
    }
    unsigned char* dev = qbuf[devid];
    long long done_off = 0;
    for (int k = 0; k < nq; ++k) {
      jobs[k].done = reinterpret_cast<int*>(dev + o_done) + done_off;
      done_off += tiles[k];
    }
    std::vector<unsigned char> host(bytes, 0);  // zero counters and status
    std::memcpy(host.data() + o_jobs, jobs.data(), sizeof(BatchJob) * nq);
    std::memcpy(host.data() + o_maps, maps.data(), sizeof(CUtensorMap) * maps.size());
    std::memcpy(host.data() + o_ent, ent.data(), sizeof(int) * ent.size());
    std::memcpy(host.data() + o_prefix, ent_prefix.data(), sizeof(long long) * (n_ent + 1));
    e = cudaMemcpyAsync(dev, host.data(), bytes, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // host image is freed on return
    if (e != cudaSuccess) return fail(SPIDER_ERR_CUDA, "batch work queue upload");
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
      attr_err = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kSmemBase + kMaxTableSmem);
      if (attr_err == cudaSuccess)  // the stage and the level buffer, not L1, take the shared memory
        attr_err = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    });
    if (attr_err != cudaSuccess) return fail(SPIDER_ERR_CUDA, "batch kernel attributes");
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel, kQueueThreads, smem_bytes);
    // No more CTAs than the largest layer has items: further CTAs would
    // mostly wait for earlier passes, holding SMs (and their shared memory)
    // that the fused passes on the side streams can use.
    const long long total_items = ent_prefix[n_ent];
    const int grid = (int)std::max<long long>(
        1, std::min({total_items, widest_layer, (long long)std::max(occ, 1) * device_sm_count()}));
    // The persistent launch is issued as a CUDA graph: the work-queue reset
    // (counter and per-tile pass counters) and the kernel, launched on the
    // caller's stream.
    const unsigned char* a_tables = dev;
    int a_tbytes = (int)tables_bytes, a_tsm = tables_in_smem, a_oe = (int)o_ent, a_op = (int)o_prefix,
        a_ne = n_ent;
    const CUtensorMap* a_maps = reinterpret_cast<const CUtensorMap*>(dev + o_maps);
    int* a_ctr = reinterpret_cast<int*>(dev + o_ctr);
    int* a_status = reinterpret_cast<int*>(dev + o_status);
    long long a_wait = wait_limit_cycles();
    long long a_drop = drop_item;
    // claim one item further ahead when the layers are much wider than the
    // grid (measured: 64-grid mix entirely in the queue 867 -> 957
    // GStencil/s, one 8192^2 radius-1 grid 1098 -> 1233; on 256 small grids,
    // whose layers are about as wide as the grid, 282 -> 234)
    const long long layers = std::max<long long>(1, layer_count);
    int a_ahead = total_items >= 8LL * grid * layers ? 1 : 0;
    void* kargs[] = {(void*)&a_tables, (void*)&a_tbytes, (void*)&a_tsm, (void*)&a_oe, (void*)&a_op, (void*)&a_ne,
                     (void*)&a_maps, (void*)&a_ctr, (void*)&a_status,
                     (void*)&a_wait, (void*)&a_drop, (void*)&a_ahead};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphCreate(&graph, 0);
    cudaGraphNode_t reset = nullptr, kern = nullptr;
    if (e == cudaSuccess) {
      cudaMemsetParams mp = {};
      mp.dst = dev + o_done;
      mp.value = 0;
      mp.elementSize = 1;
      mp.width = bytes - o_done;
      mp.height = 1;
      mp.pitch = 0;
      e = cudaGraphAddMemsetNode(&reset, graph, nullptr, 0, &mp);
    }
    if (e == cudaSuccess) {
      cudaKernelNodeParams kp = {};
      kp.func = reinterpret_cast<void*>(batch_kernel);
      kp.gridDim = dim3(grid);
      kp.blockDim = dim3(kQueueThreads);
      kp.sharedMemBytes = smem_bytes;
      kp.kernelParams = kargs;
      e = cudaGraphAddKernelNode(&kern, graph, &reset, 1, &kp);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, stream);
    side.join();  // the fused grids ran beside the queue; the wait below covers them
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, a_status, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (graph) cudaGraphDestroy(graph);
    if (e == cudaSuccess && status == 0 && drop_item < 0 && make_key(replay->key) == SPIDER_OK) {
      // the key as the image was built (padded grids allocated on the way)
      replay->exec = exec;
      replay->status = a_status;
    } else if (exec) {
      cudaGraphExecDestroy(exec);
    }
    if (e != cudaSuccess) return fail(SPIDER_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    if (status != 0) return fail(SPIDER_ERR_TIMEOUT, "a dependency wait in the batch queue ran out");
  }
  side.join();
  for (int i : direct) {
    std::lock_guard<std::mutex> lock(plans[i]->mu);
    spider_status s = run_device(plans[i], ins[i], outs[i], steps[i], stream);
    if (s != SPIDER_OK) return s;
  }
  const cudaError_t e = cudaStreamSynchronize(stream);  // synchronous: every grid is done
  if (e != cudaSuccess) return fail(SPIDER_ERR_CUDA, std::string("batch: ") + cudaGetErrorString(e));
  return SPIDER_OK;
}
