/*
 * spider.h -- C ABI of the GB300 (sm_103a) SPIDER stencil library.
 *
 * SPIDER (Sparse Tensor Cores for stencils via strided swapping) computes the
 * stencil sweep
 *
 *     u_{t+1}[i] = sum_{o in S} w[o] * u_t[i + o]            (Sec. 1, Sec. 2.2)
 *
 * by lowering every kernel row to a banded matrix product Y = K X
 * (Sec. 3.1.1), permuting K's columns ahead of time so that it has the 2:4
 * (and 1:2) structured-sparse form Sparse Tensor Cores accept (Sec. 3.1.2),
 * and applying the matching row permutation to the input while it is moved
 * from shared memory to registers (Sec. 3.2).  The result is the same
 * stencil; only rounding differs.
 *
 * Conventions for every entry point:
 *  - Grids are float32, C-contiguous, x (last extent) fastest.  Outside the
 *    grid the field is 0 at every step (zero Dirichlet halo); every point of
 *    the grid is updated.
 *  - Device pointers are CUDA device (or managed) memory of the current
 *    device; the library never frees memory it does not own.  A plan owns its
 *    packed operands and one scratch grid (allocated on first use).
 *  - Calls that take a stream are asynchronous on that stream.  A status of
 *    SPIDER_OK means the work was enqueued; faults detected by the device
 *    (e.g. a wait that ran out) are reported by the next call on that plan
 *    or by spider_plan_sync.
 *  - No C++ exception crosses this boundary.  On error the call returns a
 *    status other than SPIDER_OK, touches neither the device nor the outputs,
 *    and spider_last_error() returns a message (thread-local).
 */
#ifndef SPIDER_H_
#define SPIDER_H_

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spider_plan_t* spider_plan;
typedef struct spider_server_t* spider_server;

typedef enum {
  SPIDER_OK = 0,
  SPIDER_ERR_INVALID = 1,      /* bad argument; nothing was done              */
  SPIDER_ERR_UNSUPPORTED = 2,  /* valid stencil outside what is built         */
  SPIDER_ERR_OOM = 3,          /* device allocation or admission budget       */
  SPIDER_ERR_CUDA = 4,         /* a CUDA runtime/driver call failed           */
  SPIDER_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out          */
  SPIDER_ERR_BUSY = 6          /* server queue full; retry later              */
} spider_status;

typedef enum { SPIDER_STAR = 0, SPIDER_BOX = 1 } spider_shape;

/* Arithmetic of the tensor-core products (accumulation is always FP32).
 *  TF32   : one sparse TF32 product per kernel row (grid and weights rounded
 *           to nearest TF32; the weights so that their sum stays as close to
 *           the FP32 sum as TF32 allows).
 *  F16X2  : grid and weights split into FP16 hi + lo parts (lo parts scaled by
 *           2^11, about 22 bits); hi*hi + hi*lo + lo*hi, each hi*hi MMA into a
 *           fresh accumulator added in FP32.  Requires |grid values| < 32768.
 *  BF16X3 : grid and weights split into three BF16 terms hi + mid + lo (24
 *           bits, FP32 range); the six products above 2^-24 relative (hi*hi,
 *           hi*mid, mid*hi, hi*lo, lo*hi, mid*mid), in two passes.
 *  The last term of every split weight is rounded so the split weights sum
 *  as close as possible to the FP32 weights.  spider_plan_error_bound gives
 *  the error each arithmetic is expected to stay within.
 *  AUTO   : TF32. */
typedef enum { SPIDER_TF32 = 0, SPIDER_F16X2 = 1, SPIDER_BF16X3 = 2, SPIDER_AUTO = 3 } spider_precision;

/* Which kernel a plan runs.  SPARSE_TC is SPIDER; the others are the
 * comparators built on the same tiling: DENSE_TC multiplies the same banded
 * K without the 2:4 compression on dense tensor cores (the paper's "SPIDER w.
 * TC" ablation, Sec. 4.4), CUDA_CORE is a direct FP32 FMA stencil, and
 * SPARSE_TC_COPY is SPIDER with the input row swap done the way Sec. 3.2
 * sets its own design against: an explicit copy of every input window, in
 * the swapped order, into a shared-memory buffer of its own, which the MMA
 * operands then load contiguously (2-D, TF32, radius 1..3, one step per
 * pass; the same products as SPARSE_TC, bit for bit).  SPARSE_TC_NO_CO is
 * SPIDER without the computing optimisations of Sec. 3.3 (the "SpTC" step
 * of the Sec. 4.4 ablation): the packed kernel matrix and metadata are
 * staged in shared memory and every MMA loads its A operand and metadata
 * from there, instead of keeping them in registers for the whole kernel
 * (2-D, TF32, radius 1..3, one step per pass; bit for bit SPARSE_TC's). */
typedef enum {
  SPIDER_ENGINE_SPARSE_TC = 0,
  SPIDER_ENGINE_DENSE_TC = 1,
  SPIDER_ENGINE_CUDA_CORE = 2,
  SPIDER_ENGINE_SPARSE_TC_COPY = 3,
  SPIDER_ENGINE_SPARSE_TC_NO_CO = 4
} spider_engine;

/* spider_plan_create -- the paper's offline transform (Sec. 3.1, Sec. 3.3.2).
 *
 * Builds, for every kernel row of the stencil (Sec. 3.1.1), the banded matrix
 * K (L = 8 outputs, a 16-wide input window), applies the strided column swap
 * that gives the 2:4 / 1:2 pattern (Sec. 3.1.2), compresses it to values plus
 * 2-bit metadata, and packs values and metadata per thread in fragment order
 * (Sec. 3.3.2).  Host work only: no device is touched until the first run.
 *
 *  ndim      1, 2 or 3.
 *  extents   ndim sizes, slowest axis first, x last; each >= 1; the product
 *            must be < 2^40.
 *  shape     SPIDER_STAR: only on-axis coefficients may be non-zero;
 *            SPIDER_BOX: any.
 *  radius    1..3; 4..7 for 1-D and 2-D stencils in TF32 with the sparse
 *            engine (windows of 16 outputs, the paper's L = 2r + 2 <= 16
 *            layout, Sec. 3.1), one time step per pass.
 *  coeffs    dense (2r+1)^ndim float32 cube, row-major [dz][dy][dx], each
 *            offset running -r..r; host memory, copied; finite values only.
 *  prec      see spider_precision.
 *  out       receives the plan (owned by the caller; free with
 *            spider_plan_destroy).
 * Errors: SPIDER_ERR_INVALID (bad ndim/extents/radius/NULL, non-finite
 * coefficients, non-zero off-axis coefficient for a star),
 * SPIDER_ERR_UNSUPPORTED (radius > 7, or radius 4..7 for 3-D or a split
 * precision). */
spider_status spider_plan_create(int ndim, const int64_t* extents, spider_shape shape, int radius,
                                 const float* coeffs, spider_precision prec, spider_plan* out);

/* Selects the kernel the plan runs (default SPIDER_ENGINE_SPARSE_TC).  The
 * comparators support SPIDER_TF32 (DENSE_TC, SPARSE_TC_COPY, SPARSE_TC_NO_CO)
 * and plain FP32 (CUDA_CORE, precision ignored), radius 1..3;
 * SPARSE_TC_COPY and SPARSE_TC_NO_CO 2-D grids only (SPIDER_ERR_UNSUPPORTED
 * otherwise). */
spider_status spider_plan_set_engine(spider_plan plan, spider_engine engine);

/* Time steps fused per pass over HBM (1 = one launch per step).  Built: 1..4
 * for 2-D stencils of radius 1..3 (1..10 for radius 1 with the sparse
 * engine in TF32: 5..10 run on small tiles, for grids too small to fill the
 * GPU), and with the sparse engine in TF32 1..4 for 3-D radius-1 and 1-D
 * plans; 1 otherwise.  Values the build does not support for the plan's
 * stencil return SPIDER_ERR_UNSUPPORTED.  A run whose input grid TMA cannot
 * read takes its first step on its own. */
spider_status spider_plan_set_steps_per_pass(spider_plan plan, int steps_per_pass);

/* Tile shape of the fused kernels.  2-D: 0 = warp units of 8 output rows and
 * two input boxes in flight; 1 = 16 rows (more independent MMAs per warp), two
 * boxes; 2 = 8 rows, one box, registers capped so three CTAs share an SM;
 * 3 = 16 rows, one box; 4 = small tiles (level 1 of 32 rows instead of 64,
 * one warp unit per warp per level) for grids that do not fill the GPU;
 * 5 = as 2 with the last level written by 16-byte stores (sparse TF32; as 2
 * elsewhere).
 * FP16/BF16 splits and the dense engine: 2 and 3 = 8 rows with registers
 * capped so two CTAs share an SM, two or one input boxes; CUDA-core engine:
 * 2 and 3 run as 0 and 1.
 * 3-D: 0 and 4 = column blocks of 16 level-1 rows, warp units of 4 rows; 1
 * and 3 = 32 rows, units of 8; 2 = as 0 with registers capped for three CTAs
 * per SM at 2 steps per pass; 5 = as 2.  Any other value returns
 * SPIDER_ERR_INVALID.
 * spider_plan_autotune sets it. */
spider_status spider_plan_set_tile_variant(spider_plan plan, int variant);

/* spider_plan_autotune -- measures the plan's configurations on the caller's
 * grids and keeps the fastest: time steps per pass (1..4 where built, see
 * spider_plan_set_steps_per_pass; up to 10, and at most `steps`, for
 * radius-1 2-D grids of at most 2^22 points) and the tile variant.  Each candidate runs
 * `steps` steps from grid_in into
 * grid_out (device grids as for spider_run; grid_out is overwritten) once to
 * warm up and twice timed with CUDA events on `stream`; the call is
 * synchronous.  Results are cached per (ndim, radius, shape, precision,
 * engine, grid-size bucket), so later plans of the same kind reuse them
 * without timing.  *steps_per_pass / *variant (nullable) receive the choice. */
spider_status spider_plan_autotune(spider_plan plan, const float* grid_in, float* grid_out, int64_t steps,
                                   cudaStream_t stream, int* steps_per_pass, int* variant);

/* spider_plan_autotune_arithmetic -- the split-depth part of the autotuner
 * (the paper states no precision; this is an addition of the library).
 * Among the arithmetics the library builds for the plan's stencil -- sparse
 * TF32, the FP16 hi/lo split (only when every |grid_in| value is below
 * 16384), the BF16 hi/mid/lo split, FP32 on CUDA cores -- it keeps those
 * whose a priori error bound for `steps` steps (spider_plan_error_bound)
 * meets err_target, autotunes each on the caller's grids (as
 * spider_plan_autotune, on a temporary plan), times `steps` steps of each
 * twice with CUDA events on `stream`, and returns the fastest in *prec /
 * *engine and its rate in *gstencil_s (GStencil/s; all nullable).  The plan
 * itself is not changed: create a plan in the chosen precision (and set its
 * engine) to run in it.  grid_out is overwritten.  Synchronous.
 * SPIDER_ERR_UNSUPPORTED when no arithmetic's bound meets the target. */
spider_status spider_plan_autotune_arithmetic(spider_plan plan, const float* grid_in, float* grid_out, int64_t steps,
                                              double err_target, cudaStream_t stream, spider_precision* prec,
                                              spider_engine* engine, double* gstencil_s);

/* Reads back the plan's packed operands (host copies) for inspection and
 * testing.  Any pointer may be NULL; sizes are in 32-bit words.
 *   n_operand_words / operand_words : tensor-core A fragments, per
 *       [split term][kernel row][lane][4] words
 *   n_meta_words / meta_words       : metadata, per [kernel row][lane]
 * Returns SPIDER_ERR_INVALID if a buffer is given with a too small capacity. */
spider_status spider_plan_operands(spider_plan plan, uint32_t* operand_words, size_t operand_capacity,
                                   size_t* n_operand_words, uint32_t* meta_words, size_t meta_capacity,
                                   size_t* n_meta_words);

/* spider_run -- advances a grid by `steps` time steps (Sec. 3.2, Sec. 3.3.1).
 *
 *  grid_in   device, the plan's extents; read only (preserved).
 *  grid_out  device, same size; must not overlap grid_in.  Receives the field
 *            after `steps` steps; for steps == 0 it receives a copy of grid_in.
 *  steps     >= 0.
 *  stream    CUDA stream (0 = legacy default stream).
 * The library ping-pongs between grid_out and a plan-owned scratch grid, so
 * any step count ends in grid_out.  When grid_out cannot be read by TMA in
 * its own layout (2-D and 3-D grids whose rows are not a multiple of 4
 * floats, or a grid_out that is not 16-byte aligned), the steps between the
 * first and the last run in two plan-owned grids whose rows are padded to a
 * multiple of 4 floats, allocated on first use (2 * ny * nz * round4(nx)
 * floats); grid_in and grid_out keep the caller's packed layout.  Calls on
 * one plan must not overlap on the GPU (its scratch grids are shared); use
 * one plan per concurrent stream. */
spider_status spider_run(spider_plan plan, const float* grid_in, float* grid_out, int64_t steps,
                         cudaStream_t stream);

/* spider_run_host -- spider_run for host buffers: copies host_in to a
 * plan-owned device grid, runs, copies the result to host_out, and waits for
 * completion.  host_in / host_out may be pageable or pinned host memory and
 * may be the same buffer. */
spider_status spider_run_host(spider_plan plan, const float* host_in, float* host_out, int64_t steps,
                              cudaStream_t stream);

/* spider_run_host_async -- spider_run_host without the wait, for a stream of
 * host grids through one plan.  The paper has no counterpart: this is an
 * addition of the library.  The call enqueues the copy of host_in into one
 * of two plan-owned device slots (on a copy stream of the plan), the steps
 * (on `stream`, after that copy) and the copy of the result to host_out (on
 * a second copy stream, after the steps), and returns.  Successive calls use
 * the two slots in turn, so the copies of one call overlap the steps of the
 * call before it (with pinned host memory; pageable memory works but the
 * copies then stage through the driver and overlap little).  host_in must
 * stay unchanged and host_out untouched until spider_plan_sync(plan,
 * stream) returns, which waits for the steps and for both copy streams;
 * host_in and host_out must not be the same buffer.  Successive calls on one
 * plan must pass the same `stream`.  The slots hold 4 * points floats of
 * device memory from the first call until the plan is destroyed. */
spider_status spider_run_host_async(spider_plan plan, const float* host_in, float* host_out, int64_t steps,
                                    cudaStream_t stream);

/* spider_run_static -- spider_run that allocates no device memory.
 * The paper has no counterpart: this is an addition of the library.
 *
 * For callers that cannot call cudaMalloc: an application whose own memory
 * pool has already reserved the GPU's memory (a further cudaMalloc would
 * fail), or a latency-critical loop that cannot accept the implicit
 * device-wide synchronisation of cudaMalloc/cudaFree.  Instead of the
 * plan-owned device buffers spider_run allocates on first use, it works in
 * fixed-size __device__ arrays of the library: a scratch grid of at most
 * 4,194,304 points (16 MiB) plus 84 KiB for packed operands, metadata and
 * coefficients.  Every GPU that loads the library holds these arrays until
 * the process exits.
 *  grid_in, grid_out, steps, stream: as for spider_run.
 * On grids TMA can read in their own layout it runs the same passes as
 * spider_run (the plan's steps per pass and tile variant); grids whose rows
 * are not a multiple of 4 floats (1-D: 8), or whose output buffer is not
 * 16-byte aligned, run one time step per pass (there are no padded grids).
 * Grids with more than 4,194,304 points return SPIDER_ERR_INVALID and nothing
 * is done.  The first call on each device looks up the arrays' device
 * addresses (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The looked-up addresses are kept for the
 * process: no call may follow a cudaDeviceReset of that device.  Each call
 * copies its plan's operands (a few KB, from the plan's host memory) into
 * the shared arrays on `stream` and clears the shared status word, and all
 * calls share one scratch grid, so calls that overlap on the GPU (other
 * streams or threads) race and corrupt each other's results.  A device-side
 * wait that runs out is not reported by this entry point. */
spider_status spider_run_static(spider_plan plan, const float* grid_in, float* grid_out, int64_t steps,
                                cudaStream_t stream);

/* Blocks until the plan's work on `stream` is done (and the copies of its
 * spider_run_host_async calls) and reports any device-side error
 * (SPIDER_ERR_TIMEOUT for an expired wait). */
spider_status spider_plan_sync(spider_plan plan, cudaStream_t stream);

/* spider_plan_error_bound -- the library's a priori bound on the relative L2
 * error, against exact arithmetic, of `steps` time steps of the plan's
 * stencil computed in precision `prec` on engine `engine` (the paper states
 * no precision; this is the library's error model, and the serving loop picks
 * with it the fastest arithmetic that meets a job's error target):
 *     bound = steps * (s + d) + f
 *  s  the plan's weight-sum error in that arithmetic: how far the weights the
 *     products use (TF32-rounded, or the FP16 / BF16 split terms) sum from
 *     the FP32 weights, relative to sum |w|.  It scales the constant mode of
 *     the field every step, so on a field of one sign the error grows by
 *     about s per step.  The plan rounds weights so that s is small.
 *  d  the rest of the per-step bias: TF32 rounds the grid to 11 bits every
 *     step, which is biased where the field is smooth (up to 5e-5 per step
 *     measured); the FP16 split's 22-bit products lose low bits inside the
 *     tensor core (4e-8); BF16 hi/mid/lo (6e-9) and FP32 (none) do not;
 *  f  the part of the error that does not grow with the step count.
 * d and f are twice the largest values measured on GB300 (radius 1..3 star
 * and box stencils in 2-D and 3-D, 10..500 steps, fields uniform on [0, 1)
 * and [-1, 1)); they assume the field does not grow, as
 * with sum |w| <= 1.  Host work only.  SPIDER_ERR_UNSUPPORTED when the
 * stencil has no kernel in that arithmetic (e.g. radius 4..7 off sparse
 * TF32). */
spider_status spider_plan_error_bound(spider_plan plan, spider_precision prec, spider_engine engine, int64_t steps,
                                      double* bound);

/* Bytes of device memory the plan owns right now: its packed operands,
 * status word, scratch and padded grids and the staging grids of
 * spider_run_host, all allocated on first use.  0 for a plan that has not
 * run through spider_run, spider_run_host, spider_batch or
 * spider_plan_autotune (spider_run_static allocates nothing). */
spider_status spider_plan_device_bytes(spider_plan plan, size_t* bytes);

void spider_plan_destroy(spider_plan plan);

/* spider_batch -- advances n independent grids in one persistent launch.
 * plans[i], ins[i], outs[i], steps[i] as for spider_run (a plan may appear
 * once).  2-D grids with TF32 sparse plans go through one persistent kernel,
 * issued as a CUDA graph: work items (pass, grid, tile) are claimed from a
 * device queue in pass-major order, and pass p of a tile starts only after
 * the tile and its eight neighbours finished pass p-1 (per-tile counters,
 * bounded waits).  A pass is two time steps on a (56 - 2r) x 120 tile (the
 * first or last pass one step when the step count needs it, and every pass
 * of a one-step grid), see spider_batch_configure; seven warps compute the
 * tiles while an eighth claims the items and loads their boxes, three
 * CTAs per SM.  Results
 * are bit-identical to spider_run's.  Such grids of at least 2^16 points
 * and more than one step run through spider_run with fused passes instead
 * (the plan's steps per pass and tile variant if it fuses, else the
 * autotuned choice of its kind of stencil, else 2 steps on variant 2), on
 * library-owned side streams concurrently with the persistent launch (they
 * start after the work already queued on `stream`).  Other plans (3-D, split precisions, comparator
 * engines, radius above 3) run through spider_run on the same stream after
 * the persistent launch.  Grids whose rows are not a multiple of 4 floats,
 * or whose buffers are not 16-byte aligned, use the plan's padded grids (see
 * spider_run).  A call whose queued grids are those of the previous call on
 * the device (same plans, buffers, step counts and routing) relaunches that
 * call's persistent launch as it was built, without rebuilding or uploading
 * its tables.  Synchronous: returns when all grids are done.  n <= 4096.
 * Concurrent calls on one device (other threads or streams) run one after
 * another: they share the library's side streams and work queue.
 * SPIDER_ERR_TIMEOUT if a dependency wait ran out. */
spider_status spider_batch(int n, const spider_plan* plans, const float* const* ins, float* const* outs,
                           const int64_t* steps, cudaStream_t stream);

/* spider_batch_configure -- routing of spider_batch.  Grids of at least
 * fuse_min_points points (with more than one step) run as fused passes of
 * their own on side streams; smaller grids run in the persistent queue, whose
 * items take queue_steps_per_item time steps (1, or 2: the fused kernel's two
 * levels on tiles of (56 - 2r) x 120 outputs).  0 restores a default (the
 * measured best: 2^16 points, 2 steps per item).  Process-wide; applies to
 * later calls. */
spider_status spider_batch_configure(long long fuse_min_points, int queue_steps_per_item);

/* ---- failure detection -------------------------------------------------------
 * The paper has no counterpart.  Every wait of the library's kernels (a TMA
 * load landing, a batch-queue item waiting for its neighbours' previous pass)
 * is bounded: when it runs out, the kernel records a timeout in a device
 * status word and finishes without touching memory it does not own, the
 * CUDA context stays usable, and the call that reads the status word
 * (spider_plan_sync, spider_run_host, spider_batch) returns
 * SPIDER_ERR_TIMEOUT.
 *
 * spider_set_wait_limit: the limit of every bounded wait, in SM clock cycles
 * (default 4e9, about two seconds at 2 GHz; >= 1000).  Process-wide; applies
 * to kernels launched after the call (run graphs captured earlier keep the
 * limit they were captured with).
 *
 * spider_batch_drop_item: a test hook.  The next spider_batch call leaves
 * item `item` of its persistent queue out (items numbered in the queue's
 * queue's order, from 0: the first items are pass 0 of every job, jobs of
 * more passes first, tiles row by row; -1 clears): the item is claimed but neither
 * loaded nor computed, and its tile's pass counter is not advanced, so the
 * items that depend on it wait until the limit runs out and the call returns
 * SPIDER_ERR_TIMEOUT (that call's results are then undefined).  The hook
 * applies to one call and resets itself. */
spider_status spider_set_wait_limit(long long cycles);
spider_status spider_batch_drop_item(long long item);

/* ---- domain decomposition: slabs with ghost planes ---------------------------
 * The paper runs one GPU and has no counterpart; this is the hook a
 * multi-GPU run builds on.  A domain cuts the grid of a plan into slabs along
 * its slowest axis (z for 3-D, y for 2-D, x for 1-D).  Each slab owns a range
 * of planes and keeps ghost planes, copies of its neighbours' outermost
 * planes (the HALO region of Sec. 1 and Sec. 3.3.1 at the slab's edge).  A
 * run alternates E time steps on every slab with an exchange of the ghost
 * planes; the result equals spider_run's bit for bit.  All slabs live on the
 * current device and the exchange is a device-to-device copy. */
typedef struct spider_domain_t* spider_domain;

/* spider_domain_create -- plans a run of `plan`'s grid as `parts` slabs.
 *  plan               stencil, extents, precision, engine, steps per pass and
 *                     tile variant of every slab (copied; the caller keeps it).
 *  parts              >= 1 and <= the extent of the slowest axis.
 *  steps_per_exchange E >= 1 time steps between exchanges; 0 selects the
 *                     plan's steps per pass.
 *  out                receives the domain (free with spider_domain_destroy).
 * Interior sides get g ghost planes, E * radius rounded up to a multiple of 8
 * (1-D) or 2 (2-D); slab boundaries are the even split rounded down to the
 * same multiple, so every point keeps its place inside the tensor-core tiles.
 * SPIDER_ERR_INVALID if a slab would own fewer than g planes (or none).
 * Host work only; device memory (two grids per slab, plus each slab plan's
 * scratch grid) is allocated on the first run. */
spider_status spider_domain_create(spider_plan plan, int parts, int steps_per_exchange, spider_domain* out);

/* Layout of slab i: first owned plane, owned planes, ghost planes below and
 * above (0 at the grid's ends).  Any output pointer may be NULL. */
spider_status spider_domain_slab(spider_domain domain, int i, int64_t* first, int64_t* owned, int64_t* ghost_lo,
                                 int64_t* ghost_hi);

/* spider_domain_run -- spider_run through the slabs: copies grid_in into the
 * slabs (owned and ghost planes), runs ceil(steps / E) periods of E steps
 * (the last may be shorter) with an exchange between periods, and copies the
 * owned planes into grid_out.  grid_in, grid_out, steps, stream as for
 * spider_run; asynchronous on `stream`.  Calls on one domain must not
 * overlap on the GPU. */
spider_status spider_domain_run(spider_domain domain, const float* grid_in, float* grid_out, int64_t steps,
                                cudaStream_t stream);

/* Blocks until the domain's work on `stream` is done and reports any
 * device-side error, as spider_plan_sync. */
spider_status spider_domain_sync(spider_domain domain, cudaStream_t stream);

void spider_domain_destroy(spider_domain domain);

/* GPU FP64 validation reductions (the only FP64 the library runs on the GPU).
 *   a    device float32 array of n values
 *   ref  device float64 array of n values, or NULL
 *   out  host double[4]: sum(a^2), sum(ref^2), sum((a-ref)^2), max|a-ref|
 *        (the last two are 0 when ref is NULL).  Synchronous on `stream`. */
spider_status spider_norms_fp64(const float* a, const double* ref, int64_t n, double* out, cudaStream_t stream);

/* Constant-field invariant check: max |a[i] - value| over the points of a
 * grid (extents as for plans) that lie farther than `margin` points from every
 * face, computed in FP64 on the GPU.  Synchronous on `stream`. */
spider_status spider_constant_check_fp64(const float* a, int ndim, const int64_t* extents, int64_t margin,
                                         double value, double* max_dev, cudaStream_t stream);

/* ---- serving: continuous batching of stencil jobs ---------------------------
 * A server owns a worker thread and its own streams.  Jobs are admitted while
 * their device memory (two grids) fits the HBM budget; jobs that arrive while
 * others run are started as memory and slots free up, and their work overlaps
 * on the device. */
spider_status spider_server_create(size_t hbm_budget_bytes, spider_server* out);

/* Submits a job.  `plan` is copied (the caller may destroy it afterwards).
 * host_in: host grid of the plan's extents, copied before return.
 * err_target: relative L2 error the caller accepts.  The job runs in the
 * plan's own precision and engine if its a priori bound
 * (spider_plan_error_bound) for `steps` steps meets the target, else in the
 * arithmetic measured fastest for this class of stencil among those whose
 * bound meets it: sparse TF32, the FP16 hi/lo split (only when every
 * |host_in| value is below 16384), FP32 on CUDA cores (radius <= 3); with
 * the plan's steps per pass if above 1, else the autotuner's choice for the
 * kind of stencil if one was measured in the process, else a measured
 * default of its class.
 * *ticket identifies the job.  SPIDER_ERR_UNSUPPORTED if no arithmetic built
 * for the stencil meets the target; SPIDER_ERR_OOM if the job alone exceeds
 * the budget; SPIDER_ERR_BUSY if the queue is full. */
spider_status spider_submit(spider_server server, spider_plan plan, const float* host_in, int64_t steps,
                            double err_target, uint64_t* ticket);

/* Polls a job.  *done = 1 once finished; then, if out != NULL, the result is
 * copied to host memory `out` and the job's record is released (a ticket can
 * be read once).  latency_s (nullable) receives submit-to-completion seconds. */
spider_status spider_poll(spider_server server, uint64_t ticket, float* out, int* done, double* latency_s);

/* The arithmetic the server chose for a job (precision, engine, time steps
 * per pass) and its a priori error bound; any pointer may be NULL.  Valid
 * until spider_poll releases the ticket. */
spider_status spider_server_job_arithmetic(spider_server server, uint64_t ticket, spider_precision* prec,
                                          spider_engine* engine, int* steps_per_pass, double* bound);

/* Waits up to timeout_s seconds for a job to finish and hands out its ticket
 * (*got = 1), each finished job once, in order of completion; *got = 0 when
 * none finished in time.  The job's record stays until spider_poll reads it,
 * so a client waits here instead of polling every ticket. */
spider_status spider_server_wait(spider_server server, double timeout_s, uint64_t* ticket, int* got);

/* Stops the worker after the jobs already submitted finish, frees everything. */
void spider_server_destroy(spider_server server);

/* spider_measure_mma_rate -- the peak issue rate, in MMAs per second, of one
 * warp-level tensor-core MMA shape on the current GPU: the denominator of the
 * tensor-pipe roofline of the stencil kernels.  The paper has no counterpart
 * (its Table 2 counts MMAs per point; this measures what one GPU sustains).
 *  kind  0 = sparse TF32 m16n8k16 (mma.sp), 1 = sparse FP16 m16n8k32,
 *        2 = sparse BF16 m16n8k32, 3 = dense TF32 m16n8k8 (mma.sync).
 * A kernel of two CTAs of eight warps per SM keeps its operands in registers
 * and issues eight independent accumulator chains per warp; the best of five
 * timed launches (CUDA events on `stream`) is reported.  Synchronous; it
 * allocates and frees a small device buffer. */
spider_status spider_measure_mma_rate(int kind, double* mma_per_s, cudaStream_t stream);

/* Message for the last failing call on this thread ("" if none). */
const char* spider_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPIDER_H_ */
