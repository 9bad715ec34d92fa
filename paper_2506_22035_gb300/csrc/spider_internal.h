// Internal definitions shared by the host plan code and the CUDA kernels.
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>
#include <mutex>

#include "spider.h"

namespace spider {

// ---------------------------------------------------------------- geometry
// Every stencil is handled as 3-D (nz, ny, nx) with per-axis radii
// (rz, ry, rx); a 2-D stencil has rz = 0 and nz = 1, a 1-D one also ry = 0.
//
// Tensor-core tile geometry (Sec. 3.1.1 with L = 8, Sec. 3.3.1):
//  * a "segment" is L = 8 consecutive outputs along x; its input window is
//    the 16 points x0-4 .. x0+11 (4 >= r points of halo on each side, which
//    keeps every window start 16-byte aligned);
//  * an MMA covers M = 16 rows = two vertically adjacent output rows (y, y+1)
//    x 8 outputs of one segment, N = 8 segments, K = the 16-point window of
//    one input row (z + dz, j).  The top half of A holds kernel row
//    dy = j - y, the bottom half dy = j - y - 1, so one B fragment of input
//    row j feeds both output rows and the accumulator never moves;
//  * "A index" a = j - y + ry runs 0 .. 2ry+1 for each dz.
// Default limit of the kernels' bounded waits: SM clock cycles (~2 s at 2 GHz).
constexpr long long kDefaultWaitCycles = 4000000000LL;
void set_wait_limit_cycles(long long cycles);

constexpr int kSeg = 8;          // L: outputs per segment
constexpr int kWin = 16;         // 2L: input window per segment
constexpr int kHaloX = 4;        // window starts 4 points left of the segment
constexpr int kMaxR = 3;
// Radii 4..7 (1-D and 2-D, sparse TF32) use the wide layout: L = 16 outputs
// per segment, 32-wide windows starting 8 points left of the segment, two
// k16 MMAs per kernel row (see wide_kernels.cuh and plan.cu).
constexpr int kMaxRWide = 7;
constexpr int kWideHalo = 8;
// Window position of K index k in K half h of the wide layout: the 1:2 pair
// (2c, 2c+1) lands on positions p and p + 16, and lane q's four B values
// (k = q + 4i) are four consecutive positions.
__host__ __device__ constexpr int phi_wide(int h, int k) {
  return 8 * h + 4 * ((k % 4) >> 1) + 16 * ((k % 4) & 1) + k / 4;
}

// Fragment-aware strided permutation.  MMA K-index k of the TF32
// m16n8k16 B fragment lives in lane q = k % 4, register i = k / 4; we place
// it at window position phi(k) = 4*sigma(q) + i, so each lane's four B
// values are four consecutive floats (one 16-byte shared-memory load), and
// the 1:2 pairs (2c, 2c+1) land on window positions 8 apart -- the strided
// swap of Sec. 3.1.2 with stride L = 8.  For FP16/BF16 m16n8k32 the same
// sigma places K-index k' = 2q + 8s + h of each 16-wide half at
// 4*sigma(q) + 2s + h, so 2:4 groups are {p, p+1, p+8, p+9}.
constexpr int kSigma[4] = {0, 2, 1, 3};
inline int phi_tf32(int k) { return 4 * kSigma[k % 4] + k / 4; }
inline int phi_16bit(int kk) {  // kk in [0, 16) within one K half
  int q = (kk % 8) / 2, s = kk / 8, h = kk % 2;
  return 4 * kSigma[q] + 2 * s + h;
}

// -------------------------------------------------------------- the plan
// A captured whole run of spider_run (see run_cached in api.cu).
struct RunGraph {
  const float* in = nullptr;
  float* out = nullptr;
  int64_t steps = 0;
  int steps_per_pass = 0, tile_variant = 0, engine = 0;
  cudaGraphExec_t exec = nullptr;  // null: seen once, not captured yet
  uint64_t last_use = 0;
};

struct DeviceState {
  int device = -1;
  std::vector<RunGraph> graphs;    // at most kMaxRunGraphs, least recently used evicted
  cudaStream_t capture_stream = nullptr;
  uint64_t graph_clock = 0;
  uint32_t* a_words = nullptr;     // packed A fragments
  uint32_t* meta_words = nullptr;  // packed metadata
  float* w_dense = nullptr;        // dense coefficient cube (CUDA-core engine)
  float* scratch = nullptr;        // ping-pong grid
  float* pad = nullptr;            // two row-padded ping-pong grids (spider_batch)
  size_t pad_bytes = 0;
  float* host_stage_in = nullptr;  // device grids for spider_run_host
  float* host_stage_out = nullptr;
  // spider_run_host_async: two staging slots used in turn, so one call's
  // copies overlap the steps of the call before it; the copies run on two
  // streams of the plan (one per direction), ordered against the steps by
  // events
  struct HostSlot {
    float* in = nullptr;
    float* out = nullptr;
    cudaEvent_t copied_in = nullptr, stepped = nullptr, copied_out = nullptr;
    bool used = false;
  };
  HostSlot host_slots[2];
  int host_next = 0;
  cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
  int* status = nullptr;           // device error word (0 = ok)
  size_t scratch_bytes = 0;
  // Stream-ordered allocation (the serving loop): when `pool` is set, every
  // buffer above comes from it through cudaMallocFromPoolAsync on
  // `pool_stream` and goes back through cudaFreeAsync on the same stream, so
  // neither allocating nor freeing waits for the device.
  cudaMemPool_t pool = nullptr;
  cudaStream_t pool_stream = nullptr;
};

// Split weights of the FP16 / BF16 precisions: w ~ hi + mid + lo_scale * lo
// (FP16: mid = 0, lo scaled by 2^11; BF16: three BF16 terms).
struct SplitWeights {
  std::vector<float> hi, mid, lo;
  double lo_scale = 1.0;
};

}  // namespace spider

struct spider_plan_t {
  int ndim = 0;
  int64_t extents[3] = {1, 1, 1};
  int64_t nz = 1, ny = 1, nx = 1;
  spider_shape shape = SPIDER_BOX;
  int r = 1, rz = 0, ry = 0, rx = 1;
  spider_precision prec = SPIDER_TF32;
  spider_engine engine = SPIDER_ENGINE_SPARSE_TC;
  int steps_per_pass = 1;
  int tile_variant = 0;                  // fused warp-unit height: 0 -> 8 rows, 1 -> 16 rows
  std::vector<float> w;                  // (2rz+1)(2ry+1)(2rx+1), [dz][dy][dx]
  // Packed operands, see plan.cu for the layouts.
  int n_arows = 0;                       // A matrices per split term = (2rz+1)(2ry+2)
  int n_combos = 0;                      // A operands actually issued per dz-plane set
  std::vector<uint32_t> a_words;         // [combo][lane][4]  (dense TF32: [arow][lane][8])
  std::vector<uint32_t> meta_words;      // [combo][lane]
  spider::SplitWeights split;            // FP16 / BF16 precisions
  // |sum of the weights as the arithmetic holds them - sum of the FP32
  // weights| / sum |w|, for TF32, FP16 hi/lo and BF16 hi/mid/lo
  double wsum_rel[3] = {0, 0, 0};
  spider::DeviceState dev;
  std::mutex mu;

  int64_t points() const { return nz * ny * nx; }
  // The wide layout (wide_kernels.cuh) serves radius 4..7 and every 1-D
  // sparse TF32 plan (its 16-output segments fill both halves of M, where the
  // 8-output layout would leave the second output row of a 1-D grid empty).
  bool wide() const {
    const bool sparse_tf32 = engine == SPIDER_ENGINE_SPARSE_TC && (prec == SPIDER_TF32 || prec == SPIDER_AUTO);
    return r > spider::kMaxR || (ndim == 1 && sparse_tf32);
  }
};

namespace spider {

// thread-local last-error message
void set_error(const std::string& msg);
spider_status fail(spider_status s, const std::string& msg);

// plan.cpp
spider_status build_operands(spider_plan_t* p);
uint32_t round_tf32_rna(float x);
float tf32_value(float x);

// plan.cu: the split weights of a 16-bit precision (sum-preserving last
// term) and the error of their sum against the FP32 weights.
SplitWeights split_weights(const std::vector<float>& w, spider_precision prec);
double split_sum_error(const std::vector<float>& w, const SplitWeights& sw);

// Number of A "combos" (register operands) for a precision, per dz plane.
int combos_per_plane(spider_precision prec, int ry);

// api.cu: enqueue `steps` steps in -> out on `stream` (plan lock held by the caller).
spider_status run_device(spider_plan_t* p, const float* in, float* out, int64_t steps, cudaStream_t stream);
// api.cu: the largest number of time steps per HBM pass built for the plan
// (fused kernels: 2-D stencils, and 3-D radius-1 stencils in sparse TF32).
int max_steps_per_pass(const spider_plan_t* p);
// api.cu: the a priori error model of an arithmetic for the plan's stencil
// (spider_plan_error_bound): bound = steps * (wsum + drift) + floor.
struct ErrorModel {
  bool built = false;
  double wsum = 0, drift = 0, floor = 0;
};
ErrorModel error_model(const spider_plan_t* p, spider_precision prec, spider_engine engine);
// api.cu: upload the plan's operands (and allocate its scratch grid) if needed.
spider_status ensure_plan_device(spider_plan_t* p, bool scratch);
// autotune.cu: the tuned (steps per pass, tile variant) of the plan's kind
// of stencil, if one has been measured.
bool autotune_lookup(const spider_plan_t* p, int* steps_per_pass, int* variant);
// api.cu: make the plan's padded ping-pong area at least `bytes` long.
spider_status ensure_plan_pad(spider_plan_t* p, size_t bytes);

}  // namespace spider
