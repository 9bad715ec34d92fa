// The wide layout (sparse TF32): radius 4..7 in 1-D and 2-D, and every
// 1-D radius.
//
// With 2r + 1 > 8 non-zeros per kernel-matrix row, a 16-wide window cannot
// be 1:2 sparse.  Here a segment holds L = 16 outputs of one row (the
// paper's L = 2r + 2 <= 16, its worked example being r = 7, Sec. 3.1) and
// its window is 32 wide, starting 8 points to its left.  The strided swap
// pairs window positions p and p + 16 (phi_wide); a band of <= 15
// consecutive positions never holds both, so each half of the window is a
// 1:2-sparse k16 operand: two sparse MMAs per kernel row, M = the 16 outputs,
// N = 8 segments (128 outputs).  A 1-D grid uses it for r <= 3 too: its
// 16-output segments fill all of M, where the 8-output layout stacks two
// output rows and a 1-D grid has only one.
//
// The kernel rows are taken in groups of up to 4, whose A operands are in
// registers together (all 2r + 1 = 15 rows of r = 7 would not fit); within a
// group every input row of the warp's unit is loaded once and feeds the MMAs
// of every (kernel row, output row) pair it belongs to, H accumulator sets.
// Each output row still receives its kernel rows in increasing order.  The
// input box is rounded to TF32 in shared memory once when the grid is not
// stored rounded already (RIN), instead of on every load.
#pragma once

#include "stencil_kernels.cuh"

namespace spider {

template <int RY_, int RX_, int WY_, int H_, int MINB_ = 1>
struct WideCfg {
  static constexpr int RZ = 0, RY = RY_, RX = RX_, WY = WY_, H = H_;
  static constexpr int kMinBlocks = MINB_;  // CTAs per SM the register budget must allow
  static constexpr int BY = WY * H, BX = 128;
  static constexpr int SY = BY + 2 * RY, SX = BX + 2 * kWideHalo;
  static constexpr int kThreads = WY * 32;
  static constexpr int kStageBytes = SY * SX * 4;
  static constexpr int kStageStride = (kStageBytes + 1023) / 1024 * 1024;
  static constexpr int kSmemBytes = 2 * kStageStride + 1024 + 64;
  static constexpr int NKR = 2 * RY + 1;  // kernel rows
  static_assert(RX >= 1 && RX <= kMaxRWide, "wide layout radius");
  static_assert(SY <= 256 && SX <= 256, "TMA box dimension limit");
};

constexpr int kWideGroup = 4;  // kernel rows whose operands share the registers

// Input row JJ of the unit (relative to its first input row) against kernel
// rows K0 .. K0+G-1: output row yy = JJ - kr.
template <class C, int K0, int G, int JJ>
__device__ __forceinline__ void wide_rows(uint32_t row0, const uint4 (&A0)[G], const uint4 (&A1)[G],
                                          const uint32_t (&E0)[G], const uint32_t (&E1)[G],
                                          float (&acc)[C::H][4]) {
  float4 v0, v1;
  asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4+%5];"
      : "=f"(v0.x), "=f"(v0.y), "=f"(v0.z), "=f"(v0.w)
      : "r"(row0), "n"(JJ * C::SX * 4)
      : "memory");
  asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4+%5];"
      : "=f"(v1.x), "=f"(v1.y), "=f"(v1.z), "=f"(v1.w)
      : "r"(row0), "n"(JJ * C::SX * 4 + 32)
      : "memory");
  const uint32_t b0[4] = {__float_as_uint(v0.x), __float_as_uint(v0.y), __float_as_uint(v0.z), __float_as_uint(v0.w)};
  const uint32_t b1[4] = {__float_as_uint(v1.x), __float_as_uint(v1.y), __float_as_uint(v1.z), __float_as_uint(v1.w)};
#pragma unroll
  for (int kk = 0; kk < G; ++kk) {
    const int yy = JJ - (K0 + kk);
    if (yy >= 0 && yy < C::H) {
      mma_sp_tf32(acc[yy], A0[kk], E0[kk], b0);
      mma_sp_tf32(acc[yy], A1[kk], E1[kk], b1);
    }
  }
  if constexpr (JJ + 1 <= K0 + G - 1 + C::H - 1) wide_rows<C, K0, G, JJ + 1>(row0, A0, A1, E0, E1, acc);
}

template <class C, int K0>
__device__ __forceinline__ void wide_groups(uint32_t row0, const StepArgs& args, int lane, float (&acc)[C::H][4]) {
  constexpr int G = (C::NKR - K0) < kWideGroup ? (C::NKR - K0) : kWideGroup;
  uint4 A0[G], A1[G];
  uint32_t E0[G], E1[G];
#pragma unroll
  for (int kk = 0; kk < G; ++kk) {
    A0[kk] = args.a_words[(size_t)(2 * (K0 + kk)) * 32 + lane];
    A1[kk] = args.a_words[(size_t)(2 * (K0 + kk) + 1) * 32 + lane];
    E0[kk] = args.meta[(size_t)(2 * (K0 + kk)) * 32 + lane];
    E1[kk] = args.meta[(size_t)(2 * (K0 + kk) + 1) * 32 + lane];
  }
  wide_rows<C, K0, G, K0>(row0, A0, A1, E0, E1, acc);
  if constexpr (K0 + G < C::NKR) wide_groups<C, K0 + G>(row0, args, lane, acc);
}

template <class C, bool RIN>
__global__ void __launch_bounds__(C::kThreads, C::kMinBlocks)
    wide_step_kernel(const __grid_constant__ CUtensorMap tmap, const StepArgs args) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t base_u32 = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024 - (base_u32 & 1023)) & 1023);
  auto stage = [&](int s) { return reinterpret_cast<float*>(smem + s * C::kStageStride); };
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * C::kStageStride);

  const int tid = threadIdx.x;
  const int lane = tid & 31, wy = tid >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int ntiles = args.tiles_x * args.tiles_y;
  const bool use_tma = args.use_tma != 0;
  auto issue = [&](int t, int s) {
    const int x0 = (t % args.tiles_x) * C::BX, y0 = (t / args.tiles_x) * C::BY;
    mbar_arrive_expect_tx(&full[s], C::kStageBytes);
    tma_load_3d(stage(s), &tmap, &full[s], x0 - kWideHalo, y0 - C::RY, 0);
  };

  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    fence_mbar_init();
  }
  griddep_wait();  // see stencil_step_kernel
  griddep_launch_dependents();
  __syncthreads();
  if (use_tma && tid == 0) {
    if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
    if ((int)(blockIdx.x + gridDim.x) < ntiles) issue(blockIdx.x + gridDim.x, 1);
  }
  // this lane's B columns: segment g's window, K half 0 (half 1 is 8 further)
  const int coff = 16 * g + phi_wide(0, q);

  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int s = it & 1;
    float* S = stage(s);
    const int x0 = (t % args.tiles_x) * C::BX, y0 = (t / args.tiles_x) * C::BY;
    if (use_tma) {
      const bool ok = mbar_wait_bounded(&full[s], (it >> 1) & 1, args.status, args.wait_cycles);
      if (!__syncthreads_and(ok)) break;
    } else {
      load_box_async(args.src, args.nx, args.ny, 1, (int64_t)x0 - kWideHalo, (int64_t)y0 - C::RY, 0, C::SX, C::SY,
                     1, S, wy, C::kThreads / 32, lane);
      __syncthreads();
    }
    if (RIN) {
      // round the box to TF32 once (the MMAs read every value up to 2r + 1 times)
      for (int i = tid; i < C::SY * C::SX; i += C::kThreads) S[i] = __uint_as_float(cvt_tf32(S[i]));
      __syncthreads();
    }

    float acc[C::H][4];
#pragma unroll
    for (int i = 0; i < C::H; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    // output row yy of the unit reads input row yy + kr for kernel row kr
    // (dy = kr - ry); rows are relative to the unit's first input row
    wide_groups<C, 0>(smem_u32(S + (wy * C::H) * C::SX + coff), args, lane, acc);
    if (args.out_tf32) {
#pragma unroll
      for (int i = 0; i < C::H; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = __uint_as_float(cvt_tf32(acc[i][j]));
    }
    // D[m][n]: c0 (g, 2q), c1 (g, 2q+1), c2 (g+8, 2q), c3 (g+8, 2q+1); output
    // m of segment n is column 16 n + m of the tile
    const int ybase = y0 + wy * C::H;
    const int xb = x0 + 32 * q + g;
    const int cols[4] = {xb, xb + 16, xb + 8, xb + 24};
    float* o = args.dst + (int64_t)ybase * args.pitch;
    const bool interior = ybase + C::H <= args.ny && x0 + C::BX <= args.nx;
#pragma unroll
    for (int yy = 0; yy < C::H; ++yy) {
      if (interior || ybase + yy < args.ny) {
        float* orow = o + (int64_t)yy * args.pitch;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (interior || cols[j] < args.nx) orow[cols[j]] = acc[yy][j];
      }
    }

    __syncthreads();  // every warp is done with stage s
    if (use_tma && tid == 0) {
      const int tn = t + 2 * (int)gridDim.x;
      if (tn < ntiles) {
        fence_proxy_async_smem();
        issue(tn, s);
      }
    }
  }
  // loads still in flight after an early exit: wait for them (bounded)
  if (use_tma && tid == 0) {
    for (int k = 0; k < 2; ++k) {
      const int t = blockIdx.x + (it + k) * gridDim.x;
      if (t < ntiles) (void)mbar_wait_bounded(&full[(it + k) & 1], ((it + k) >> 1) & 1, args.status, args.wait_cycles);
    }
  }
}

}  // namespace spider

namespace spider {

// 1-D grids in the wide layout, several 128-point rows per warp.  The array
// is taken as consecutive rows of 128 points; a tile of BY rows is one
// contiguous chunk [X0 - 8, X0 + 128 BY + 8) in shared memory, so the window
// of a row's last segment runs into the next row's first points, which are
// its true neighbours.  The chunk is loaded by TMA through a 2-D view of the
// array as rows of 8 floats, zero outside the array: two boxes of 8 BY + 4
// such rows, so that the second box starts on a 128-byte boundary of shared
// memory (48 floats beyond the chunk are loaded and not used).  Arrays whose
// length is not a multiple of 8 load the chunk with cp.async.
template <int RX_, int H_, int NW_>
struct Wide1DCfg {
  static constexpr int RZ = 0, RY = 0, RX = RX_, H = H_, NW = NW_;
  static constexpr int kMinBlocks = 1;
  static constexpr int SX = 128;                  // row pitch in shared memory (no halo columns)
  static constexpr int BY = NW * H, NT = BY * SX;  // rows and points per tile
  static constexpr int kChunk = NT + 2 * kWideHalo;  // points the tile reads
  static constexpr int kBoxRows = 8 * BY + 4;          // rows of 8 floats per TMA box (two boxes)
  static constexpr int kThreads = NW * 32;
  static constexpr int kStageBytes = 2 * kBoxRows * 8 * 4;
  static constexpr int kStageStride = (kStageBytes + 1023) / 1024 * 1024;
  static constexpr int kSmemBytes = 2 * kStageStride + 1024 + 64;
  static constexpr int NKR = 1;
  static_assert(2 * kBoxRows * 8 >= kChunk && (kBoxRows * 32) % 128 == 0 && kBoxRows <= 256, "TMA boxes");
  static_assert(RX >= 1 && RX <= kMaxRWide, "wide layout radius");
};

template <class C, bool RIN>
__global__ void __launch_bounds__(C::kThreads)
    wide1d_kernel(const __grid_constant__ CUtensorMap tmap, const StepArgs args) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t base_u32 = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024 - (base_u32 & 1023)) & 1023);
  auto stage = [&](int s) { return reinterpret_cast<float*>(smem + s * C::kStageStride); };
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * C::kStageStride);

  const int tid = threadIdx.x;
  const int lane = tid & 31, wy = tid >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int64_t n = args.nx;
  const int ntiles = args.tiles_x;
  const bool use_tma = args.use_tma != 0;
  auto issue = [&](int t, int s) {
    // chunk start X0 - 8 is a multiple of 8: row (X0 - 8) / 8 of the 8-float view
    const int row8 = (int)(((int64_t)t * C::NT - kWideHalo) / 8);
    mbar_arrive_expect_tx(&full[s], C::kStageBytes);
    tma_load_3d(stage(s), &tmap, &full[s], 0, row8, 0);
    tma_load_3d(stage(s) + C::kBoxRows * 8, &tmap, &full[s], 0, row8 + C::kBoxRows, 0);
  };

  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    fence_mbar_init();
  }
  griddep_wait();  // see stencil_step_kernel
  griddep_launch_dependents();
  __syncthreads();
  if (use_tma && tid == 0) {
    if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
    if ((int)(blockIdx.x + gridDim.x) < ntiles) issue(blockIdx.x + gridDim.x, 1);
  }
  const int coff = 16 * g + phi_wide(0, q);

  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int s = it & 1;
    float* S = stage(s);
    const int64_t x0 = (int64_t)t * C::NT;
    if (use_tma) {
      const bool ok = mbar_wait_bounded(&full[s], (it >> 1) & 1, args.status, args.wait_cycles);
      if (!__syncthreads_and(ok)) break;
    } else {
      load_box_async(args.src, n, 1, 1, x0 - kWideHalo, 0, 0, C::kChunk, 1, 1, S, wy, C::kThreads / 32, lane);
      __syncthreads();
    }
    if (RIN) {
      for (int i = tid; i < C::kChunk; i += C::kThreads) S[i] = __uint_as_float(cvt_tf32(S[i]));
      __syncthreads();
    }
    float acc[C::H][4];
#pragma unroll
    for (int i = 0; i < C::H; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    wide_groups<C, 0>(smem_u32(S + (wy * C::H) * C::SX + coff), args, lane, acc);
    if (args.out_tf32) {
#pragma unroll
      for (int i = 0; i < C::H; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = __uint_as_float(cvt_tf32(acc[i][j]));
    }
    // row yy of this warp starts at point x0 + (wy H + yy) 128; output m of
    // segment n sits 16 n + m further (fragment map as in wide_step_kernel)
    const int64_t xw = x0 + (int64_t)(wy * C::H) * C::SX + 32 * q + g;
    const bool interior = x0 + C::NT <= n;
#pragma unroll
    for (int yy = 0; yy < C::H; ++yy) {
      float* o = args.dst + xw + yy * C::SX;
      const int64_t xr = xw + yy * C::SX;
      const int offs[4] = {0, 16, 8, 24};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (interior || xr + offs[j] < n) o[offs[j]] = acc[yy][j];
    }

    __syncthreads();  // every warp is done with stage s
    if (use_tma && tid == 0) {
      const int tn = t + 2 * (int)gridDim.x;
      if (tn < ntiles) {
        fence_proxy_async_smem();
        issue(tn, s);
      }
    }
  }
  if (use_tma && tid == 0) {
    for (int k = 0; k < 2; ++k) {
      const int t = blockIdx.x + (it + k) * gridDim.x;
      if (t < ntiles) (void)mbar_wait_bounded(&full[(it + k) & 1], ((it + k) >> 1) & 1, args.status, args.wait_cycles);
    }
  }
}

}  // namespace spider

namespace spider {

// 1-D temporal fusion: T steps per pass.  A tile of BY output rows of 128
// points computes every level on BY + 2 rows -- its own plus one neighbour
// row on each side -- so all level buffers share one layout: index
// i <-> point X0 - 136 + i, 8 unused margin points at each end (always 0).
// The windows of level t read level t-1 through the same 128-point row
// trick as wide1d_kernel.  A level value depends on level t-1 within r
// points only, so the garbage that enters from the margins creeps inward
// r points per level and never reaches the BY output rows while
// (T - 1) r <= 128.  Points outside the array are stored as 0 at every
// level (the zero Dirichlet halo of every step) and intermediate levels are
// stored rounded to TF32 as the next level's MMA reads them: bit-identical
// to T single steps.  The input chunk is loaded by TMA (the 8-float view,
// two boxes) into a ring of two stages.
template <int RX_, int T_, int BY_, int NW_>
struct Wide1DFusedCfg {
  static constexpr int RZ = 0, RY = 0, RX = RX_, T = T_, NW = NW_;
  static constexpr int kMinBlocks = 1;
  static constexpr int BY = BY_;                  // output rows per tile
  static constexpr int LR = BY + 2;               // rows of every level
  static constexpr int H = LR / NW;               // level rows per warp
  static constexpr int SX = 128;
  static constexpr int NT = BY * SX;              // output points per tile
  static constexpr int kOff = SX + kWideHalo;     // buffer index of point X0
  static constexpr int kBuf = LR * SX + 2 * kWideHalo;  // floats of every level buffer
  static constexpr int kBoxRows = ((kBuf / 8 + 1) / 2 + 3) / 4 * 4;  // two boxes, 128-byte aligned
  static constexpr int kInBytes = 2 * kBoxRows * 8 * 4;
  static constexpr int kInStride = (kInBytes + 1023) / 1024 * 1024;
  static constexpr int kLvStride = (kBuf * 4 + 1023) / 1024 * 1024;
  static constexpr int kThreads = NW * 32;
  static constexpr int kSmemBytes = 2 * kInStride + 2 * kLvStride + 1024 + 64;
  static constexpr int NKR = 1;
  static_assert(LR % NW == 0 && H >= 1, "level rows split evenly over the warps");
  static_assert((T - 1) * RX <= SX, "margin garbage must not reach the output rows");
  static_assert(2 * kBoxRows * 8 >= kBuf && (kBoxRows * 32) % 128 == 0 && kBoxRows <= 256, "TMA boxes");
  static_assert(T >= 2 && T <= 4, "steps per pass");
};

template <class C, bool RIN>
__global__ void __launch_bounds__(C::kThreads)
    wide1d_fused_kernel(const __grid_constant__ CUtensorMap tmap, const StepArgs args) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t base_u32 = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024 - (base_u32 & 1023)) & 1023);
  auto in_stage = [&](int s) { return reinterpret_cast<float*>(smem + s * C::kInStride); };
  float* lv[2] = {reinterpret_cast<float*>(smem + 2 * C::kInStride),
                  reinterpret_cast<float*>(smem + 2 * C::kInStride + C::kLvStride)};
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * C::kInStride + 2 * C::kLvStride);

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int64_t n = args.nx;
  const int ntiles = args.tiles_x;
  auto issue = [&](int t, int s) {
    // buffer index 0 is point X0 - 136, a multiple of 8
    const int row8 = (int)(((int64_t)t * C::NT - C::kOff) / 8);
    mbar_arrive_expect_tx(&full[s], C::kInBytes);
    tma_load_3d(in_stage(s), &tmap, &full[s], 0, row8, 0);
    tma_load_3d(in_stage(s) + C::kBoxRows * 8, &tmap, &full[s], 0, row8 + C::kBoxRows, 0);
  };

  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    fence_mbar_init();
  }
  // level buffers: zero margins (never written afterwards)
  for (int i = tid; i < C::kBuf; i += C::kThreads) lv[0][i] = lv[1][i] = 0.f;
  griddep_wait();  // see stencil_step_kernel
  griddep_launch_dependents();
  __syncthreads();
  if (tid == 0) {
    if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
    if ((int)(blockIdx.x + gridDim.x) < ntiles) issue(blockIdx.x + gridDim.x, 1);
  }
  const int coff = 16 * g + phi_wide(0, q);

  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int s = it & 1;
    float* S = in_stage(s);
    const int64_t x0 = (int64_t)t * C::NT;
    const bool ok = mbar_wait_bounded(&full[s], (it >> 1) & 1, args.status, args.wait_cycles);
    if (!__syncthreads_and(ok)) break;
    if (RIN) {
      for (int i = tid; i < C::kBuf; i += C::kThreads) S[i] = __uint_as_float(cvt_tf32(S[i]));
      __syncthreads();
    }
    // this warp's level rows warp*H .. warp*H+H-1; level row i covers points
    // x0 - 128 + 128 i .. +127 and reads the buffer from index 128 i
    const int64_t xw = x0 - C::SX + (int64_t)(warp * C::H) * C::SX + 32 * q + g;
    const int offs[4] = {0, 16, 8, 24};
#pragma unroll 1
    for (int level = 1; level <= C::T; ++level) {
      const float* src = level == 1 ? S : lv[(level - 2) & 1];
      float acc[C::H][4];
#pragma unroll
      for (int i = 0; i < C::H; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
      wide_groups<C, 0>(smem_u32(src + (warp * C::H) * C::SX + coff), args, lane, acc);
      if (level < C::T) {
        float* d = lv[(level - 1) & 1] + kWideHalo + (warp * C::H) * C::SX + 32 * q + g;
#pragma unroll
        for (int yy = 0; yy < C::H; ++yy)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int64_t x = xw + yy * C::SX + offs[j];
            d[yy * C::SX + offs[j]] = (x >= 0 && x < n) ? __uint_as_float(cvt_tf32(acc[yy][j])) : 0.f;
          }
      } else {
        if (args.out_tf32) {
#pragma unroll
          for (int i = 0; i < C::H; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = __uint_as_float(cvt_tf32(acc[i][j]));
        }
#pragma unroll
        for (int yy = 0; yy < C::H; ++yy) {
          const int row = warp * C::H + yy;  // output rows are level rows 1 .. BY
          if (row < 1 || row > C::BY) continue;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int64_t x = xw + yy * C::SX + offs[j];
            if (x < n) args.dst[x] = acc[yy][j];
          }
        }
      }
      __syncthreads();  // level complete before the next one reads it
      if (level == 1 && tid == 0) {
        // the input stage is no longer read: load the tile two ahead into it
        const int tn = t + 2 * (int)gridDim.x;
        if (tn < ntiles) {
          fence_proxy_async_smem();
          issue(tn, s);
        }
      }
    }
  }
  if (tid == 0) {
    for (int k = 0; k < 2; ++k) {
      const int t = blockIdx.x + (it + k) * gridDim.x;
      if (t < ntiles) (void)mbar_wait_bounded(&full[(it + k) & 1], ((it + k) >> 1) & 1, args.status, args.wait_cycles);
    }
  }
}

}  // namespace spider
