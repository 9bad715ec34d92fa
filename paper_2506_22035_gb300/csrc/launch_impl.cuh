// Template launcher shared by the per-mode dispatch translation units.
#pragma once

#include <type_traits>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "launch.h"
#include "fused_kernels.cuh"
#include "stencil_kernels.cuh"
#include "stream3d_fused_kernels.cuh"
#include "stream3d_kernels.cuh"
#include "wide_kernels.cuh"

namespace spider {

// Row pitches of a pass's grids (LaunchCtx pitch 0 = nx) and the source's
// tensor map in that layout.
inline int64_t src_pitch(const LaunchCtx& ctx) { return ctx.src_pitch ? ctx.src_pitch : ctx.plan->nx; }
inline int64_t dst_pitch(const LaunchCtx& ctx) { return ctx.dst_pitch ? ctx.dst_pitch : ctx.plan->nx; }
inline bool make_src_map(CUtensorMap* map, const LaunchCtx& ctx, int64_t nz, int box_x, int box_y, int box_z) {
  const spider_plan_t* p = ctx.plan;
  return make_tensor_map_pitched(map, ctx.src, p->nx, p->ny, nz, src_pitch(ctx), box_x, box_y, box_z);
}

// Launch with programmatic stream serialization: the kernel may begin while
// the previous kernel on the stream drains; the kernels wait (griddep_wait)
// before touching the grids.
template <class K>
cudaError_t launch_pdl(K kern, int grid, int threads, int smem, cudaStream_t stream, const CUtensorMap& map,
                       const StepArgs& a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, map, a);
}

template <class C, Mode MODE, bool RIN, bool STAR>
cudaError_t launch_cfg_k(const LaunchCtx& ctx) {
  const spider_plan_t* p = ctx.plan;
  auto kern = stencil_step_kernel<C, MODE, RIN, STAR>;
  // Per-device one-time setup: opt into the dynamic shared memory and read
  // the occupancy that sizes the persistent grid.
  static std::mutex mu;
  static int occ_by_dev[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int occ;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (occ_by_dev[dev] == 0) {
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, step_smem_bytes<C, MODE>());
      if (err != cudaSuccess) return err;
      int o = 0;
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, C::kThreads, step_smem_bytes<C, MODE>());
      if (err != cudaSuccess) return err;
      occ_by_dev[dev] = std::max(o, 1);
    }
    occ = occ_by_dev[dev];
  }
  StepArgs a;
  a.src = ctx.src;
  a.dst = ctx.dst;
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  a.pitch = dst_pitch(ctx);
  a.tiles_x = (int)((p->nx + C::BX - 1) / C::BX);
  a.tiles_y = (int)((p->ny + C::BY - 1) / C::BY);
  a.tiles_z = (int)((p->nz + C::BZ - 1) / C::BZ);
  a.a_words = reinterpret_cast<const uint4*>(p->dev.a_words);
  a.meta = p->dev.meta_words;
  a.w = p->dev.w_dense;
  a.status = p->dev.status;
  a.wait_cycles = wait_limit_cycles();
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  a.use_tma = make_src_map(&map, ctx, p->nz, C::SX, C::SY, C::SZ) ? 1 : 0;
  if (!a.use_tma && src_pitch(ctx) != p->nx) return cudaErrorNotSupported;  // the loader reads packed rows
  a.out_tf32 = ctx.out_tf32 ? 1 : 0;
  const long long ntiles = (long long)a.tiles_x * a.tiles_y * a.tiles_z;
  if (ntiles > (1LL << 31) - 1) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>(ntiles, (long long)occ * ctx.sms);
  return launch_pdl(kern, grid, C::kThreads, step_smem_bytes<C, MODE>(), ctx.stream, map, a);
}

// TF32 modes read a grid stored already rounded (ctx.in_tf32) with the
// kernel that skips the operand rounding.
template <class C, Mode MODE, bool STAR = false>
cudaError_t launch_cfg(const LaunchCtx& ctx) {
  if constexpr (is_tf32_mode(MODE)) {
    if (ctx.in_tf32) return launch_cfg_k<C, MODE, false, STAR>(ctx);
  }
  return launch_cfg_k<C, MODE, true, STAR>(ctx);
}

// Number of z chunks per column block for the z-streaming kernels.  Items
// (column, chunk) of equal length run in waves of `slots` resident CTAs; a
// chunk of c planes costs c + `halo` plane times (its halo planes are read,
// or recomputed, twice).  The count minimises waves x (nz / chunks + halo)
// over chunks of at least `min_planes` planes: one wave of long chunks when
// the columns fill the slots evenly, more waves of shorter chunks when one
// wave would leave many slots idle.
inline long long choose_z_chunks(long long ncol, long long slots, long long nz, long long halo, long long min_planes) {
  const long long max_chunks = std::max<long long>(1, nz / min_planes);
  long long best = 1;
  double best_cost = 1e300;
  for (long long c = 1; c <= max_chunks; ++c) {
    const long long waves = (ncol * c + slots - 1) / slots;
    const double cost = (double)waves * ((double)nz / (double)c + (double)halo);
    if (cost < best_cost * (1.0 - 1e-9)) {
      best_cost = cost;
      best = c;
    }
  }
  return best;
}

// 3-D z-streaming launch (TMA-describable grids); cudaErrorNotSupported
// otherwise, and the caller uses the cube-tiled kernel.
template <class C, Mode MODE, bool RIN, bool STAR>
cudaError_t launch_stream3d_k(const LaunchCtx& ctx) {
  const spider_plan_t* p = ctx.plan;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  if (!make_src_map(&map, ctx, p->nz, C::SX, C::SY, 1)) return cudaErrorNotSupported;
  auto kern = stream3d_kernel<C, MODE, RIN, STAR>;
  static std::mutex mu;
  static int occ_by_dev[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int occ;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (occ_by_dev[dev] == 0) {
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
      if (err != cudaSuccess) return err;
      int o = 0;
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, C::kThreads, C::kSmemBytes);
      if (err != cudaSuccess) return err;
      occ_by_dev[dev] = std::max(o, 1);
    }
    occ = occ_by_dev[dev];
  }
  StepArgs a;
  a.src = ctx.src;
  a.dst = ctx.dst;
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  a.pitch = dst_pitch(ctx);
  a.tiles_x = (int)((p->nx + C::BX - 1) / C::BX);
  a.tiles_y = (int)((p->ny + C::BY - 1) / C::BY);
  a.tiles_z = 1;
  a.a_words = reinterpret_cast<const uint4*>(p->dev.a_words);
  a.meta = p->dev.meta_words;
  a.w = p->dev.w_dense;
  a.status = p->dev.status;
  a.wait_cycles = wait_limit_cycles();
  a.use_tma = 1;
  a.out_tf32 = ctx.out_tf32 ? 1 : 0;
  const long long ncol = (long long)a.tiles_x * a.tiles_y;
  const long long slots = (long long)occ * ctx.sms;
  // z chunks of >= 8 planes, 2r halo planes each (on 512^3 TF32 this is one
  // wave of 73-plane chunks; four short chunks per CTA re-read 11 % of the
  // planes)
  const long long nchunks = choose_z_chunks(ncol, slots, p->nz, 2 * C::RZ, 8);
  if (ncol * nchunks > (1LL << 31) - 1) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>(ncol * nchunks, slots);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(C::kThreads);
  cfg.dynamicSmemBytes = C::kSmemBytes;
  cfg.stream = ctx.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, map, a, (int)nchunks);
}

template <class C, Mode MODE, bool STAR = false>
cudaError_t launch_stream3d(const LaunchCtx& ctx) {
  if constexpr (is_tf32_mode(MODE)) {
    if (ctx.in_tf32) return launch_stream3d_k<C, MODE, false, STAR>(ctx);
  }
  return launch_stream3d_k<C, MODE, true, STAR>(ctx);
}

// Tile shapes per stencil class: 1-D, 2-D (64 x 128 outputs, 8 warps),
// 3-D (z-streaming 32 x 128 column blocks; cube tiles of planes x 16 x 128
// outputs when the grid's rows are not TMA-describable).  The 3-D column
// block of radius 1 is 4 warps of 16 rows (its ring of 4 planes leaves room
// for two to three CTAs per SM).  Radius 2 and 3 keep 6 and 8 planes in
// flight, one CTA per SM, and there 8 warps of 8 rows run faster (GStencil/s
// at 160^3 / 320^3, 4 -> 8 warps: FP16 split radius-3 box 35 -> 42 / 46 ->
// 56, star 57 -> 88 / 79 -> 124; CUDA cores radius-3 star 131 -> 158 / 201
// -> 248), except for TF32 at radius 3, whose 16-row warp tiles feed more
// MMAs per row load (box 85 / 115 with 4 warps against 63 / 81 with 8).
template <int R, Mode MODE>
using Stream3DCfg = typename std::conditional<R >= 2 && !(R == 3 && is_tf32_mode(MODE)), StreamCfg<R, 4, 2, 8, 0>,
                                              StreamCfg<R, 2, 2, 16, 0>>::type;

template <int R, Mode MODE>
cudaError_t launch_class(int cls, const LaunchCtx& ctx) {
  if (cls == 1) return launch_cfg<TileCfg<0, 0, R, 1, 1, 2, 2>, MODE>(ctx);
  if (cls == 2) return launch_cfg<TileCfg<0, R, R, 1, 4, 2, 16>, MODE>(ctx);
  if (cls == 3) {
    // star stencils skip the zero operands (CUDA cores: the zero weights)
    // of the off-centre planes (the cube tiles, for grids TMA cannot read,
    // in TF32 only)
    {
      if (ctx.plan->shape == SPIDER_STAR) {
        const cudaError_t e = launch_stream3d<Stream3DCfg<R, MODE>, MODE, true>(ctx);
        if (e != cudaErrorNotSupported) return e;
        if constexpr (is_tf32_mode(MODE)) return launch_cfg<TileCfg<R, R, R, (R <= 2 ? 4 : 2), 1, 2, 16>, MODE, true>(ctx);
      }
    }
    const cudaError_t e = launch_stream3d<Stream3DCfg<R, MODE>, MODE>(ctx);
    if (e != cudaErrorNotSupported) return e;
    return launch_cfg<TileCfg<R, R, R, (R <= 2 ? 4 : 2), 1, 2, 16>, MODE>(ctx);
  }
  return cudaErrorNotSupported;
}

template <Mode MODE>
cudaError_t launch_mode(int cls, int r, const LaunchCtx& ctx) {
  switch (r) {
    case 1: return launch_class<1, MODE>(cls, ctx);
    case 2: return launch_class<2, MODE>(cls, ctx);
    case 3: return launch_class<3, MODE>(cls, ctx);
    default: return cudaErrorNotSupported;
  }
}

// ---- temporal fusion (2-D) ----------------------------------------------
template <class F, Mode MODE, bool RIN>
cudaError_t launch_fused_cfg_k(const LaunchCtx& ctx) {
  const spider_plan_t* p = ctx.plan;
  if (p->ndim != 2) return cudaErrorNotSupported;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  if (!make_src_map(&map, ctx, 1, F::width(0), F::rows(0), 1)) return cudaErrorNotSupported;
  auto kern = fused_step_kernel<F, MODE, RIN>;
  static std::mutex mu;
  static int occ_by_dev[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int occ;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (occ_by_dev[dev] == 0) {
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, F::kSmemBytes);
      if (err != cudaSuccess) return err;
      int o = 0;
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, F::kThreads, F::kSmemBytes);
      if (err != cudaSuccess) return err;
      occ_by_dev[dev] = std::max(o, 1);
    }
    occ = occ_by_dev[dev];
  }
  StepArgs a;
  a.src = ctx.src;
  a.dst = ctx.dst;
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = 1;
  a.pitch = dst_pitch(ctx);
  a.tiles_x = (int)((p->nx + F::BX - 1) / F::BX);
  a.tiles_y = (int)((p->ny + F::BY - 1) / F::BY);
  a.tiles_z = 1;
  a.a_words = reinterpret_cast<const uint4*>(p->dev.a_words);
  a.meta = p->dev.meta_words;
  a.w = p->dev.w_dense;
  a.status = p->dev.status;
  a.wait_cycles = wait_limit_cycles();
  a.use_tma = 1;
  a.out_tf32 = ctx.out_tf32 ? 1 : 0;
  const long long ntiles = (long long)a.tiles_x * a.tiles_y;
  if (ntiles > (1LL << 31) - 1) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>(ntiles, (long long)occ * ctx.sms);
  return launch_pdl(kern, grid, F::kThreads, F::kSmemBytes, ctx.stream, map, a);
}

template <class F, Mode MODE>
cudaError_t launch_fused_cfg(const LaunchCtx& ctx) {
  if constexpr (is_tf32_mode(MODE)) {
    if (ctx.in_tf32) return launch_fused_cfg_k<F, MODE, false>(ctx);
  }
  return launch_fused_cfg_k<F, MODE, true>(ctx);
}

// Fused tile shapes: level 1 is 64 rows x 16 segments (two N-tiles), so the
// output tile is BY = 64 - 2r(T-1) rows x BX = 8 (17 - T) columns; 8 warps;
// warp units of H rows x 8 segments.  Variants:
//   0: H = 8,  two input boxes in flight      1: H = 16, two input boxes
//   2: H = 8,  one input box, registers capped for 3 CTAs per SM
//   3: H = 16, one input box
template <int R, int T, int H, int MINB, int INS, int L1 = 64, int VEC = 0>
using FusedTile = FuseCfg<R, T, L1 - 2 * R * (T - 1), 8 * (17 - T), H, 8, MINB, INS, VEC>;

template <Mode MODE, int R, int H, int MINB, int INS, int L1 = 64, int VEC = 0>
cudaError_t launch_fused_rh(int T, const LaunchCtx& ctx) {
  switch (T) {
    case 2: return launch_fused_cfg<FusedTile<R, 2, H, MINB, INS, L1, VEC>, MODE>(ctx);
    case 3: return launch_fused_cfg<FusedTile<R, 3, H, MINB, INS, L1, VEC>, MODE>(ctx);
    case 4: return launch_fused_cfg<FusedTile<R, 4, H, MINB, INS, L1, VEC>, MODE>(ctx);
    default: return cudaErrorNotSupported;
  }
}

// Variants 2 and 3 differ by mode.  Sparse TF32: 2 = H 8 with registers
// capped for three CTAs per SM, 3 = H 16 with one input box.  FP16/BF16
// splits and dense TF32 (150..190 registers uncapped, one CTA per SM):
// 2 and 3 = H 8 with registers capped for two CTAs per SM, two or one input
// boxes (124..128 registers, at most a few spilled words).  CUDA cores (W
// in registers): 2 and 3 run as 0 and 1.  Variant 4 is the small tile: level
// 1 of 32 rows, one warp unit per warp per level, four times the tiles of
// the 64-row shapes -- for grids too small to fill the GPU, where a pass is
// the latency of one tile's levels.  Variant 5 (sparse TF32): variant 2 with
// the final level written by 16-byte stores after a transpose of the
// accumulator fragments within groups of four lanes (other modes: as 2).
template <Mode MODE, int R>
cudaError_t launch_fused_r(int T, const LaunchCtx& ctx) {
  int v = ctx.plan->tile_variant;
  if (v == 4) return launch_fused_rh<MODE, R, 8, 1, 2, 32>(T, ctx);
  if constexpr (MODE == Mode::SpTF32) {
    if (v == 5) return launch_fused_rh<MODE, R, 8, 3, 1, 64, 1>(T, ctx);
    if (v == 2) return launch_fused_rh<MODE, R, 8, 3, 1>(T, ctx);
    if (v == 3) return launch_fused_rh<MODE, R, 16, 1, 1>(T, ctx);
  } else if constexpr (MODE != Mode::CudaCore) {
    if (v == 2 || v == 5) return launch_fused_rh<MODE, R, 8, 2, 2>(T, ctx);
    if (v == 3) return launch_fused_rh<MODE, R, 8, 2, 1>(T, ctx);
  } else {
    if (v == 5) v = 2;
    if (v >= 2) v -= 2;
  }
  return v == 1 ? launch_fused_rh<MODE, R, 16, 1, 2>(T, ctx) : launch_fused_rh<MODE, R, 8, 1, 2>(T, ctx);
}

// Deep fusion (radius 1): T = 5..10 levels on a 16 x 64 output tile (level 1
// is 16 + 2R(T-1) rows x 64 + 8(T-1) columns; one unit per warp on the last
// levels).  For grids too small to fill the GPU a pass costs about one
// tile's T levels, so fewer, deeper passes finish a run sooner although the
// levels' halos repeat work.
template <int R, int T>
using DeepTile = FuseCfg<R, T, 16, 64, 8, 8, 1, 2>;

template <Mode MODE, int R>
cudaError_t launch_fused_deep(int T, const LaunchCtx& ctx) {
  if (T > max_deep_steps(R)) return cudaErrorNotSupported;
  switch (T) {
    case 5: return launch_fused_cfg<DeepTile<R, 5>, MODE>(ctx);
    case 6: return launch_fused_cfg<DeepTile<R, 6>, MODE>(ctx);
    case 7: return launch_fused_cfg<DeepTile<R, 7>, MODE>(ctx);
    case 8: return launch_fused_cfg<DeepTile<R, 8>, MODE>(ctx);
    case 9: return launch_fused_cfg<DeepTile<R, 9>, MODE>(ctx);
    case 10: return launch_fused_cfg<DeepTile<R, 10>, MODE>(ctx);
    default: return cudaErrorNotSupported;
  }
}

template <Mode MODE>
cudaError_t launch_fused_mode(int r, int T, const LaunchCtx& ctx) {
  switch (r) {
    case 1: return launch_fused_r<MODE, 1>(T, ctx);
    case 2: return launch_fused_r<MODE, 2>(T, ctx);
    case 3: return launch_fused_r<MODE, 3>(T, ctx);
    default: return cudaErrorNotSupported;
  }
}


// ---- temporal fusion (3-D, z-streaming) -----------------------------------
template <class F, Mode MODE, bool RIN, bool STAR>
cudaError_t launch_fused3d_k(const LaunchCtx& ctx) {
  const spider_plan_t* p = ctx.plan;
  if (p->ndim != 3) return cudaErrorNotSupported;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  if (!make_src_map(&map, ctx, p->nz, F::width(0), F::rows(0), 1)) return cudaErrorNotSupported;
  auto kern = stream3d_fused_kernel<F, MODE, RIN, STAR>;
  static std::mutex mu;
  static int occ_by_dev[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int occ;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (occ_by_dev[dev] == 0) {
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, F::kSmemBytes);
      if (err != cudaSuccess) return err;
      int o = 0;
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, F::kThreads, F::kSmemBytes);
      if (err != cudaSuccess) return err;
      occ_by_dev[dev] = std::max(o, 1);
    }
    occ = occ_by_dev[dev];
  }
  StepArgs a;
  a.src = ctx.src;
  a.dst = ctx.dst;
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  a.pitch = dst_pitch(ctx);
  a.tiles_x = (int)((p->nx + F::BX - 1) / F::BX);
  a.tiles_y = (int)((p->ny + F::BY - 1) / F::BY);
  a.tiles_z = 1;
  a.a_words = reinterpret_cast<const uint4*>(p->dev.a_words);
  a.meta = p->dev.meta_words;
  a.w = p->dev.w_dense;
  a.status = p->dev.status;
  a.wait_cycles = wait_limit_cycles();
  a.use_tma = 1;
  a.out_tf32 = ctx.out_tf32 ? 1 : 0;
  const long long ncol = (long long)a.tiles_x * a.tiles_y;
  const long long slots = (long long)occ * ctx.sms;
  // z chunks of >= 32 planes; a chunk reads 2rT extra input planes and
  // recomputes 2r(T-t) planes of level t at its ends
  const long long nchunks = choose_z_chunks(ncol, slots, p->nz, 2 * F::R * F::T, 32);
  if (ncol * nchunks > (1LL << 31) - 1) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>(ncol * nchunks, slots);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(F::kThreads);
  cfg.dynamicSmemBytes = F::kSmemBytes;
  cfg.stream = ctx.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, map, a, (int)nchunks);
}

template <class F, Mode MODE>
cudaError_t launch_fused3d_cfg(const LaunchCtx& ctx) {
  const bool star = ctx.plan->shape == SPIDER_STAR;
  if (ctx.in_tf32) {
    return star ? launch_fused3d_k<F, MODE, false, true>(ctx) : launch_fused3d_k<F, MODE, false, false>(ctx);
  }
  return star ? launch_fused3d_k<F, MODE, true, true>(ctx) : launch_fused3d_k<F, MODE, true, false>(ctx);
}

// 3-D fused column blocks (r = 1): level 1 is L1Y rows x 128 columns.
//   variant 0: L1Y = 16, warp units of 4 rows, 8 warps, registers for 2 CTAs
//              per SM (1 for T = 4, whose rings need 114 KB)
//   variant 1, 3: L1Y = 32, warp units of 8 rows, 8 warps, one CTA per SM
//   variant 2: as 0 with registers capped for 3 CTAs per SM at T = 2
//   variant 4: as 0
template <Mode MODE, int T>
cudaError_t launch_fused3d_t(const LaunchCtx& ctx) {
  constexpr int kMinB = T == 4 ? 1 : 2;
  const int v = ctx.plan->tile_variant == 5 ? 2 : ctx.plan->tile_variant;
  if (v % 2 == 1) return launch_fused3d_cfg<Fuse3Cfg<1, T, 32, 8, 8, 1>, MODE>(ctx);
  if (T == 2 && v == 2) return launch_fused3d_cfg<Fuse3Cfg<1, T, 16, 4, 8, 3>, MODE>(ctx);
  return launch_fused3d_cfg<Fuse3Cfg<1, T, 16, 4, 8, kMinB>, MODE>(ctx);
}

template <Mode MODE>
cudaError_t launch_fused3d_mode(int r, int T, const LaunchCtx& ctx) {
  if (r != 1) return cudaErrorNotSupported;
  switch (T) {
    case 2: return launch_fused3d_t<MODE, 2>(ctx);
    case 3: return launch_fused3d_t<MODE, 3>(ctx);
    case 4: return launch_fused3d_t<MODE, 4>(ctx);
    default: return cudaErrorNotSupported;
  }
}


// ---- wide layout, radius 4..7 ---------------------------------------------
template <class C, bool RIN>
cudaError_t launch_wide_k(const LaunchCtx& ctx) {
  const spider_plan_t* p = ctx.plan;
  auto kern = wide_step_kernel<C, RIN>;
  static std::mutex mu;
  static int occ_by_dev[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int occ;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (occ_by_dev[dev] == 0) {
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
      if (err != cudaSuccess) return err;
      int o = 0;
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, C::kThreads, C::kSmemBytes);
      if (err != cudaSuccess) return err;
      occ_by_dev[dev] = std::max(o, 1);
    }
    occ = occ_by_dev[dev];
  }
  StepArgs a;
  a.src = ctx.src;
  a.dst = ctx.dst;
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = 1;
  a.pitch = dst_pitch(ctx);
  a.tiles_x = (int)((p->nx + C::BX - 1) / C::BX);
  a.tiles_y = (int)((p->ny + C::BY - 1) / C::BY);
  a.tiles_z = 1;
  a.a_words = reinterpret_cast<const uint4*>(p->dev.a_words);
  a.meta = p->dev.meta_words;
  a.w = p->dev.w_dense;
  a.status = p->dev.status;
  a.wait_cycles = wait_limit_cycles();
  a.out_tf32 = ctx.out_tf32 ? 1 : 0;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  a.use_tma = make_src_map(&map, ctx, 1, C::SX, C::SY, 1) ? 1 : 0;
  if (!a.use_tma && src_pitch(ctx) != p->nx) return cudaErrorNotSupported;  // the loader reads packed rows
  const long long ntiles = (long long)a.tiles_x * a.tiles_y;
  if (ntiles > (1LL << 31) - 1) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>(ntiles, (long long)occ * ctx.sms);
  return launch_pdl(kern, grid, C::kThreads, C::kSmemBytes, ctx.stream, map, a);
}

// 1-D: tiles of 16 rows of 128 points (8 warps x 2 rows), chunks loaded by
// TMA through a view of the array as rows of 8 floats.
template <class C, bool RIN>
cudaError_t launch_wide1d_k(const LaunchCtx& ctx) {
  const spider_plan_t* p = ctx.plan;
  auto kern = wide1d_kernel<C, RIN>;
  static std::mutex mu;
  static int occ_by_dev[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int occ;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (occ_by_dev[dev] == 0) {
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
      if (err != cudaSuccess) return err;
      int o = 0;
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, C::kThreads, C::kSmemBytes);
      if (err != cudaSuccess) return err;
      occ_by_dev[dev] = std::max(o, 1);
    }
    occ = occ_by_dev[dev];
  }
  StepArgs a;
  a.src = ctx.src;
  a.dst = ctx.dst;
  a.nx = p->nx;
  a.ny = 1;
  a.nz = 1;
  a.pitch = dst_pitch(ctx);
  a.tiles_x = (int)((p->nx + C::NT - 1) / C::NT);
  a.tiles_y = 1;
  a.tiles_z = 1;
  a.a_words = reinterpret_cast<const uint4*>(p->dev.a_words);
  a.meta = p->dev.meta_words;
  a.w = p->dev.w_dense;
  a.status = p->dev.status;
  a.wait_cycles = wait_limit_cycles();
  a.out_tf32 = ctx.out_tf32 ? 1 : 0;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  // the array as rows of 8 floats (needs a length that is a multiple of 8;
  // a padded source is src_pitch long, its tail beyond nx zero)
  const int64_t len = src_pitch(ctx);
  a.use_tma = (len % 8 == 0 && make_tensor_map(&map, ctx.src, 8, len / 8, 1, 8, C::kBoxRows, 1)) ? 1 : 0;
  if (!a.use_tma && len != p->nx) return cudaErrorNotSupported;  // the loader reads nx points
  const int grid = (int)std::min<long long>(a.tiles_x, (long long)occ * ctx.sms);
  return launch_pdl(kern, grid, C::kThreads, C::kSmemBytes, ctx.stream, map, a);
}

// 1-D fused passes: tiles of 14 output rows of 128 points, every level on
// 16 rows (8 warps x 2); needs the 8-float TMA view (length a multiple of 8).
template <class C, bool RIN>
cudaError_t launch_wide1d_fused_k(const LaunchCtx& ctx) {
  const spider_plan_t* p = ctx.plan;
  const int64_t len = src_pitch(ctx);  // a padded source: its tail beyond nx is zero
  if (len % 8 != 0) return cudaErrorNotSupported;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  if (!make_tensor_map(&map, ctx.src, 8, len / 8, 1, 8, C::kBoxRows, 1)) return cudaErrorNotSupported;
  auto kern = wide1d_fused_kernel<C, RIN>;
  static std::mutex mu;
  static int occ_by_dev[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int occ;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (occ_by_dev[dev] == 0) {
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
      if (err != cudaSuccess) return err;
      int o = 0;
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, C::kThreads, C::kSmemBytes);
      if (err != cudaSuccess) return err;
      occ_by_dev[dev] = std::max(o, 1);
    }
    occ = occ_by_dev[dev];
  }
  StepArgs a;
  a.src = ctx.src;
  a.dst = ctx.dst;
  a.nx = p->nx;
  a.ny = 1;
  a.nz = 1;
  a.pitch = dst_pitch(ctx);
  a.tiles_x = (int)((p->nx + C::NT - 1) / C::NT);
  a.tiles_y = 1;
  a.tiles_z = 1;
  a.a_words = reinterpret_cast<const uint4*>(p->dev.a_words);
  a.meta = p->dev.meta_words;
  a.w = p->dev.w_dense;
  a.status = p->dev.status;
  a.wait_cycles = wait_limit_cycles();
  a.use_tma = 1;
  a.out_tf32 = ctx.out_tf32 ? 1 : 0;
  const int grid = (int)std::min<long long>(a.tiles_x, (long long)occ * ctx.sms);
  return launch_pdl(kern, grid, C::kThreads, C::kSmemBytes, ctx.stream, map, a);
}

template <int R>
cudaError_t launch_wide1d_fused_r(int T, const LaunchCtx& ctx) {
  auto go = [&](auto cfg) -> cudaError_t {
    using C = decltype(cfg);
    return ctx.in_tf32 ? launch_wide1d_fused_k<C, false>(ctx) : launch_wide1d_fused_k<C, true>(ctx);
  };
  switch (T) {
    case 2: return go(Wide1DFusedCfg<R, 2, 14, 8>());
    case 3: return go(Wide1DFusedCfg<R, 3, 14, 8>());
    case 4: return go(Wide1DFusedCfg<R, 4, 14, 8>());
    default: return cudaErrorNotSupported;
  }
}

// 2-D: 8 warps x 8 rows x 128 columns, registers for 2 CTAs per SM; 1-D:
// tiles of 16 rows of 128 points.
template <int R>
cudaError_t launch_wide_r(int cls, const LaunchCtx& ctx) {
  if (cls == 2) {
    if constexpr (R <= kMaxR) return cudaErrorNotSupported;  // 2-D radius 1..3: the 8-output layout
    using C = WideCfg<R, R, 8, 8, 2>;
    return ctx.in_tf32 ? launch_wide_k<C, false>(ctx) : launch_wide_k<C, true>(ctx);
  }
  if (cls == 1) {
    using C = Wide1DCfg<R, 2, 8>;
    return ctx.in_tf32 ? launch_wide1d_k<C, false>(ctx) : launch_wide1d_k<C, true>(ctx);
  }
  return cudaErrorNotSupported;
}

}  // namespace spider
