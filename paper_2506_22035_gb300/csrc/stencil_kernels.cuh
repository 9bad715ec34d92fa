// One fused stencil time step on GB300: TMA-staged halo tiles, the SPIDER
// sparse tensor-core product (and the dense tensor-core and CUDA-core
// comparators on the same tiling), coalesced write-back.
//
// Tiling (Sec. 3.3.1).  A CTA owns a block tile of BZ x BY x BX outputs
// (planes x rows x columns) and stages the input box
// (BZ + 2rz) x (BY + 2ry) x (BX + 8) in shared memory with one TMA tile load;
// points outside the grid arrive as zeros (zero Dirichlet halo).  CTAs are
// persistent and double-buffer their tiles: the load of the next tile is in
// flight while the current one is computed.  Each warp owns a warp tile of
// 1 plane x H rows x 64 columns; at the MMA level one m16n8k16 (TF32) covers
// two output rows x 8 segments of 8 outputs.
//
// Kernel matrix in registers (Sec. 3.3.1): the compressed A operands and their
// metadata are loaded once per CTA (per dz plane in 3-D) with coalesced
// 16-byte loads from the plan's packed buffers (Sec. 3.3.2) and stay in
// registers.
//
// Row swap on the fly (Sec. 3.2): lane (g, q) takes the window of segment g
// at positions 4*sigma(q) .. 4*sigma(q)+3 with one 16-byte shared-memory load;
// which of those values meets which kernel coefficient is fixed by the
// plan's strided permutation, so the swap costs no instruction: it is only
// the choice of address.  Every B fragment of input row j feeds all output
// row pairs that row j reaches.
#pragma once

#include <cstdint>
#include <cuda.h>

#include "device_common.cuh"
#include "spider_internal.h"

namespace spider {

enum class Mode : int { SpTF32 = 0, SpF16x2 = 1, SpBF16x3 = 2, DenseTF32 = 3, CudaCore = 4 };

struct StepArgs {
  const float* src;        // source grid (generic loader only)
  float* dst;              // destination grid
  int64_t nx, ny, nz;
  int64_t pitch;           // destination row pitch in floats (>= nx); planes are ny * pitch apart
  int tiles_x, tiles_y, tiles_z;
  const uint4* a_words;    // packed A operands
  const uint32_t* meta;    // packed metadata
  const float* w;          // coefficient cube (CUDA-core mode), float32
  int* status;             // device status word
  int use_tma;             // 1: TMA tile loads from `tmap`; 0: cooperative loads from src
  int out_tf32;            // TF32 modes: store the outputs rounded to TF32 (the grid feeds another step)
};

// TF32 modes round every B operand to TF32 (round to nearest, ties to even)
// before the MMA.  A grid written for another step of the same run can hold
// its values already rounded that way: the reading step then passes the raw
// bits to the MMA (kernel template flag RIN = false) and gets bit-identical
// results, at one rounding per stored point instead of one per operand
// load (each input value is loaded about 2.75 times by overlapping windows
// and warp tiles).
__host__ __device__ constexpr bool is_tf32_mode(Mode m) { return m == Mode::SpTF32 || m == Mode::DenseTF32; }

template <int N>
__device__ __forceinline__ void round_tf32_inplace(float (&acc)[N][4]) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = __uint_as_float(cvt_tf32(acc[i][j]));
}

template <int RZ_, int RY_, int RX_, int WZ_, int WY_, int WX_, int H_>
struct TileCfg {
  static constexpr int RZ = RZ_, RY = RY_, RX = RX_, WZ = WZ_, WY = WY_, WX = WX_, H = H_;
  static constexpr int BZ = WZ, BY = WY * H, BX = WX * 64;
  static constexpr int SZ = BZ + 2 * RZ, SY = BY + 2 * RY, SX = BX + 2 * kHaloX;
  static constexpr int kThreads = WZ * WY * WX * 32;
  static constexpr int kStageFloats = SZ * SY * SX;
  static constexpr int kStageBytes = kStageFloats * 4;
  static constexpr int kStageStride = (kStageBytes + 1023) / 1024 * 1024;
  static constexpr int kSmemBytes = 2 * kStageStride + 1024 /*alignment slack*/ + 64 /*barriers*/;
  static constexpr int NA = 2 * RY + 2;  // A indices per plane
  static_assert(H % 2 == 0, "warp tile height must be even");
  static_assert(SX <= 256 && SY <= 256 && SZ <= 256, "TMA box dimension limit");
  static_assert(RX <= kHaloX && RX <= kMaxR, "radius too large for the 16-wide window");
};

// --------------------------------------------------------------------------
// Per-warp compute for one dz plane.  `row0` points at this lane's first
// input value (plane, first input row of the warp tile); rows are SX floats
// apart.  acc[pp] accumulates output rows (2pp, 2pp+1) of the warp tile.

// ROUND = false when the source already holds TF32 values (fused
// intermediate levels), so the 13 low mantissa bits are already zero.
// Only the A indices AMIN..AMAX are applied (all of them by default); row
// pair pp reads input rows 2pp + AMIN .. 2pp + AMAX, so the rows loaded are
// AMIN .. H - 2 + AMAX.
template <class C, int SP, bool ROUND, int JJ, int AMIN, int AMAX>
__device__ __forceinline__ void sp_tf32_row(uint32_t addr, const uint4 (&A)[C::NA], const uint32_t (&E)[C::NA],
                                            float (&acc)[C::H / 2][4]) {
  const float4 v = lds128_at<JJ * SP * 4>(addr);
  const uint32_t b[4] = {ROUND ? cvt_tf32(v.x) : __float_as_uint(v.x), ROUND ? cvt_tf32(v.y) : __float_as_uint(v.y),
                         ROUND ? cvt_tf32(v.z) : __float_as_uint(v.z), ROUND ? cvt_tf32(v.w) : __float_as_uint(v.w)};
#pragma unroll
  for (int pp = 0; pp < C::H / 2; ++pp) {
    const int a = JJ - 2 * pp;
    if (a >= AMIN && a <= AMAX) mma_sp_tf32(acc[pp], A[a], E[a], b);
  }
  if constexpr (JJ + 1 <= C::H - 2 + AMAX) sp_tf32_row<C, SP, ROUND, JJ + 1, AMIN, AMAX>(addr, A, E, acc);
}

template <class C, int SP = C::SX, bool ROUND = true, int AMIN = 0, int AMAX = C::NA - 1>
__device__ __forceinline__ void plane_sp_tf32(const float* row0, const uint4 (&A)[C::NA],
                                              const uint32_t (&E)[C::NA], float (&acc)[C::H / 2][4]) {
  sp_tf32_row<C, SP, ROUND, AMIN, AMIN, AMAX>(smem_u32(row0), A, E, acc);
}

template <class C, int SP, bool ROUND, int JJ, int AMIN, int AMAX>
__device__ __forceinline__ void dense_tf32_row(uint32_t addr, const uint4 (&A)[C::NA][2], float (&acc)[C::H / 2][4]) {
  const float4 v = lds128_at<JJ * SP * 4>(addr);
  const uint32_t b[4] = {ROUND ? cvt_tf32(v.x) : __float_as_uint(v.x), ROUND ? cvt_tf32(v.y) : __float_as_uint(v.y),
                         ROUND ? cvt_tf32(v.z) : __float_as_uint(v.z), ROUND ? cvt_tf32(v.w) : __float_as_uint(v.w)};
#pragma unroll
  for (int pp = 0; pp < C::H / 2; ++pp) {
    const int a = JJ - 2 * pp;
    if (a >= AMIN && a <= AMAX) {
      mma_tf32(acc[pp], A[a][0], b[0], b[1]);
      mma_tf32(acc[pp], A[a][1], b[2], b[3]);
    }
  }
  if constexpr (JJ + 1 <= C::H - 2 + AMAX) dense_tf32_row<C, SP, ROUND, JJ + 1, AMIN, AMAX>(addr, A, acc);
}

template <class C, int SP = C::SX, bool ROUND = true, int AMIN = 0, int AMAX = C::NA - 1>
__device__ __forceinline__ void plane_dense_tf32(const float* row0, const uint4 (&A)[C::NA][2],
                                                 float (&acc)[C::H / 2][4]) {
  dense_tf32_row<C, SP, ROUND, AMIN, AMIN, AMAX>(smem_u32(row0), A, acc);
}

// 3-D star stencils: a dz plane other than the centre holds only the
// coefficient w[dz][0][0], i.e. kernel row dy = 0, which is A index ry for
// the top output row and ry + 1 for the bottom one; the other A operands of
// that plane are zero and are skipped (one MMA per input row instead of up
// to ry + 1, and H input rows instead of H + 2ry).
template <class C, int SP, bool ROUND>
__device__ __forceinline__ void plane_sp_tf32_centre(const float* row0, const uint4 (&A)[C::NA],
                                                     const uint32_t (&E)[C::NA], float (&acc)[C::H / 2][4]) {
  plane_sp_tf32<C, SP, ROUND, C::RY, C::RY + 1>(row0, A, E, acc);
}
template <class C, int SP, bool ROUND>
__device__ __forceinline__ void plane_dense_tf32_centre(const float* row0, const uint4 (&A)[C::NA][2],
                                                        float (&acc)[C::H / 2][4]) {
  plane_dense_tf32<C, SP, ROUND, C::RY, C::RY + 1>(row0, A, acc);
}

// Split precisions (FP16 hi/lo with the lo parts scaled by 2^11, or BF16
// hi/lo): value v = hi + lo.  Per pair of input rows (j, j+1) one k32 MMA
// takes hi*hi for both rows, and per row one k32 MMA takes
// hi(w)*lo(v) + lo(w)*hi(v).
template <class C, bool BF16>
__device__ __forceinline__ void split4(const float4& v, uint32_t (&hi)[2], uint32_t (&lo)[2]) {
  if (BF16) {
    hi[0] = pack_bf162(v.x, v.y);
    hi[1] = pack_bf162(v.z, v.w);
    const float2 h01 = unpack_bf162(hi[0]), h23 = unpack_bf162(hi[1]);
    lo[0] = pack_bf162(v.x - h01.x, v.y - h01.y);
    lo[1] = pack_bf162(v.z - h23.x, v.w - h23.y);
  } else {
    hi[0] = pack_half2(v.x, v.y);
    hi[1] = pack_half2(v.z, v.w);
    const float2 h01 = unpack_half2(hi[0]), h23 = unpack_half2(hi[1]);
    lo[0] = pack_half2((v.x - h01.x) * 2048.0f, (v.y - h01.y) * 2048.0f);
    lo[1] = pack_half2((v.z - h23.x) * 2048.0f, (v.w - h23.y) * 2048.0f);
  }
}

template <class C, bool BF16>
__device__ __forceinline__ void mma_k32(float (&d)[4], const uint4& a, uint32_t e, uint32_t b0, uint32_t b1,
                                        uint32_t b2, uint32_t b3) {
  if (BF16) mma_sp_bf16_k32(d, a, e, b0, b1, b2, b3);
  else mma_sp_f16_k32(d, a, e, b0, b1, b2, b3);
}

template <class C, bool BF16, int SP, int JJ>
__device__ __forceinline__ void sp_split_rows(uint32_t addr, const uint4 (&Am)[C::RY + 1],
                                              const uint32_t (&Em)[C::RY + 1], const uint4 (&Ac)[C::NA],
                                              const uint32_t (&Ec)[C::NA], float (&accM)[C::H / 2][4],
                                              float (&accC)[C::H / 2][4]) {
  uint32_t hi0[2], lo0[2], hi1[2], lo1[2];
  split4<C, BF16>(lds128_at<JJ * SP * 4>(addr), hi0, lo0);
  split4<C, BF16>(lds128_at<(JJ + 1) * SP * 4>(addr), hi1, lo1);
#pragma unroll
  for (int pp = 0; pp < C::H / 2; ++pp) {
    const int a0 = JJ - 2 * pp;  // even; rows JJ, JJ+1 use A indices a0, a0+1
    if (a0 >= 0 && a0 + 1 < C::NA) {
      mma_k32<C, BF16>(accM[pp], Am[a0 / 2], Em[a0 / 2], hi0[0], hi0[1], hi1[0], hi1[1]);
      mma_k32<C, BF16>(accC[pp], Ac[a0], Ec[a0], lo0[0], lo0[1], hi0[0], hi0[1]);
      mma_k32<C, BF16>(accC[pp], Ac[a0 + 1], Ec[a0 + 1], lo1[0], lo1[1], hi1[0], hi1[1]);
    }
  }
  if constexpr (JJ + 2 < C::H + 2 * C::RY) sp_split_rows<C, BF16, SP, JJ + 2>(addr, Am, Em, Ac, Ec, accM, accC);
}

template <class C, bool BF16, int SP = C::SX>
__device__ __forceinline__ void plane_sp_split(const float* row0, const uint4 (&Am)[C::RY + 1],
                                               const uint32_t (&Em)[C::RY + 1], const uint4 (&Ac)[C::NA],
                                               const uint32_t (&Ec)[C::NA], float (&accM)[C::H / 2][4],
                                               float (&accC)[C::H / 2][4]) {
  sp_split_rows<C, BF16, SP, 0>(smem_u32(row0), Am, Em, Ac, Ec, accM, accC);
}

// --------------------------------------------------------------------------
template <class C, Mode MODE, bool RIN = true, bool STAR = false>
__global__ void __launch_bounds__(C::kThreads)
    stencil_step_kernel(const __grid_constant__ CUtensorMap tmap, const StepArgs args) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t base_u32 = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024 - (base_u32 & 1023)) & 1023);
  auto stage = [&](int s) { return reinterpret_cast<float*>(smem + s * C::kStageStride); };
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * C::kStageStride);

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int wx = warp % C::WX, wy = (warp / C::WX) % C::WY, wz = warp / (C::WX * C::WY);
  const int ntiles = args.tiles_x * args.tiles_y * args.tiles_z;
  const bool use_tma = args.use_tma != 0;

  auto coords = [&](int t, int& x0, int& y0, int& z0) {
    const int tx = t % args.tiles_x;
    const int ty = (t / args.tiles_x) % args.tiles_y;
    const int tz = t / (args.tiles_x * args.tiles_y);
    x0 = tx * C::BX;
    y0 = ty * C::BY;
    z0 = tz * C::BZ;
  };
  auto issue = [&](int t, int s) {
    int x0, y0, z0;
    coords(t, x0, y0, z0);
    mbar_arrive_expect_tx(&full[s], C::kStageBytes);
    tma_load_3d(stage(s), &tmap, &full[s], x0 - kHaloX, y0 - C::RY, z0 - C::RZ);
  };

  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    fence_mbar_init();
  }
  // the previous step's kernel may still be running: wait before reading the
  // source grid or writing the destination (which it may be reading)
  griddep_wait();
  griddep_launch_dependents();
  __syncthreads();
  if (use_tma && tid == 0) {
    if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
    if ((int)(blockIdx.x + gridDim.x) < ntiles) issue(blockIdx.x + gridDim.x, 1);
  }

  // Kernel-matrix operands resident in registers (2-D: for the whole kernel).
  constexpr int NA = C::NA;
  constexpr int CPP = (MODE == Mode::SpF16x2 || MODE == Mode::SpBF16x3) ? (C::RY + 1) + NA : NA;
  uint4 A[NA];
  uint32_t E[NA];
  uint4 Ad[NA][2];
  uint4 Am[C::RY + 1];
  uint32_t Em[C::RY + 1];
  float W[(2 * C::RY + 1) * (2 * C::RX + 1)];
  auto load_operands = [&](int dzi) {
    if (MODE == Mode::SpTF32) {
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        if (STAR && dzi != C::RZ && a != C::RY && a != C::RY + 1) continue;  // zero operands
        A[a] = args.a_words[(size_t)(dzi * CPP + a) * 32 + lane];
        E[a] = args.meta[(size_t)(dzi * CPP + a) * 32 + lane];
      }
    } else if (MODE == Mode::DenseTF32) {
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        if (STAR && dzi != C::RZ && a != C::RY && a != C::RY + 1) continue;
        Ad[a][0] = args.a_words[((size_t)(dzi * NA + a) * 32 + lane) * 2 + 0];
        Ad[a][1] = args.a_words[((size_t)(dzi * NA + a) * 32 + lane) * 2 + 1];
      }
    } else if (MODE == Mode::SpF16x2 || MODE == Mode::SpBF16x3) {
#pragma unroll
      for (int c = 0; c <= C::RY; ++c) {
        Am[c] = args.a_words[(size_t)(dzi * CPP + c) * 32 + lane];
        Em[c] = args.meta[(size_t)(dzi * CPP + c) * 32 + lane];
      }
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        A[a] = args.a_words[(size_t)(dzi * CPP + C::RY + 1 + a) * 32 + lane];
        E[a] = args.meta[(size_t)(dzi * CPP + C::RY + 1 + a) * 32 + lane];
      }
    } else {
      constexpr int NW = (2 * C::RY + 1) * (2 * C::RX + 1);
#pragma unroll
      for (int i = 0; i < NW; ++i) W[i] = args.w[(size_t)dzi * NW + i];
    }
  };
  if (C::RZ == 0) load_operands(0);

  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int s = it & 1;
    float* S = stage(s);
    int x0, y0, z0;
    coords(t, x0, y0, z0);
    if (use_tma) {
      const bool ok = mbar_wait_bounded(&full[s], (it >> 1) & 1, args.status);
      if (!__syncthreads_and(ok)) break;
    } else {
      // Asynchronous copies (grids whose rows are not 16-byte aligned).
      load_box_async(args.src, args.nx, args.ny, args.nz, (int64_t)x0 - kHaloX, (int64_t)y0 - C::RY,
                     (int64_t)z0 - C::RZ, C::SX, C::SY, C::SZ, S, warp, C::kThreads / 32, lane);
      __syncthreads();
    }

    const int64_t z = (int64_t)z0 + wz;
    const int ybase = y0 + wy * C::H;
    const int xbase = x0 + wx * 64;
    if (MODE == Mode::CudaCore) {
      float acc[C::H][2];
#pragma unroll
      for (int i = 0; i < C::H; ++i) acc[i][0] = acc[i][1] = 0.f;
#pragma unroll 1
      for (int dzi = 0; dzi < 2 * C::RZ + 1; ++dzi) {
        if (C::RZ != 0) load_operands(dzi);
        const float* pl = S + (size_t)(wz + dzi) * C::SY * C::SX + (size_t)(wy * C::H) * C::SX + wx * 64 +
                          kHaloX + lane - C::RX;
#pragma unroll
        for (int jj = 0; jj < C::H + 2 * C::RY; ++jj) {
          float in0[2 * C::RX + 1], in1[2 * C::RX + 1];
#pragma unroll
          for (int k = 0; k < 2 * C::RX + 1; ++k) {
            in0[k] = pl[jj * C::SX + k];
            in1[k] = pl[jj * C::SX + 32 + k];
          }
#pragma unroll
          for (int yy = 0; yy < C::H; ++yy) {
            const int dy = jj - C::RY - yy;
            if (dy >= -C::RY && dy <= C::RY) {
#pragma unroll
              for (int k = 0; k < 2 * C::RX + 1; ++k) {
                const float wv = W[(dy + C::RY) * (2 * C::RX + 1) + k];
                acc[yy][0] = fmaf(wv, in0[k], acc[yy][0]);
                acc[yy][1] = fmaf(wv, in1[k], acc[yy][1]);
              }
            }
          }
        }
      }
      if (z < args.nz) {
        float* o = args.dst + (z * args.ny + ybase) * args.pitch + xbase + lane;
        const int pitch = (int)args.pitch;
        const int ylim = (int)(args.ny - ybase < C::H ? args.ny - ybase : C::H);
        const int xlim = (int)(args.nx - xbase < 64 ? args.nx - xbase : 64);
#pragma unroll
        for (int yy = 0; yy < C::H; ++yy) {
          if (yy < ylim) {
#pragma unroll
            for (int c = 0; c < 2; ++c)
              if (lane + 32 * c < xlim) o[(size_t)yy * pitch + 32 * c] = acc[yy][c];
          }
        }
      }
    } else {
      float acc[C::H / 2][4];
      float accC[C::H / 2][4];
#pragma unroll
      for (int i = 0; i < C::H / 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = accC[i][j] = 0.f;
#pragma unroll 1
      for (int dzi = 0; dzi < 2 * C::RZ + 1; ++dzi) {
        if (C::RZ != 0) load_operands(dzi);
        const float* row0 = S + (size_t)(wz + dzi) * C::SY * C::SX + (size_t)(wy * C::H) * C::SX + wx * 64 +
                            8 * g + 4 * ((q == 1) ? 2 : (q == 2) ? 1 : q);
        const bool centre_only = STAR && dzi != C::RZ;
        if (MODE == Mode::SpTF32) {
          if (centre_only) plane_sp_tf32_centre<C, C::SX, RIN>(row0, A, E, acc);
          else plane_sp_tf32<C, C::SX, RIN>(row0, A, E, acc);
        } else if (MODE == Mode::DenseTF32) {
          if (centre_only) plane_dense_tf32_centre<C, C::SX, RIN>(row0, Ad, acc);
          else plane_dense_tf32<C, C::SX, RIN>(row0, Ad, acc);
        } else if (MODE == Mode::SpF16x2) {
          plane_sp_split<C, false>(row0, Am, Em, A, E, acc, accC);
        } else {
          plane_sp_split<C, true>(row0, Am, Em, A, E, acc, acc);
        }
      }
      if (MODE == Mode::SpF16x2) {
#pragma unroll
        for (int i = 0; i < C::H / 2; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(accC[i][j], 1.0f / 2048.0f, acc[i][j]);
      }
      if (is_tf32_mode(MODE) && args.out_tf32) round_tf32_inplace(acc);
      if (z < args.nz) {
        float* o = args.dst + (z * args.ny + ybase) * args.pitch + xbase + 16 * q + g;
        const int pitch = (int)args.pitch;
        if (ybase + C::H <= args.ny && xbase + 64 <= args.nx) {
          // interior warp tile: no bounds checks
#pragma unroll
          for (int pp = 0; pp < C::H / 2; ++pp) {
#pragma unroll
            for (int sr = 0; sr < 2; ++sr) {
              float* orow = o + (size_t)(2 * pp + sr) * pitch;
              orow[0] = acc[pp][2 * sr];
              orow[8] = acc[pp][2 * sr + 1];
            }
          }
        } else {
          const int ylim = (int)(args.ny - ybase < C::H ? args.ny - ybase : C::H);
          const int xlim = (int)(args.nx - xbase < 64 ? args.nx - xbase : 64);
#pragma unroll
          for (int pp = 0; pp < C::H / 2; ++pp) {
#pragma unroll
            for (int sr = 0; sr < 2; ++sr) {
              if (2 * pp + sr < ylim) {
#pragma unroll
                for (int c = 0; c < 2; ++c)
                  if (16 * q + 8 * c + g < xlim) o[(size_t)(2 * pp + sr) * pitch + 8 * c] = acc[pp][2 * sr + c];
              }
            }
          }
        }
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
  // Loads still in flight after an early exit: wait for them (bounded) so no
  // copy targets shared memory of a finished CTA.
  if (use_tma && tid == 0) {
    for (int k = 0; k < 2; ++k) {
      const int t = blockIdx.x + (it + k) * gridDim.x;
      if (t < ntiles) {
        (void)mbar_wait_bounded(&full[(it + k) & 1], ((it + k) >> 1) & 1, args.status);
      }
    }
  }
}

}  // namespace spider
