// Temporal fusion for 2-D stencils: T time steps per pass over HBM.
//
// A CTA loads one input box with a halo of T*r rows and 4*T columns on each
// side (TMA, zero outside the grid), then computes T levels in shared memory:
// level t covers the output tile grown by r*(T-t) rows and 4*(T-t) columns on
// each side, reading level t-1.  Points of an intermediate level that lie
// outside the grid are stored as 0, so every fused step sees the zero
// Dirichlet halo exactly as separate steps would; only level T is written to
// HBM.  Each level is computed with the same per-warp unit as the one-step
// kernel (H rows x 8 segments of 8 outputs), so results are bit-identical to
// T separate steps -- except for the FP16/BF16 splits at odd r: their hi*hi
// MMA adds two input rows at once, and an intermediate level that starts on
// an odd row groups those products differently (same accuracy; the last bits
// may differ).  The input buffer is free once level 1 has read it: the next
// tile's TMA load is issued then and overlaps levels 2..T.
//
// Tile heights are chosen so that every level splits into the same number of
// warp units (level 1 is 64 rows; BY = 64 - 2r(T-1)), keeping the warps
// balanced between the level barriers.  Intermediate levels are stored with an
// XOR swizzle (bit 3 of the column flips in odd 32-column blocks), which
// spreads the fragment-order stores over all 32 banks and keeps every 4-float
// chunk contiguous for the 16-byte loads of the next level.
#pragma once

#include "stencil_kernels.cuh"

namespace spider {

template <int R_, int T_, int BY_, int BX_, int H_, int NW_, int MINB_ = 1, int INS_ = 1, int VEC_ = 0>
struct FuseCfg {
  static constexpr int RZ = 0, RY = R_, RX = R_, T = T_, BY = BY_, BX = BX_, H = H_, NW = NW_;
  static constexpr int kMinBlocks = MINB_;  // CTAs per SM the register budget must allow
  static constexpr int kInStages = INS_;    // input boxes in flight: 1, or 2 (prefetch a whole tile ahead)
  static constexpr bool kVecStore = VEC_ != 0;  // final level: 16-byte stores after a quad transpose
  static constexpr int NA = 2 * RY + 2;
  static constexpr int kThreads = NW * 32;
  // level t: 0 = input box, T = output tile
  __host__ __device__ static constexpr int rows(int t) { return BY + 2 * RY * (T - t); }
  __host__ __device__ static constexpr int width(int t) { return BX + 8 * (T - t); }
  __host__ __device__ static constexpr int segs(int t) { return width(t) / 8; }
  // Row pitch in shared memory: the TMA box is dense (level 0); intermediate
  // levels round up to 16 columns so the swizzle stays inside the row.
  __host__ __device__ static constexpr int pitch(int t) { return t == 0 ? width(0) : (width(t) + 15) / 16 * 16; }
  __host__ __device__ static constexpr int align1k(int b) { return (b + 1023) / 1024 * 1024; }
  static constexpr int kInBytes = rows(0) * width(0) * 4;
  static constexpr int kInStride = align1k(kInBytes);
  static constexpr int kPStride = T >= 2 ? align1k(rows(1) * pitch(1) * 4) : 0;  // odd levels
  static constexpr int kQStride = T >= 3 ? align1k(rows(2) * pitch(2) * 4) : 0;  // even levels
  static constexpr int kSmemBytes = kInStages * kInStride + kPStride + kQStride + 1024 + 64;
  // T = 1 describes a one-level pass on a fused tile's geometry (the batch
  // queue's single-step passes of a job that otherwise takes two steps per
  // pass); the stand-alone fused kernel is launched for T >= 2 only
  static_assert(T >= 1, "at least one level");
  static_assert(BX % 8 == 0 && BX >= 64, "tile width");
  static_assert(width(0) <= 256 && rows(0) <= 256, "TMA box dimension limit");
  static_assert(H % 2 == 0 && rows(T) >= H, "warp tile height");
  static_assert(RX <= kHaloX, "radius too large for the 16-wide window");
};

__device__ __forceinline__ int swz(int col) { return col ^ (((col >> 5) & 1) << 3); }

// 4 x 4 transpose across the four lanes of a warp that share q and have
// g = 4a .. 4a + 3 (lanes 4 apart; i = g mod 4).  Lane i holds v_c for the
// four (row, segment) combinations c of its output g; afterwards it holds,
// for combination i, the outputs of the four lanes in order (four consecutive
// x positions).  Two butterfly rounds of two shuffles each.
__device__ __forceinline__ void quad_transpose(float& v0, float& v1, float& v2, float& v3, int i) {
  const bool b0 = (i & 1) != 0, b1 = (i & 2) != 0;
  float t0 = b0 ? v0 : v1, t1 = b0 ? v2 : v3;
  t0 = __shfl_xor_sync(0xffffffffu, t0, 4);
  t1 = __shfl_xor_sync(0xffffffffu, t1, 4);
  if (b0) { v0 = t0; v2 = t1; } else { v1 = t0; v3 = t1; }
  float u0 = b1 ? v0 : v2, u1 = b1 ? v1 : v3;
  u0 = __shfl_xor_sync(0xffffffffu, u0, 8);
  u1 = __shfl_xor_sync(0xffffffffu, u1, 8);
  if (b1) { v0 = u0; v1 = u1; } else { v2 = u0; v3 = u1; }
}

struct FusedCtx {
  const StepArgs* args;
  int x0, y0;
  int lane, warp, g, q;
};

// One level LV: reads `src` (level LV-1), writes `dst` (level LV, shared
// memory) or the output grid (LV == T).
template <class F, Mode MODE, bool RIN, int LV>
__device__ __forceinline__ void fused_level(const FusedCtx& c, const float* src, float* dst, const uint4 (&A)[F::NA],
                                            const uint32_t (&E)[F::NA], const uint4 (&Ad)[F::NA][2],
                                            const uint4 (&Am)[F::RY + 1], const uint32_t (&Em)[F::RY + 1],
                                            const float (&W)[(2 * F::RY + 1) * (2 * F::RX + 1)]) {
  constexpr int SP = F::pitch(LV - 1), DP = F::pitch(LV);
  constexpr int R = F::rows(LV), S = F::segs(LV);
  constexpr int NR = (R + F::H - 1) / F::H, NS = (S + 7) / 8, U = NR * NS;
  constexpr int GY = F::RY * (F::T - LV), GX = 4 * (F::T - LV);  // level LV origin = tile origin - (GY, GX)
  const StepArgs& args = *c.args;
  for (int u = c.warp; u < U; u += F::NW) {
    const int r0 = min((u / NS) * F::H, R - F::H);
    const int s0 = min((u % NS) * 8, S - 8);
    if (MODE == Mode::CudaCore) {
      // lane l: columns 2l, 2l + 1 of the unit, inputs loaded as 8-byte
      // pairs (v[e] = source column 8 s0 + 2l + e; the swizzle keeps pairs
      // adjacent), as in the one-step kernel
      constexpr int E0 = (4 - F::RX) / 2, E1 = (5 + F::RX) / 2;
      float acc[F::H][2];
#pragma unroll
      for (int i = 0; i < F::H; ++i) acc[i][0] = acc[i][1] = 0.f;
      const float* pl = src + r0 * SP;
      const int cb = 8 * s0 + 2 * c.lane;  // first column this lane's pairs start at
#pragma unroll
      for (int jj = 0; jj < F::H + 2 * F::RY; ++jj) {
        float v[10];
#pragma unroll
        for (int m = E0; m <= E1; ++m) {
          const int col = cb + 2 * m;
          const float2 t = *reinterpret_cast<const float2*>(pl + jj * SP + (LV >= 2 ? swz(col) : col));
          v[2 * m] = t.x;
          v[2 * m + 1] = t.y;
        }
#pragma unroll
        for (int yy = 0; yy < F::H; ++yy) {
          const int dy = jj - F::RY - yy;
          if (dy >= -F::RY && dy <= F::RY) {
#pragma unroll
            for (int k = 0; k < 2 * F::RX + 1; ++k) {
              const float wv = W[(dy + F::RY) * (2 * F::RX + 1) + k];
              acc[yy][0] = fmaf(wv, v[4 - F::RX + k], acc[yy][0]);
              acc[yy][1] = fmaf(wv, v[5 - F::RX + k], acc[yy][1]);
            }
          }
        }
      }
      const int gy0 = c.y0 - GY + r0, gx0 = c.x0 - GX + 8 * s0;  // unit origin in the grid
      const bool interior = gy0 >= 0 && gy0 + F::H <= (int)args.ny && gx0 >= 0 && gx0 + 64 <= (int)args.nx;
      if (LV < F::T) {
        float* d = dst + r0 * DP;
        const int p0 = swz(8 * s0 + 2 * c.lane);  // the pair stays adjacent after the swizzle
#pragma unroll
        for (int yy = 0; yy < F::H; ++yy)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const bool in = interior || ((unsigned)(gy0 + yy) < (unsigned)args.ny &&
                                         (unsigned)(gx0 + 2 * c.lane + h) < (unsigned)args.nx);
            d[yy * DP + p0 + h] = in ? acc[yy][h] : 0.f;
          }
      } else {
        float* o = args.dst + (int64_t)gy0 * args.pitch + gx0 + 2 * c.lane;
#pragma unroll
        for (int yy = 0; yy < F::H; ++yy)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const bool in = interior || ((unsigned)(gy0 + yy) < (unsigned)args.ny &&
                                         (unsigned)(gx0 + 2 * c.lane + h) < (unsigned)args.nx);
            if (in) o[(int64_t)yy * args.pitch + h] = acc[yy][h];
          }
      }
    } else {
      float acc[F::H / 2][4];
      float accC[F::H / 2][4];
#pragma unroll
      for (int i = 0; i < F::H / 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = accC[i][j] = 0.f;
      const int ccol = 8 * (s0 + c.g) + 4 * ((c.q == 1) ? 2 : (c.q == 2) ? 1 : c.q);
      const float* row0 = src + r0 * SP + (LV >= 2 ? swz(ccol) : ccol);
      // levels >= 2 read values this kernel stored already rounded to TF32;
      // level 1 reads the input grid, rounded already when RIN is false
      if (MODE == Mode::SpTF32) plane_sp_tf32<F, SP, LV == 1 && RIN>(row0, A, E, acc);
      else if (MODE == Mode::DenseTF32) plane_dense_tf32<F, SP, LV == 1 && RIN>(row0, Ad, acc);
      else if (MODE == Mode::SpF16x2) plane_sp_split<F, false, 0, SP>(row0, Am, Em, A, E, acc, accC);
      else {
        // BF16 hi/mid/lo: two passes, each with its own operands
        uint4 Am2[F::RY + 1], A2[F::NA];
        uint32_t Em2[F::RY + 1], E2[F::NA];
        plane_split<F, MODE, SP>(args, 0, c.lane, row0, Am2, Em2, A2, E2, acc, accC);
      }
      if (MODE == Mode::SpF16x2 || MODE == Mode::SpBF16x3) combine_split<MODE>(acc, accC);
      constexpr bool kStoreTF32 = (MODE == Mode::SpTF32 || MODE == Mode::DenseTF32);
      const int gy0 = c.y0 - GY + r0, gx0 = c.x0 - GX + 8 * s0;  // unit origin in the grid
      const bool interior = gy0 >= 0 && gy0 + F::H <= (int)args.ny && gx0 >= 0 && gx0 + 64 <= (int)args.nx;
      const int lx = 16 * c.q + c.g;  // this lane's column (h = 0) within the unit
      if (LV < F::T) {
        // intermediate level: zero outside the grid; TF32 modes store the
        // value already rounded as the next level's MMA will read it
        float* d = dst + r0 * DP;
        const int p0 = swz(8 * s0 + lx), p1 = swz(8 * s0 + lx + 8);
        if (interior) {
#pragma unroll
          for (int pp = 0; pp < F::H / 2; ++pp)
#pragma unroll
            for (int sr = 0; sr < 2; ++sr)
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const float v = kStoreTF32 ? __uint_as_float(cvt_tf32(acc[pp][2 * sr + h])) : acc[pp][2 * sr + h];
                d[(2 * pp + sr) * DP + (h ? p1 : p0)] = v;
              }
        } else {
          const bool xin0 = (unsigned)(gx0 + lx) < (unsigned)args.nx;
          const bool xin1 = (unsigned)(gx0 + lx + 8) < (unsigned)args.nx;
#pragma unroll
          for (int pp = 0; pp < F::H / 2; ++pp)
#pragma unroll
            for (int sr = 0; sr < 2; ++sr) {
              const bool yin = (unsigned)(gy0 + 2 * pp + sr) < (unsigned)args.ny;
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const float v = kStoreTF32 ? __uint_as_float(cvt_tf32(acc[pp][2 * sr + h])) : acc[pp][2 * sr + h];
                d[(2 * pp + sr) * DP + (h ? p1 : p0)] = (yin && (h ? xin1 : xin0)) ? v : 0.f;
              }
            }
        }
      } else {
        if (kStoreTF32 && args.out_tf32) round_tf32_inplace(acc);
        float* o = args.dst + (int64_t)gy0 * args.pitch + gx0 + lx;
        const int pitch = (int)args.pitch;
        // 16-byte stores need rows that start on 16-byte boundaries
        const bool vec = F::kVecStore && (args.pitch & 3) == 0 && (reinterpret_cast<uintptr_t>(args.dst) & 15) == 0;
        if (interior && vec) {
          // lane (g, q) holds output g of segments 2q, 2q + 1 in rows 2pp,
          // 2pp + 1; after the transpose lane i = g mod 4 holds combination
          // i (row 2pp + i / 2, segment 2q + i mod 2) at x = 4 (g / 4) .. + 3
          const int i = c.g & 3;
          float* ob = args.dst + (int64_t)gy0 * args.pitch + gx0 + 16 * c.q + 8 * (i & 1) + (c.g & 4);
#pragma unroll
          for (int pp = 0; pp < F::H / 2; ++pp) {
            float v0 = acc[pp][0], v1 = acc[pp][1], v2 = acc[pp][2], v3 = acc[pp][3];
            quad_transpose(v0, v1, v2, v3, i);
            *reinterpret_cast<float4*>(ob + (int64_t)(2 * pp + (i >> 1)) * pitch) = make_float4(v0, v1, v2, v3);
          }
        } else if (interior) {
#pragma unroll
          for (int pp = 0; pp < F::H / 2; ++pp)
#pragma unroll
            for (int sr = 0; sr < 2; ++sr) {
              float* orow = o + (size_t)(2 * pp + sr) * pitch;
              orow[0] = acc[pp][2 * sr];
              orow[8] = acc[pp][2 * sr + 1];
            }
        } else {
          const bool xin0 = (unsigned)(gx0 + lx) < (unsigned)args.nx;
          const bool xin1 = (unsigned)(gx0 + lx + 8) < (unsigned)args.nx;
#pragma unroll
          for (int pp = 0; pp < F::H / 2; ++pp)
#pragma unroll
            for (int sr = 0; sr < 2; ++sr) {
              if ((unsigned)(gy0 + 2 * pp + sr) < (unsigned)args.ny) {
                float* orow = o + (size_t)(2 * pp + sr) * pitch;
                if (xin0) orow[0] = acc[pp][2 * sr];
                if (xin1) orow[8] = acc[pp][2 * sr + 1];
              }
            }
        }
      }
    }
  }
}

template <class F, Mode MODE, bool RIN, int LV>
struct LevelRunner {
  template <class... Ops>
  __device__ __forceinline__ static void run(const FusedCtx& c, float* in, float* P, float* Q, uint64_t* bar,
                                             const CUtensorMap* tmap, int refill_tile, Ops&... ops);
};

// `in`/`bar`: the input box of this tile and its barrier; once level 1 has
// read it, the box is refilled with `refill_tile` (if any).
template <class F, Mode MODE, bool RIN, int LV>
template <class... Ops>
__device__ __forceinline__ void LevelRunner<F, MODE, RIN, LV>::run(const FusedCtx& c, float* in, float* P, float* Q,
                                                              uint64_t* bar, const CUtensorMap* tmap, int refill_tile,
                                                              Ops&... ops) {
  const float* src = (LV == 1) ? in : ((LV - 1) % 2 == 1 ? P : Q);
  float* dst = (LV == F::T) ? nullptr : (LV % 2 == 1 ? P : Q);
  fused_level<F, MODE, RIN, LV>(c, src, dst, ops...);
  __syncthreads();
  if (LV == 1 && threadIdx.x == 0 && refill_tile >= 0) {
    // the input box is no longer read: prefetch a later tile into it
    const StepArgs& args = *c.args;
    const int tx = refill_tile % args.tiles_x, ty = refill_tile / args.tiles_x;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, F::kInBytes);
    tma_load_3d(in, tmap, bar, tx * F::BX - 4 * F::T, ty * F::BY - F::RY * F::T, 0);
  }
  if constexpr (LV < F::T) LevelRunner<F, MODE, RIN, LV + 1>::run(c, in, P, Q, bar, tmap, refill_tile, ops...);
}

template <class F, Mode MODE, bool RIN = true>
__global__ void __launch_bounds__(F::kThreads, F::kMinBlocks)
    fused_step_kernel(const __grid_constant__ CUtensorMap tmap, const StepArgs args) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t base_u32 = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024 - (base_u32 & 1023)) & 1023);
  constexpr int NS = F::kInStages;
  float* P = reinterpret_cast<float*>(smem + NS * F::kInStride);
  float* Q = reinterpret_cast<float*>(smem + NS * F::kInStride + F::kPStride);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NS * F::kInStride + F::kPStride + F::kQStride);
  auto in_box = [&](int s) { return reinterpret_cast<float*>(smem + s * F::kInStride); };

  FusedCtx c;
  c.args = &args;
  const int tid = threadIdx.x;
  c.lane = tid & 31;
  c.warp = tid >> 5;
  c.g = c.lane >> 2;
  c.q = c.lane & 3;
  const int ntiles = args.tiles_x * args.tiles_y;

  if (tid == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&bar[k], 1);
    fence_mbar_init();
  }
  griddep_wait();  // see stencil_step_kernel
  griddep_launch_dependents();
  __syncthreads();
  if (tid == 0) {
    for (int k = 0; k < NS; ++k) {
      const int t = blockIdx.x + k * gridDim.x;
      if (t >= ntiles) break;
      const int tx = t % args.tiles_x, ty = t / args.tiles_x;
      mbar_arrive_expect_tx(&bar[k], F::kInBytes);
      tma_load_3d(in_box(k), &tmap, &bar[k], tx * F::BX - 4 * F::T, ty * F::BY - F::RY * F::T, 0);
    }
  }

  constexpr int NA = F::NA;
  constexpr int CPP = MODE == Mode::SpF16x2 ? (F::RY + 1) + NA : NA;
  uint4 A[NA];
  uint32_t E[NA];
  uint4 Ad[NA][2];
  uint4 Am[F::RY + 1];
  uint32_t Em[F::RY + 1];
  float W[(2 * F::RY + 1) * (2 * F::RX + 1)];
  if (MODE == Mode::SpTF32) {
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      A[a] = args.a_words[(size_t)a * 32 + c.lane];
      E[a] = args.meta[(size_t)a * 32 + c.lane];
    }
  } else if (MODE == Mode::DenseTF32) {
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      Ad[a][0] = args.a_words[((size_t)a * 32 + c.lane) * 2 + 0];
      Ad[a][1] = args.a_words[((size_t)a * 32 + c.lane) * 2 + 1];
    }
  } else if (MODE == Mode::SpF16x2) {
    load_split_operands<F>(args, 0, c.lane, Am, Em, A, E);
  } else if (MODE == Mode::SpBF16x3) {
    // two passes of operands, loaded per warp unit (see fused_level)
  } else {
#pragma unroll
    for (int i = 0; i < (2 * F::RY + 1) * (2 * F::RX + 1); ++i) W[i] = args.w[i];
  }
  (void)CPP;

  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int st = it % NS;
    const uint32_t parity = (uint32_t)((it / NS) & 1);
    const bool ok = mbar_wait_bounded(&bar[st], parity, args.status, args.wait_cycles);
    if (!__syncthreads_and(ok)) {
      // the load we gave up on may still land: wait for it once more (bounded)
      if (tid == 0) (void)mbar_wait_bounded(&bar[st], parity, args.status, args.wait_cycles);
      break;
    }
    c.x0 = (t % args.tiles_x) * F::BX;
    c.y0 = (t / args.tiles_x) * F::BY;
    const int refill = t + NS * (int)gridDim.x < ntiles ? t + NS * (int)gridDim.x : -1;
    LevelRunner<F, MODE, RIN, 1>::run(c, in_box(st), P, Q, &bar[st], &tmap, refill, A, E, Ad, Am, Em, W);
  }
}

}  // namespace spider
