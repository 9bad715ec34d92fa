// Temporal fusion for 3-D stencils: T time steps per pass over HBM, streamed
// along z.
//
// A CTA owns a column block of BY x BX outputs and a chunk of z planes.  It
// streams the input planes of the block (grown by T*r rows and 4*T columns on
// each side, TMA, zero outside the grid) through a ring of 2r + 2 slots, and
// keeps for every intermediate level t = 1..T-1 a ring of the 2r + 1 most
// recent planes of that level, each covering the block grown by r*(T-t) rows
// and 4*(T-t) columns.  When input plane zi has landed, level t computes its
// plane zi - t*r from the 2r + 1 planes of level t-1 around it, for
// t = 1..T in turn; level T is the output and goes to HBM.  A level plane
// outside the grid (z < 0 or z >= nz) is all zero, and points of a level
// plane outside the grid in x or y are stored as zero, so every fused step
// sees the zero Dirichlet halo exactly as separate steps do.  The per-warp
// unit is the one-step kernel's (Sec. 3.1-3.3), so results are bit-identical
// to T separate steps.
//
// Only level 1 reads the TMA ring: its oldest slot is free after level 1 and
// the load of the plane 2r + 2 ahead goes there, overlapping levels 2..T.
#pragma once

#include "fused_kernels.cuh"

namespace spider {

template <int R_, int T_, int L1Y_, int H_, int NW_, int MINB_>
struct Fuse3Cfg {
  static constexpr int R = R_, RZ = R_, RY = R_, RX = R_, T = T_, H = H_, NW = NW_;
  static constexpr int kMinBlocks = MINB_;
  static constexpr int NA = 2 * RY + 2;
  static constexpr int kThreads = NW * 32;
  // output block; level 1 is L1Y rows x 128 columns (two N-tiles)
  static constexpr int BY = L1Y_ - 2 * R * (T - 1), BX = 8 * (17 - T);
  // level t: 0 = input planes, T = output planes
  __host__ __device__ static constexpr int rows(int t) { return BY + 2 * R * (T - t); }
  __host__ __device__ static constexpr int width(int t) { return BX + 8 * (T - t); }
  __host__ __device__ static constexpr int segs(int t) { return width(t) / 8; }
  __host__ __device__ static constexpr int pitch(int t) { return t == 0 ? width(0) : (width(t) + 15) / 16 * 16; }
  static constexpr int SX = 136;  // unused default row pitch of the plane helpers
  static constexpr int NP0 = 2 * R + 2;  // input ring slots
  static constexpr int NPL = 2 * R + 1;  // ring slots of each intermediate level
  static constexpr int kInBytes = rows(0) * width(0) * 4;
  static constexpr int kInStride = (kInBytes + 127) / 128 * 128;
  static constexpr int kLvStride = (rows(1) * pitch(1) * 4 + 127) / 128 * 128;
  static constexpr int kSmemBytes = NP0 * kInStride + (T - 1) * NPL * kLvStride + 1024 + 128;
  static_assert(T >= 2, "use the z-streaming one-step kernel for T = 1");
  static_assert(width(0) == 136 && rows(0) <= 256, "TMA box");
  static_assert(H % 2 == 0 && rows(T) >= H, "warp tile height");
  static_assert(R <= kMaxR, "radius");
};

struct Fuse3Ctx {
  const StepArgs* args;
  unsigned char* smem;
  uint64_t* bar;
  const CUtensorMap* tmap;
  int x0, y0, z0, zstart, zend, rot;
  int lane, warp, g, q, tid;
  uint32_t* phases;
  uint32_t* pending;
};

template <class C>
__device__ __forceinline__ float* f3_in_slot(const Fuse3Ctx& c, int s) {
  return reinterpret_cast<float*>(c.smem + s * C::kInStride);
}
template <class C>
__device__ __forceinline__ float* f3_lv_slot(const Fuse3Ctx& c, int lv, int s) {
  return reinterpret_cast<float*>(c.smem + C::NP0 * C::kInStride + ((lv - 1) * C::NPL + s) * C::kLvStride);
}
template <class C>
__device__ __forceinline__ int f3_slot0(const Fuse3Ctx& c, int zi) {
  return (zi - c.zstart + c.rot) % C::NP0;
}
__device__ __forceinline__ int f3_slotl(int z, int n) { return ((z % n) + n) % n; }

template <class C>
__device__ __forceinline__ void f3_issue(Fuse3Ctx& c, int zi) {
  const int s = f3_slot0<C>(c, zi);
  mbar_arrive_expect_tx(&c.bar[s], C::kInBytes);
  tma_load_3d(f3_in_slot<C>(c, s), c.tmap, &c.bar[s], c.x0 - 4 * C::T, c.y0 - C::R * C::T, zi);
  *c.pending |= 1u << s;
}

// Level LV of input step zi: computes level plane zi - LV*r if the chunk
// needs it, then the next level.
template <class C, Mode MODE, bool RIN, bool STAR, int LV>
__device__ __forceinline__ void f3_level(Fuse3Ctx& c, int zi, const uint4 (&A)[2 * C::R + 1][C::NA],
                                         const uint32_t (&E)[2 * C::R + 1][C::NA],
                                         const uint4 (&Ad)[2 * C::R + 1][C::NA][2]) {
  constexpr int R = C::R, T = C::T, H = C::H;
  constexpr int SP = C::pitch(LV - 1), DP = C::pitch(LV);
  constexpr int NRW = C::rows(LV), NSG = C::segs(LV);
  constexpr int NR = (NRW + H - 1) / H, NS = (NSG + 7) / 8, U = NR * NS;
  constexpr int GY = R * (T - LV), GX = 4 * (T - LV);  // level origin = block origin - (GY, GX)
  constexpr bool kRound = (LV == 1) && RIN;  // levels >= 2 read values stored rounded
  const StepArgs& args = *c.args;
  const int zt = zi - LV * R;
  if (zt < c.z0 - (T - LV) * R) return;  // this level (and the ones above) not started yet
  const bool inside = zt >= 0 && zt < (int)args.nz;
  if (!inside) {
    if constexpr (LV < T) {
      float4* d = reinterpret_cast<float4*>(f3_lv_slot<C>(c, LV, f3_slotl(zt, C::NPL)));
      for (int i = c.tid; i < C::rows(LV) * DP / 4; i += C::kThreads) d[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  } else {
    for (int u = c.warp; u < U; u += C::NW) {
      const int r0 = min((u / NS) * H, NRW - H);
      const int s0 = min((u % NS) * 8, NSG - 8);
      float acc[H / 2][4];
#pragma unroll
      for (int i = 0; i < H / 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
      const int ccol = 8 * (s0 + c.g) + 4 * ((c.q == 1) ? 2 : (c.q == 2) ? 1 : c.q);
#pragma unroll
      for (int dzi = 0; dzi <= 2 * R; ++dzi) {
        const int zs = zt - R + dzi;
        const float* src = (LV == 1) ? f3_in_slot<C>(c, f3_slot0<C>(c, zs))
                                     : f3_lv_slot<C>(c, LV - 1, f3_slotl(zs, C::NPL));
        const float* row0 = src + r0 * SP + (LV >= 2 ? swz(ccol) : ccol);
        const bool centre_only = STAR && dzi != R;
        if (MODE == Mode::SpTF32) {
          if (centre_only) plane_sp_tf32_centre<C, SP, kRound>(row0, A[dzi], E[dzi], acc);
          else plane_sp_tf32<C, SP, kRound>(row0, A[dzi], E[dzi], acc);
        } else {
          if (centre_only) plane_dense_tf32_centre<C, SP, kRound>(row0, Ad[dzi], acc);
          else plane_dense_tf32<C, SP, kRound>(row0, Ad[dzi], acc);
        }
      }
      const int gy0 = c.y0 - GY + r0, gx0 = c.x0 - GX + 8 * s0;  // unit origin in the grid
      const bool interior = gy0 >= 0 && gy0 + H <= (int)args.ny && gx0 >= 0 && gx0 + 64 <= (int)args.nx;
      const int lx = 16 * c.q + c.g;  // this lane's column (h = 0) within the unit
      if constexpr (LV < T) {
        // stored rounded to TF32 as the next level's MMA reads it; zero outside the grid
        float* d = f3_lv_slot<C>(c, LV, f3_slotl(zt, C::NPL)) + r0 * DP;
        const int p0 = swz(8 * s0 + lx), p1 = swz(8 * s0 + lx + 8);
        if (interior) {
#pragma unroll
          for (int pp = 0; pp < H / 2; ++pp)
#pragma unroll
            for (int sr = 0; sr < 2; ++sr)
#pragma unroll
              for (int h = 0; h < 2; ++h)
                d[(2 * pp + sr) * DP + (h ? p1 : p0)] = __uint_as_float(cvt_tf32(acc[pp][2 * sr + h]));
        } else {
          const bool xin0 = (unsigned)(gx0 + lx) < (unsigned)args.nx;
          const bool xin1 = (unsigned)(gx0 + lx + 8) < (unsigned)args.nx;
#pragma unroll
          for (int pp = 0; pp < H / 2; ++pp)
#pragma unroll
            for (int sr = 0; sr < 2; ++sr) {
              const bool yin = (unsigned)(gy0 + 2 * pp + sr) < (unsigned)args.ny;
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const float v = __uint_as_float(cvt_tf32(acc[pp][2 * sr + h]));
                d[(2 * pp + sr) * DP + (h ? p1 : p0)] = (yin && (h ? xin1 : xin0)) ? v : 0.f;
              }
            }
        }
      } else {
        if (args.out_tf32) round_tf32_inplace(acc);
        float* o = args.dst + ((int64_t)zt * args.ny + gy0) * args.pitch + gx0 + lx;
        const int pitch = (int)args.pitch;
        if (interior) {
#pragma unroll
          for (int pp = 0; pp < H / 2; ++pp)
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
          for (int pp = 0; pp < H / 2; ++pp)
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
  __syncthreads();  // level LV plane zt complete; level LV-1 planes read
  if (LV == 1 && c.tid == 0) {
    // the input plane zi - 2r is no longer read: load plane zi + 2 into its slot
    const int zn = zi + 2;
    if (zn >= c.zstart + C::NP0 && zn <= c.zend) {
      fence_proxy_async_smem();
      f3_issue<C>(c, zn);
    }
  }
  if constexpr (LV < T) f3_level<C, MODE, RIN, STAR, LV + 1>(c, zi, A, E, Ad);
}

template <class C, Mode MODE, bool RIN = true, bool STAR = false>
__global__ void __launch_bounds__(C::kThreads, C::kMinBlocks)
    stream3d_fused_kernel(const __grid_constant__ CUtensorMap tmap, const StepArgs args, int nchunks) {
  static_assert(is_tf32_mode(MODE), "3-D fusion is built for the TF32 modes");
  extern __shared__ unsigned char smem_raw[];
  const uint32_t base_u32 = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024 - (base_u32 & 1023)) & 1023);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::NP0 * C::kInStride + (C::T - 1) * C::NPL * C::kLvStride);

  uint32_t phases = 0;   // parity of the next completion of each input slot
  uint32_t pending = 0;  // input slots with a load issued and not yet waited for (thread 0)
  Fuse3Ctx c;
  c.args = &args;
  c.smem = smem;
  c.bar = bar;
  c.tmap = &tmap;
  c.tid = threadIdx.x;
  c.lane = c.tid & 31;
  c.warp = c.tid >> 5;
  c.g = c.lane >> 2;
  c.q = c.lane & 3;
  c.phases = &phases;
  c.pending = &pending;
  c.rot = 0;
  const int ncol = args.tiles_x * args.tiles_y;
  const int nitems = ncol * nchunks;

  if (c.tid == 0) {
    for (int k = 0; k < C::NP0; ++k) mbar_init(&bar[k], 1);
    fence_mbar_init();
  }
  griddep_wait();
  griddep_launch_dependents();
  __syncthreads();

  constexpr int NZ = 2 * C::R + 1, NA = C::NA;
  uint4 A[NZ][NA];
  uint32_t E[NZ][NA];
  uint4 Ad[NZ][NA][2];
#pragma unroll
  for (int dzi = 0; dzi < NZ; ++dzi)
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      if (STAR && dzi != C::R && a != C::RY && a != C::RY + 1) continue;  // zero operands
      if (MODE == Mode::SpTF32) {
        A[dzi][a] = args.a_words[(size_t)(dzi * NA + a) * 32 + c.lane];
        E[dzi][a] = args.meta[(size_t)(dzi * NA + a) * 32 + c.lane];
      } else {
        Ad[dzi][a][0] = args.a_words[((size_t)(dzi * NA + a) * 32 + c.lane) * 2 + 0];
        Ad[dzi][a][1] = args.a_words[((size_t)(dzi * NA + a) * 32 + c.lane) * 2 + 1];
      }
    }

  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int col = item % ncol, chunk = item / ncol;
    c.x0 = (col % args.tiles_x) * C::BX;
    c.y0 = (col / args.tiles_x) * C::BY;
    c.z0 = (int)((int64_t)chunk * args.nz / nchunks);
    const int z1 = (int)((int64_t)(chunk + 1) * args.nz / nchunks);
    c.zstart = c.z0 - C::T * C::R;
    c.zend = z1 - 1 + C::T * C::R;
    if (c.tid == 0) {
      fence_proxy_async_smem();
      for (int zi = c.zstart; zi <= c.zend && zi < c.zstart + C::NP0; ++zi) f3_issue<C>(c, zi);
    }
    bool ok = true;
    for (int zi = c.zstart; zi <= c.zend; ++zi) {
      const int s = f3_slot0<C>(c, zi);
      ok = ok && mbar_wait_bounded(&bar[s], (phases >> s) & 1, args.status, args.wait_cycles);
      phases ^= 1u << s;
      pending &= ~(1u << s);
      if (!__syncthreads_and(ok)) break;
      f3_level<C, MODE, RIN, STAR, 1>(c, zi, A, E, Ad);
    }
    if (!ok) {
      // loads still in flight after a wait ran out: wait for them (bounded)
      if (c.tid == 0)
        for (int s = 0; s < C::NP0; ++s)
          if ((pending >> s) & 1) (void)mbar_wait_bounded(&bar[s], (phases >> s) & 1, args.status, args.wait_cycles);
      break;
    }
    c.rot = (c.rot + (c.zend - c.zstart + 1)) % C::NP0;
  }
}

}  // namespace spider
