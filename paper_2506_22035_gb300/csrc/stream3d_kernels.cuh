// 3-D stencils streamed along z.
//
// A CTA owns a column block of BY x BX outputs and a chunk of ZC planes.  It
// keeps a ring of 2r+2 input planes in shared memory, each the (BY + 2r) x
// (BX + 8) box of one input plane loaded by TMA (zero outside the grid): the
// 2r+1 planes output plane z reads, plus the next plane in flight.  Every
// input plane is loaded once per chunk (plus 2r halo planes at the chunk
// ends), instead of 1 + 2r/BZ times as with cube tiles, and the ring is small
// enough for several CTAs per SM.  The per-warp work is the one-step kernel's
// (Sec. 3.1-3.3): for each dz plane, one 16-byte load per lane per input row
// feeding the sparse MMAs of the row pairs it reaches.
#pragma once

#include "stencil_kernels.cuh"

namespace spider {

template <int R_, int WY_, int WX_, int H_, int ZC_>
struct StreamCfg {
  static constexpr int RZ = R_, RY = R_, RX = R_, WY = WY_, WX = WX_, H = H_, ZC = ZC_;
  static constexpr int BY = WY * H, BX = WX * 64;
  static constexpr int SY = BY + 2 * RY, SX = BX + 2 * kHaloX;
  static constexpr int NP = 2 * RZ + 2;  // ring slots
  static constexpr int kThreads = WY * WX * 32;
  static constexpr int kPlaneBytes = SY * SX * 4;
  static constexpr int kPlaneStride = (kPlaneBytes + 127) / 128 * 128;
  static constexpr int kSmemBytes = NP * kPlaneStride + 1024 + 128;
  static constexpr int NA = 2 * RY + 2;
  // A operands of every dz plane stay in registers when they fit
  static constexpr bool kAllOperands = (2 * RZ + 1) * NA <= 12;
  static_assert(SX <= 256 && SY <= 256, "TMA box dimension limit");
};

template <class C, Mode MODE, bool RIN = true, bool STAR = false>
__global__ void __launch_bounds__(C::kThreads) stream3d_kernel(const __grid_constant__ CUtensorMap tmap,
                                                               const StepArgs args, int nchunks) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t base_u32 = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024 - (base_u32 & 1023)) & 1023);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::NP * C::kPlaneStride);
  auto slot_ptr = [&](int s) { return reinterpret_cast<float*>(smem + s * C::kPlaneStride); };

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int wx = warp % C::WX, wy = warp / C::WX;
  const int ncol = args.tiles_x * args.tiles_y;
  const int nitems = ncol * nchunks;

  if (tid == 0) {
    for (int k = 0; k < C::NP; ++k) mbar_init(&bar[k], 1);
    fence_mbar_init();
  }
  griddep_wait();
  griddep_launch_dependents();
  __syncthreads();

  constexpr int NA = C::NA;
  constexpr int CPP = MODE == Mode::SpF16x2 ? (C::RY + 1) + NA : NA;
  constexpr int NZ = 2 * C::RZ + 1;
  constexpr int NWT = (2 * C::RY + 1) * (2 * C::RX + 1);
  // operands: all dz planes (small stencils) or one plane at a time.  The
  // FP16 split of a star keeps one plane's (143 instead of 244 registers,
  // three CTAs per SM instead of two: Heat-3D 447 against 428 GStencil/s);
  // for a box, loading the larger operand sets plane by plane costs more than
  // the third CTA gains (Box-3D 377 against 408)
  constexpr bool kAll = C::kAllOperands && !(MODE == Mode::SpF16x2 && STAR);
  constexpr int NPL = kAll ? NZ : 1;
  uint4 A[NPL][NA];
  uint32_t E[NPL][NA];
  uint4 Ad[NPL][NA][2];
  uint4 Am[NPL][C::RY + 1];
  uint32_t Em[NPL][C::RY + 1];
  float W[NWT];
  auto load_operands = [&](int dzi, int k) {
    if (MODE == Mode::SpTF32) {
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        if (STAR && dzi != C::RZ && a != C::RY && a != C::RY + 1) continue;  // zero operands
        A[k][a] = args.a_words[(size_t)(dzi * CPP + a) * 32 + lane];
        E[k][a] = args.meta[(size_t)(dzi * CPP + a) * 32 + lane];
      }
    } else if (MODE == Mode::DenseTF32) {
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        if (STAR && dzi != C::RZ && a != C::RY && a != C::RY + 1) continue;
        Ad[k][a][0] = args.a_words[((size_t)(dzi * NA + a) * 32 + lane) * 2 + 0];
        Ad[k][a][1] = args.a_words[((size_t)(dzi * NA + a) * 32 + lane) * 2 + 1];
      }
    } else if (MODE == Mode::SpF16x2) {
      if (STAR && dzi != C::RZ) {
        // off-centre plane of a star: the two-row combos and the cross
        // combos of A indices ry, ry + 1 (the others are zero and not applied)
#pragma unroll
        for (int c = 0; c <= C::RY; ++c) {
          if (2 * c + 1 < C::RY || 2 * c > C::RY + 1) continue;
          Am[k][c] = args.a_words[(size_t)(dzi * CPP + c) * 32 + lane];
          Em[k][c] = args.meta[(size_t)(dzi * CPP + c) * 32 + lane];
        }
#pragma unroll
        for (int a = C::RY; a <= C::RY + 1; ++a) {
          A[k][a] = args.a_words[(size_t)(dzi * CPP + C::RY + 1 + a) * 32 + lane];
          E[k][a] = args.meta[(size_t)(dzi * CPP + C::RY + 1 + a) * 32 + lane];
        }
      } else {
        load_split_operands<C>(args, dzi * CPP, lane, Am[k], Em[k], A[k], E[k]);
      }
    } else if (MODE == Mode::SpBF16x3) {
      // two passes of operands, loaded by plane_split
    } else {
#pragma unroll
      for (int i = 0; i < NWT; ++i) W[i] = args.w[(size_t)dzi * NWT + i];
    }
  };
  if (kAll) {
#pragma unroll
    for (int dzi = 0; dzi < NZ; ++dzi) load_operands(dzi, dzi);
  }

  uint32_t phases = 0;   // parity of the next completion of each ring slot
  uint32_t pending = 0;  // slots with a load issued and not yet waited for (thread 0)
  int rot = 0;          // ring position of the first plane of the current item
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int col = item % ncol, chunk = item / ncol;
    const int x0 = (col % args.tiles_x) * C::BX, y0 = (col / args.tiles_x) * C::BY;
    const int z0 = (int)((int64_t)chunk * args.nz / nchunks), z1 = (int)((int64_t)(chunk + 1) * args.nz / nchunks);
    // plane zi (input z coordinate) lives in slot (zi - (z0 - RZ) + rot) % NP
    auto slot_of = [&](int zi) { return (zi - (z0 - C::RZ) + rot) % C::NP; };
    auto issue = [&](int zi) {
      const int s = slot_of(zi);
      mbar_arrive_expect_tx(&bar[s], C::kPlaneBytes);
      tma_load_3d(slot_ptr(s), &tmap, &bar[s], x0 - kHaloX, y0 - C::RY, zi);
    };
    if (tid == 0) {
      fence_proxy_async_smem();
      for (int zi = z0 - C::RZ; zi <= min(z0 + C::RZ + 1, z1 - 1 + C::RZ); ++zi) {
        issue(zi);
        pending |= 1u << slot_of(zi);
      }
    }
    bool ok = true;
    for (int z = z0; z < z1; ++z) {
      // planes z-r .. z+r must have landed; z+r is the newest
      const int sn = slot_of(z + C::RZ);
      if (z == z0) {
        for (int zi = z0 - C::RZ; zi <= z0 + C::RZ; ++zi) {
          const int s = slot_of(zi);
          ok = ok && mbar_wait_bounded(&bar[s], (phases >> s) & 1, args.status, args.wait_cycles);
          phases ^= 1u << s;
          pending &= ~(1u << s);
        }
      } else {
        ok = ok && mbar_wait_bounded(&bar[sn], (phases >> sn) & 1, args.status, args.wait_cycles);
        phases ^= 1u << sn;
        pending &= ~(1u << sn);
      }
      if (!__syncthreads_and(ok)) break;

      const int ybase = y0 + wy * C::H, xbase = x0 + wx * 64;
      const int coff = 8 * g + 4 * ((q == 1) ? 2 : (q == 2) ? 1 : q);
      if (MODE == Mode::CudaCore) {
        // FP32 FMA stencil: lane l computes columns 2l and 2l + 1 of its
        // warp's 64; per input row it loads the 2r + 2 floats those read as
        // 8-byte pairs (v[e] = box column 2l + e of the warp, e = 0..9; the
        // block's column c sits at box column c + 4)
        constexpr int E0 = (4 - C::RX) / 2, E1 = (5 + C::RX) / 2;  // pairs e = 2m, 2m + 1 for m in [E0, E1]
        float acc[C::H][2];
#pragma unroll
        for (int i = 0; i < C::H; ++i) acc[i][0] = acc[i][1] = 0.f;
#pragma unroll 1
        for (int dzi = 0; dzi < NZ; ++dzi) {
          if (!kAll) load_operands(dzi, 0);
          const float* pl = slot_ptr(slot_of(z - C::RZ + dzi)) + (wy * C::H) * C::SX + wx * 64 + 2 * lane;
          if (STAR && dzi != C::RZ) {
            // off-centre plane of a star: its one non-zero weight, the
            // centre; the other products are exact zeros in the box loop
            // below, so skipping them keeps the result bit for bit
            const float wv = args.w[(size_t)dzi * NWT + C::RY * (2 * C::RX + 1) + C::RX];
#pragma unroll
            for (int yy = 0; yy < C::H; ++yy) {
              const float2 c = *reinterpret_cast<const float2*>(pl + (yy + C::RY) * C::SX + kHaloX);
              acc[yy][0] = fmaf(wv, c.x, acc[yy][0]);
              acc[yy][1] = fmaf(wv, c.y, acc[yy][1]);
            }
            continue;
          }
          // the weights of this dz plane (a star's centre plane: row dy = 0
          // and column dx = 0 only)
          float Wd[NWT];
#pragma unroll
          for (int i = 0; i < NWT; ++i) Wd[i] = args.w[(size_t)dzi * NWT + i];
#pragma unroll
          for (int jj = 0; jj < C::H + 2 * C::RY; ++jj) {
            // a star reads the whole row only where it is some output's dy = 0 row
            const bool full_row = !STAR || (jj >= C::RY && jj < C::RY + C::H);
            float v[10];
#pragma unroll
            for (int m = E0; m <= E1; ++m) {
              if (!full_row && m != 2) continue;  // the centre columns are v[4], v[5]
              const float2 t = *reinterpret_cast<const float2*>(pl + jj * C::SX + 2 * m);
              v[2 * m] = t.x;
              v[2 * m + 1] = t.y;
            }
#pragma unroll
            for (int yy = 0; yy < C::H; ++yy) {
              const int dy = jj - C::RY - yy;
              if (dy >= -C::RY && dy <= C::RY) {
#pragma unroll
                for (int kx = 0; kx < 2 * C::RX + 1; ++kx) {
                  if (STAR && dy != 0 && kx != C::RX) continue;
                  const float wv = Wd[(dy + C::RY) * (2 * C::RX + 1) + kx];
                  acc[yy][0] = fmaf(wv, v[4 - C::RX + kx], acc[yy][0]);
                  acc[yy][1] = fmaf(wv, v[5 - C::RX + kx], acc[yy][1]);
                }
              }
            }
          }
        }
        float* o = args.dst + ((int64_t)z * args.ny + ybase) * args.pitch + xbase + 2 * lane;
        const int ylim = (int)(args.ny - ybase < C::H ? args.ny - ybase : C::H);
        const int xlim = (int)(args.nx - xbase < 64 ? args.nx - xbase : 64);
#pragma unroll
        for (int yy = 0; yy < C::H; ++yy)
          if (yy < ylim) {
#pragma unroll
            for (int c = 0; c < 2; ++c)
              if (2 * lane + c < xlim) o[(size_t)yy * args.pitch + c] = acc[yy][c];
          }
      } else {
        float acc[C::H / 2][4];
        float accC[C::H / 2][4];
#pragma unroll
        for (int i = 0; i < C::H / 2; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = accC[i][j] = 0.f;
#pragma unroll
        for (int dzi = 0; dzi < NZ; ++dzi) {
          if (!kAll) load_operands(dzi, 0);
          const int k = kAll ? dzi : 0;
          const float* row0 = slot_ptr(slot_of(z - C::RZ + dzi)) + (wy * C::H) * C::SX + wx * 64 + coff;
          const bool centre_only = STAR && dzi != C::RZ;  // see plane_sp_tf32_centre
          if (MODE == Mode::SpTF32) {
            if (centre_only) plane_sp_tf32_centre<C, C::SX, RIN>(row0, A[k], E[k], acc);
            else plane_sp_tf32<C, C::SX, RIN>(row0, A[k], E[k], acc);
          } else if (MODE == Mode::DenseTF32) {
            if (centre_only) plane_dense_tf32_centre<C, C::SX, RIN>(row0, Ad[k], acc);
            else plane_dense_tf32<C, C::SX, RIN>(row0, Ad[k], acc);
          } else if (centre_only) {
            plane_split<C, MODE, C::SX, C::RY, C::RY + 1>(args, dzi, lane, row0, Am[k], Em[k], A[k], E[k], acc,
                                                          accC);
          } else {
            plane_split<C, MODE>(args, dzi, lane, row0, Am[k], Em[k], A[k], E[k], acc, accC);
          }
        }
        if (MODE == Mode::SpF16x2 || MODE == Mode::SpBF16x3) combine_split<MODE>(acc, accC);
        if (is_tf32_mode(MODE) && args.out_tf32) round_tf32_inplace(acc);
        float* o = args.dst + ((int64_t)z * args.ny + ybase) * args.pitch + xbase + 16 * q + g;
        const int pitch = (int)args.pitch;
        if (ybase + C::H <= args.ny && xbase + 64 <= args.nx) {
#pragma unroll
          for (int pp = 0; pp < C::H / 2; ++pp)
#pragma unroll
            for (int sr = 0; sr < 2; ++sr) {
              float* orow = o + (size_t)(2 * pp + sr) * pitch;
              orow[0] = acc[pp][2 * sr];
              orow[8] = acc[pp][2 * sr + 1];
            }
        } else {
          const int ylim = (int)(args.ny - ybase < C::H ? args.ny - ybase : C::H);
          const int xlim = (int)(args.nx - xbase < 64 ? args.nx - xbase : 64);
#pragma unroll
          for (int pp = 0; pp < C::H / 2; ++pp)
#pragma unroll
            for (int sr = 0; sr < 2; ++sr)
              if (2 * pp + sr < ylim) {
#pragma unroll
                for (int c = 0; c < 2; ++c)
                  if (16 * q + 8 * c + g < xlim) o[(size_t)(2 * pp + sr) * pitch + 8 * c] = acc[pp][2 * sr + c];
              }
        }
      }
      __syncthreads();  // every warp is done with plane z - r
      if (tid == 0 && z + C::RZ + 2 <= z1 - 1 + C::RZ) {
        fence_proxy_async_smem();
        issue(z + C::RZ + 2);  // into the slot plane z - r just left
        pending |= 1u << slot_of(z + C::RZ + 2);
      }
    }
    if (!ok) {
      // loads still in flight after a wait ran out: wait for them (bounded)
      if (tid == 0)
        for (int s = 0; s < C::NP; ++s)
          if ((pending >> s) & 1) (void)mbar_wait_bounded(&bar[s], (phases >> s) & 1, args.status, args.wait_cycles);
      break;
    }
    rot = (rot + (z1 - z0) + 2 * C::RZ) % C::NP;
  }
}

}  // namespace spider
