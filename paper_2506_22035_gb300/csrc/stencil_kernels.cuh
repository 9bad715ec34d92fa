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

// SpTF32Copy: SpTF32 with the input row swap done by an explicit copy of
// every window into a buffer of its own (the baseline of Sec. 3.2).
// SpTF32NoCO: SpTF32 without the computing optimisations of Sec. 3.3: the
// kernel-matrix operands and metadata are staged in shared memory and every
// MMA loads its own from there instead of keeping them in registers.
enum class Mode : int {
  SpTF32 = 0,
  SpF16x2 = 1,
  SpBF16x3 = 2,
  DenseTF32 = 3,
  CudaCore = 4,
  SpTF32Copy = 5,
  SpTF32NoCO = 6
};

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
  long long wait_cycles;   // limit of every bounded wait (SM cycles)
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
__host__ __device__ constexpr bool is_tf32_mode(Mode m) {
  return m == Mode::SpTF32 || m == Mode::DenseTF32 || m == Mode::SpTF32Copy || m == Mode::SpTF32NoCO;
}
__host__ __device__ constexpr bool is_sp_tf32(Mode m) {
  return m == Mode::SpTF32 || m == Mode::SpTF32Copy || m == Mode::SpTF32NoCO;
}

// Shared memory of the one-step kernel: two input stages, barriers and, for
// SpTF32Copy, the buffer of swapped windows (every row's BX / 8 windows of 16
// points, twice the row: consecutive windows overlap by 8 points); for
// SpTF32NoCO, the packed operands and metadata of every A index of a plane.
template <class C, Mode MODE>
__host__ __device__ constexpr int step_window_bytes() {
  return MODE == Mode::SpTF32Copy   ? C::SY * C::SZ * (C::BX / 8) * 16 * 4
         : MODE == Mode::SpTF32NoCO ? C::NA * 32 * (16 + 4)
                                    : 0;
}
template <class C, Mode MODE>
__host__ __device__ constexpr int step_smem_bytes() {
  return C::kSmemBytes + step_window_bytes<C, MODE>();
}

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

// SpTF32NoCO: as sp_tf32_row, with every MMA's A operand and metadata read
// from shared memory: this lane's uint4 of A index a at ops_a + 512 a, its
// metadata word at ops_e + 128 a (the packed layout, 32 lanes per index).
// The loads are volatile, so the compiler cannot keep the operands in
// registers across tiles.
template <class C, int SP, bool ROUND, int JJ>
__device__ __forceinline__ void sp_tf32_row_smem_ops(uint32_t addr, uint32_t ops_a, uint32_t ops_e,
                                                     float (&acc)[C::H / 2][4]) {
  const float4 v = lds128_at<JJ * SP * 4>(addr);
  const uint32_t b[4] = {ROUND ? cvt_tf32(v.x) : __float_as_uint(v.x), ROUND ? cvt_tf32(v.y) : __float_as_uint(v.y),
                         ROUND ? cvt_tf32(v.z) : __float_as_uint(v.z), ROUND ? cvt_tf32(v.w) : __float_as_uint(v.w)};
#pragma unroll
  for (int pp = 0; pp < C::H / 2; ++pp) {
    const int a = JJ - 2 * pp;
    if (a >= 0 && a < C::NA) {
      uint4 av;
      uint32_t e;
      asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(av.x), "=r"(av.y), "=r"(av.z), "=r"(av.w)
                   : "r"(ops_a + (uint32_t)(a * 32 * 16)));
      asm volatile("ld.shared.u32 %0, [%1];" : "=r"(e) : "r"(ops_e + (uint32_t)(a * 32 * 4)));
      mma_sp_tf32(acc[pp], av, e, b);
    }
  }
  if constexpr (JJ + 1 <= C::H - 2 + C::NA - 1) sp_tf32_row_smem_ops<C, SP, ROUND, JJ + 1>(addr, ops_a, ops_e, acc);
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

// Split precisions.  FP16 hi/lo: v = hi + lo * 2^-11 (lo scaled by 2^11);
// BF16 hi/mid/lo: v = hi + mid + lo, 24 significant bits.  The products kept
// are those above 2^-24 relative: FP16 hi*hi, hi*lo, lo*hi; BF16 hi*hi,
// hi*mid, mid*hi, hi*lo, lo*hi, mid*mid.  They run in passes over the input
// rows; pass P applies
//  * per pair of input rows (j, j+1) one k32 MMA [K_x(a) | K_x(a+1)] x
//    [X_x(j); X_x(j+1)] with x = hi in pass 0 (BF16 pass 1: x = mid);
//  * per input row one k32 MMA [K_hi(a) | K_y(a)] x [X_y(j); X_hi(j)] with
//    y = lo for FP16, y = mid in BF16 pass 0 and lo in pass 1.
// The hi*hi products go to accM, each MMA into a fresh zero accumulator
// that is then added in FP32: the tensor core adds a chain's products to its
// running sum with fewer bits below the sum's leading digit than an FP32
// add keeps, which shrinks the result by a few units in the last place per
// step (measured: a relative error growing linearly with the step count on
// fields of one sign); a fresh accumulator is the size of the products.
// Everything else goes to accC, two to three orders of magnitude smaller.
template <bool BF16, int PASS>
__device__ __forceinline__ void split_terms(const float4& v, uint32_t (&two)[2], uint32_t (&cross)[2],
                                            uint32_t (&hi)[2]) {
  if (!BF16) {
    hi[0] = pack_half2(v.x, v.y);
    hi[1] = pack_half2(v.z, v.w);
    const float2 h01 = unpack_half2(hi[0]), h23 = unpack_half2(hi[1]);
    cross[0] = pack_half2((v.x - h01.x) * 2048.0f, (v.y - h01.y) * 2048.0f);
    cross[1] = pack_half2((v.z - h23.x) * 2048.0f, (v.w - h23.y) * 2048.0f);
    two[0] = hi[0];
    two[1] = hi[1];
  } else {
    hi[0] = pack_bf162(v.x, v.y);
    hi[1] = pack_bf162(v.z, v.w);
    const float2 h01 = unpack_bf162(hi[0]), h23 = unpack_bf162(hi[1]);
    // v - hi is exact in FP32 (hi holds v's leading 8 bits), and so is
    // v - hi - mid below
    const float r0 = v.x - h01.x, r1 = v.y - h01.y, r2 = v.z - h23.x, r3 = v.w - h23.y;
    uint32_t mid[2] = {pack_bf162(r0, r1), pack_bf162(r2, r3)};
    if (PASS == 0) {
      two[0] = hi[0];
      two[1] = hi[1];
      cross[0] = mid[0];
      cross[1] = mid[1];
    } else {
      const float2 m01 = unpack_bf162(mid[0]), m23 = unpack_bf162(mid[1]);
      two[0] = mid[0];
      two[1] = mid[1];
      cross[0] = pack_bf162(r0 - m01.x, r1 - m01.y);
      cross[1] = pack_bf162(r2 - m23.x, r3 - m23.y);
    }
  }
}

template <class C, bool BF16>
__device__ __forceinline__ void mma_k32(float (&d)[4], const uint4& a, uint32_t e, uint32_t b0, uint32_t b1,
                                        uint32_t b2, uint32_t b3) {
  if (BF16) mma_sp_bf16_k32(d, a, e, b0, b1, b2, b3);
  else mma_sp_f16_k32(d, a, e, b0, b1, b2, b3);
}

// Whether rows JJ, JJ + 1 (JJ even) feed a two-row combo (a0, a0 + 1),
// a0 = JJ - 2pp, that touches the applied A indices AMIN..AMAX.
template <class C, int AMIN, int AMAX>
__host__ __device__ constexpr bool split_rows_needed(int jj) {
  for (int pp = 0; pp < C::H / 2; ++pp) {
    const int a0 = jj - 2 * pp;
    if (a0 >= 0 && a0 + 1 < C::NA && a0 <= AMAX && a0 + 1 >= AMIN) return true;
  }
  return false;
}

// Only the A indices AMIN..AMAX are applied (all by default; a 3-D star's
// off-centre planes apply ry, ry + 1): a two-row combo runs when one of its
// two kernel rows is applied (the other one is zero in the packed operand),
// a cross combo only for an applied index, and rows no combo reads are not
// loaded.
template <class C, bool BF16, int PASS, int SP, int JJ, int AMIN, int AMAX>
__device__ __forceinline__ void sp_split_rows(uint32_t addr, const uint4 (&Am)[C::RY + 1],
                                              const uint32_t (&Em)[C::RY + 1], const uint4 (&Ac)[C::NA],
                                              const uint32_t (&Ec)[C::NA], float (&accM)[C::H / 2][4],
                                              float (&accC)[C::H / 2][4]) {
  if constexpr (split_rows_needed<C, AMIN, AMAX>(JJ)) {
    uint32_t t0[2], c0[2], h0[2], t1[2], c1[2], h1[2];
    split_terms<BF16, PASS>(lds128_at<JJ * SP * 4>(addr), t0, c0, h0);
    split_terms<BF16, PASS>(lds128_at<(JJ + 1) * SP * 4>(addr), t1, c1, h1);
#pragma unroll
    for (int pp = 0; pp < C::H / 2; ++pp) {
      const int a0 = JJ - 2 * pp;  // even; rows JJ, JJ+1 use A indices a0, a0+1
      if (a0 >= 0 && a0 + 1 < C::NA && a0 <= AMAX && a0 + 1 >= AMIN) {
        if (PASS == 0) {
          float f[4] = {0.f, 0.f, 0.f, 0.f};
          mma_k32<C, BF16>(f, Am[a0 / 2], Em[a0 / 2], t0[0], t0[1], t1[0], t1[1]);
#pragma unroll
          for (int i = 0; i < 4; ++i) accM[pp][i] += f[i];
        } else {
          mma_k32<C, BF16>(accC[pp], Am[a0 / 2], Em[a0 / 2], t0[0], t0[1], t1[0], t1[1]);
        }
        if (a0 >= AMIN) mma_k32<C, BF16>(accC[pp], Ac[a0], Ec[a0], c0[0], c0[1], h0[0], h0[1]);
        if (a0 + 1 <= AMAX) mma_k32<C, BF16>(accC[pp], Ac[a0 + 1], Ec[a0 + 1], c1[0], c1[1], h1[0], h1[1]);
      }
    }
  }
  if constexpr (JJ + 2 < C::H + 2 * C::RY)
    sp_split_rows<C, BF16, PASS, SP, JJ + 2, AMIN, AMAX>(addr, Am, Em, Ac, Ec, accM, accC);
}

template <class C, bool BF16, int PASS = 0, int SP = C::SX, int AMIN = 0, int AMAX = C::NA - 1>
__device__ __forceinline__ void plane_sp_split(const float* row0, const uint4 (&Am)[C::RY + 1],
                                               const uint32_t (&Em)[C::RY + 1], const uint4 (&Ac)[C::NA],
                                               const uint32_t (&Ec)[C::NA], float (&accM)[C::H / 2][4],
                                               float (&accC)[C::H / 2][4]) {
  sp_split_rows<C, BF16, PASS, SP, 0, AMIN, AMAX>(smem_u32(row0), Am, Em, Ac, Ec, accM, accC);
}

// Packed combos of one pass of a split precision: (RY + 1) two-row combos,
// then NA one-row combos, starting at combo `first`.
template <class C>
__device__ __forceinline__ void load_split_operands(const StepArgs& args, int first, int lane,
                                                    uint4 (&Am)[C::RY + 1], uint32_t (&Em)[C::RY + 1],
                                                    uint4 (&A)[C::NA], uint32_t (&E)[C::NA]) {
#pragma unroll
  for (int c = 0; c <= C::RY; ++c) {
    Am[c] = args.a_words[(size_t)(first + c) * 32 + lane];
    Em[c] = args.meta[(size_t)(first + c) * 32 + lane];
  }
#pragma unroll
  for (int a = 0; a < C::NA; ++a) {
    A[a] = args.a_words[(size_t)(first + C::RY + 1 + a) * 32 + lane];
    E[a] = args.meta[(size_t)(first + C::RY + 1 + a) * 32 + lane];
  }
}

// The whole split product of one dz plane (index dzi) into accM / accC:
// FP16 one pass with the operands already in registers; BF16 two passes,
// each loading its operands first.  AMIN..AMAX: the applied A indices.
template <class C, Mode MODE, int SP = C::SX, int AMIN = 0, int AMAX = C::NA - 1>
__device__ __forceinline__ void plane_split(const StepArgs& args, int dzi, int lane, const float* row0,
                                            uint4 (&Am)[C::RY + 1], uint32_t (&Em)[C::RY + 1], uint4 (&A)[C::NA],
                                            uint32_t (&E)[C::NA], float (&accM)[C::H / 2][4],
                                            float (&accC)[C::H / 2][4]) {
  constexpr int kPass = (C::RY + 1) + C::NA;
  if (MODE == Mode::SpF16x2) {
    plane_sp_split<C, false, 0, SP, AMIN, AMAX>(row0, Am, Em, A, E, accM, accC);
  } else {
    // a loop the compiler keeps: one pass's operands live at a time
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      load_split_operands<C>(args, (2 * dzi + pass) * kPass, lane, Am, Em, A, E);
      if (pass == 0) plane_sp_split<C, true, 0, SP, AMIN, AMAX>(row0, Am, Em, A, E, accM, accC);
      else plane_sp_split<C, true, 1, SP, AMIN, AMAX>(row0, Am, Em, A, E, accM, accC);
    }
  }
}

// accM + accC with accC's scale: 2^-11 for FP16, 1 for BF16.
template <Mode MODE, int N>
__device__ __forceinline__ void combine_split(float (&accM)[N][4], const float (&accC)[N][4]) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      accM[i][j] = MODE == Mode::SpF16x2 ? fmaf(accC[i][j], 1.0f / 2048.0f, accM[i][j]) : accM[i][j] + accC[i][j];
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
  constexpr int CPP = MODE == Mode::SpF16x2 ? (C::RY + 1) + NA : NA;
  uint4 A[NA];
  uint32_t E[NA];
  uint4 Ad[NA][2];
  uint4 Am[C::RY + 1];
  uint32_t Em[C::RY + 1];
  float W[(2 * C::RY + 1) * (2 * C::RX + 1)];
  auto load_operands = [&](int dzi) {
    if (MODE == Mode::SpTF32NoCO) {
      // staged in shared memory below and read there by every MMA
    } else if (is_sp_tf32(MODE)) {
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
    } else if (MODE == Mode::SpF16x2) {
      load_split_operands<C>(args, dzi * CPP, lane, Am, Em, A, E);
    } else if (MODE == Mode::SpBF16x3) {
      // two passes of operands, loaded by plane_split
    } else {
      constexpr int NW = (2 * C::RY + 1) * (2 * C::RX + 1);
#pragma unroll
      for (int i = 0; i < NW; ++i) W[i] = args.w[(size_t)dzi * NW + i];
    }
  };
  if (C::RZ == 0) load_operands(0);
  // SpTF32NoCO (2-D): the plane's packed operands, then its metadata words
  const uint32_t ops_smem = smem_u32(smem + 2 * C::kStageStride + 64);
  if constexpr (MODE == Mode::SpTF32NoCO) {
    static_assert(C::RZ == 0, "2-D only");
    uint4* oa = reinterpret_cast<uint4*>(smem + 2 * C::kStageStride + 64);
    uint32_t* oe = reinterpret_cast<uint32_t*>(oa + NA * 32);
    for (int i = tid; i < NA * 32; i += C::kThreads) {
      oa[i] = args.a_words[i];
      oe[i] = args.meta[i];
    }
    __syncthreads();
  }
  (void)ops_smem;

  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int s = it & 1;
    float* S = stage(s);
    int x0, y0, z0;
    coords(t, x0, y0, z0);
    if (use_tma) {
      const bool ok = mbar_wait_bounded(&full[s], (it >> 1) & 1, args.status, args.wait_cycles);
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
      // FP32 FMA stencil: lane l computes columns 2l and 2l + 1 of its
      // warp's 64 and loads the inputs of a row as 8-byte pairs (v[e] = tile
      // row column 2l + e of the warp, e = 0..9; output column c reads
      // v[c - 2l + 4 - r .. + r])
      constexpr int E0 = (4 - C::RX) / 2, E1 = (5 + C::RX) / 2;
      float acc[C::H][2];
#pragma unroll
      for (int i = 0; i < C::H; ++i) acc[i][0] = acc[i][1] = 0.f;
#pragma unroll 1
      for (int dzi = 0; dzi < 2 * C::RZ + 1; ++dzi) {
        if (C::RZ != 0) load_operands(dzi);
        const float* pl = S + (size_t)(wz + dzi) * C::SY * C::SX + (size_t)(wy * C::H) * C::SX + wx * 64 + 2 * lane;
#pragma unroll
        for (int jj = 0; jj < C::H + 2 * C::RY; ++jj) {
          float v[10];
#pragma unroll
          for (int m = E0; m <= E1; ++m) {
            const float2 t = *reinterpret_cast<const float2*>(pl + jj * C::SX + 2 * m);
            v[2 * m] = t.x;
            v[2 * m + 1] = t.y;
          }
#pragma unroll
          for (int yy = 0; yy < C::H; ++yy) {
            const int dy = jj - C::RY - yy;
            if (dy >= -C::RY && dy <= C::RY) {
#pragma unroll
              for (int k = 0; k < 2 * C::RX + 1; ++k) {
                const float wv = W[(dy + C::RY) * (2 * C::RX + 1) + k];
                acc[yy][0] = fmaf(wv, v[4 - C::RX + k], acc[yy][0]);
                acc[yy][1] = fmaf(wv, v[5 - C::RX + k], acc[yy][1]);
              }
            }
          }
        }
      }
      if (z < args.nz) {
        float* o = args.dst + (z * args.ny + ybase) * args.pitch + xbase + 2 * lane;
        const int pitch = (int)args.pitch;
        const int ylim = (int)(args.ny - ybase < C::H ? args.ny - ybase : C::H);
        const int xlim = (int)(args.nx - xbase < 64 ? args.nx - xbase : 64);
#pragma unroll
        for (int yy = 0; yy < C::H; ++yy) {
          if (yy < ylim) {
#pragma unroll
            for (int c = 0; c < 2; ++c)
              if (2 * lane + c < xlim) o[(size_t)yy * pitch + c] = acc[yy][c];
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
        if (MODE == Mode::SpTF32Copy) {
          // the explicit row-swap copy: every window of 16 input points (8
          // apart, overlapping) goes to a buffer of its own in the order the
          // MMA's K index wants, four 16-byte chunks per window with chunk c
          // taken from window chunk sigma(c); the operands then load 16
          // contiguous bytes per lane from it
          constexpr int NSEG = C::BX / 8, WP = NSEG * 16;
          float* Wb = reinterpret_cast<float*>(smem + 2 * C::kStageStride + 64);
          const float* Sp = S + (size_t)(wz + dzi) * C::SY * C::SX;
          for (int e = tid; e < C::SY * NSEG * 4; e += C::kThreads) {
            const int row = e / (NSEG * 4), seg = (e / 4) % NSEG, cc = e % 4;
            const int sig = (cc == 1) ? 2 : (cc == 2) ? 1 : cc;
            *reinterpret_cast<float4*>(Wb + row * WP + seg * 16 + 4 * cc) =
                *reinterpret_cast<const float4*>(Sp + row * C::SX + 8 * seg + 4 * sig);
          }
          __syncthreads();
          const float* wrow0 = Wb + (wy * C::H) * WP + (wx * 8 + g) * 16 + 4 * q;
          plane_sp_tf32<C, WP, RIN>(wrow0, A, E, acc);
          __syncthreads();  // the buffer is rewritten for the next plane or tile
        } else if (MODE == Mode::SpTF32NoCO) {
          sp_tf32_row_smem_ops<C, C::SX, RIN, 0>(smem_u32(row0), ops_smem + 16u * lane,
                                                 ops_smem + (uint32_t)(NA * 32 * 16) + 4u * lane, acc);
        } else if (MODE == Mode::SpTF32) {
          if (centre_only) plane_sp_tf32_centre<C, C::SX, RIN>(row0, A, E, acc);
          else plane_sp_tf32<C, C::SX, RIN>(row0, A, E, acc);
        } else if (MODE == Mode::DenseTF32) {
          if (centre_only) plane_dense_tf32_centre<C, C::SX, RIN>(row0, Ad, acc);
          else plane_dense_tf32<C, C::SX, RIN>(row0, Ad, acc);
        } else {
          plane_split<C, MODE>(args, dzi, lane, row0, Am, Em, A, E, acc, accC);
        }
      }
      if (MODE == Mode::SpF16x2 || MODE == Mode::SpBF16x3) combine_split<MODE>(acc, accC);
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
        (void)mbar_wait_bounded(&full[(it + k) & 1], ((it + k) >> 1) & 1, args.status, args.wait_cycles);
      }
    }
  }
}

}  // namespace spider
