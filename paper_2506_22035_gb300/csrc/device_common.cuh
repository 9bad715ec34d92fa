// Device helpers: shared-memory addressing, mbarrier waits with a time limit,
// TMA tile loads, TF32 / FP16 / BF16 conversion and the tensor-core MMAs.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

namespace spider {

// Device status word values (DeviceState::status).
constexpr int kStatusOk = 0;
constexpr int kStatusTimeout = 1;

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may start while the previous kernel in the
// stream finishes; it must wait here before touching any grid the previous
// kernel reads or writes.  launch_dependents lets the next kernel's CTAs be
// scheduled early (they wait in griddep_wait in turn).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of the barrier; returns false (and records a
// timeout in *status) if it has not completed within `limit` SM cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) {
      atomicExch(status, kStatusTimeout);
      return false;
    }
  }
  return true;
}

// 3-D tiled TMA load of the box at (x, y, z) (elements) into shared memory,
// completing on `bar`.  Out-of-range elements of the box read as zero (the
// tensor map is encoded with zero OOB fill), which is the zero Dirichlet halo.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                            int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ float4 lds128(const float* p) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(smem_u32(p))
               : "memory");
  return v;
}

// 16-byte shared-memory load at shared-window address `addr` + OFF bytes;
// the constant offset folds into the instruction.  Not volatile: the
// compiler may schedule it early (the memory clobber keeps it on the right
// side of barriers and stores).
template <int OFF>
__device__ __forceinline__ float4 lds128_at(uint32_t addr) {
  float4 v;
  asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4+%5];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr), "n"(OFF)
               : "memory");
  return v;
}

// Asynchronous 4-byte global -> shared copy; src_bytes = 0 writes a zero
// (the source address is then not read, but it is kept inside the grid).
__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gsrc, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(smem_dst)), "l"(gsrc),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Loads the box of SZ x SY x SX floats whose first element is grid point
// (z0, y0, x0) into shared memory (row pitch SX), zero outside the
// nz x ny x nx grid, for grids whose rows TMA cannot describe.  Rows are
// spread over the warps, columns over the lanes (coalesced); every thread
// keeps many copies in flight.  The caller waits with a barrier afterwards.
__device__ __forceinline__ void load_box_async(const float* __restrict__ src, int64_t nx, int64_t ny, int64_t nz,
                                               int64_t x0, int64_t y0, int64_t z0, int SX, int SY, int SZ, float* S,
                                               int warp, int nwarps, int lane) {
  for (int row = warp; row < SY * SZ; row += nwarps) {
    const int zz = row / SY, yy = row - zz * SY;
    const int64_t gz = z0 + zz, gy = y0 + yy;
    const bool row_ok = gz >= 0 && gz < nz && gy >= 0 && gy < ny;
    const float* srow = src + (row_ok ? (gz * ny + gy) * nx : 0);
    float* drow = S + row * SX;
    for (int xx = lane; xx < SX; xx += 32) {
      const int64_t gx = x0 + xx;
      const bool ok = row_ok && gx >= 0 && gx < nx;
      cp_async4(drow + xx, ok ? srow + gx : src, ok);
    }
  }
  cp_async_wait_all();
}

// FP32 -> TF32, round to nearest, ties to even (NaN stays NaN).  The
// ties-away form (cvt.rna) measured three times the instructions for the
// same nearest rounding; the two differ only on exact ties.
__device__ __forceinline__ uint32_t cvt_tf32(float x) {
  uint32_t r;
  asm("cvt.rn.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
  __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack_bf162(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float2 unpack_half2(uint32_t v) {
  __half2 h = *reinterpret_cast<__half2*>(&v);
  return __half22float2(h);
}
__device__ __forceinline__ float2 unpack_bf162(uint32_t v) {
  // bf16 -> f32 is exact: the 16 bits become the high half of the f32.
  return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xFFFF0000u));
}

// The MMA wrappers are not volatile: each is a pure function of its operands,
// so the compiler is free to interleave them with the loads of later rows.

// D += A(sparse 1:2, TF32) * B, m16n8k16.
__device__ __forceinline__ void mma_sp_tf32(float (&d)[4], const uint4& a, uint32_t e, const uint32_t (&b)[4]) {
  asm(
      "mma.sp::ordered_metadata.sync.aligned.m16n8k16.row.col.f32.tf32.tf32.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9,%10,%11}, {%0,%1,%2,%3}, %12, 0x0;"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(e));
}

// D += A(dense TF32) * B, m16n8k8.
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint4& a, uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// D += A(sparse 2:4, FP16) * B, m16n8k32.
__device__ __forceinline__ void mma_sp_f16_k32(float (&d)[4], const uint4& a, uint32_t e, uint32_t b0, uint32_t b1,
                                               uint32_t b2, uint32_t b3) {
  asm(
      "mma.sp::ordered_metadata.sync.aligned.m16n8k32.row.col.f32.f16.f16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9,%10,%11}, {%0,%1,%2,%3}, %12, 0x0;"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1), "r"(b2), "r"(b3), "r"(e));
}

// D += A(sparse 2:4, BF16) * B, m16n8k32.
__device__ __forceinline__ void mma_sp_bf16_k32(float (&d)[4], const uint4& a, uint32_t e, uint32_t b0, uint32_t b1,
                                                uint32_t b2, uint32_t b3) {
  asm(
      "mma.sp::ordered_metadata.sync.aligned.m16n8k32.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9,%10,%11}, {%0,%1,%2,%3}, %12, 0x0;"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1), "r"(b2), "r"(b3), "r"(e));
}

}  // namespace spider
