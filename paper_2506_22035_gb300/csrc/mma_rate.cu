// Peak issue rate of the warp-level tensor-core MMAs the stencil kernels use,
// measured on the running GPU: the denominator of their tensor-pipe roofline.
//
// Every warp keeps its A, B and metadata operands in registers and issues
// eight independent accumulator chains per loop iteration, so neither memory
// nor a dependency chain limits the rate; two CTAs of eight warps per SM.
#include <algorithm>
#include <string>

#include "device_common.cuh"
#include "launch.h"
#include "spider_internal.h"

namespace spider {
namespace {

constexpr int kChains = 8;
constexpr int kRateThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kRateThreads) mma_rate_kernel(int iters, float* sink) {
  const uint32_t lane = threadIdx.x & 31;
  // small operands (no overflow over the loop); metadata nibble 0b0100 keeps
  // elements 0 and 1 of every group, valid for the 1:2 and 2:4 forms
  const uint32_t one16 = KIND == 2 ? 0x3F803F80u : 0x3C003C00u;  // (1, 1) in BF16 / FP16
  const uint32_t tiny16 = KIND == 2 ? 0x3A803A80u : 0x14001400u; // (2^-10, 2^-10)
  const uint32_t av = KIND == 0 || KIND == 3 ? 0x3F800000u : one16;
  const uint32_t bv = KIND == 0 || KIND == 3 ? (0x3A800000u ^ (lane << 13)) : (tiny16 ^ lane);
  const uint4 a = make_uint4(av, av, av, av);
  const uint32_t b[4] = {bv, bv, bv, bv};
  const uint32_t e = 0x44444444u;
  float acc[kChains][4];
#pragma unroll
  for (int k = 0; k < kChains; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[k][j] = 0.f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if (KIND == 0) mma_sp_tf32(acc[k], a, e, b);
      else if (KIND == 1) mma_sp_f16_k32(acc[k], a, e, b[0], b[1], b[2], b[3]);
      else if (KIND == 2) mma_sp_bf16_k32(acc[k], a, e, b[0], b[1], b[2], b[3]);
      else mma_tf32(acc[k], a, b[0], b[1]);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += acc[k][0] + acc[k][1] + acc[k][2] + acc[k][3];
  sink[blockIdx.x * kRateThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace spider

using namespace spider;

extern "C" spider_status spider_measure_mma_rate(int kind, double* mma_per_s, cudaStream_t stream) {
  set_error("");
  if (!mma_per_s) return fail(SPIDER_ERR_INVALID, "mma_per_s is NULL");
  if (kind < 0 || kind > 3) return fail(SPIDER_ERR_INVALID, "kind must be 0..3");
  void (*kern)(int, float*) = kind == 0   ? mma_rate_kernel<0>
                              : kind == 1 ? mma_rate_kernel<1>
                              : kind == 2 ? mma_rate_kernel<2>
                                          : mma_rate_kernel<3>;
  const int grid = 2 * device_sm_count();
  const int iters = 4096;
  float* sink = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaMalloc(&sink, (size_t)grid * kRateThreads * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float best_ms = 0.f;
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {  // the first launch warms up
    e = cudaEventRecord(t0, stream);
    if (e == cudaSuccess) {
      kern<<<grid, kRateThreads, 0, stream>>>(iters, sink);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t1, stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess && rep > 0) best_ms = best_ms == 0.f ? ms : std::min(best_ms, ms);
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return fail(SPIDER_ERR_CUDA, std::string("mma rate: ") + cudaGetErrorString(e));
  const double mmas = (double)grid * (kRateThreads / 32) * kChains * (double)iters;
  *mma_per_s = mmas / (best_ms * 1e-3);
  return SPIDER_OK;
}
