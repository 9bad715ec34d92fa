// GPU FP64 validation reductions: norms and error against an FP64 reference,
// and the constant-field invariant check.  These are the only FP64 kernels of
// the library; the stencil itself never computes in FP64.
#include <algorithm>
#include <cmath>
#include <string>

#include "spider_internal.h"

namespace spider {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Per-block partial results: [block][4] = sum a^2, sum ref^2, sum (a-ref)^2, max |a-ref|.
__global__ void norms_partial(const float* __restrict__ a, const double* __restrict__ ref, int64_t n,
                              double* __restrict__ partial) {
  double saa = 0, srr = 0, sdd = 0, md = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = (double)a[i];
    saa += x * x;
    if (ref) {
      const double r = ref[i], d = x - r;
      srr += r * r;
      sdd += d * d;
      md = fmax(md, fabs(d));
    }
  }
  __shared__ double sh[4][kThreads / 32];
  saa = warp_sum(saa);
  srr = warp_sum(srr);
  sdd = warp_sum(sdd);
  md = warp_max(md);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) { sh[0][w] = saa; sh[1][w] = srr; sh[2][w] = sdd; sh[3][w] = md; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int k = 0; k < kThreads / 32; ++k) {
      t[0] += sh[0][k]; t[1] += sh[1][k]; t[2] += sh[2][k]; t[3] = fmax(t[3], sh[3][k]);
    }
    for (int k = 0; k < 4; ++k) partial[(size_t)blockIdx.x * 4 + k] = t[k];
  }
}

__global__ void norms_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t[4] = {0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b) {
    t[0] += partial[b * 4 + 0]; t[1] += partial[b * 4 + 1]; t[2] += partial[b * 4 + 2];
    t[3] = fmax(t[3], partial[b * 4 + 3]);
  }
  for (int k = 0; k < 4; ++k) out[k] = t[k];
}

__global__ void constant_partial(const float* __restrict__ a, int64_t nz, int64_t ny, int64_t nx, int64_t mz,
                                 int64_t my, int64_t mx, double value, double* __restrict__ partial) {
  double md = 0;
  const int64_t n = nz * ny * nx;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
    if (x < mx || x >= nx - mx || y < my || y >= ny - my || z < mz || z >= nz - mz) continue;
    md = fmax(md, fabs((double)a[i] - value));
  }
  __shared__ double sh[kThreads / 32];
  md = warp_max(md);
  if (threadIdx.x % 32 == 0) sh[threadIdx.x / 32] = md;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < kThreads / 32; ++k) t = fmax(t, sh[k]);
    partial[blockIdx.x] = t;
  }
}

__global__ void max_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0;
  for (int b = 0; b < nblocks; ++b) t = fmax(t, partial[b]);
  out[0] = t;
}

int reduction_blocks(int64_t n) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
}

spider_status cuda_status(cudaError_t e, const char* what) {
  return fail(SPIDER_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace
}  // namespace spider

using namespace spider;

extern "C" spider_status spider_norms_fp64(const float* a, const double* ref, int64_t n, double* out,
                                           cudaStream_t stream) {
  set_error("");
  if (!a || !out || n < 1) return fail(SPIDER_ERR_INVALID, "bad arguments");
  const int nb = reduction_blocks(n);
  double* buf = nullptr;  // [nb][4] partials + [4] result
  cudaError_t e = cudaMalloc(&buf, sizeof(double) * ((size_t)nb * 4 + 4));
  if (e != cudaSuccess) { cudaGetLastError(); return fail(SPIDER_ERR_OOM, "reduction buffer"); }
  norms_partial<<<nb, kThreads, 0, stream>>>(a, ref, n, buf);
  norms_final<<<1, 32, 0, stream>>>(buf, nb, buf + (size_t)nb * 4);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, buf + (size_t)nb * 4, sizeof(double) * 4, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_status(e, "norm reduction");
  return SPIDER_OK;
}

extern "C" spider_status spider_constant_check_fp64(const float* a, int ndim, const int64_t* extents, int64_t margin,
                                                    double value, double* max_dev, cudaStream_t stream) {
  set_error("");
  if (!a || !extents || !max_dev || ndim < 1 || ndim > 3 || margin < 0) return fail(SPIDER_ERR_INVALID, "bad arguments");
  int64_t nx = extents[ndim - 1], ny = ndim >= 2 ? extents[ndim - 2] : 1, nz = ndim >= 3 ? extents[0] : 1;
  if (nx < 1 || ny < 1 || nz < 1) return fail(SPIDER_ERR_INVALID, "bad extents");
  const int64_t mx = margin, my = ndim >= 2 ? margin : 0, mz = ndim >= 3 ? margin : 0;
  const int64_t n = nx * ny * nz;
  const int nb = reduction_blocks(n);
  double* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, sizeof(double) * ((size_t)nb + 1));
  if (e != cudaSuccess) { cudaGetLastError(); return fail(SPIDER_ERR_OOM, "reduction buffer"); }
  constant_partial<<<nb, kThreads, 0, stream>>>(a, nz, ny, nx, mz, my, mx, value, buf);
  max_final<<<1, 32, 0, stream>>>(buf, nb, buf + nb);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(max_dev, buf + nb, sizeof(double), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_status(e, "constant check");
  return SPIDER_OK;
}
