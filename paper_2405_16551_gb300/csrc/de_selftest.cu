// de_selftest.cu -- self-tests with no counterpart in the paper:
//   * the library's own FP64 -> FP32 rounding (to_f32_rn, used for the
//     split-precision operands) against the GPU's conversion instruction,
//     so that tests can check the integer rounding bit for bit;
//   * the device's FP64 fused multiply-add throughput, the measured peak the
//     FP64 kernels are reported against.
#include <cuda_runtime.h>

#include <algorithm>

#include "de.h"
#include "de_device.cuh"

namespace de {

__global__ void k_selftest_f32(const double* __restrict__ x, long long n, unsigned long long* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float a = to_f32_rn(x[i]);
    const float b = (float)x[i];
    const bool both_nan = a != a && b != b;
    if (!both_nan && __float_as_uint(a) != __float_as_uint(b)) atomicAdd(bad, 1ull);
  }
}

// Independent multiply-add chains per thread (enough in flight to keep the
// FP64 pipe busy); the result is stored only under a condition that never
// holds, so the chains stay live.
constexpr int kDfmaChains = 8;
__global__ void k_dfma_rate(int iters, double* __restrict__ sink) {
  double a[kDfmaChains];
#pragma unroll
  for (int k = 0; k < kDfmaChains; ++k) a[k] = 1.0 + 1e-9 * (double)(threadIdx.x + k);
  const double b = 0.9999999999, c = 1e-12;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kDfmaChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kDfmaChains; ++k) s += a[k];
  if (s == -1.0) sink[0] = s;
}

}  // namespace de

extern "C" DE_API double de_selftest_fp64_rate(void) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return -1.0;
  }
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double best = -1.0;
  const int iters = 1024, threads = 256, blocks = nsm * 4;
  if (cudaMalloc(&sink, sizeof(double)) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
      cudaEventCreate(&e1) == cudaSuccess) {
    de::k_dfma_rate<<<blocks, threads>>>(iters, sink);  // warm-up
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0);
      de::k_dfma_rate<<<blocks, threads>>>(iters, sink);
      cudaEventRecord(e1);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) {
        best = -1.0;
        break;
      }
      const double flops = 2.0 * de::kDfmaChains * (double)iters * (double)threads * (double)blocks;
      best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
  }
  if (cudaGetLastError() != cudaSuccess) best = -1.0;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  return best;
}

extern "C" DE_API int64_t de_selftest_f32_rounding(const double* x_host, int64_t n) {
  if (!x_host || n < 0) return -1;
  if (n == 0) return 0;
  double* dx = nullptr;
  unsigned long long* dbad = nullptr;
  unsigned long long bad = 0;
  int64_t out = -1;
  if (cudaMalloc(&dx, (size_t)n * sizeof(double)) == cudaSuccess &&
      cudaMalloc(&dbad, sizeof(unsigned long long)) == cudaSuccess &&
      cudaMemcpy(dx, x_host, (size_t)n * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
      cudaMemset(dbad, 0, sizeof(unsigned long long)) == cudaSuccess) {
    de::k_selftest_f32<<<152 * 4, 256>>>(dx, (long long)n, dbad);
    if (cudaGetLastError() == cudaSuccess &&
        cudaMemcpy(&bad, dbad, sizeof bad, cudaMemcpyDeviceToHost) == cudaSuccess)
      out = (int64_t)bad;
  }
  if (dx) cudaFree(dx);
  if (dbad) cudaFree(dbad);
  return out;
}
