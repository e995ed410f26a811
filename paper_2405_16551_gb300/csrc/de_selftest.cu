// de_selftest.cu -- self-test of the library's own FP64 -> FP32 rounding
// (to_f32_rn, used for the split-precision operands) against the GPU's
// conversion instruction.  The paper has no counterpart; the entry point
// exists so that tests can check the integer rounding bit for bit.
#include <cuda_runtime.h>

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

}  // namespace de

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
