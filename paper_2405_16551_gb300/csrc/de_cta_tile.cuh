// de_cta_tile.cuh -- building blocks of the split-precision persistent
// kernels in which a CTA runs the tensor-core products of its own targets
// (k_persist_cta for one run, k_persist_batch for a batch): operand sizes, the
// split store of y into the 16-row B operand, the copy of the split M into the
// 128-row A operand, and the whole-CTA FP64 evaluation of the rows the split
// error bound cannot decide.
#pragma once
#include <cuda_runtime.h>

#include "de_device.cuh"
#include "de_tcgen05.cuh"

namespace de {

constexpr int kCtaRowsMax = 16;  // targets per CTA tile (two row groups of the y operand)

// Bytes of one part (high or low) of the 16-row y operand: k-groups of 16
// bytes, each holding two 8-row core matrices (k-group stride 256 bytes).
__host__ __device__ inline uint32_t cta_y_part(const RunDesc& R) { return (uint32_t)(R.kpad * R.esz / 16) * 256u; }
// ... and of the 128-row M operand (k-group stride 16 x 128 = 2048 bytes).
__host__ __device__ inline uint32_t cta_m_part(const RunDesc& R) { return (uint32_t)(R.kpad * R.esz / 16) * 2048u; }
// Row stride (floats) of the accumulator rows in shared memory.
__host__ __device__ inline int cta_zstride(const RunDesc& R) { return R.ntn + 4; }

// y[0..3] (coordinates j0..j0+3 of row m < 16 of the y operand) as high and
// low parts.
template <int ESZ>
__device__ __forceinline__ void cta_store_split4(uint8_t* A, uint32_t a_part, int m, int j0, const float y[4]) {
  const int rg = m >> 3, rr = m & 7;
  if constexpr (ESZ == 2) {
    __nv_bfloat16 hi[4], lo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      hi[q] = __float2bfloat16_rn(y[q]);
      lo[q] = __float2bfloat16_rn(y[q] - __bfloat162float(hi[q]));  // exact residual, then rounded
    }
    const uint32_t off = (uint32_t)(j0 >> 3) * 256u + (uint32_t)rg * 128u + (uint32_t)rr * 16u + (uint32_t)(j0 & 7) * 2u;
    *reinterpret_cast<uint2*>(A + off) = *reinterpret_cast<const uint2*>(hi);
    *reinterpret_cast<uint2*>(A + a_part + off) = *reinterpret_cast<const uint2*>(lo);
  } else {
    float4 hi, lo;
    hi.x = to_tf32(y[0]);
    hi.y = to_tf32(y[1]);
    hi.z = to_tf32(y[2]);
    hi.w = to_tf32(y[3]);
    lo.x = to_tf32(y[0] - hi.x);
    lo.y = to_tf32(y[1] - hi.y);
    lo.z = to_tf32(y[2] - hi.z);
    lo.w = to_tf32(y[3] - hi.w);
    const uint32_t off = (uint32_t)(j0 >> 2) * 256u + (uint32_t)rg * 128u + (uint32_t)rr * 16u;
    *reinterpret_cast<float4*>(A + off) = hi;
    *reinterpret_cast<float4*>(A + a_part + off) = lo;
  }
}

// FP64 fitness of the shifted vector y (shared memory, d values) by the
// whole CTA: z_j = sum_k M_jk y_k (M^T read at L2, two accumulator chains),
// the objective terms per coordinate, then a fixed-order sum (per warp an
// xor tree, then the warps in order).  Every thread returns the value.
__device__ __forceinline__ double cta_fitness_fp64(const RunDesc& R, const double* sy, double* red) {
  const int d = R.d, obj = R.obj, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ double s_zv[129];
  if (tid < d) {
    double z;
    if (R.rotate) {
      double p0 = 0.0, p1 = 0.0;
      int k = 0;
      for (; k + 1 < d; k += 2) {
        p0 = fma(__ldcg(R.MT + (size_t)k * d + tid), sy[k], p0);
        p1 = fma(__ldcg(R.MT + (size_t)(k + 1) * d + tid), sy[k + 1], p1);
      }
      if (k < d) p0 = fma(__ldcg(R.MT + (size_t)k * d + tid), sy[k], p0);
      z = p0 + p1;
    } else {
      z = sy[tid];
    }
    s_zv[tid] = z;
  }
  __syncthreads();
  double t1 = 0.0, t2 = 0.0;
  if (tid < d) {
    const double z = s_zv[tid];
    if (obj == kObjSphere) {
      t1 = z * z;
    } else if (obj == kObjRastrigin) {
      t1 = z * z - 10.0 * cos2pi_f64(z) + 10.0;
    } else if (obj == kObjAckley) {
      t1 = z * z;
      t2 = cos2pi_f64(z);
    } else if (tid + 1 < d) {  // Rosenbrock at t = z + 1
      const double t0 = z + 1.0, tn = s_zv[tid + 1] + 1.0;
      const double a = tn - t0 * t0, b = t0 - 1.0;
      t1 = 100.0 * a * a + b * b;
    }
  }
  t1 = warp_sum(t1);
  t2 = warp_sum(t2);
  if (lane == 0) {
    red[warp] = t1;
    red[8 + warp] = t2;
  }
  __syncthreads();
  double s1 = 0.0, s2 = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    s1 += red[w];
    s2 += red[8 + w];
  }
  __syncthreads();  // red and s_zv are reused by the next call
  return obj == kObjAckley ? 20.0 + 2.718281828459045 - 20.0 * exp(-0.2 * sqrt(s1 / d)) - exp(s2 / d) : s1;
}

// The split M (global copy: ntn rows, k-group stride ntn / 8 x 128 bytes) as
// the products' 128-row A operand in shared memory (k-group stride 2048
// bytes, rows past ntn zero), by all threads of the CTA.
template <int ESZ>
__device__ __forceinline__ void cta_load_m(const RunDesc& R, uint8_t* sMop, uint32_t m_part) {
  const int nkg = R.kpad * ESZ / 16, rgs = R.ntn / 8;
  const size_t gpart = (size_t)R.b_tile_bytes / 2;
  for (int u = threadIdx.x; u < 2 * nkg * 128; u += blockDim.x) {
    const int part = u / (nkg * 128), rem = u % (nkg * 128);
    const int kg = rem / 128, rg = (rem / 8) % 16, rr = rem % 8;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (rg < rgs) v = __ldg(reinterpret_cast<const uint4*>(R.B + part * gpart + (size_t)(kg * rgs + rg) * 128 + rr * 16));
    *reinterpret_cast<uint4*>(sMop + part * m_part + (uint32_t)kg * 2048u + (uint32_t)rg * 128u + (uint32_t)rr * 16u) = v;
  }
}

}  // namespace de
