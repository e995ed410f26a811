// de_tcgen05.cuh -- tensor-core building blocks shared by the split-precision
// kernels: PTX wrappers for mbarriers, bulk async copies, tcgen05.mma /
// tcgen05.ld, the split of y into high and low parts in the operand layout,
// and the FP32 objective epilogue over TMEM columns.
//
// Operand layout (no swizzle, K-major): a "core matrix" is 8 rows x 16 bytes,
// stored as 128 contiguous bytes.  Core matrix (kg, rg) -- k-group kg of 16
// bytes, row group rg of 8 rows -- sits at byte (kg * RG + rg) * 128, where RG
// is the number of row groups (16 for a 128-row A tile, ntn / 8 for an N tile
// of B).  In the instruction's shared-memory descriptor the leading byte offset
// is the stride between k-groups (RG * 128) and the stride byte offset the one
// between row groups (128).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "de_device.cuh"

namespace de {

constexpr int kTileM = 128;
constexpr int kFitThreads = 256;
constexpr int kStageBudget = 96 * 1024;
constexpr size_t kSingleStageMax = 216 * 1024;  // dynamic shared memory of one whole-K stage
constexpr int kMaxStages = 8;                   // stages of the fitness kernel's K pipeline
constexpr size_t kFitSmemMax = 200 * 1024;      // dynamic shared memory of all stages
constexpr size_t kBandSmem = 160 * 1024;        // M rows staged by one FP64 band work item
constexpr long long kWaitLimit = 1LL << 22;

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the sm_100 family; no swizzle, base offset 0
  return d;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

template <int ESZ>
__device__ __forceinline__ void mma_split(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (ESZ == 2) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}

// The same product with A in tensor memory (a_tmem: lane 0, first column of
// the K step; rows of A in lanes, K along columns, two 16-bit elements or one
// 32-bit element per column).
template <int ESZ>
__device__ __forceinline__ void mma_split_ta(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (ESZ == 2) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ float tmem_ld1(uint32_t taddr) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  return __uint_as_float(r);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// TMEM -> registers: 32, 16 or 8 consecutive columns of this warp's 32 lanes,
// load and wait in one statement.
__device__ __forceinline__ void tmem_ld_cols32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void tmem_ld_cols16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// cos(2 pi z) in FP32: 2z = k + r with k = rint(2z) and |r| <= 1/2 exact, so
// cos(2 pi z) = (-1)^k cos(pi r), and the hardware cosine sees |pi r| <= pi/2.
__device__ __forceinline__ float cos2pi(float z) {
  const float tz = 2.0f * z;
  const float k = rintf(tz);
  const float c = __cosf(3.14159265358979f * (tz - k));
  return (((int)k) & 1) ? -c : c;
}

// Write y[0..3] (coordinates j0..j0+3 of tile row m) as high and low parts
// into the A tile (hi part at Ahi, lo part at Ahi + a_part).
template <int ESZ>
__device__ __forceinline__ void store_split4(uint8_t* Ahi, uint32_t a_part, int m, int j0, const float y[4]) {
  const int rg = m >> 3, rr = m & 7;
  if constexpr (ESZ == 2) {
    __nv_bfloat16 hi[4], lo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      hi[q] = __float2bfloat16_rn(y[q]);
      lo[q] = __float2bfloat16_rn(y[q] - __bfloat162float(hi[q]));  // exact residual, then rounded
    }
    const size_t off = ((size_t)(j0 >> 3) * 16 + rg) * 128 + rr * 16 + (j0 & 7) * 2;
    *reinterpret_cast<uint2*>(Ahi + off) = *reinterpret_cast<const uint2*>(hi);
    *reinterpret_cast<uint2*>(Ahi + a_part + off) = *reinterpret_cast<const uint2*>(lo);
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
    const size_t off = ((size_t)(j0 >> 2) * 16 + rg) * 128 + rr * 16;
    *reinterpret_cast<float4*>(Ahi + off) = hi;
    *reinterpret_cast<float4*>(Ahi + a_part + off) = lo;
  }
}

// ------------------------------------------------------------------ epilogue terms
// Objective terms of up to 32 consecutive columns (w of them valid) of one
// row, starting at output coordinate nb; the array index is a compile-time
// constant after unrolling, so the columns stay in registers.
struct EpiAcc {
  float a1, a2, a3, aS, aG, prev_t;
};

template <int OBJ>
__device__ __forceinline__ void epi_cols(const float* v, int w, int nb, int d, bool first, EpiAcc& A) {
#pragma unroll
  for (int e = 0; e < 32; ++e) {
    const int n = nb + e;
    const float z = v[e];
    if (e < w && n < d) {
      if constexpr (OBJ == kObjSphere) {
        A.a1 = fmaf(z, z, A.a1);
        A.aG += 2.f * fabsf(z);
      } else if constexpr (OBJ == kObjRastrigin) {
        const float cz = cos2pi_f32(z);
        A.a1 += fmaf(z, z, fmaf(-10.f, cz, 10.f));
        A.aS += fmaf(z, z, fmaf(10.f, fabsf(cz), 10.f));
        A.aG += fmaf(2.f, fabsf(z), 62.83185307f);
      } else if constexpr (OBJ == kObjAckley) {
        const float cz = cos2pi_f32(z);
        A.a1 = fmaf(z, z, A.a1);
        A.a2 += cz;
        A.a3 += fabsf(z);
        A.aS += fabsf(cz);
      } else {  // Rosenbrock at t = z + 1: the term of coordinate n - 1
        const float t = z + 1.f;
        if (!(first && e == 0)) {
          const float aa = t - A.prev_t * A.prev_t, bb = A.prev_t - 1.f;
          A.a1 += fmaf(100.f * aa, aa, bb * bb);
          A.aG += 400.f * fabsf(A.prev_t) * fabsf(aa) + 2.f * fabsf(bb) + 200.f * fabsf(aa);
        }
        A.prev_t = t;
      }
    }
  }
}

__device__ __forceinline__ void epi_dispatch(int obj, const float* v, int w, int nb, int d, bool first, EpiAcc& A) {
  if (obj == kObjSphere) epi_cols<kObjSphere>(v, w, nb, d, first, A);
  else if (obj == kObjRastrigin) epi_cols<kObjRastrigin>(v, w, nb, d, first, A);
  else if (obj == kObjAckley) epi_cols<kObjAckley>(v, w, nb, d, first, A);
  else epi_cols<kObjRosenbrock>(v, w, nb, d, first, A);
}

// The same terms over one accumulator row held in shared memory, the
// columns j = sub, sub + 16, ... of one of 16 threads (each term in the order
// of epi_cols; Rosenbrock's term of coordinate j pairs z_j with z_{j+1}).
template <int OBJ>
__device__ __forceinline__ void epi_strided(const float* z, int sub, int d, EpiAcc& A) {
  for (int j = sub; j < d; j += 16) {
    const float zj = z[j];
    if constexpr (OBJ == kObjSphere) {
      A.a1 = fmaf(zj, zj, A.a1);
      A.aG += 2.f * fabsf(zj);
    } else if constexpr (OBJ == kObjRastrigin) {
      const float cz = cos2pi_f32(zj);
      A.a1 += fmaf(zj, zj, fmaf(-10.f, cz, 10.f));
      A.aS += fmaf(zj, zj, fmaf(10.f, fabsf(cz), 10.f));
      A.aG += fmaf(2.f, fabsf(zj), 62.83185307f);
    } else if constexpr (OBJ == kObjAckley) {
      const float cz = cos2pi_f32(zj);
      A.a1 = fmaf(zj, zj, A.a1);
      A.a2 += cz;
      A.a3 += fabsf(zj);
      A.aS += fabsf(cz);
    } else {  // Rosenbrock at t = z + 1
      if (j + 1 < d) {
        const float t = zj + 1.f, tn = z[j + 1] + 1.f;
        const float aa = tn - t * t, bb = t - 1.f;
        A.a1 += fmaf(100.f * aa, aa, bb * bb);
        A.aG += 400.f * fabsf(t) * fabsf(aa) + 2.f * fabsf(bb) + 200.f * fabsf(aa);
      }
    }
  }
}

__device__ __forceinline__ void epi_strided_dispatch(int obj, const float* z, int sub, int d, EpiAcc& A) {
  if (obj == kObjSphere) epi_strided<kObjSphere>(z, sub, d, A);
  else if (obj == kObjRastrigin) epi_strided<kObjRastrigin>(z, sub, d, A);
  else if (obj == kObjAckley) epi_strided<kObjAckley>(z, sub, d, A);
  else epi_strided<kObjRosenbrock>(z, sub, d, A);
}

}  // namespace de
