// de_common.cuh -- device-side building blocks of the DE generation step.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written
// from the published round function.  The paper's GPU DEs draw from cuRAND
// (Sec. 4.4, Sec. 6.2.1); a counter-based generator makes every draw a pure
// function of (seed, generation, individual, draw), so the result does not
// depend on the launch shape.
//
// Stream layout:
//   key = (seed low 32 bits, seed high 32 bits)
//   ctr = (draw / 4, individual, generation, run_id << 12 | cand << 4 | purpose)
//   draw d is word d % 4 of its block.
// Trial of target i at generation g (purpose STEP): draws 0, 1, 2 pick r1, r2,
// r3 (Eq. 2), draw 3 picks j_rand, draw 4 + j is rand_j of coordinate j (Eq. 3).
// Initial population (purpose INIT, generation 0): parameter j of individual i
// takes draws 2j and 2j + 1.
#pragma once
#include <stdint.h>

namespace de {

constexpr uint32_t kPurposeInit = 1u;
constexpr uint32_t kPurposeStep = 2u;
constexpr uint32_t kPurposeJde = 6u;  // jDE: draws 0..3 of (i, g) decide F_i and CR_i

constexpr int kObjSphere = 0;
constexpr int kObjRastrigin = 1;
constexpr int kObjRosenbrock = 2;
constexpr int kObjAckley = 3;
constexpr int kObjOde = 4;

struct U32x4 {
  uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ U32x4 philox4x32_10(U32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
#if defined(__CUDA_ARCH__)
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
#else
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
#endif
    c = U32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Block `blk` of the stream (purpose, run_id, cand, generation, individual).
__host__ __device__ __forceinline__ U32x4 draw_block(uint64_t seed, uint32_t purpose, uint32_t run_id,
                                                     uint32_t cand, uint32_t generation, uint32_t individual,
                                                     uint32_t blk) {
  U32x4 c{blk, individual, generation, (run_id << 12) | ((cand & 0xFFu) << 4) | (purpose & 0xFu)};
  return philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}

__host__ __device__ __forceinline__ uint32_t word_of(const U32x4& b, int k) {
  return k == 0 ? b.x : (k == 1 ? b.y : (k == 2 ? b.z : b.w));
}

// Multiply-shift map of a 32-bit word onto [0, n).
__host__ __device__ __forceinline__ uint32_t map_to_range(uint32_t u, uint32_t n) {
  return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

// 53-bit uniform double in [0, 1) from two words.
__host__ __device__ __forceinline__ double unit_double(uint32_t hi, uint32_t lo) {
  const uint64_t bits = ((((uint64_t)hi) << 32) | (uint64_t)lo) >> 11;
  return (double)bits * 0x1.0p-53;
}

// Eq. 2 needs r1, r2, r3 distinct and != i.  Draw the k-th one uniformly over
// the np - k indices not yet taken and step it past the taken ones in
// ascending order: exactly three draws for the uniform ordered triple.
__host__ __device__ __forceinline__ void mutant_indices(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t i,
                                                        uint32_t np, uint32_t& r1, uint32_t& r2,
                                                        uint32_t& r3) {
  r1 = map_to_range(w0, np - 1u);
  r1 += (r1 >= i);
  // taken = {i, r1} ascending
  uint32_t a = i < r1 ? i : r1, b = i < r1 ? r1 : i;
  r2 = map_to_range(w1, np - 2u);
  r2 += (r2 >= a);
  r2 += (r2 >= b);
  // taken = {a, b, r2} ascending
  uint32_t s0 = a, s1 = b, s2 = r2;
  if (s2 < s1) { uint32_t t = s1; s1 = s2; s2 = t; }
  if (s1 < s0) { uint32_t t = s0; s0 = s1; s1 = t; }
  r3 = map_to_range(w2, np - 3u);
  r3 += (r3 >= s0);
  r3 += (r3 >= s1);
  r3 += (r3 >= s2);
}

// rand_j <= CR with rand_j = u / 2^32 holds exactly when u <= floor(CR 2^32).
__host__ __device__ __forceinline__ uint64_t cr_threshold(double cr) {
  return (uint64_t)(cr * 4294967296.0);
}

}  // namespace de
