// de_device.cuh -- device helpers shared by the FP64 and the tensor-core
// kernels: objective of a row in FP64, the FP64 rotation of a tile, the
// best-record reduction, and the construction of one trial vector.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>
#include <string.h>

#include "de_common.cuh"
#include "de_internal.cuh"

namespace de {

// Programmatic dependent launch: a kernel launched with the programmatic
// serialization attribute may start while its predecessor finishes; it must
// wait before touching the predecessor's results.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }

// ------------------------------------------------------------------ cos(2 pi z)
// 2z = k + r with k the nearest integer, found exactly by adding and removing
// 1.5 * 2^(p-1) (p the significand width); |r| <= 1/2 and r is exact.  Then
// cos(2 pi z) = (-1)^k cos(pi r), and cos(pi r) is its Taylor series in
// u = r^2, sum_n (-1)^n pi^(2n) u^n / (2n)!, truncated where the next term is
// below the format's rounding (u <= 1/4): 7 terms in FP32 (next term 6e-9),
// 11 terms in FP64 (next term 2e-17).  The FP64 sum is evaluated by Estrin's
// scheme (dependency depth 5 instead of 10: a dependent FP64 operation costs
// tens of cycles on this part).
__host__ __device__ constexpr double cospi_taylor(int n) {
  double c = 1.0;
  for (int k = 1; k <= n; ++k) c *= -9.8696044010893586188 / ((2.0 * k - 1.0) * (2.0 * k));  // pi^2
  return c;
}

__device__ __forceinline__ double cos2pi_f64(double z) {
  const double sh = 6755399441055744.0;  // 1.5 * 2^52
  const double tz = 2.0 * z;
  const double t1 = __dadd_rn(tz, sh);
  const double r = __dsub_rn(tz, __dsub_rn(t1, sh));
  const bool odd = __double_as_longlong(t1) & 1;
  const double u = r * r, u2 = u * u, u4 = u2 * u2, u8 = u4 * u4;
  const double p01 = fma(cospi_taylor(1), u, cospi_taylor(0));
  const double p23 = fma(cospi_taylor(3), u, cospi_taylor(2));
  const double p45 = fma(cospi_taylor(5), u, cospi_taylor(4));
  const double p67 = fma(cospi_taylor(7), u, cospi_taylor(6));
  const double p89 = fma(cospi_taylor(9), u, cospi_taylor(8));
  const double q0 = fma(p23, u2, p01);
  const double q1 = fma(p67, u2, p45);
  const double q2 = fma(cospi_taylor(10), u2, p89);
  const double c = fma(q2, u8, fma(q1, u4, q0));
  return odd ? -c : c;
}

// Same series by Horner's rule: fewer FP64 instructions than Estrin's
// scheme, for kernels bound by FP64 throughput rather than latency.
__device__ __forceinline__ double cos2pi_f64_horner(double z) {
  const double sh = 6755399441055744.0;  // 1.5 * 2^52
  const double tz = 2.0 * z;
  const double t1 = __dadd_rn(tz, sh);
  const double r = __dsub_rn(tz, __dsub_rn(t1, sh));
  const bool odd = __double_as_longlong(t1) & 1;
  const double u = r * r;
  double c = cospi_taylor(10);
#pragma unroll
  for (int n = 9; n >= 0; --n) c = fma(c, u, cospi_taylor(n));
  return odd ? -c : c;
}

__device__ __forceinline__ float cos2pi_f32(float z) {
  const float sh = 12582912.0f;  // 1.5 * 2^23
  const float tz = 2.0f * z;
  const float t1 = __fadd_rn(tz, sh);
  const float r = __fsub_rn(tz, __fsub_rn(t1, sh));
  const bool odd = __float_as_int(t1) & 1;
  const float u = r * r;
  float c = (float)cospi_taylor(6);
  c = fmaf(c, u, (float)cospi_taylor(5));
  c = fmaf(c, u, (float)cospi_taylor(4));
  c = fmaf(c, u, (float)cospi_taylor(3));
  c = fmaf(c, u, (float)cospi_taylor(2));
  c = fmaf(c, u, (float)cospi_taylor(1));
  c = fmaf(c, u, 1.0f);
  return odd ? -c : c;
}

// Ordering key of a fitness value for the best-record reductions: the
// integer image of the double (monotone for finite values), NaN last.
__device__ __forceinline__ long long fit_key(double f) {
  const long long k = __double_as_longlong(f);
  if ((k & 0x7FF0000000000000LL) == 0x7FF0000000000000LL && (k & 0x000FFFFFFFFFFFFFLL)) return 0x7FFFFFFFFFFFFFFFLL;
  return k >= 0 ? k : -(k & 0x7FFFFFFFFFFFFFFFLL);
}

// ------------------------------------------------------------------ objective
// Objective of one row held in shared memory (z, length d); the calling warp
// returns the same value in every lane.  Terms are summed per lane in
// coordinate order, then across lanes by a fixed xor tree.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ ODE objective
// The expensive objective of the surrogate-assisted workload.  The paper
// motivates costly objectives (Abstract) but defines none; this one is a
// reading.  Ten unit masses in a chain: springs k_i to ground, dampers c_i,
// unit springs between neighbours, walls at both ends.
//   dq_i/dt = p_i,  dp_i/dt = (q_{i-1} + q_{i+1}) - (k_i + 2) q_i - c_i p_i
// Parameters from x in [-100, 100]^20:
//   k_i = 0.5 + 4.5 (x_i + 100) / 200,  c_i = 0.01 + 0.49 (x_{10+i} + 100) / 200.
// Classical RK4 with dt = 1e-3 for 2000 steps from q(0) = e_1, p(0) = 0.
// f = mean over steps and masses of (q - q_ref)^2, where q_ref is the
// trajectory of the hidden parameter vector (the run's shift o).
// One warp per parameter vector; lane i < 10 carries mass i and its
// neighbours come by shuffles.  Rounding: one IEEE operation per step of the
// stated order (explicit __fma_rn / __dadd_rn), so a trajectory is a pure
// function of x and f(o) = 0 exactly.
constexpr int kOdeN = 10;
constexpr int kOdeSteps = 2000;
constexpr double kOdeDt = 1e-3;

__device__ __forceinline__ double ode_neighbours(double q, int lane) {
  const double l = __shfl_up_sync(0xffffffffu, q, 1);
  const double r = __shfl_down_sync(0xffffffffu, q, 1);
  return __dadd_rn(lane == 0 ? 0.0 : l, lane >= kOdeN - 1 ? 0.0 : r);
}

// Integrates the chain of x (20 parameters).  Returns this lane's sum of
// (q - ref)^2 over the steps when ref is not NULL (0 in lanes >= 10); writes
// the positions to out[step * 10 + lane] when out is not NULL.  All 32 lanes
// must call it.
static __device__ __forceinline__ double ode_chain(const double* __restrict__ x, int lane, const double* __restrict__ ref,
                                         double* __restrict__ out) {
  const bool on = lane < kOdeN;
  const int li = on ? lane : 0;
  const double uk = __ddiv_rn(__dadd_rn(x[li], 100.0), 200.0);
  const double uc = __ddiv_rn(__dadd_rn(x[kOdeN + li], 100.0), 200.0);
  const double k = __dadd_rn(0.5, __dmul_rn(4.5, uk));
  const double c = __dadd_rn(0.01, __dmul_rn(0.49, uc));
  const double nk2 = -__dadd_rn(k, 2.0), nc = -c;
  const double h = kOdeDt, hh = kOdeDt * 0.5, h6 = kOdeDt / 6.0;
  double q = lane == 0 ? 1.0 : 0.0, p = 0.0, acc = 0.0;
  // the reference position of step s is loaded one step ahead, off the
  // integration's dependency chain
  double rv = (ref && on) ? __ldg(ref + lane) : 0.0;
  for (int s = 0; s < kOdeSteps; ++s) {
    const double rv_next = (ref && on && s + 1 < kOdeSteps) ? __ldg(ref + (s + 1) * kOdeN + lane) : 0.0;
    const double a1 = __fma_rn(nc, p, __fma_rn(nk2, q, ode_neighbours(q, lane)));
    const double q2 = __fma_rn(hh, p, q), p2 = __fma_rn(hh, a1, p);
    const double a2 = __fma_rn(nc, p2, __fma_rn(nk2, q2, ode_neighbours(q2, lane)));
    const double q3 = __fma_rn(hh, p2, q), p3 = __fma_rn(hh, a2, p);
    const double a3 = __fma_rn(nc, p3, __fma_rn(nk2, q3, ode_neighbours(q3, lane)));
    const double q4 = __fma_rn(h, p3, q), p4 = __fma_rn(h, a3, p);
    const double a4 = __fma_rn(nc, p4, __fma_rn(nk2, q4, ode_neighbours(q4, lane)));
    const double mq = __dadd_rn(p2, p3), mp = __dadd_rn(a2, a3);
    q = __fma_rn(h6, __dadd_rn(__dadd_rn(p, p4), __dadd_rn(mq, mq)), q);
    p = __fma_rn(h6, __dadd_rn(__dadd_rn(a1, a4), __dadd_rn(mp, mp)), p);
    if (on) {
      if (ref) {
        const double r = __dsub_rn(q, rv);
        acc = __fma_rn(r, r, acc);
      }
      if (out) out[s * kOdeN + lane] = q;
    }
    rv = rv_next;
  }
  return acc;
}

__device__ __forceinline__ double row_objective_fp64(int obj, const double* __restrict__ z, int d, int lane) {
  double s1 = 0.0, s2 = 0.0;
  if (obj == kObjSphere) {
    for (int j = lane; j < d; j += 32) s1 += z[j] * z[j];
  } else if (obj == kObjRastrigin) {
    for (int j = lane; j < d; j += 32) {
      const double zj = z[j];
      s1 += zj * zj - 10.0 * cos2pi_f64_horner(zj) + 10.0;
    }
  } else if (obj == kObjRosenbrock) {
    for (int j = lane; j + 1 < d; j += 32) {
      const double t0 = z[j] + 1.0, t1 = z[j + 1] + 1.0;
      const double a = t1 - t0 * t0, b = t0 - 1.0;
      s1 += 100.0 * a * a + b * b;
    }
  } else if (obj == kObjAckley) {
    for (int j = lane; j < d; j += 32) {
      const double zj = z[j];
      s1 += zj * zj;
      s2 += cos2pi_f64_horner(zj);
    }
  } else {
    s1 = CUDART_NAN;
  }
  s1 = warp_sum(s1);
  if (obj == kObjAckley) {
    s2 = warp_sum(s2);
    const double inv_d = 1.0 / (double)d;
    return 20.0 + 2.718281828459045 - 20.0 * exp(-0.2 * sqrt(s1 * inv_d)) - exp(s2 * inv_d);
  }
  return s1;
}

// Z[r][j] = sum_k M[j][k] Y[r][k] for the rows of a tile (ROWS rows of stride
// dp in shared memory).  Thread t owns output columns t, t + blockDim, ...
template <int ROWS>
__device__ __forceinline__ void tile_rotate_fp64(const double* __restrict__ MT, const double* __restrict__ Y,
                                                 double* __restrict__ Z, int d, int dp) {
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    double acc[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) acc[r] = 0.0;
    const double* mcol = MT + j;
    int k = 0;
    for (; k + 4 <= d; k += 4) {
      const double m0 = __ldg(mcol + (size_t)(k + 0) * d);
      const double m1 = __ldg(mcol + (size_t)(k + 1) * d);
      const double m2 = __ldg(mcol + (size_t)(k + 2) * d);
      const double m3 = __ldg(mcol + (size_t)(k + 3) * d);
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        const double* y = Y + r * dp + k;
        acc[r] = fma(m0, y[0], acc[r]);
        acc[r] = fma(m1, y[1], acc[r]);
        acc[r] = fma(m2, y[2], acc[r]);
        acc[r] = fma(m3, y[3], acc[r]);
      }
    }
    for (; k < d; ++k) {
      const double m = __ldg(mcol + (size_t)k * d);
#pragma unroll
      for (int r = 0; r < ROWS; ++r) acc[r] = fma(m, Y[r * dp + k], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) Z[r * dp + j] = acc[r];
  }
}

__device__ __forceinline__ void tile_rotate_dispatch(int rows, const double* MT, const double* Y, double* Z, int d,
                                                     int dp) {
  if (rows <= 1) tile_rotate_fp64<1>(MT, Y, Z, d, dp);
  else if (rows <= 2) tile_rotate_fp64<2>(MT, Y, Z, d, dp);
  else if (rows <= 4) tile_rotate_fp64<4>(MT, Y, Z, d, dp);
  else if (rows <= 8) tile_rotate_fp64<8>(MT, Y, Z, d, dp);
  else tile_rotate_fp64<16>(MT, Y, Z, d, dp);
}

// ------------------------------------------------------------------ best record
// Running best (f, index) of a reduction.  The ordered integer key of f is
// computed once per offered value; comparisons and shuffles then use the key
// (smaller key wins, then the lower index; a NaN, key INT64_MAX, never wins).
struct Best {
  double f;
  long long k;
  int i;
  __device__ __forceinline__ void init() {
    f = CUDART_INF;
    k = 0x7FFFFFFFFFFFFFFFLL;
    i = -1;
  }
  __device__ __forceinline__ void take(double fo, long long ko, int io) {
    if (io >= 0 && ko != 0x7FFFFFFFFFFFFFFFLL && (i < 0 || ko < k || (ko == k && io < i))) {
      f = fo;
      k = ko;
      i = io;
    }
  }
  __device__ __forceinline__ void offer(double fo, int io) { take(fo, fit_key(fo), io); }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double fo = __shfl_xor_sync(0xffffffffu, f, o);
      const long long ko = __shfl_xor_sync(0xffffffffu, k, o);
      const int io = __shfl_xor_sync(0xffffffffu, i, o);
      take(fo, ko, io);
    }
  }
};

// Finish a generation of a run: called by the last CTA to arrive.  Reduces
// the tile partials in order (and, for the split precisions, the rows decided
// in FP64 this generation, which carry no partial),
// advances the counters and evaluates the stop rule (Sec. 7.3.4).  The best
// vector itself is read from the population when a caller asks for it.
__device__ __forceinline__ void finish_generation(const RunDesc& R, int64_t g, int nparts, const BestPartial* part,
                                                  const double* Xn, const BandEntry* band = nullptr, int nband = 0,
                                                  int run = -1, const double* fcur = nullptr) {
  __shared__ double sf[32];
  __shared__ long long sk[32];
  __shared__ int si[32];
  Best b;
  b.init();
  for (int t = threadIdx.x; t < nparts; t += blockDim.x) b.offer(__ldcg(&part[t].f), __ldcg(&part[t].idx));
  for (int t = threadIdx.x; t < nband; t += blockDim.x) {
    if (__ldcg(&band[t].run) != run) continue;
    const int i = __ldcg(&band[t].row);
    b.offer(__ldcg(&fcur[i]), i);
  }
  b.warp_reduce();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sf[warp] = b.f; sk[warp] = b.k; si[warp] = b.i; }
  __syncthreads();
  if (threadIdx.x == 0) {
    b.init();
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b.take(sf[w], sk[w], si[w]);
    const double bf = b.f;
    const int bi = b.i;
    RunState* st = R.st;
    if (bi >= 0) {
      st->best_f = bf;
      st->best_idx = bi;
    } else {
      st->err |= kErrNonFinite;
    }
    st->gen = g;
    st->evals += R.np;
    int stop = 0;
    if (R.target > 0.0 && st->best_idx >= 0 && st->best_f < R.target) stop = 1;
    else if (R.max_evals > 0 && st->evals >= R.max_evals) stop = 2;
    else if (g >= R.max_gens) stop = 3;
    st->stop = stop;
    st->ticket = 0;
    st->band_n = 0;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ trial row
// Construction of the trial of target i at generation g (Eq. 2 and Eq. 3,
// with bound repair), split so that the FP64 and the tensor-core trial
// kernels share it.  A warp handles one target; lane L owns coordinates
// 128c + 4L .. 128c + 4L + 3 of chunk c.
// Total order of finite doubles as 64-bit integers (-0 and +0 map to 0), so
// that the bound tests below run on the integer pipe instead of the slow
// FP64 pipe; exact for every finite value.
__host__ __device__ __forceinline__ long long ordered_key(double x) {
#if defined(__CUDA_ARCH__)
  const long long k = __double_as_longlong(x);
#else
  long long k;
  memcpy(&k, &x, sizeof k);
#endif
  return k >= 0 ? k : -(k & 0x7FFFFFFFFFFFFFFFLL);
}

// The same order on the high 32 bits alone: a <= b implies
// hi_key32(a) <= hi_key32(b) for finite a, b (the high word of a
// magnitude is monotone in it, and -0, +0 and the tiniest values of either
// sign map to 0).  So hi_key32(x) < hi_key32(lo) proves x < lo, and
// hi_key32(lo) < hi_key32(x) < hi_key32(hi) proves lo < x < hi; only equal
// high words need the 64-bit keys.  The trial kernels test bounds with it:
// the 64-bit key and its compare cost one FP64-pipe instruction per
// coordinate on this part (counted with sm__inst_executed_pipe_fp64), the
// 32-bit form none.
__host__ __device__ __forceinline__ int hi_key32(double x) {
#if defined(__CUDA_ARCH__)
  const int h = __double2hiint(x);
#else
  long long k;
  memcpy(&k, &x, sizeof k);
  const int h = (int)(k >> 32);
#endif
  return h >= 0 ? h : -(h & 0x7FFFFFFF);
}

// FP64 -> FP32 rounding to nearest, ties to even, on the integer pipe (the
// conversion instruction occupies the FP64 pipe, which bounds the trial
// kernels on this part).  Normal results: the 29 dropped significand bits
// decide the increment, whose carry runs into the exponent field (and to
// infinity past the largest float).  Results below the normal range: the
// 53-bit significand shifted to units of 2^-149 with the same rounding (a
// carry gives the smallest normal).  Infinities and NaNs stay so; finite
// inputs beyond the float range round to infinity.
__device__ __forceinline__ float to_f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int ex = (int)((b >> 52) & 0x7FF);
  const int e = ex - 1023 + 127;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFULL;
  unsigned int r;
  if (e >= 1 && e <= 254) {
    const unsigned int mant = (unsigned int)(m >> 29);
    const unsigned int rem = (unsigned int)(m & 0x1FFFFFFFULL);
    r = sign | ((unsigned int)e << 23) | mant;
    if (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) r += 1u;
  } else if (ex == 0x7FF) {
    r = sign | 0x7F800000u | (m ? 0x400000u | (unsigned int)(m >> 29) : 0u);
  } else if (e > 254) {
    r = sign | 0x7F800000u;
  } else {
    // x = (2^52 + m) 2^(ex - 1075); in units of 2^-149 that is a right shift
    // by sh = 926 - ex >= 30 bits (double subnormals are far below 2^-150)
    const int sh = 926 - ex;
    unsigned int k = 0u;
    if (ex != 0 && sh < 64) {
      const unsigned long long sig = (1ULL << 52) | m;
      const unsigned long long rem = sig & ((1ULL << sh) - 1ULL), half = 1ULL << (sh - 1);
      k = (unsigned int)(sig >> sh);
      if (rem > half || (rem == half && (k & 1u))) k += 1u;
    }
    r = sign | k;
  }
  return __uint_as_float(r);
}

// FP32 -> FP64 (exact) on the integer pipe.
__device__ __forceinline__ double f64_of_f32(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int ex = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  const unsigned long long m = u & 0x7FFFFFu;
  unsigned long long r;
  if (ex != 0u && ex != 0xFFu) {
    r = sign | ((unsigned long long)(ex + 896u) << 52) | (m << 29);
  } else if (ex == 0xFFu) {
    r = sign | (0x7FFULL << 52) | (m << 29);
  } else if (m == 0u) {
    r = sign;
  } else {
    // subnormal: m 2^-149 with the leading one at bit p
    const int p = 31 - __clz((unsigned int)m);
    r = sign | ((unsigned long long)(p - 149 + 1023) << 52) | ((m << (52 - p)) & 0xFFFFFFFFFFFFFULL);
  }
  return __longlong_as_double((long long)r);
}

// y = (t - o) s with the scale known at compile time to be 1 (UNIT: no
// multiplication on the FP64 pipe, which bounds the trial kernels) or not
template <bool UNIT>
__device__ __forceinline__ double shifted_as(double t, double o, double s) {
  const double y = __dsub_rn(t, o);
  return UNIT ? y : __dmul_rn(y, s);
}

// y = (t - o) s, rounded once per operation as written
__device__ __forceinline__ double shifted(double t, double o, const RunDesc& R) {
  const double y = __dsub_rn(t, o);
  return R.unit_scale ? y : __dmul_rn(y, R.scale);
}

struct TrialSetup {
  uint32_t r1, r2, r3, jr;
};

// Draws 0..3 of the STEP stream: mutant indices (Eq. 2) and j_rand (Eq. 3).
// cand selects the candidate stream (0: plain DE; 1, 2, ...: the extra
// candidate trials a surrogate screens); record = false skips the debug copy.
__device__ __forceinline__ TrialSetup trial_setup(const RunDesc& R, uint32_t i, int64_t g, int lane,
                                                  uint32_t cand = 0u, bool record = true) {
  const U32x4 b0 = draw_block(R.seed, kPurposeStep, R.run_id, cand, (uint32_t)g, i, 0u);
  TrialSetup s;
  mutant_indices(b0.x, b0.y, b0.z, i, (uint32_t)R.np, s.r1, s.r2, s.r3);
  s.jr = map_to_range(b0.w, (uint32_t)R.d);
  if (record && R.dbg_idx && lane == 0) {
    R.dbg_idx[3 * i + 0] = (int32_t)s.r1;
    R.dbg_idx[3 * i + 1] = (int32_t)s.r2;
    R.dbg_idx[3 * i + 2] = (int32_t)s.r3;
    R.dbg_jrand[i] = (int32_t)s.jr;
  }
  return s;
}

// Inputs of one 4-coordinate chunk of a trial: the target's and the three
// donors' coordinates and the chunk's Philox block (rand_j of Eq. 3).
struct ChunkIn {
  double xi[4], x1[4], x2[4], x3[4];
  U32x4 u;
};

// Issue the loads of chunk j0 (j0 < d, j0 % 4 == 0) and draw its block.
// The rows are read at L2 (ld.global.cg): the persistent kernels read, in
// generation g, population rows other CTAs wrote in generation g - 1, so the
// loads must not come from a non-coherent per-SM cache.
__device__ __forceinline__ void trial_load(const RunDesc& R, const double* X, const TrialSetup& s,
                                           uint32_t i, int64_t g, int j0, ChunkIn& c, uint32_t cand = 0u) {
  c.u = draw_block(R.seed, kPurposeStep, R.run_id, cand, (uint32_t)g, i, 1u + (uint32_t)(j0 >> 2));
  const double* rows[4] = {X + (size_t)i * R.dp + j0, X + (size_t)s.r1 * R.dp + j0, X + (size_t)s.r2 * R.dp + j0,
                           X + (size_t)s.r3 * R.dp + j0};
  double* dst[4] = {c.xi, c.x1, c.x2, c.x3};
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const double2 a = __ldcg(reinterpret_cast<const double2*>(rows[r]));
    const double2 b = __ldcg(reinterpret_cast<const double2*>(rows[r] + 2));
    dst[r][0] = a.x;
    dst[r][1] = a.y;
    dst[r][2] = b.x;
    dst[r][3] = b.y;
  }
}

// Coordinates j0 .. j0+3 of the trial from loaded inputs with weight F and
// crossover threshold thr; entries at j >= d are 0.  L = 0: binomial
// crossover (Eq. 3); L >= 1: exponential crossover of the cyclic block
// j_rand .. j_rand + L - 1.  Returns the crossed-coordinate bits (bit m for
// j0 + m).
__device__ __forceinline__ uint32_t trial_compute(const RunDesc& R, const TrialSetup& s, int j0, const ChunkIn& c,
                                                  double t[4], double F, uint64_t thr, int L) {
  const int d = R.d;
  const uint32_t u[4] = {c.u.x, c.u.y, c.u.z, c.u.w};
  // u <= thr on 32 bits (thr = 2^32, CR = 1, crosses every coordinate, as
  // does the largest 32-bit value)
  const uint32_t thr32 = thr > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)thr;
  // per slot: below lo / above hi by the high words alone, or a high word
  // equal to a bound's (decided on all 64 bits below)
  uint32_t bits = 0, lowm = 0, highm = 0, eqm = 0;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int j = j0 + m;
    t[m] = 0.0;
    if (j < d) {
      bool crossed;
      if (L > 0) {
        int off = j - (int)s.jr;
        if (off < 0) off += d;
        crossed = off < L;
      } else {
        crossed = ((uint32_t)j == s.jr) || (u[m] <= thr32);
      }
      if (crossed) {
        // Eq. 2: y = x_r1 + F (x_r2 - x_r3), one rounding for the product-sum
        const double v = __fma_rn(F, __dsub_rn(c.x2[m], c.x3[m]), c.x1[m]);
        t[m] = v;
        bits |= 1u << m;
        // non-finite values land above hi (+NaN, +inf) or below lo
        const int hk = hi_key32(v);
        lowm |= (uint32_t)(hk < R.lo_hk) << m;
        highm |= (uint32_t)(hk > R.hi_hk) << m;
        eqm |= (uint32_t)(hk == R.lo_hk || hk == R.hi_hk) << m;
      } else {
        t[m] = c.xi[m];
      }
    }
  }
  // bound repair: a crossed coordinate outside [lo, hi] goes half way from
  // the target's coordinate to the violated bound (the paper leaves bounds
  // handling open).  (x_i + b) / 2 rounded once equals fma(0.5, x_i, b / 2):
  // halving commutes with rounding away from the subnormal range, and b / 2 is
  // exact, so the repair is one FP64 instruction per slot.  It runs only when
  // some lane of the warp needs it (one vote per chunk: a vote per slot cost
  // the FP64 generation kernel more than the instructions it saved), and the
  // 64-bit keys only when some lane has a high word equal to a bound's (their
  // compare costs an FP64-pipe instruction per slot).
  if (__any_sync(__activemask(), (lowm | highm | eqm) != 0u)) {
    if (__any_sync(__activemask(), eqm != 0u)) {
#pragma unroll
      for (int m = 0; m < 4; ++m)
        if ((eqm >> m) & 1u) {
          const long long kv = ordered_key(t[m]);
          lowm |= (uint32_t)(kv < R.lo_key) << m;
          highm |= (uint32_t)(kv > R.hi_key) << m;
        }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (((lowm | highm) >> m) & 1u) t[m] = __fma_rn(0.5, c.xi[m], ((lowm >> m) & 1u) ? R.lo_half : R.hi_half);
  }
  return bits;
}

// DE/rand/1/bin with the run's F and CR.
__device__ __forceinline__ uint32_t trial_compute(const RunDesc& R, const TrialSetup& s, int j0, const ChunkIn& c,
                                                  double t[4]) {
  return trial_compute(R, s, j0, c, t, R.F, R.cr_thr, 0);
}

// Coordinates j0 .. j0+3 (j0 < d, j0 % 4 == 0) of the trial; entries at
// j >= d are 0.  Returns the crossed-coordinate bits (bit m for j0 + m).
__device__ __forceinline__ uint32_t trial_chunk(const RunDesc& R, const double* __restrict__ X, const TrialSetup& s,
                                                uint32_t i, int64_t g, int j0, double t[4], uint32_t cand = 0u) {
  ChunkIn c;
  trial_load(R, X, s, i, g, j0, c, cand);
  return trial_compute(R, s, j0, c, t);
}

// ------------------------------------------------------------------ variants
// Control parameters of one trial under the strategy variants and jDE.
struct TrialVar {
  double F;      // weight of the difference vector
  double CR;     // crossover rate (stored into jCR on acceptance)
  uint64_t thr;  // floor(CR 2^32): rand_j <= thr crosses coordinate j
  int L;         // exponential crossover: block length (0: binomial)
};

// jDE (Brest et al.'s self-adaptation, the adaptive variant of Sec. 2): draws
// a0..a3 of the JDE stream of (i, g); with probability 0.1 each
// (a1 resp. a3 below floor(0.1 2^32)) F_i = 0.1 + 0.9 a0 / 2^32 (one
// rounding) and CR_i = a2 / 2^32, otherwise the stored values.
__device__ __forceinline__ void jde_params(const RunDesc& R, uint32_t i, int64_t g, const double* jF,
                                           const double* jCR, double& F, double& CR) {
  const uint32_t tau = 429496729u;  // floor(0.1 * 2^32)
  const U32x4 a = draw_block(R.seed, kPurposeJde, R.run_id, 0u, (uint32_t)g, i, 0u);
  F = a.y < tau ? __fma_rn(0.9, (double)a.x * 0x1p-32, 0.1) : __ldcg(jF + i);
  CR = a.w < tau ? (double)a.z * 0x1p-32 : __ldcg(jCR + i);
}

// Exponential crossover length (Sec. 2): L = 1 + the number of leading
// crossover draws rand_0, rand_1, ... (draw 4 + m of the STEP stream, the
// ones binomial crossover gives coordinate m) that are <= thr, capped at d.
// Called by the whole warp; lane q tests draws 128c + 4q .. 128c + 4q + 3.
// The warp may hold several targets: lpt lanes per target (a power of two,
// aligned segments), the lane's position in its segment is lane % lpt, and
// the segment's draws are tested 4 lpt at a time.  Every lane runs the same
// number of rounds (d is the run's), so the ballots stay warp-wide.
__device__ __forceinline__ int exp_length(const RunDesc& R, uint32_t i, int64_t g, int lane, uint64_t thr,
                                          int lpt = 32) {
  const int d = R.d;
  const int sub = lane & (lpt - 1), base = lane - sub;
  const uint32_t seg = lpt == 32 ? 0xffffffffu : (((1u << lpt) - 1u) << base);
  int L = d;
  bool found = false;
  for (int m0 = 0; m0 <= d - 2; m0 += 4 * lpt) {
    const int mb = m0 + 4 * sub;
    uint32_t fail = 0;
    if (mb <= d - 2 && !found) {
      const U32x4 b = draw_block(R.seed, kPurposeStep, R.run_id, 0u, (uint32_t)g, i, 1u + (uint32_t)(mb >> 2));
      const uint32_t u[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (mb + q <= d - 2 && (uint64_t)u[q] > thr) fail |= 1u << q;
    }
    const uint32_t any = __ballot_sync(0xffffffffu, fail != 0u) & seg;
    const int fl = any ? __ffs(any) - 1 : lane;
    const uint32_t fb = __shfl_sync(0xffffffffu, fail, fl);
    if (any && !found) {
      L = m0 + 4 * (fl - base) + (__ffs(fb) - 1) + 1;
      found = true;
    }
    if (lpt == 32 && found) break;  // the whole warp is one target: a uniform exit
  }
  return L;
}

// Trial setup under the run's strategy and jDE: records the drawn donors,
// then for DE/best/1 takes the base from row `best` and the difference from
// the first two drawn donors.  Called by the whole warp.
__device__ __forceinline__ TrialSetup trial_setup_var(const RunDesc& R, uint32_t i, int64_t g, int lane, int best,
                                                      const double* jF, const double* jCR, TrialVar& v,
                                                      int lpt = 32, bool record = true) {
  TrialSetup s = trial_setup(R, i, g, lane & (lpt - 1), 0u, record);
  if (R.strategy == 1) {
    s.r3 = s.r2;
    s.r2 = s.r1;
    s.r1 = (uint32_t)best;
  }
  v.F = R.F;
  v.CR = R.CR;
  v.thr = R.cr_thr;
  if (R.jde) {
    jde_params(R, i, g, jF, jCR, v.F, v.CR);
    v.thr = (uint64_t)floor(__dmul_rn(v.CR, 4294967296.0));
  }
  v.L = R.strategy == 2 ? exp_length(R, i, g, lane, v.thr, lpt) : 0;
  return s;
}

// Debug capture of one chunk: trial values and the crossover mask word.
// Called by every lane of the warp (the mask word is assembled by shuffles
// within each target's lpt lanes); `valid` lanes write.
__device__ __forceinline__ void trial_debug(const RunDesc& R, uint32_t i, int j0, int lane, uint32_t bits,
                                            const double t[4], int lpt = 32, bool valid = true) {
  const int d = R.d;
  if (valid && j0 < d) {
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (j0 + m < d) R.dbg_trial[(size_t)i * d + j0 + m] = t[m];
  }
  // lanes 8w .. 8w+7 of a target's chunk cover mask word 4c + w
  uint32_t word = (j0 < d) ? (bits << (j0 & 31)) : 0u;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1)
    if (o < lpt) word |= __shfl_xor_sync(0xffffffffu, word, o);
  const int wi = j0 >> 5;
  if (valid && (lane & 7 & (lpt - 1)) == 0 && wi < R.nw) R.dbg_mask[(size_t)i * R.nw + wi] = word;
}

// FP64 path: build the trial row into T and Y = (T - o) s (rows of length dp).
// VAR: the run may use a strategy variant or jDE (best: the current best row;
// jF, jCR: the current jDE parameters).
// UNIT: the run's domain scale is 1 (the shift without a multiplication)
template <bool VAR, bool UNIT = false>
__device__ __forceinline__ void build_trial_row(const RunDesc& R, const double* X, uint32_t i,
                                                int64_t g, int lane, double* __restrict__ Trow,
                                                double* __restrict__ Yrow, int best = 0,
                                                const double* jF = nullptr, const double* jCR = nullptr) {
  TrialVar v;
  const TrialSetup s = VAR ? trial_setup_var(R, i, g, lane, best, jF, jCR, v) : trial_setup(R, i, g, lane);
  const bool dbg = R.dbg_trial != nullptr;
  const int nchunks = (R.d + 127) / 128;
  for (int c = 0; c < nchunks; ++c) {
    const int j0 = 128 * c + 4 * lane;
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    uint32_t bits = 0;
    if (j0 < R.d) {
      if (VAR) {
        ChunkIn ci;
        trial_load(R, X, s, i, g, j0, ci);
        bits = trial_compute(R, s, j0, ci, t, v.F, v.thr, v.L);
      } else {
        bits = trial_chunk(R, X, s, i, g, j0, t);
      }
      double y[4];
#pragma unroll
      for (int m = 0; m < 4; ++m)
        y[m] = (j0 + m < R.d) ? (UNIT ? shifted_as<true>(t[m], R.o[j0 + m], 1.0) : shifted(t[m], R.o[j0 + m], R)) : 0.0;
      *reinterpret_cast<double2*>(Trow + j0) = make_double2(t[0], t[1]);
      *reinterpret_cast<double2*>(Trow + j0 + 2) = make_double2(t[2], t[3]);
      *reinterpret_cast<double2*>(Yrow + j0) = make_double2(y[0], y[1]);
      *reinterpret_cast<double2*>(Yrow + j0 + 2) = make_double2(y[2], y[3]);
    }
    if (dbg) trial_debug(R, i, j0, lane, bits, t);
  }
}

}  // namespace de
