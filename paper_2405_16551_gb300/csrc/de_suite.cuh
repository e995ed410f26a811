// de_suite.cuh -- the benchmark the paper proposes for GPU DEs (Sec. 7.3,
// Table 2) on the FP64 path: its basic functions on a warp, the hybrid
// functions (Sec. 7.3.2: one shift, one rotation, a permutation, parts
// evaluated by different basic functions) and the composition functions
// (Sec. 7.3.3: n shifted and rotated basic functions mixed by distance
// weights).
//
// Every basic function g has g = 0 at z = 0 (with the offsets written next to
// it).  The definitions are the published CEC'14 / CEC'17 ones the paper
// names; the shift, rotation and permutation data are the run's.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>

#include "de_common.cuh"
#include "de_device.cuh"
#include "de_internal.cuh"

namespace de {

constexpr int kObjZakharov = 5, kObjSchwefel = 6, kObjBentCigar = 7, kObjHGBat = 8, kObjSchafferF6 = 9;
constexpr int kObjKatsuura = 10, kObjHappyCat = 11, kObjGriewankRosenbrock = 12, kObjElliptic = 13;
constexpr int kObjGriewank = 14, kObjHybrid1 = 15, kObjHybrid3 = 17, kObjComposition1 = 18;
constexpr int kObjComposition3 = 20;

__device__ __forceinline__ bool suite_objective(int obj) { return obj >= kObjZakharov && obj <= kObjComposition3; }

__device__ __forceinline__ double warp_prod(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// modified Schwefel term of t = z + 420.9687462275036: t sin sqrt|t| inside
// [-500, 500]; outside, the value folded back with fmod plus the penalty
// (t -+ 500)^2 / (10^4 n)
__device__ __forceinline__ double schwefel_term(double t, int n) {
  if (t > 500.0) {
    const double m = fmod(t, 500.0);
    return (500.0 - m) * sin(sqrt(500.0 - m)) - (t - 500.0) * (t - 500.0) / (10000.0 * n);
  }
  if (t < -500.0) {
    const double m = fmod(-t, 500.0);
    return (m - 500.0) * sin(sqrt(500.0 - m)) - (t + 500.0) * (t + 500.0) / (10000.0 * n);
  }
  return t * sin(sqrt(fabs(t)));
}

// The costly part of coordinate l's term of basic function fn (the FP64
// transcendental functions), at w = w_l and v = w_{next(l)} (the cyclic
// neighbour, for the pair functions); 0 where fn has none.  The whole CTA
// computes these for a tile before one warp per row sums the terms.  kex:
// Katsuura's exponent 10 / n^1.2 for this n (computed once per part).
__device__ __forceinline__ double basic_costly(int fn, double w, double v, int l, int n, double kex) {
  switch (fn) {
    case kObjRastrigin:
    case kObjAckley: return cos2pi_f64_horner(w);
    case kObjSchwefel: return schwefel_term(w + 420.9687462275036, n);
    case kObjSchafferF6: {
      const double s = w * w + v * v;
      const double sn = sin(sqrt(s));
      const double den = 1.0 + 0.001 * s;
      return 0.5 + (sn * sn - 0.5) / (den * den);
    }
    case kObjKatsuura: {
      // 1 + i sum_{j=1}^{32} |2^j w - nearest integer| / 2^j, to the power 10 / n^1.2;
      // 2^j w, its rounding and the difference are exact
      double s = 0.0, p2 = 1.0;
      for (int j = 1; j <= 32; ++j) {
        p2 *= 2.0;
        const double t = p2 * w;
        s += fabs(t - rint(t)) / p2;
      }
      return pow(1.0 + (double)(l + 1) * s, kex);
    }
    case kObjGriewankRosenbrock: {
      // Griewank's 1-D term of Rosenbrock's 2-D term of the cyclic pair, at t = w + 1
      const double u = w + 1.0, vv = v + 1.0;
      const double a = u * u - vv, b = u - 1.0;
      const double r = 100.0 * a * a + b * b;
      return r * r / 4000.0 - cos(r) + 1.0;
    }
    case kObjElliptic: return n > 1 ? pow(1e6, (double)l / (double)(n - 1)) : 1.0;
    case kObjGriewank: return cos(w / sqrt((double)(l + 1)));
    default: return 0.0;
  }
}

__device__ __forceinline__ bool basic_has_costly(int fn) {
  return fn == kObjRastrigin || fn == kObjAckley || fn == kObjSchwefel || fn == kObjSchafferF6 ||
         fn == kObjKatsuura || fn == kObjGriewankRosenbrock || fn == kObjElliptic || fn == kObjGriewank;
}

// g of basic function fn on the n-vector w_l = sc * z[src(l)], src(l) =
// idx[base + l] (idx != NULL: a hybrid part) or base + l; position i = l + 1;
// E[l] holds basic_costly of coordinate l.  Called by a whole warp: lane k
// sums the terms of l = k, k + 32, ... in order, then a fixed xor tree; every
// lane returns g.
static __device__ __noinline__ double basic_fn_warp(int fn, const double* __restrict__ z,
                                                    const int32_t* __restrict__ idx, int base, int n, double sc,
                                                    const double* __restrict__ E, int lane) {
  auto W = [&](int l) { return sc * z[idx ? idx[base + l] : base + l]; };
  double s1 = 0.0, s2 = 0.0, p = 1.0;
  for (int l = lane; l < n; l += 32) {
    const double w = W(l);
    switch (fn) {
      case kObjSphere: s1 += w * w; break;
      case kObjRastrigin: s1 += w * w - 10.0 * E[l] + 10.0; break;
      case kObjRosenbrock:
        if (l + 1 < n) {
          const double t0 = w + 1.0, t1 = W(l + 1) + 1.0;
          const double a = t1 - t0 * t0, b = t0 - 1.0;
          s1 += 100.0 * a * a + b * b;
        }
        break;
      case kObjAckley:
        s1 += w * w;
        s2 += E[l];
        break;
      case kObjZakharov:
        // sum w^2 + (sum 0.5 i w_i)^2 + (sum 0.5 i w_i)^4
        s1 += w * w;
        s2 += 0.5 * (double)(l + 1) * w;
        break;
      case kObjSchwefel:
      case kObjSchafferF6:
      case kObjGriewankRosenbrock: s1 += E[l]; break;
      case kObjBentCigar: s1 += (l == 0 ? 1.0 : 1e6) * (w * w); break;
      case kObjHGBat:
      case kObjHappyCat: {
        const double x = w - 1.0;  // minimum at w = 0
        s1 += x * x;
        s2 += x;
        break;
      }
      case kObjKatsuura: p *= E[l]; break;
      case kObjElliptic: s1 += E[l] * (w * w); break;
      case kObjGriewank:
        s1 += w * w / 4000.0;
        p *= E[l];
        break;
      default: s1 = CUDART_NAN;
    }
  }
  s1 = warp_sum(s1);
  switch (fn) {
    case kObjAckley: {
      s2 = warp_sum(s2);
      return 20.0 + 2.718281828459045 - 20.0 * exp(-0.2 * sqrt(s1 / n)) - exp(s2 / n);
    }
    case kObjZakharov: {
      s2 = warp_sum(s2);
      const double b2 = s2 * s2;
      return s1 + b2 + b2 * b2;
    }
    case kObjSchwefel: return 418.9828872724338 * n - s1;
    case kObjHGBat: {
      // |a^2 - b^2|^(1/2) + (0.5 a + b) / n + 0.5, a = sum x^2, b = sum x
      s2 = warp_sum(s2);
      return sqrt(fabs(s1 * s1 - s2 * s2)) + (0.5 * s1 + s2) / n + 0.5;
    }
    case kObjHappyCat: {
      // |a - n|^(1/4) + (0.5 a + b) / n + 0.5
      s2 = warp_sum(s2);
      return pow(fabs(s1 - n), 0.25) + (0.5 * s1 + s2) / n + 0.5;
    }
    case kObjKatsuura: {
      p = warp_prod(p);
      const double c = 10.0 / ((double)n * n);
      return c * p - c;
    }
    case kObjGriewank: {
      p = warp_prod(p);
      return s1 - p + 1.0;
    }
    default: return s1;
  }
}

// Rotation of the tile's nrows rows with a given transposed matrix: thread
// t owns output columns t, t + blockDim, ... and runs one accumulator chain
// per row (each MT element loaded once serves every row of the tile).
__device__ __forceinline__ void suite_rotate(const double* __restrict__ MT, const double* __restrict__ Y,
                                             double* __restrict__ Z, int nrows, int d, int dp) {
  switch (nrows) {
    case 1: tile_rotate_fp64<1>(MT, Y, Z, d, dp); break;
    case 2: tile_rotate_fp64<2>(MT, Y, Z, d, dp); break;
    case 3: tile_rotate_fp64<3>(MT, Y, Z, d, dp); break;
    case 4: tile_rotate_fp64<4>(MT, Y, Z, d, dp); break;
    case 5: tile_rotate_fp64<5>(MT, Y, Z, d, dp); break;
    case 6: tile_rotate_fp64<6>(MT, Y, Z, d, dp); break;
    case 7: tile_rotate_fp64<7>(MT, Y, Z, d, dp); break;
    default: tile_rotate_fp64<8>(MT, Y, Z, d, dp); break;
  }
}

// Rotation of every component of a composition function at once:
// Z_c[r][j] = sum_k MT_c[k][j] Y_c[r][k] for c < nc, with Y_c and Z_c the
// c-th blocks of ROWS x dp rows.  Thread t owns (component, column) pairs
// t, t + blockDim, ... and runs one accumulator chain per row, as
// tile_rotate_fp64 does for one matrix (the same sums in the same order).
template <int ROWS>
__device__ __forceinline__ void comp_rotate(const double* __restrict__ MT, const double* __restrict__ Y,
                                            double* __restrict__ Z, int nc, int d, int dp) {
  const size_t blk = (size_t)ROWS * dp;
  for (int cj = threadIdx.x; cj < nc * d; cj += blockDim.x) {
    const int c = cj / d, j = cj - c * d;
    const double* mcol = MT + (size_t)c * d * d + j;
    const double* Yc = Y + c * blk;
    double acc[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) acc[r] = 0.0;
    int k = 0;
    for (; k + 4 <= d; k += 4) {
      const double m0 = __ldg(mcol + (size_t)(k + 0) * d);
      const double m1 = __ldg(mcol + (size_t)(k + 1) * d);
      const double m2 = __ldg(mcol + (size_t)(k + 2) * d);
      const double m3 = __ldg(mcol + (size_t)(k + 3) * d);
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        const double* y = Yc + r * dp + k;
        acc[r] = fma(m0, y[0], acc[r]);
        acc[r] = fma(m1, y[1], acc[r]);
        acc[r] = fma(m2, y[2], acc[r]);
        acc[r] = fma(m3, y[3], acc[r]);
      }
    }
    for (; k < d; ++k) {
      const double m = __ldg(mcol + (size_t)k * d);
#pragma unroll
      for (int r = 0; r < ROWS; ++r) acc[r] = fma(m, Yc[r * dp + k], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) Z[c * blk + r * dp + j] = acc[r];
  }
}

// Objective of the suite for nrows rows of src (row stride ld, in shared or
// global memory); the whole CTA calls it.  Y, Z: shared buffers of
// nrows x dp doubles, nc times that for a composition function;
// f[r] receives row r's value; comp: per row, the composition's g_c and
// D_c (kSuiteMaxRows x 10).
//   basic (5..14):  g(M ((x - o) s)), s the run's scale
//   hybrid:         z = M ((x - o) s), part p = the positions seg_p ..
//                   seg_{p+1} - 1 of the permuted z, scaled by the part's
//                   domain scale and evaluated as an n_p-dimensional function
//   composition:    sum_c omega_c (lambda_c g_c(M_c ((x - o_c) s_c)) + bias_c)
//                   with omega_c = w_c / sum w, w_c = exp(-D_c / (2 d
//                   sigma_c^2)) / sqrt(D_c), D_c = |x - o_c|^2, normalised in
//                   logarithms; at x = o_c the weight is 1 for the first such c.
constexpr int kSuiteMaxRows = 8;

static __device__ __noinline__ void suite_tile(const RunDesc& R, const double* src, int64_t ld, int nrows,
                                              double* __restrict__ Y, double* __restrict__ Z, double* __restrict__ f,
                                              double (*comp)[10]) {
  const int d = R.d, dp = R.dp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const bool is_comp = R.obj >= kObjComposition1;
  const bool is_hyb = R.obj >= kObjHybrid1 && R.obj <= kObjHybrid3;
  if (is_comp) {
    // every component at once: Y_c = (x - o_c) s_c, Z_c = M_c Y_c (blocks of
    // nrows x dp), then g_c and D_c = |x - o_c|^2 for every (row, component)
    const int nc = R.nc;
    const int blk = nrows * dp;
    for (int e = threadIdx.x; e < nc * blk; e += blockDim.x) {
      const int c = e / blk, rem = e - c * blk, r = rem / dp, j = rem - r * dp;
      double y = 0.0;
      if (j < d) y = __dmul_rn(__dsub_rn(src[(size_t)r * ld + j], R.o[(size_t)c * dp + j]), R.sscale[c]);
      Y[e] = y;
    }
    __syncthreads();
    if (R.rotate) {
      switch (nrows) {
        case 1: comp_rotate<1>(R.MT, Y, Z, nc, d, dp); break;
        case 2: comp_rotate<2>(R.MT, Y, Z, nc, d, dp); break;
        case 3: comp_rotate<3>(R.MT, Y, Z, nc, d, dp); break;
        case 4: comp_rotate<4>(R.MT, Y, Z, nc, d, dp); break;
        case 5: comp_rotate<5>(R.MT, Y, Z, nc, d, dp); break;
        case 6: comp_rotate<6>(R.MT, Y, Z, nc, d, dp); break;
        case 7: comp_rotate<7>(R.MT, Y, Z, nc, d, dp); break;
        default: comp_rotate<8>(R.MT, Y, Z, nc, d, dp); break;
      }
    } else {
      for (int e = threadIdx.x; e < nc * blk; e += blockDim.x) Z[e] = Y[e];
    }
    __syncthreads();
    // the costly parts of every (component, row, coordinate) over the whole
    // CTA, into Y (free after the rotation)
    for (int e = threadIdx.x; e < nc * blk; e += blockDim.x) {
      const int c = e / blk, rem = e - c * blk, r = rem / dp, j = rem - r * dp;
      if (j >= d || !basic_has_costly(R.sfn[c])) continue;
      const double* zr = Z + (size_t)c * blk + r * dp;
      Y[e] = basic_costly(R.sfn[c], zr[j], zr[j + 1 < d ? j + 1 : 0], j, d, R.skex[c]);
    }
    __syncthreads();
    for (int p = warp; p < nc * nrows; p += nwarps) {
      const int c = p / nrows, r = p - c * nrows;
      const double g =
          basic_fn_warp(R.sfn[c], Z + (size_t)c * blk + r * dp, nullptr, 0, d, 1.0, Y + (size_t)c * blk + r * dp, lane);
      const double* oc = R.o + (size_t)c * dp;
      double dd = 0.0;
      for (int j = lane; j < d; j += 32) {
        const double t = __dsub_rn(src[(size_t)r * ld + j], oc[j]);
        dd += t * t;
      }
      dd = warp_sum(dd);
      if (lane == 0) {
        comp[r][c] = g;
        comp[r][5 + c] = dd;
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
      int hit = -1;
      for (int c = 0; c < nc; ++c)
        if (comp[r][5 + c] == 0.0 && hit < 0) hit = c;
      double om[5], m = -CUDART_INF, sum = 0.0;
      for (int c = 0; c < nc; ++c) {
        const double D = comp[r][5 + c];
        om[c] = -0.5 * log(D) - D / (2.0 * d * R.ssigma[c] * R.ssigma[c]);
        m = fmax(m, om[c]);
      }
      for (int c = 0; c < nc; ++c) {
        om[c] = hit >= 0 ? (c == hit ? 1.0 : 0.0) : exp(om[c] - m);
        sum += om[c];
      }
      double acc = 0.0;
      for (int c = 0; c < nc; ++c) acc += om[c] / sum * (R.slambda[c] * comp[r][c] + R.sbias[c]);
      f[r] = acc;
    }
    __syncthreads();
    return;
  }
  // basic and hybrid functions: one shift and one rotation
  for (int e = threadIdx.x; e < nrows * dp; e += blockDim.x) {
    const int r = e / dp, j = e - r * dp;
    double y = 0.0;
    if (j < d) y = __dmul_rn(__dsub_rn(src[(size_t)r * ld + j], R.o[j]), R.scale);
    Y[e] = y;
  }
  __syncthreads();
  if (R.rotate) suite_rotate(R.MT, Y, Z, nrows, d, dp);
  else
    for (int e = threadIdx.x; e < nrows * dp; e += blockDim.x) Z[e] = Y[e];
  __syncthreads();
  // the costly parts of every (row, position) over the whole CTA, into Y
  // (free after the rotation)
  if (is_hyb) {
    // part q takes positions seg_q .. seg_{q+1} - 1 of the permuted row; its
    // nrows x n_q terms form chunks of 32, and warps take chunks, so that the
    // lanes of a warp evaluate one basic function
    int nch = 0, cst[6];
    for (int q = 0; q < R.nc; ++q) {
      cst[q] = nch;
      nch += basic_has_costly(R.sfn[q]) ? (nrows * (R.seg[q + 1] - R.seg[q]) + 31) / 32 : 0;
    }
    cst[R.nc] = nch;
    for (int ch = warp; ch < nch; ch += nwarps) {
      int q = 0;
      while (ch >= cst[q + 1]) ++q;
      const int b0 = R.seg[q], n = R.seg[q + 1] - b0;
      const int k = (ch - cst[q]) * 32 + lane;
      if (k >= nrows * n) continue;
      const int r = k / n, l = k - r * n;
      const double* zr = Z + r * dp;
      const double sc = R.sscale[q];
      Y[r * dp + b0 + l] =
          basic_costly(R.sfn[q], sc * zr[R.perm[b0 + l]], sc * zr[R.perm[b0 + (l + 1 < n ? l + 1 : 0)]], l, n, R.skex[q]);
    }
  } else if (basic_has_costly(R.obj)) {
    for (int e = threadIdx.x; e < nrows * dp; e += blockDim.x) {
      const int r = e / dp, j = e - r * dp;
      if (j >= d) continue;
      const double* zr = Z + r * dp;
      Y[e] = basic_costly(R.obj, zr[j], zr[j + 1 < d ? j + 1 : 0], j, d, R.skex[0]);
    }
  }
  __syncthreads();
  for (int r = warp; r < nrows; r += nwarps) {
    const double* zr = Z + r * dp;
    const double* er = Y + r * dp;
    double g = 0.0;
    if (is_hyb) {
      for (int q = 0; q < R.nc; ++q)
        g += basic_fn_warp(R.sfn[q], zr, R.perm, R.seg[q], R.seg[q + 1] - R.seg[q], R.sscale[q], er + R.seg[q], lane);
    } else {
      g = basic_fn_warp(R.obj, zr, nullptr, 0, d, 1.0, er, lane);
    }
    if (lane == 0) f[r] = g;
  }
  __syncthreads();
}

}  // namespace de
