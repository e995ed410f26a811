// de_fp64.cu -- FP64 kernels of the DE/rand/1/bin generation step.
//
//   k_init_population   Sec. 2 / Sec. 6.2.1: uniform initial population
//   k_eval_rows         Sec. 7.3.1: z = M((x - o) s), objective of each row
//   k_best_init         best record, stop flag and counters after (re)initialisation
//   k_gen_fp64          one whole generation, fused: mutant indices (Eq. 2),
//                       mutation (Eq. 2), binomial crossover (Eq. 3), bound
//                       repair, shift + rotation + objective (Sec. 7.3.1),
//                       greedy selection (Sec. 2, Sec. 6.2.5), best-so-far and
//                       stop test (Sec. 7.3.4)
//
// One CTA owns a tile of `rows` targets of one run.  A warp builds one trial
// at a time: lane L holds coordinates 128c + 4L .. 128c + 4L + 3, so a row is
// read with 32-byte vector loads per lane and each lane needs exactly one
// Philox block per 4 coordinates.  Trials, shifted vectors and rotated
// vectors of the tile live in shared memory; the population stays in
// HBM/L2.  The rotation is a DFMA contraction of the tile with M^T (row k of
// M^T is one coalesced read shared by all rows of the tile).  The last CTA of
// a run to finish (atomic ticket) reduces the per-tile best partials in tile
// order, so the best record is deterministic.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>

#include "de_common.cuh"
#include "de_internal.cuh"
#include "de_kernels.h"

namespace de {

// ------------------------------------------------------------------ objective
// Objective of one row held in shared memory (z, length d); the calling warp
// returns the same value in every lane.  Terms are summed per lane in
// coordinate order, then across lanes by a fixed xor tree.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double row_objective_fp64(int obj, const double* __restrict__ z, int d, int lane) {
  double s1 = 0.0, s2 = 0.0;
  if (obj == kObjSphere) {
    for (int j = lane; j < d; j += 32) s1 += z[j] * z[j];
  } else if (obj == kObjRastrigin) {
    for (int j = lane; j < d; j += 32) {
      const double zj = z[j];
      s1 += zj * zj - 10.0 * cospi(2.0 * zj) + 10.0;
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
      s2 += cospi(2.0 * zj);
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

// ------------------------------------------------------------------ init
// Parameter j of individual i: x = lo + (hi - lo) u with u from draws 2j, 2j+1
// of the INIT stream; one Philox block serves parameters 2b and 2b + 1.
__global__ void k_init_population(const RunDesc* __restrict__ runs, int run) {
  const RunDesc& R = runs[run];
  const int64_t nblk = (int64_t)R.np * (R.dp / 2);
  const double span = R.hi - R.lo;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nblk; t += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(t / (R.dp / 2));
    const uint32_t b = (uint32_t)(t % (R.dp / 2));
    const uint32_t j = 2u * b;
    double2 v = make_double2(0.0, 0.0);
    if ((int)j < R.d) {
      const U32x4 w = draw_block(R.seed, kPurposeInit, R.run_id, 0u, 0u, i, b);
      v.x = __fma_rn(span, unit_double(w.x, w.y), R.lo);
      if ((int)j + 1 < R.d) v.y = __fma_rn(span, unit_double(w.z, w.w), R.lo);
    }
    reinterpret_cast<double2*>(R.X[0] + (size_t)i * R.dp)[b] = v;
  }
}

// ------------------------------------------------------------------ eval
// f of n rows of x (row stride ld) with run `run`'s objective; CTA per tile
// of `rows` rows.  Shared memory: 2 * rows * dp doubles.
__global__ void k_eval_rows(const RunDesc* __restrict__ runs, int run, const double* __restrict__ x, int64_t ld,
                            int n, int rows, double* __restrict__ fout, uint8_t* __restrict__ fx_out) {
  extern __shared__ __align__(16) double sm[];
  const RunDesc& R = runs[run];
  const int d = R.d, dp = R.dp;
  double* Y = sm;
  double* Z = Y + rows * dp;
  const int row0 = blockIdx.x * rows;
  const int nrows = min(rows, n - row0);
  if (nrows <= 0) return;
  for (int e = threadIdx.x; e < rows * dp; e += blockDim.x) {
    const int r = e / dp, j = e % dp;
    double y = 0.0;
    if (r < nrows && j < d) y = __dmul_rn(__dsub_rn(x[(size_t)(row0 + r) * ld + j], R.o[j]), R.scale);
    Y[e] = y;
  }
  __syncthreads();
  const double* Zr = Y;
  if (R.rotate) {
    tile_rotate_dispatch(rows, R.MT, Y, Z, d, dp);
    Zr = Z;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int r = warp; r < nrows; r += nwarps) {
    const double f = row_objective_fp64(R.obj, Zr + r * dp, d, lane);
    if (lane == 0) {
      fout[row0 + r] = f;
      if (fx_out) fx_out[row0 + r] = 1;
    }
  }
}

// ------------------------------------------------------------------ best record
__device__ __forceinline__ bool better(double fa, int ia, double fb, int ib) {
  // a beats b: smaller f, or equal f and lower index; NaN never wins
  if (fa != fa) return false;
  if (ib < 0 || fb != fb) return true;
  return fa < fb || (fa == fb && ia < ib);
}

// Reduce f[0..np) of the current generation into the run's best record and
// set the stop flag; single CTA per run.  Used after (re)initialisation.
__global__ void k_best_init(const RunDesc* __restrict__ runs, int run) {
  const RunDesc& R = runs[run];
  RunState* st = R.st;
  const int cur = (int)(st->gen & 1);
  const double* f = R.f[cur];
  __shared__ double sf[32];
  __shared__ int si[32];
  double bf = CUDART_INF;
  int bi = -1;
  for (int i = threadIdx.x; i < R.np; i += blockDim.x)
    if (better(f[i], i, bf, bi)) { bf = f[i]; bi = i; }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double of = __shfl_xor_sync(0xffffffffu, bf, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (oi >= 0 && better(of, oi, bf, bi)) { bf = of; bi = oi; }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sf[warp] = bf; si[warp] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    bf = CUDART_INF;
    bi = -1;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      if (si[w] >= 0 && better(sf[w], si[w], bf, bi)) { bf = sf[w]; bi = si[w]; }
    st->best_f = bf;
    st->best_idx = bi;
    st->ticket = 0;
    st->ticket2 = 0;
    int stop = 0;
    if (R.target > 0.0 && bi >= 0 && bf < R.target) stop = 1;
    else if (R.max_evals > 0 && st->evals >= R.max_evals) stop = 2;
    else if (st->gen >= R.max_gens) stop = 3;
    st->stop = stop;
    if (bi < 0) st->err |= kErrNonFinite;
  }
  __syncthreads();
  const int best = st->best_idx;
  if (best >= 0)
    for (int j = threadIdx.x; j < R.dp; j += blockDim.x) R.best_x[j] = R.X[cur][(size_t)best * R.dp + j];
}

// Finish a generation of a run: called by the last CTA to arrive.  Reduces
// the tile partials in order, copies the best row, advances the counters and
// evaluates the stop rule (Sec. 7.3.4).
__device__ void finish_generation(const RunDesc& R, int64_t g, int nparts, const BestPartial* part,
                                  const double* Xn) {
  __shared__ double sf[32];
  __shared__ int si[32];
  double bf = CUDART_INF;
  int bi = -1;
  for (int t = threadIdx.x; t < nparts; t += blockDim.x) {
    const double pf = __ldcg(&part[t].f);
    const int pi = __ldcg(&part[t].idx);
    if (pi >= 0 && better(pf, pi, bf, bi)) { bf = pf; bi = pi; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double of = __shfl_xor_sync(0xffffffffu, bf, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (oi >= 0 && better(of, oi, bf, bi)) { bf = of; bi = oi; }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sf[warp] = bf; si[warp] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    bf = CUDART_INF;
    bi = -1;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      if (si[w] >= 0 && better(sf[w], si[w], bf, bi)) { bf = sf[w]; bi = si[w]; }
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
    si[0] = st->best_idx;
  }
  __syncthreads();
  const int best = si[0];
  if (best >= 0)
    for (int j = threadIdx.x; j < R.dp; j += blockDim.x) R.best_x[j] = __ldcg(Xn + (size_t)best * R.dp + j);
  __syncthreads();
  if (threadIdx.x == 0) R.st->ticket = 0;
}

// ------------------------------------------------------------------ trial row
// Build the trial of target i (Eq. 2 and Eq. 3 with bound repair) with one
// warp; writes T (trial) and Y = (T - o) s rows of length dp.
__device__ __forceinline__ double repair(double v, double x, double lo, double hi) {
  // a coordinate that leaves [lo, hi] goes half way from the target's
  // coordinate to the violated bound (the paper leaves bounds handling open)
  if (v < lo) return __dmul_rn(__dadd_rn(x, lo), 0.5);
  if (v > hi) return __dmul_rn(__dadd_rn(x, hi), 0.5);
  return v;
}

__device__ __forceinline__ void build_trial_row(const RunDesc& R, const double* __restrict__ X, uint32_t i,
                                                int64_t g, int lane, double* __restrict__ Trow,
                                                double* __restrict__ Yrow, float* ynorm2) {
  const int d = R.d;
  const U32x4 b0 = draw_block(R.seed, kPurposeStep, R.run_id, 0u, (uint32_t)g, i, 0u);
  uint32_t r1, r2, r3;
  mutant_indices(b0.x, b0.y, b0.z, i, (uint32_t)R.np, r1, r2, r3);
  const uint32_t jr = map_to_range(b0.w, (uint32_t)d);
  const double* xi = X + (size_t)i * R.dp;
  const double* x1 = X + (size_t)r1 * R.dp;
  const double* x2 = X + (size_t)r2 * R.dp;
  const double* x3 = X + (size_t)r3 * R.dp;
  const bool dbg = R.dbg_trial != nullptr;
  if (dbg && lane == 0) {
    R.dbg_idx[3 * i + 0] = (int32_t)r1;
    R.dbg_idx[3 * i + 1] = (int32_t)r2;
    R.dbg_idx[3 * i + 2] = (int32_t)r3;
    R.dbg_jrand[i] = (int32_t)jr;
  }
  float yn2 = 0.f;
  const int nchunks = (d + 127) / 128;
  for (int c = 0; c < nchunks; ++c) {
    const int j0 = 128 * c + 4 * lane;
    uint32_t bits = 0;
    if (j0 < d) {
      const U32x4 bc = draw_block(R.seed, kPurposeStep, R.run_id, 0u, (uint32_t)g, i, 1u + (uint32_t)(j0 >> 2));
      const double2 xa = *reinterpret_cast<const double2*>(xi + j0);
      const double2 xb = *reinterpret_cast<const double2*>(xi + j0 + 2);
      const double2 a1 = *reinterpret_cast<const double2*>(x1 + j0);
      const double2 b1 = *reinterpret_cast<const double2*>(x1 + j0 + 2);
      const double2 a2 = *reinterpret_cast<const double2*>(x2 + j0);
      const double2 b2 = *reinterpret_cast<const double2*>(x2 + j0 + 2);
      const double2 a3 = *reinterpret_cast<const double2*>(x3 + j0);
      const double2 b3 = *reinterpret_cast<const double2*>(x3 + j0 + 2);
      const double tx[4] = {xa.x, xa.y, xb.x, xb.y};
      const double v1[4] = {a1.x, a1.y, b1.x, b1.y};
      const double v2[4] = {a2.x, a2.y, b2.x, b2.y};
      const double v3[4] = {a3.x, a3.y, b3.x, b3.y};
      const uint32_t u[4] = {bc.x, bc.y, bc.z, bc.w};
      double t[4], y[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int j = j0 + m;
        t[m] = 0.0;
        y[m] = 0.0;
        if (j < d) {
          const bool crossed = ((uint32_t)j == jr) || ((uint64_t)u[m] <= R.cr_thr);
          if (crossed) {
            // Eq. 2: y = x_r1 + F (x_r2 - x_r3), one rounding for the product-sum
            const double v = __fma_rn(R.F, __dsub_rn(v2[m], v3[m]), v1[m]);
            t[m] = repair(v, tx[m], R.lo, R.hi);
            bits |= 1u << m;
          } else {
            t[m] = tx[m];
          }
          y[m] = __dmul_rn(__dsub_rn(t[m], R.o[j]), R.scale);
          yn2 += (float)y[m] * (float)y[m];
        }
      }
      *reinterpret_cast<double2*>(Trow + j0) = make_double2(t[0], t[1]);
      *reinterpret_cast<double2*>(Trow + j0 + 2) = make_double2(t[2], t[3]);
      if (Yrow) {
        *reinterpret_cast<double2*>(Yrow + j0) = make_double2(y[0], y[1]);
        *reinterpret_cast<double2*>(Yrow + j0 + 2) = make_double2(y[2], y[3]);
      }
      if (dbg) {
#pragma unroll
        for (int m = 0; m < 4; ++m)
          if (j0 + m < d) R.dbg_trial[(size_t)i * d + j0 + m] = t[m];
      }
    }
    if (dbg) {
      // lanes 8w .. 8w+7 of this chunk cover mask word 4c + w
      uint32_t word = (j0 < d) ? (bits << (j0 & 31)) : 0u;
      word |= __shfl_xor_sync(0xffffffffu, word, 1);
      word |= __shfl_xor_sync(0xffffffffu, word, 2);
      word |= __shfl_xor_sync(0xffffffffu, word, 4);
      const int wi = j0 >> 5;
      if ((lane & 7) == 0 && wi < R.nw) R.dbg_mask[(size_t)i * R.nw + wi] = word;
    }
  }
  if (ynorm2) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) yn2 += __shfl_xor_sync(0xffffffffu, yn2, o);
    *ynorm2 = yn2;
  }
}

// ------------------------------------------------------------------ generation
// Shared memory: T, Y, Z tiles of rows x dp doubles (Z aliases Y when there
// is no rotation).
__global__ void __launch_bounds__(256) k_gen_fp64(const RunDesc* __restrict__ runs,
                                                  const int2* __restrict__ items) {
  extern __shared__ __align__(16) double sm[];
  __shared__ int s_stop, s_last;
  __shared__ long long s_gen;
  __shared__ double s_bf[8];
  __shared__ int s_bi[8];
  const int2 it = items[blockIdx.x];
  const RunDesc& R = runs[it.x];
  RunState* st = R.st;
  if (threadIdx.x == 0) {
    s_stop = *(volatile int32_t*)&st->stop;
    s_gen = *(volatile int64_t*)&st->gen;
  }
  __syncthreads();
  if (s_stop) return;
  const int64_t g = s_gen + 1;
  const int cur = (int)(s_gen & 1), nxt = cur ^ 1;
  const double* __restrict__ X = R.X[cur];
  double* __restrict__ Xn = R.X[nxt];
  const double* __restrict__ fX = R.f[cur];
  double* __restrict__ fn = R.f[nxt];
  const int d = R.d, dp = R.dp, rows = R.rows;
  const int row0 = it.y * rows;
  const int nrows = min(rows, R.np - row0);
  double* T = sm;
  double* Y = T + rows * dp;
  double* Z = R.rotate ? Y + rows * dp : Y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;

  // rows of the tile past the population end contribute zeros to the GEMM
  for (int e = nrows * dp + threadIdx.x; e < rows * dp; e += blockDim.x) Y[e] = 0.0;
  for (int rl = warp; rl < nrows; rl += nwarps)
    build_trial_row(R, X, (uint32_t)(row0 + rl), g, lane, T + rl * dp, Y + rl * dp, nullptr);
  __syncthreads();
  if (R.rotate) tile_rotate_dispatch(rows, R.MT, Y, Z, d, dp);
  __syncthreads();

  double bf = CUDART_INF;
  int bi = -1;
  for (int rl = warp; rl < nrows; rl += nwarps) {
    const int i = row0 + rl;
    const double ft = row_objective_fp64(R.obj, Z + rl * dp, d, lane);
    const double fi = fX[i];
    const bool acc = ft <= fi;  // false for a NaN trial
    const double* src = acc ? (T + rl * dp) : (X + (size_t)i * dp);
    double2* dst = reinterpret_cast<double2*>(Xn + (size_t)i * dp);
    for (int j = lane; j < dp / 2; j += 32) dst[j] = reinterpret_cast<const double2*>(src)[j];
    const double fnew = acc ? ft : fi;
    if (lane == 0) {
      fn[i] = fnew;
      if (R.dbg_ftrial) {
        R.dbg_ftrial[i] = ft;
        R.dbg_accept[i] = acc ? 1 : 0;
        R.dbg_fp64[i] = 1;
      }
    }
    if (better(fnew, i, bf, bi)) { bf = fnew; bi = i; }
  }
  if (lane == 0) { s_bf[warp] = bf; s_bi[warp] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    bf = CUDART_INF;
    bi = -1;
    for (int w = 0; w < nwarps; ++w)
      if (s_bi[w] >= 0 && better(s_bf[w], s_bi[w], bf, bi)) { bf = s_bf[w]; bi = s_bi[w]; }
    R.part[it.y].f = bf;
    R.part[it.y].idx = bi;
    __threadfence();
    const uint32_t t = atomicAdd(&st->ticket, 1u);
    s_last = (t == (uint32_t)R.ntiles - 1u);
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    finish_generation(R, g, R.ntiles, R.part, Xn);
  }
}

}  // namespace de

// ------------------------------------------------------------------ launchers
namespace de {

void k_configure(size_t smem_gen) {
  cudaFuncSetAttribute(k_gen_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem_gen, 1));
  cudaFuncSetAttribute(k_eval_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

void k_gen_fp64_launch(const RunDesc* runs, const int2* items, int nitems, int threads, size_t smem,
                       cudaStream_t s) {
  k_gen_fp64<<<nitems, threads, smem, s>>>(runs, items);
}

void k_init_population_launch(const RunDesc* runs, int run, int np, int dp, cudaStream_t s) {
  const long long n = (long long)np * (dp / 2);
  const int threads = 256;
  const int blocks = (int)std::min<long long>((n + threads - 1) / threads, 152LL * 16);
  k_init_population<<<blocks, threads, 0, s>>>(runs, run);
}

void k_eval_rows_launch(const RunDesc* runs, int run, const double* x, int64_t ld, int n, int dp, int rotate,
                        double* f, uint8_t* fx, cudaStream_t s) {
  int rows = 8;
  while (rows > 1 && (size_t)2 * rows * dp * sizeof(double) > 200 * 1024) rows >>= 1;
  (void)rotate;
  const size_t smem = (size_t)2 * rows * dp * sizeof(double);
  k_eval_rows<<<(n + rows - 1) / rows, 256, smem, s>>>(runs, run, x, ld, n, rows, f, fx);
}

void k_best_init_launch(const RunDesc* runs, int run, cudaStream_t s) { k_best_init<<<1, 256, 0, s>>>(runs, run); }

}  // namespace de
