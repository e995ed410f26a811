// de_fp64.cu -- FP64 kernels of the DE/rand/1/bin generation step.
//
//   k_init_population   Sec. 2 / Sec. 6.2.1: uniform initial population
//   k_eval_rows         Sec. 7.3.1: z = M((x - o) s), objective of each row
//   k_best_init         best record, stop flag and counters after (re)initialisation
//   k_ode_reference     trajectory of the hidden parameters of the ODE objective
//   k_jde_init          jDE: initial F_i and CR_i
//   k_gen_fp64          one whole generation, fused: mutant indices (Eq. 2),
//                       mutation (Eq. 2), binomial crossover (Eq. 3), bound
//                       repair, shift + rotation + objective (Sec. 7.3.1),
//                       greedy selection (Sec. 2, Sec. 6.2.5), best-so-far and
//                       stop test (Sec. 7.3.4); also the DE/best/1/bin and
//                       DE/rand/1/exp strategies and jDE (Sec. 2)
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
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>

#include "de_common.cuh"
#include "de_internal.cuh"
#include "de_device.cuh"
#include "de_island_dev.cuh"
#include "de_kernels.h"
#include "de_suite.cuh"

namespace cg = cooperative_groups;

namespace de {

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
  // a composition function keeps every component's rows at once
  const int ncomp = R.obj >= kObjComposition1 ? R.nc : 1;
  double* Y = sm;
  double* Z = Y + ncomp * rows * dp;
  const int row0 = blockIdx.x * rows;
  const int nrows = min(rows, n - row0);
  if (nrows <= 0) return;
  if (suite_objective(R.obj)) {
    // the proposed benchmark's functions (Sec. 7.3, Table 2)
    __shared__ double s_f[kSuiteMaxRows];
    __shared__ double s_comp[kSuiteMaxRows][10];
    suite_tile(R, x + (size_t)row0 * ld, ld, nrows, Y, Z, s_f, s_comp);
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
      fout[row0 + r] = s_f[r];
      if (fx_out) fx_out[row0 + r] = 1;
    }
    return;
  }
  if (R.obj == kObjOde) {
    // a warp integrates one row's chain
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int r = warp; r < nrows; r += nwarps) {
      const double s = warp_sum(ode_chain(x + (size_t)(row0 + r) * ld, lane, R.ode_ref, nullptr));
      if (lane == 0) {
        fout[row0 + r] = s / (double)(kOdeSteps * kOdeN);
        if (fx_out) fx_out[row0 + r] = 1;
      }
    }
    return;
  }
  for (int e = threadIdx.x; e < rows * dp; e += blockDim.x) {
    const int r = e / dp, j = e % dp;
    double y = 0.0;
    if (r < nrows && j < d) y = shifted(x[(size_t)(row0 + r) * ld + j], R.o[j], R);
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

// jDE: every F_i and CR_i of generation 0 set to the run's F and CR.
__global__ void k_jde_init(const RunDesc* __restrict__ runs, int run) {
  const RunDesc& R = runs[run];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < R.np) {
    R.jF[0][i] = R.F;
    R.jCR[0][i] = R.CR;
  }
}

// Trajectory of the hidden parameter vector o of an ODE run (one warp).
__global__ void k_ode_reference(const RunDesc* __restrict__ runs, int run, double* __restrict__ ref) {
  const RunDesc& R = runs[run];
  ode_chain(R.o, threadIdx.x & 31, nullptr, ref);
}

// Reduce f[0..np) of the current generation into the run's best record and
// set the stop flag; single CTA per run.  Used after (re)initialisation.
__global__ void k_best_init(const RunDesc* __restrict__ runs, int run) {
  const RunDesc& R = runs[run];
  RunState* st = R.st;
  // double-buffered paths alternate buffers by generation; the three-kernel
  // split path updates X[0] in place
  const int cur = R.dbuf ? (int)(st->gen & 1) : 0;
  const double* f = R.f[cur];
  __shared__ double sf[32];
  __shared__ long long sk[32];
  __shared__ int si[32];
  Best b;
  b.init();
  for (int i = threadIdx.x; i < R.np; i += blockDim.x) b.offer(f[i], i);
  b.warp_reduce();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sf[warp] = b.f; sk[warp] = b.k; si[warp] = b.i; }
  __syncthreads();
  if (threadIdx.x == 0) {
    b.init();
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b.take(sf[w], sk[w], si[w]);
    const double bf = b.f;
    const int bi = b.i;
    st->best_f = bf;
    st->best_idx = bi;
    st->ticket = 0;
    st->band_n = 0;
    st->band_left = 0;
    int stop = 0;
    // the target test takes FP64 values only (a split-precision initial value
    // below the target leaves the decision to the first generation's FP64 band)
    if (R.target > 0.0 && bi >= 0 && bf < R.target && R.fx[cur][bi]) stop = 1;
    else if (R.max_evals > 0 && st->evals >= R.max_evals) stop = 2;
    else if (st->gen >= R.max_gens) stop = 3;
    st->stop = stop;
    if (bi < 0) st->err |= kErrNonFinite;
  }
}

// ------------------------------------------------------------------ generation
// Q groups of 32 flattened outputs (row r, coordinate j) of the tile's
// rotation, one per accumulator chain: z[r][j] = sum_k M^T[k][j] y[r][k].
template <int Q>
__device__ __forceinline__ void rotate_groups(const RunDesc& R, const double* __restrict__ Y, double* __restrict__ Z,
                                              int w0, int stride, int lane, int nout, int dp) {
  const int d = R.d;
  int rr[Q], jj[Q];
  bool ok[Q];
  double acc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int e = (w0 + q * stride) * 32 + lane;
    ok[q] = e < nout;
    const int ec = ok[q] ? e : nout - 1;
    rr[q] = ec / d;
    jj[q] = ec - rr[q] * d;
    acc[q] = 0.0;
  }
  for (int k = 0; k < d; ++k) {
    const double* mk = R.MT + (size_t)k * d;
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = fma(__ldg(mk + jj[q]), Y[rr[q] * dp + k], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < Q; ++q)
    if (ok[q]) Z[rr[q] * dp + jj[q]] = acc[q];
}

// One tile of generation g: the trials of targets row0 .. row0 + nrows - 1
// (a warp per target), their fitness, and greedy selection into the other
// population buffer.  Shared memory sm: T (trials), Y (shifted trials), Z
// (rotated), W (second term sum of Ackley), each rows_max x dp doubles.
// best: the current population's best row (DE/best/1).  Returns the calling
// warp's best (f, index) over the tile's new population rows (the same in
// every lane).  Population rows, fitness and jDE parameters of generation
// g - 1 are read at L2.
// VAR / SUITE: strategy variants and jDE / the benchmark suite's objectives.
template <bool VAR, bool SUITE>
__device__ __forceinline__ Best gen_tile(const RunDesc& R, int64_t g, int row0, int nrows, int rows_max, int best,
                                         double* sm, double* s_fsuite, double (*s_comp)[10]) {
  const int cur = (int)((g - 1) & 1), nxt = cur ^ 1;
  const double* X = R.X[cur];
  double* __restrict__ Xn = R.X[nxt];
  const double* fX = R.f[cur];
  double* __restrict__ fn = R.f[nxt];
  const int d = R.d, dp = R.dp;
  double* T = sm;
  double* Y = T + rows_max * dp;
  double* Z = Y + rows_max * dp;
  double* W = Z + rows_max * dp;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;

  // ---- trials (a warp per target)
  const bool var = VAR && (R.strategy != 0 || R.jde);
  const double* jFc = VAR && R.jde ? R.jF[cur] : nullptr;
  const double* jCRc = VAR && R.jde ? R.jCR[cur] : nullptr;
  if (var) {
    for (int rl = warp; rl < nrows; rl += nwarps)
      build_trial_row<true>(R, X, (uint32_t)(row0 + rl), g, lane, T + rl * dp, Y + rl * dp, best, jFc, jCRc);
  } else if (R.unit_scale) {
    // a unit domain scale: no multiplication on the FP64 pipe (the compiler
    // would otherwise run it speculatively)
    for (int rl = warp; rl < nrows; rl += nwarps)
      build_trial_row<false, true>(R, X, (uint32_t)(row0 + rl), g, lane, T + rl * dp, Y + rl * dp);
  } else {
    for (int rl = warp; rl < nrows; rl += nwarps)
      build_trial_row<false>(R, X, (uint32_t)(row0 + rl), g, lane, T + rl * dp, Y + rl * dp);
  }
  __syncthreads();

  const int nout = nrows * d;
  const bool suite = SUITE && suite_objective(R.obj);
  if (suite) {
    // ---- the proposed benchmark's functions (Sec. 7.3, Table 2)
    const int ncomp = R.obj >= kObjComposition1 ? R.nc : 1;  // Y and Z hold every component of the tile
    suite_tile(R, T, dp, nrows, Y, Y + (size_t)ncomp * rows_max * dp, s_fsuite, s_comp);
  } else if (R.obj == kObjOde) {
    // ---- ODE objective: a warp integrates one trial's chain; f to W[row][0]
    for (int rl = warp; rl < nrows; rl += nwarps) {
      const double s = warp_sum(ode_chain(T + rl * dp, lane, R.ode_ref, nullptr));
      if (lane == 0) W[rl * dp] = s / (double)(kOdeSteps * kOdeN);
    }
    __syncthreads();
  } else {
    // ---- rotation, flattened over (row, output): output e = 32 w + lane of
    // warp-group w; a warp takes groups warp, warp + 8, ... and runs up to four
    // of them at once (independent accumulator chains)
    if (R.rotate) {
      const int ngroups = (nout + 31) / 32;
      for (int w0 = warp; w0 < ngroups; w0 += 4 * nwarps) {
        const int qn = min(4, (ngroups - w0 + nwarps - 1) / nwarps);  // uniform in the warp
        if (qn == 4) rotate_groups<4>(R, Y, Z, w0, nwarps, lane, nout, dp);
        else if (qn == 3) rotate_groups<3>(R, Y, Z, w0, nwarps, lane, nout, dp);
        else if (qn == 2) rotate_groups<2>(R, Y, Z, w0, nwarps, lane, nout, dp);
        else rotate_groups<1>(R, Y, Z, w0, nwarps, lane, nout, dp);
      }
    } else {
      for (int e = tid; e < nout; e += blockDim.x) {
        const int r = e / d, j = e - r * d;
        Z[r * dp + j] = Y[r * dp + j];
      }
    }
    __syncthreads();

    // ---- objective terms, flattened; Y and W receive the per-coordinate terms
    for (int e = tid; e < nout; e += blockDim.x) {
      const int r = e / d, j = e - r * d;
      const double z = Z[r * dp + j];
      double t1 = 0.0, t2 = 0.0;
      if (R.obj == kObjSphere) {
        t1 = z * z;
      } else if (R.obj == kObjRastrigin) {
        t1 = z * z - 10.0 * cos2pi_f64_horner(z) + 10.0;
      } else if (R.obj == kObjAckley) {
        t1 = z * z;
        t2 = cos2pi_f64_horner(z);
      } else if (R.obj == kObjRosenbrock) {
        if (j + 1 < d) {
          const double t0 = z + 1.0, tn = Z[r * dp + j + 1] + 1.0;
          const double a = tn - t0 * t0, b = t0 - 1.0;
          t1 = 100.0 * a * a + b * b;
        }
      } else {
        t1 = CUDART_NAN;
      }
      Y[r * dp + j] = t1;
      W[r * dp + j] = t2;
    }
    __syncthreads();
  }

  // ---- row sums, greedy selection, best partial (a warp per row)
  Best bb;
  bb.init();
  for (int rl = warp; rl < nrows; rl += nwarps) {
    const int i = row0 + rl;
    double ft;
    if (suite) {
      ft = s_fsuite[rl];
    } else if (R.obj == kObjOde) {
      ft = W[rl * dp];
    } else {
      double s1 = 0.0, s2 = 0.0;
      for (int j = lane; j < d; j += 32) {
        s1 += Y[rl * dp + j];
        s2 += W[rl * dp + j];
      }
      s1 = warp_sum(s1);
      s2 = warp_sum(s2);
      ft = R.obj == kObjAckley ? 20.0 + 2.718281828459045 - 20.0 * exp(-0.2 * sqrt(s1 / d)) - exp(s2 / d) : s1;
    }
    const double fi = __ldcg(fX + i);
    const bool acc = fit_key(ft) <= fit_key(fi) && fit_key(ft) != 0x7FFFFFFFFFFFFFFFLL;  // ft <= fi, NaN never
    double2* dst = reinterpret_cast<double2*>(Xn + (size_t)i * dp);
    if (acc) {
      const double2* src = reinterpret_cast<const double2*>(T + rl * dp);
      for (int j = lane; j < dp / 2; j += 32) dst[j] = src[j];
    } else {
      const double2* src = reinterpret_cast<const double2*>(X + (size_t)i * dp);
      for (int j = lane; j < dp / 2; j += 32) dst[j] = __ldcg(src + j);
    }
    const double fnew = acc ? ft : fi;
    if (VAR && R.jde && lane == 0) {
      // jDE: an accepted trial passes its F_i and CR_i on
      double Fi = __ldcg(jFc + i), CRi = __ldcg(jCRc + i);
      if (acc) jde_params(R, (uint32_t)i, g, jFc, jCRc, Fi, CRi);
      R.jF[nxt][i] = Fi;
      R.jCR[nxt][i] = CRi;
    }
    if (lane == 0) {
      fn[i] = fnew;
      if (R.dbg_ftrial) {
        R.dbg_ftrial[i] = ft;
        R.dbg_accept[i] = acc ? 1 : 0;
        R.dbg_fp64[i] = 1;
      }
    }
    bb.offer(fnew, i);
  }
  return bb;
}

// Copy of a run descriptor into shared memory (its fields are read in every
// phase, after barriers that would force global reloads).
__device__ __forceinline__ void load_desc(RunDesc& sR, const RunDesc* src) {
  for (int q = threadIdx.x; q < (int)(sizeof(RunDesc) / 8); q += blockDim.x)
    reinterpret_cast<uint64_t*>(&sR)[q] = reinterpret_cast<const uint64_t*>(src)[q];
}

// items: (run, tile, first row, rows); the rows of all runs are spread over
// about one CTA per SM so that every SM's FP64 pipe gets the same work.
// VAR: some run of the launch uses a strategy variant or jDE; SUITE: some
// run uses a function of the proposed benchmark (objectives 5..20).  Separate
// instances, so that plain DE/rand/1/bin keeps its register allocation.
template <bool VAR, bool SUITE>
__global__ void __launch_bounds__(256) k_gen_fp64(const RunDesc* __restrict__ runs,
                                                  const int4* __restrict__ items) {
  extern __shared__ __align__(16) double sm[];
  __shared__ int s_stop, s_last, s_best;
  __shared__ long long s_gen;
  __shared__ double s_bf[8];
  __shared__ long long s_bk[8];
  __shared__ int s_bi[8];
  __shared__ double s_fsuite[kSuiteMaxRows];
  __shared__ double s_comp[kSuiteMaxRows][10];
  const int4 it = items[blockIdx.x];
  __shared__ RunDesc sR;
  load_desc(sR, runs + it.x);
  const RunDesc& R = sR;
  pdl_launch_dependents();
  pdl_wait();
  __syncthreads();
  RunState* st = R.st;
  if (threadIdx.x == 0) {
    s_stop = *(volatile int32_t*)&st->stop;
    s_gen = *(volatile int64_t*)&st->gen;
    // DE/best/1: the lowest-index best of the current population (row 0
    // when no fitness is finite)
    s_best = max(*(volatile int32_t*)&st->best_idx, 0);
  }
  __syncthreads();
  if (s_stop) return;
  const int64_t g = s_gen + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
  Best bb = gen_tile<VAR, SUITE>(R, g, it.z, it.w, R.rows, s_best, sm, s_fsuite, s_comp);
  if (lane == 0) { s_bf[warp] = bb.f; s_bk[warp] = bb.k; s_bi[warp] = bb.i; }
  __syncthreads();
  if (tid == 0) {
    bb.init();
    for (int w = 0; w < nwarps; ++w) bb.take(s_bf[w], s_bk[w], s_bi[w]);
    R.part[it.y].f = bb.f;
    R.part[it.y].idx = bb.i;
    __threadfence();
    const uint32_t t = atomicAdd(&st->ticket, 1u);
    s_last = (t == (uint32_t)R.ntiles - 1u);
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    finish_generation(R, g, R.ntiles, R.part, R.X[g & 1]);
  }
}

// The generation loop of FP64 runs in one cooperative launch: CTA t owns
// item t's targets for every generation; after its tile it arrives at a grid
// barrier (bounded spin on a global counter), then every CTA of a run reduces
// that run's tile partials (double buffered by generation parity) itself, so
// that all of them take the same best record and stop decision; the run's
// tile 0 publishes the run state.  Population rows written by other CTAs in
// generation g - 1 are read at L2 (gen_tile).
//
// The CTAs of a stopped run keep arriving at the barrier until every run has
// stopped.  A run that stops at iteration k is counted (by its tile 0) in
// ctl->stopped[k % 3]; every CTA reads that slot after barrier k + 1, when
// it is complete and no longer written, so all CTAs see the same count and
// leave at the same iteration; CTA 0 clears slot (k + 1) % 3 after barrier k
// (every CTA read it after barrier k - 1; it is next written after barrier
// k + 1).  Runs stopped before the launch are counted in
// slot 2 (iteration -1).  With one run every CTA takes the stop decision
// itself and the launch ends at once.
//
// clustered = 1: the launch is one thread-block cluster (a single run of at
// most 8 tiles); the hardware cluster barrier, whose release / acquire covers
// the global writes of every thread, replaces the counter.
constexpr long long kFp64Spin = 1LL << 22;

// ISL: the runs are islands (an instance of its own, so that the other
// instances keep their register allocation)
template <bool VAR, bool SUITE, bool ISL>
__global__ void __launch_bounds__(256) k_gen_fp64_persist(const RunDesc* __restrict__ runs,
                                                          const int4* __restrict__ items, int nruns,
                                                          PersistCtl* ctl, long long gens, int clustered,
                                                          IslandCtl* isl, IslandStage stage) {
  extern __shared__ __align__(16) double sm[];
  __shared__ int s_stop, s_best, s_abort, s_done;
  __shared__ unsigned s_below;
  __shared__ long long s_gen, s_evals;
  __shared__ double s_bestf;
  __shared__ double s_bf[8];
  __shared__ long long s_bk[8];
  __shared__ int s_bi[8];
  __shared__ double s_fsuite[kSuiteMaxRows];
  __shared__ double s_comp[kSuiteMaxRows][10];
  const int4 it = items[blockIdx.x];
  __shared__ RunDesc sR;
  load_desc(sR, runs + it.x);
  __syncthreads();
  const RunDesc& R = sR;
  RunState* st = R.st;
  const unsigned nct = gridDim.x;
  const int ntiles = R.ntiles;
  if (threadIdx.x == 0) {
    s_stop = st->stop;
    s_gen = st->gen;
    s_evals = st->evals;
    s_bestf = st->best_f;
    s_best = st->best_idx;
    s_abort = 0;
    s_done = 0;
    s_below = 0u;
    if (blockIdx.x == 0) ctl->gen0 = s_gen;
    if (s_stop && it.y == 0 && nruns > 1) atomicAdd(&ctl->stopped[2], 1u);
  }
  __syncthreads();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
  if (nruns == 1 && s_stop) return;
  unsigned nstopped = 0;  // runs known stopped (thread 0)
  // the failure-detection test (off in normal launches): this CTA may leave
  // out its first arrival, and the barrier may give up sooner
  const bool test_skip = ctl->test_skip == (int)blockIdx.x + 1;
  const long long spin_limit = ctl->test_spin > 0 ? ctl->test_spin : kFp64Spin;
  // grid barrier number nbar + 1 (warp 0; the whole warp polls the counter,
  // one load per poll, no divergent spin)
  unsigned nbar = 0;
  auto grid_sync = [&]() -> bool {
    if (lane == 0 && !(test_skip && nbar == 0)) {
      // release: the CTA's writes before the barrier are visible to every
      // CTA that observes the count
      asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(&ctl->bar), "r"(1u) : "memory");
    }
    __syncwarp();
    const unsigned target = (nbar + 1u) * nct;
    bool ok = false;
    for (long long k = 0; k < spin_limit; ++k) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&ctl->bar) : "memory");
      if (v >= target) {
        ok = true;
        break;
      }
      // the abort flag every 16th poll (a read after every poll doubles
      // the round trips per poll)
      if ((k & 15) == 15 && *(volatile int*)&ctl->abort) break;
    }
    __syncwarp();
    ++nbar;
    return ok;
  };
  // a grid barrier of the whole CTA (island migration steps); the CTA
  // barrier first orders every warp's writes (the posted migrants) before
  // warp 0's release
  auto full_sync = [&]() {
    __syncthreads();
    if (warp == 0) {
      const bool ok = grid_sync();
      if (!ok && lane == 0) {
        atomicExch(&ctl->abort, 1);
        atomicOr(&st->err, kErrTimeout);
        s_abort = 1;
      }
    }
    __syncthreads();
  };
  for (long long itg = 0; itg < gens; ++itg) {
    const bool live = !s_stop;
    const int64_t g = s_gen + 1;
    if (live) {
      Best bb = gen_tile<VAR, SUITE>(R, g, it.z, it.w, R.rows, max(s_best, 0), sm, s_fsuite, s_comp);
      if (lane == 0) { s_bf[warp] = bb.f; s_bk[warp] = bb.k; s_bi[warp] = bb.i; }
      __syncthreads();
      if (tid == 0) {
        bb.init();
        for (int w = 0; w < nwarps; ++w) bb.take(s_bf[w], s_bk[w], s_bi[w]);
        BestPartial* pp = R.part + (size_t)(g & 1) * ntiles + it.y;
        pp->f = bb.f;
        pp->idx = bb.i;
        // island model: the model stops as a whole once any island's best is
        // below the target (counted before the barrier, read after it)
        if (ISL && R.target > 0.0 && bb.i >= 0 && bb.f < R.target) atomicAdd(&ctl->below[itg % 3], 1u);
      }
    }
    if (clustered) {
      cg::this_cluster().sync();
    } else if (warp == 0) {
      // arrive, then wait for every CTA of this iteration
      const bool ok = grid_sync();
      if (lane == 0) {
        if (!ok) {
          atomicExch(&ctl->abort, 1);
          atomicOr(&st->err, kErrTimeout);
          s_abort = 1;
        } else if (nruns > 1) {
          // runs stopped at iteration itg - 1 (complete after this barrier)
          nstopped += __ldcg(&ctl->stopped[(itg + 2) % 3]);
          // every CTA read slot (itg + 1) % 3 after the previous barrier; it is
          // next written at iteration itg + 1, after the next barrier
          if (blockIdx.x == 0) ctl->stopped[(itg + 1) % 3] = 0u;
          if (nstopped >= (unsigned)nruns) s_done = 1;
        }
        if (ISL && ok) {
          s_below = __ldcg(&ctl->below[itg % 3]);
          // every CTA read slot (itg + 2) % 3 before arriving at this barrier;
          // it is next counted at iteration itg + 2
          if (blockIdx.x == 0) ctl->below[(itg + 2) % 3] = 0u;
        }
      }
    }
    __syncthreads();
    if (s_abort || s_done) break;
    if (live) {
      // the best record and the stop rule of generation g, the same in every
      // CTA of the run: the whole CTA reduces the run's tile partials
      Best b;
      b.init();
      const BestPartial* q = R.part + (size_t)(g & 1) * ntiles;
      for (int t = tid; t < ntiles; t += blockDim.x) b.offer(__ldcg(&q[t].f), __ldcg(&q[t].idx));
      b.warp_reduce();
      if (lane == 0) { s_bf[warp] = b.f; s_bk[warp] = b.k; s_bi[warp] = b.i; }
      __syncthreads();
      if (tid == 0) {
        b.init();
        for (int w = 0; w < nwarps; ++w) b.take(s_bf[w], s_bk[w], s_bi[w]);
        const bool have = b.i >= 0;
        if (have) {
          s_bestf = b.f;
          s_best = b.i;
        }
        const int64_t evals = s_evals + R.np;
        int stop = 0;
        if (ISL && s_below > 0u) stop = 1;  // some island is below the target
        else if (R.target > 0.0 && s_best >= 0 && s_bestf < R.target) stop = 1;
        else if (R.max_evals > 0 && evals >= R.max_evals) stop = 2;
        else if (g >= R.max_gens) stop = 3;
        s_evals = evals;
        s_stop = stop;
        s_gen = g;
        if (it.y == 0) {
          if (have) {
            st->best_f = b.f;
            st->best_idx = b.i;
          } else {
            atomicOr(&st->err, kErrNonFinite);
          }
          st->gen = g;
          st->evals = evals;
          st->stop = stop;
          if (stop && nruns > 1) atomicAdd(&ctl->stopped[itg % 3], 1u);
        }
      }
      __syncthreads();
      if (nruns == 1 && s_stop) break;
    }
    if constexpr (ISL) {
      if (!(live && isl->interval > 0 && g % isl->interval == 0)) continue;
      // island model: migration after generation g (the islands advance
      // together, so every CTA takes this branch).  The CTA of each island's
      // tile 0 exchanges; a grid barrier then keeps every tile from building
      // generation g + 1 before the migrants are in place.
      const int cur = (int)(g & 1);
      const bool owner = it.y == 0;
      if (isl->async) {
        // one interval late, through the mailbox (k_island_async's rule)
        const int64_t ep = g / isl->interval;
        // post_gen is written by CTA 0 after an earlier migration's barrier: read at L2
        const long long pg = *(volatile long long*)&isl->post_gen;
        const bool take = pg >= 0 && pg == g - isl->interval;
        if (owner)
          island_exchange(R, it.x, isl->m, isl->nmig, cur, stage, true, (size_t)(ep & 1) * stage.slot, take,
                          (size_t)((ep & 1) ^ 1) * stage.slot);
      } else {
        // every island posts before any island takes
        if (owner) island_exchange(R, it.x, isl->m, isl->nmig, cur, stage, true, 0, false, 0);
        full_sync();
        if (s_abort) break;
        if (owner) island_exchange(R, it.x, isl->m, isl->nmig, cur, stage, false, 0, true, 0);
      }
      full_sync();
      if (s_abort) break;
      if (tid == 0) {
        // the island's best record after the exchange (DE/best/1's base)
        s_best = *(volatile int32_t*)&st->best_idx;
        s_bestf = *(volatile double*)&st->best_f;
        if (blockIdx.x == 0) {
          isl->mig_gen = g;
          if (isl->async) isl->post_gen = g;
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace de

// ------------------------------------------------------------------ launchers
namespace de {

void k_configure(size_t smem_gen) {
  const int smem = (int)std::max<size_t>(smem_gen, 1);
  cudaFuncSetAttribute(k_gen_fp64<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_gen_fp64<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_gen_fp64<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_gen_fp64<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_gen_fp64_persist<false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_gen_fp64_persist<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_gen_fp64_persist<false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_gen_fp64_persist<true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_gen_fp64_persist<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_gen_fp64_persist<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_eval_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t k_gen_fp64_persist_launch(const RunDesc* runs, const int4* items, int nitems, int nruns, int threads,
                                      size_t smem, bool var, bool suite, PersistCtl* ctl, long long gens,
                                      cudaStream_t s, int test_skip, IslandCtl* isl, const IslandStage* stage) {
  cudaError_t e = persist_ctl_reset(ctl, test_skip, s);
  if (e != cudaSuccess) return e;
  int clustered = 0;
  IslandStage st{};
  if (stage) st = *stage;
  void* args[] = {(void*)&runs, (void*)&items, (void*)&nruns, (void*)&ctl, (void*)&gens, (void*)&clustered,
                  (void*)&isl, (void*)&st};
  const dim3 grid((unsigned)nitems), block((unsigned)threads);
  if (isl && suite) return cudaErrorInvalidValue;  // islands of the suite's objectives run generation by generation
  const void* k = isl ? (var ? (const void*)k_gen_fp64_persist<true, false, true>
                             : (const void*)k_gen_fp64_persist<false, false, true>)
                  : var && suite ? (const void*)k_gen_fp64_persist<true, true, false>
                  : var          ? (const void*)k_gen_fp64_persist<true, false, false>
                  : suite        ? (const void*)k_gen_fp64_persist<false, true, false>
                                 : (const void*)k_gen_fp64_persist<false, false, false>;
  return cudaLaunchCooperativeKernel(k, grid, block, args, smem, s);
}

// The same kernel as one cluster of nitems CTAs (nitems <= 8, one run).
template <bool VAR, bool SUITE>
static cudaError_t fp64_cluster_launch(const RunDesc* runs, const int4* items, int nitems, int threads, size_t smem,
                                       PersistCtl* ctl, long long gens, cudaStream_t s, bool query_only,
                                       int* nclusters) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nitems);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)nitems;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (query_only) return cudaOccupancyMaxActiveClusters(nclusters, k_gen_fp64_persist<VAR, SUITE, false>, &cfg);
  const int nruns = 1, clustered = 1;
  IslandCtl* isl = nullptr;
  const IslandStage stage{};
  return cudaLaunchKernelEx(&cfg, k_gen_fp64_persist<VAR, SUITE, false>, runs, items, nruns, ctl, gens, clustered, isl,
                            stage);
}

cudaError_t k_gen_fp64_cluster_launch(const RunDesc* runs, const int4* items, int nitems, int threads, size_t smem,
                                      bool var, bool suite, PersistCtl* ctl, long long gens, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(PersistCtl), s);
  if (e != cudaSuccess) return e;
  if (var && suite) return fp64_cluster_launch<true, true>(runs, items, nitems, threads, smem, ctl, gens, s, false, nullptr);
  if (var) return fp64_cluster_launch<true, false>(runs, items, nitems, threads, smem, ctl, gens, s, false, nullptr);
  if (suite) return fp64_cluster_launch<false, true>(runs, items, nitems, threads, smem, ctl, gens, s, false, nullptr);
  return fp64_cluster_launch<false, false>(runs, items, nitems, threads, smem, ctl, gens, s, false, nullptr);
}

bool k_gen_fp64_cluster_fits(int nitems, int threads, size_t smem, bool var, bool suite) {
  if (nitems < 1 || nitems > 8) return false;
  int n = 0;
  cudaError_t e;
  if (var && suite) e = fp64_cluster_launch<true, true>(nullptr, nullptr, nitems, threads, smem, nullptr, 0, 0, true, &n);
  else if (var) e = fp64_cluster_launch<true, false>(nullptr, nullptr, nitems, threads, smem, nullptr, 0, 0, true, &n);
  else if (suite) e = fp64_cluster_launch<false, true>(nullptr, nullptr, nitems, threads, smem, nullptr, 0, 0, true, &n);
  else e = fp64_cluster_launch<false, false>(nullptr, nullptr, nitems, threads, smem, nullptr, 0, 0, true, &n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n >= 1;
}

int k_gen_fp64_persist_capacity(int threads, size_t smem, bool var, bool suite, bool isl) {
  int per_sm = 0, dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (isl && suite) return 0;  // islands of the suite's objectives run generation by generation
  const void* f = isl ? (var ? (const void*)k_gen_fp64_persist<true, false, true>
                             : (const void*)k_gen_fp64_persist<false, false, true>)
                  : var && suite ? (const void*)k_gen_fp64_persist<true, true, false>
                  : var          ? (const void*)k_gen_fp64_persist<true, false, false>
                  : suite        ? (const void*)k_gen_fp64_persist<false, true, false>
                                 : (const void*)k_gen_fp64_persist<false, false, false>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * nsm;
}

void k_gen_fp64_launch(const RunDesc* runs, const int4* items, int nitems, int threads, size_t smem, bool var,
                       bool suite, cudaStream_t s) {
  // programmatic stream serialization: generation g + 1 is scheduled while
  // generation g drains, and waits (griddepcontrol.wait) before reading it
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nitems);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (var && suite) cudaLaunchKernelEx(&cfg, k_gen_fp64<true, true>, runs, items);
  else if (var) cudaLaunchKernelEx(&cfg, k_gen_fp64<true, false>, runs, items);
  else if (suite) cudaLaunchKernelEx(&cfg, k_gen_fp64<false, true>, runs, items);
  else cudaLaunchKernelEx(&cfg, k_gen_fp64<false, false>, runs, items);
}

void k_init_population_launch(const RunDesc* runs, int run, int np, int dp, cudaStream_t s) {
  const long long n = (long long)np * (dp / 2);
  const int threads = 256;
  const int blocks = (int)std::min<long long>((n + threads - 1) / threads, 152LL * 16);
  k_init_population<<<blocks, threads, 0, s>>>(runs, run);
}

void k_eval_rows_launch(const RunDesc* runs, int run, const RunDesc& Rh, const double* x, int64_t ld, int n,
                        double* f, uint8_t* fx, cudaStream_t s) {
  if (n <= 0) return;
  if (Rh.obj == kObjOde) {
    // a warp per row, few rows per CTA: the rows spread over every SM (an
    // SM's FP64 pipe, not the latency of one chain, bounds a CTA of 8 chains)
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int rows = std::max(1, std::min(8, (n + nsm - 1) / std::max(nsm, 1)));
    k_eval_rows<<<(n + rows - 1) / rows, 32 * rows, 0, s>>>(runs, run, x, ld, n, rows, f, fx);
    return;
  }
  const int dp = Rh.dp, ncomp = suite_comps(Rh);
  int rows = 8;
  while (rows > 1 && (size_t)2 * ncomp * rows * dp * sizeof(double) > 200 * 1024) rows >>= 1;
  const size_t smem = (size_t)2 * ncomp * rows * dp * sizeof(double);
  k_eval_rows<<<(n + rows - 1) / rows, 256, smem, s>>>(runs, run, x, ld, n, rows, f, fx);
}

void k_best_init_launch(const RunDesc* runs, int run, cudaStream_t s) { k_best_init<<<1, 256, 0, s>>>(runs, run); }

void k_jde_init_launch(const RunDesc* runs, int run, int np, cudaStream_t s) {
  k_jde_init<<<(np + 255) / 256, 256, 0, s>>>(runs, run);
}

void k_ode_reference_launch(const RunDesc* runs, int run, double* ref, cudaStream_t s) {
  k_ode_reference<<<1, 32, 0, s>>>(runs, run, ref);
}

}  // namespace de
