// de_tc.cu -- split-precision generation step on the tcgen05 tensor cores.
//
// One generation is three launches:
//
//   k_trial_split  a warp per target: mutant indices, mutation, binomial
//                  crossover and bound repair (Eq. 2, Eq. 3) in FP64, exactly as
//                  in the FP64 path; the trial row goes to T (FP64) and its
//                  shifted vector y = (t - o) s, rounded to FP32 and split into
//                  a high and a low part (bf16 + bf16, or tf32 + tf32), goes
//                  straight into the tensor-core operand layout of its
//                  128-row tile.
//
//   k_fit_tc       a CTA per 128-row tile: the rotation z = M y of Sec. 7.3.1
//                  as Z = Y M^T on tcgen05 (kind::f16 for bf16, kind::tf32),
//                  three products yh Mh + yh Ml + yl Mh accumulated in FP32 in
//                  tensor memory; operands arrive by bulk async copies through
//                  a two-stage shared-memory pipeline; the objective terms are
//                  evaluated from TMEM on the CUDA cores in FP32; then greedy
//                  selection (Sec. 2) where the split-precision values decide
//                  it within their error bound; accepted trials are copied
//                  over their targets in place (the trial kernel of this
//                  generation has finished reading donors).  Rows the split
//                  values cannot decide, and trials that could become the new
//                  best, go to a list for the FP64 band kernel.
//
//   k_band_fp64    the listed rows, spread over the whole GPU: FP64 rotation
//                  and objective of the trial (and of the target when its
//                  stored fitness is not FP64) in 32-column chunks, then the
//                  FP64 selection decision.  The last CTA to finish a run's
//                  rows (or the last fitness CTA, when none was listed)
//                  reduces the best record and evaluates the stop rule
//                  (Sec. 7.3.4); the best record is therefore always FP64.
//
// Operand layout (no swizzle, K-major): a "core matrix" is 8 rows x 16 bytes,
// stored as 128 contiguous bytes.  Core matrix (kg, rg) -- k-group kg of 16
// bytes, row group rg of 8 rows -- sits at byte (kg * RG + rg) * 128, where RG
// is the number of row groups (16 for a 128-row A tile, ntn / 8 for an N tile
// of B).  In the instruction's shared-memory descriptor the leading byte offset
// is the stride between k-groups (RG * 128) and the stride byte offset the one
// between row groups (128).  A K chunk of the operand is therefore one
// contiguous byte range, moved by one cp.async.bulk.
//
// Every wait on an mbarrier is bounded; on expiry the kernel records
// kErrTimeout in the run state, waits (bounded) for its copies and MMAs, frees
// its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "de_device.cuh"
#include "de_kernels.h"
#include "de_tcgen05.cuh"

namespace de {

// ------------------------------------------------------------------ trial kernel
// items: (run, group); a warp holds 32 / R.lpt targets, R.lpt lanes each
// (lane L: coordinates 4 (L % lpt) .. + 3 of each 4 lpt-wide chunk), so that
// short rows do not leave most lanes of the FP64 instructions idle; warp w of
// the CTA takes targets (group * warps + w) * (32 / lpt) + L / lpt.
// VAR: some run uses a strategy variant or jDE (a separate instance).
// OCC: an instance held to 85 registers a thread (three 256-thread CTAs' worth
// of warps per SM), which spills a little but keeps more loads in flight; the
// other is held to 128 (no spills; left unbounded the compiler takes ~150 and
// a quarter of the warps).  The autotuner times both on the handle's problem.
template <int ESZ, bool VAR, bool OCC>
__global__ void __launch_bounds__(256, OCC ? 3 : 2)
    k_trial_split(const RunDesc* __restrict__ runs, const int2* __restrict__ items) {
  __shared__ int s_stop, s_best;
  __shared__ long long s_gen;
  const int2 it = items[blockIdx.x];
  const RunDesc& R = runs[it.x];
  pdl_launch_dependents();
  pdl_wait();
  // the previous generation's FP64 band kernel has finished: empty its list
  if (blockIdx.x == 0 && threadIdx.x == 0) *R.band_cnt = 0u;
  if (threadIdx.x == 0) {
    s_stop = *(volatile int32_t*)&R.st->stop;
    s_gen = *(volatile int64_t*)&R.st->gen;
    s_best = max(*(volatile int32_t*)&R.st->best_idx, 0);  // DE/best/1 base (row 0 when none is finite)
  }
  __syncthreads();
  if (s_stop) return;
  const int64_t g = s_gen + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lpt = R.lpt, sub = lane & (lpt - 1);
  const int i0 = (it.y * (int)(blockDim.x >> 5) + warp) * (32 / lpt);
  if (i0 >= R.np) return;  // the whole warp
  const int iraw = i0 + lane / lpt;
  const bool valid = iraw < R.np;
  const int i = valid ? iraw : R.np - 1;  // idle segments repeat a valid target without writing
  const double* X = R.X[0];
  TrialVar v;
  TrialSetup s;
  if constexpr (VAR) s = trial_setup_var(R, (uint32_t)i, g, lane, s_best, R.jde ? R.jF[0] : nullptr,
                                         R.jde ? R.jCR[0] : nullptr, v, lpt, valid);
  else s = trial_setup(R, (uint32_t)i, g, sub, 0u, valid);
  uint8_t* Ahi = R.A + (size_t)(i >> 7) * R.a_tile_bytes;
  const uint32_t a_part = (uint32_t)(R.a_tile_bytes / 2);
  const int m = i & 127;
  float yn2 = 0.f;
  const bool dbg = R.dbg_trial != nullptr;
  const int cw = 4 * lpt;  // coordinates per chunk
  const int nchunks = (R.kpad + cw - 1) / cw;
  // the loads of chunk c + 1 are issued before chunk c is computed; the loop
  // is compiled twice, for a unit domain scale (no multiplication) and any other
  ChunkIn cur, nxt;
  if (4 * sub < R.d) trial_load(R, X, s, (uint32_t)i, g, 4 * sub, cur);
  auto chunks = [&](auto unit) {
  constexpr bool UNIT = decltype(unit)::value;
  for (int c = 0; c < nchunks; ++c) {
    const int j0 = cw * c + 4 * sub;
    if (c + 1 < nchunks && j0 + cw < R.d) trial_load(R, X, s, (uint32_t)i, g, j0 + cw, nxt);
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    uint32_t bits = 0;
    if (j0 < R.d) {
      if constexpr (VAR) bits = trial_compute(R, s, j0, cur, t, v.F, v.thr, v.L);
      else bits = trial_compute(R, s, j0, cur, t);
      if (valid) {
        double* Trow = R.T + (size_t)i * R.dp + j0;
        *reinterpret_cast<double2*>(Trow) = make_double2(t[0], t[1]);
        *reinterpret_cast<double2*>(Trow + 2) = make_double2(t[2], t[3]);
      }
    }
    if (j0 < R.kpad) {
      float y[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        y[q] = (j0 + q < R.d) ? to_f32_rn(shifted_as<UNIT>(t[q], R.o[j0 + q], R.scale)) : 0.f;
        yn2 += y[q] * y[q];
      }
      if (valid) store_split4<ESZ>(Ahi, a_part, m, j0, y);
    }
    if (dbg) trial_debug(R, (uint32_t)i, j0, lane, bits, t, lpt, valid);
    cur = nxt;
  }
  };
  if (R.unit_scale) chunks(std::true_type{});
  else chunks(std::false_type{});
  for (int o = lpt >> 1; o > 0; o >>= 1) yn2 += __shfl_xor_sync(0xffffffffu, yn2, o);
  if (valid && sub == 0) R.ynorm[i] = sqrtf(yn2);
}

// Rows of caller memory -> A operand tiles and |y| (evaluation mode).
template <int ESZ>
__global__ void __launch_bounds__(256) k_prep_rows(const RunDesc* __restrict__ runs, int run,
                                                   const double* __restrict__ x, int64_t ld, int n) {
  const RunDesc& R = runs[run];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  if (i >= n) return;
  uint8_t* Ahi = R.A + (size_t)(i >> 7) * R.a_tile_bytes;
  const uint32_t a_part = (uint32_t)(R.a_tile_bytes / 2);
  float yn2 = 0.f;
  for (int j0 = 4 * lane; j0 < R.kpad; j0 += 128) {
    float y[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + q;
      y[q] = (j < R.d) ? to_f32_rn(shifted(x[(size_t)i * ld + j], R.o[j], R)) : 0.f;
      yn2 += y[q] * y[q];
    }
    store_split4<ESZ>(Ahi, a_part, i & 127, j0, y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) yn2 += __shfl_xor_sync(0xffffffffu, yn2, o);
  if (lane == 0) R.ynorm[i] = sqrtf(yn2);
}

// ------------------------------------------------------------------ fitness + selection kernel
// mode 0: one generation (items = (run, 128-row tile)); mode 1: evaluation of
// n_eval rows already converted by k_prep_rows, f written to fout; mode 2:
// the same for the run's own population (n_eval = np), written as the
// population's split fitness values with their error bounds (f, fx = 0, tau).
template <int ESZ>
__global__ void __launch_bounds__(kFitThreads, 1)
    k_fit_tc(const RunDesc* __restrict__ runs, const int2* __restrict__ items, int mode, double* __restrict__ fout,
             int n_eval) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[2 * kMaxStages + 1];  // full[S], done[S], acc
  __shared__ uint32_t s_tmem;
  __shared__ int s_stop, s_err, s_nlist, s_nacc, s_last;
  __shared__ long long s_gen;
  __shared__ double s_bestprev;
  __shared__ float s_part[5][kTileM];
  __shared__ double s_fnew[kTileM];
  __shared__ double s_ftrial[kTileM];
  __shared__ float s_taunew[kTileM];
  __shared__ uint8_t s_flag[kTileM];  // bit 0 accept, bit 1 decided in FP64
  __shared__ int s_list[kTileM];
  __shared__ int s_acc[kTileM];
  __shared__ double s_bf[8];
  __shared__ long long s_bk[8];
  __shared__ int s_bi[8];

  const int2 it = items[blockIdx.x];
  const RunDesc& R = runs[it.x];  // run descriptors are written once, at set-up
  // several N tiles: with gridDim.y > 1, CTA (tile, y) computes N tile y only
  // and the tile's last CTA combines the per-row partial sums in N-tile order
  if ((int)blockIdx.y >= R.nn) return;  // the grid covers the largest N-tile count of the batch
  const bool split = gridDim.y > 1 && R.nn > 1;
  const int nt_lo = split ? (int)blockIdx.y : 0, nt_hi = split ? nt_lo + 1 : R.nn;
  RunState* st = R.st;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  pdl_launch_dependents();

  // ---- set-up that does not depend on the previous kernel: barriers, tensor
  // memory, and the constant B operand of the first pipeline stages
  // S-stage K pipeline: stage s is filled when full[s] completes and free
  // again when done[s] (the commit of its products) completes
  const int S = R.nstage;
  auto full_bar = [&](int sg) { return smem_u32(&bars[sg]); };
  auto done_bar = [&](int sg) { return smem_u32(&bars[kMaxStages + sg]); };
  const uint32_t b_acc = smem_u32(&bars[2 * kMaxStages]);
  if (tid == 0) {
    for (int k = 0; k < 2 * kMaxStages + 1; ++k) mbar_init(smem_u32(&bars[k]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_err = 0;
    s_nlist = 0;
    s_nacc = 0;
  }
  const uint32_t ncols = R.ntn <= 32 ? 32u : (R.ntn <= 64 ? 64u : (R.ntn <= 128 ? 128u : 256u));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  // ---- geometry of the K pipeline
  const int kc = R.kc;
  const int nkc = (R.kpad + kc - 1) / kc;
  const int nseq = (nt_hi - nt_lo) * nkc;
  const uint32_t a_part = (uint32_t)(R.a_tile_bytes / 2);
  const uint32_t b_part = (uint32_t)(R.b_tile_bytes / 2);
  const uint32_t kg_chunk = (uint32_t)(kc * ESZ / 16);  // k-groups per full chunk
  const uint32_t a_chunk = kg_chunk * 16u * 128u;
  const uint32_t bk = (uint32_t)(R.ntn / 8) * 128u;     // B k-group stride
  const uint32_t b_chunk = kg_chunk * bk;
  const uint32_t stage_bytes = 2 * a_chunk + 2 * b_chunk;
  const uint8_t* Atile = R.A + (size_t)it.y * R.a_tile_bytes;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t fmt = ESZ == 2 ? 1u : 2u;
  const uint32_t idesc =
      (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(R.ntn >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);

  auto chunk_len = [&](int kci) { return min(kc, R.kpad - kci * kc); };
  // B half of stage load q (counts the bytes of both halves on the barrier)
  auto issue_load_b = [&](int q) {
    const int nt = nt_lo + q / nkc, kci = q % nkc, sg = q % S;
    const uint32_t kgs = (uint32_t)(chunk_len(kci) * ESZ / 16);
    const uint32_t ab = kgs * 16u * 128u, bb = kgs * bk;
    const uint32_t base = sbase + (uint32_t)sg * stage_bytes;
    const uint32_t bar = full_bar(sg);
    mbar_expect_tx(bar, 2 * ab + 2 * bb);
    const size_t b_off = (size_t)kci * b_chunk;
    const uint8_t* Bt = R.B + (size_t)nt * R.b_tile_bytes;
    bulk_g2s(base + 2 * a_chunk, Bt + b_off, bb, bar);
    bulk_g2s(base + 2 * a_chunk + b_chunk, Bt + b_part + b_off, bb, bar);
  };
  auto issue_load_a = [&](int q) {
    const int kci = q % nkc, sg = q % S;
    const uint32_t kgs = (uint32_t)(chunk_len(kci) * ESZ / 16);
    const uint32_t ab = kgs * 16u * 128u;
    const uint32_t base = sbase + (uint32_t)sg * stage_bytes;
    const uint32_t bar = full_bar(sg);
    const size_t a_off = (size_t)kci * a_chunk;
    bulk_g2s(base, Atile + a_off, ab, bar);
    bulk_g2s(base + a_chunk, Atile + a_part + a_off, ab, bar);
  };
  const int npro = min(nseq, S);
  if (tid == 0)
    for (int q = 0; q < npro; ++q) issue_load_b(q);

  // ---- from here on the previous kernel's results are needed
  pdl_wait();
  if (tid == 0) {
    s_stop = mode == 0 ? *(volatile int32_t*)&st->stop : 0;
    s_gen = *(volatile int64_t*)&st->gen;
    s_bestprev = *(volatile double*)&st->best_f;
    for (int q = 0; q < npro; ++q) issue_load_a(q);
  }
  __syncthreads();
  if (s_stop) {
    // the run has stopped: let the prologue copies land, free TMEM, leave
    if (tid == 0)
      for (int q = 0; q < npro; ++q) mbar_wait(full_bar(q), 0u);
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    return;
  }
  const int row0 = it.y * kTileM;
  const int nrows = min(kTileM, (mode == 0 ? R.np : n_eval) - row0);

  // per-thread epilogue state: row m (TMEM lane), column half h
  const int m = 32 * (warp & 3) + lane;
  const int h = warp >> 2;
  const int half = R.ntn / 2;
  const int cb = h * half;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  EpiAcc acc_{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int obj = R.obj, d = R.d;
  // the selection inputs of this row, fetched while the tensor cores work
  double pf_fi = 0.0;
  float pf_tau = 0.f, pf_yn = 0.f;
  uint8_t pf_fx = 1;
  if (h == 0 && m < nrows) {
    const int i = row0 + m;
    pf_yn = R.ynorm[i];
    if (mode == 0) {
      pf_fi = R.f[0][i];
      pf_fx = R.fx[0][i];
      pf_tau = R.tau[i];
    }
  }

  int loads_issued = npro, mmas_committed = 0;
  int q = 0;
  for (int nt = nt_lo; nt < nt_hi; ++nt) {
    if (tid == 0 && !s_err) {
      bool ok = true;
      for (int kci = 0; kci < nkc; ++kci, ++q) {
        const int sg = q % S;
        ok = mbar_wait(full_bar(sg), (uint32_t)((q / S) & 1));
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = sbase + (uint32_t)sg * stage_bytes;
        const int ksteps = chunk_len(kci) * ESZ / 32;
        for (int ks = 0; ks < ksteps; ++ks) {
#pragma unroll
          for (int pass = 0; pass < 3; ++pass) {
            const uint32_t a = base + (pass == 2 ? a_chunk : 0u) + (uint32_t)ks * 2u * 2048u;
            const uint32_t b = base + 2 * a_chunk + (pass == 1 ? b_chunk : 0u) + (uint32_t)ks * 2u * bk;
            const uint32_t accum = (kci > 0 || ks > 0 || pass > 0) ? 1u : 0u;
            mma_split<ESZ>(tmem, smem_desc(a, 2048u, 128u), smem_desc(b, bk, 128u), idesc, accum);
          }
        }
        mma_commit(done_bar(sg));
        ++mmas_committed;
        // refill the stage of chunk q - 1 (its products done) with chunk q - 1 + S
        if (q >= 1 && q - 1 + S < nseq) {
          const int pq = q - 1;
          ok = mbar_wait(done_bar(pq % S), (uint32_t)((pq / S) & 1));
          if (!ok) break;
          issue_load_b(pq + S);
          issue_load_a(pq + S);
          ++loads_issued;
        }
      }
      mma_commit(b_acc);
      if (!ok) s_err = 1;
    }
    __syncthreads();
    bool have = false;
    if (!s_err) {
      have = mbar_wait(b_acc, (uint32_t)((nt - nt_lo) & 1));
      if (!have) atomicOr(&s_err, 1);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (have) {
      // ---- epilogue of N tile nt: objective terms from TMEM (FP32), 32 or 16
      // columns per load
      const int nbase = nt * R.ntn + cb;
      for (int c = 0; c < half; c += 32) {
        float v[32];
        const int w = min(32, half - c);  // a multiple of 8
        const uint32_t ta = tmem + lane_base + (uint32_t)(cb + c);
        // constant offsets only, so that v stays in registers
        if (w == 32) {
          tmem_ld_cols32(ta, v);
        } else if (w == 24) {
          tmem_ld_cols16(ta, v);
          tmem_ld8(ta + 16u, v + 16);
        } else if (w == 16) {
          tmem_ld_cols16(ta, v);
        } else {
          tmem_ld8(ta, v);
        }
        epi_dispatch(obj, v, w, nbase + c, d, c == 0, acc_);
      }
      if (obj == kObjRosenbrock && h == 0 && half < R.ntn && half < d) {
        // the term of the last column of this half needs the next column
        const float t = tmem_ld1(tmem + lane_base + (uint32_t)half) + 1.f;
        const float aa = t - acc_.prev_t * acc_.prev_t, bb = acc_.prev_t - 1.f;
        acc_.a1 += fmaf(100.f * aa, aa, bb * bb);
        acc_.aG += 400.f * fabsf(acc_.prev_t) * fabsf(aa) + 2.f * fabsf(bb) + 200.f * fabsf(aa);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }

  // ---- error path: wait (bounded) for outstanding copies and MMAs; in
  // evaluation mode the tile's outputs become NaN, so that a caller who
  // cannot read the run state still sees that these rows were not evaluated
  if (s_err) {
    if (tid == 0) {
      atomicOr(&st->err, kErrTimeout);
      for (int k = 0; k < loads_issued; ++k) mbar_wait(full_bar(k % S), (uint32_t)((k / S) & 1));
      for (int k = 0; k < mmas_committed; ++k) mbar_wait(done_bar(k % S), (uint32_t)((k / S) & 1));
    }
    if (mode == 1 && tid < nrows) fout[row0 + tid] = __longlong_as_double(0x7FF8000000000000LL);
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    return;
  }
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));

  // ---- combine the two column halves of each row (fixed order)
  if (h == 1) {
    s_part[0][m] = acc_.a1;
    s_part[1][m] = acc_.a2;
    s_part[2][m] = acc_.a3;
    s_part[3][m] = acc_.aS;
    s_part[4][m] = acc_.aG;
  }
  __syncthreads();
  float t1 = 0.f, t2 = 0.f, t3 = 0.f, tS = 0.f, tG = 0.f;
  if (h == 0) {
    t1 = acc_.a1 + s_part[0][m];
    t2 = acc_.a2 + s_part[1][m];
    t3 = acc_.a3 + s_part[2][m];
    tS = acc_.aS + s_part[3][m];
    tG = acc_.aG + s_part[4][m];
  }
  if (split) {
    // partial sums of this N tile -> global; the tile's last CTA adds them up
    // in N-tile order (the same order whichever CTA finishes last)
    const size_t pstride = (size_t)5 * kTileM;
    float* P = R.npart + ((size_t)it.y * R.nn + nt_lo) * pstride;
    if (h == 0) {
      P[0 * kTileM + m] = t1;
      P[1 * kTileM + m] = t2;
      P[2 * kTileM + m] = t3;
      P[3 * kTileM + m] = tS;
      P[4 * kTileM + m] = tG;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const uint32_t tk = atomicAdd(&R.nticket[it.y], 1u);
      s_last = (tk == (uint32_t)R.nn - 1u);
      if (s_last) R.nticket[it.y] = 0u;  // every CTA of this tile has counted itself
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (h == 0) {
      const float* Q = R.npart + (size_t)it.y * R.nn * pstride;
      t1 = t2 = t3 = tS = tG = 0.f;
      for (int k = 0; k < R.nn; ++k, Q += pstride) {
        t1 += __ldcg(Q + 0 * kTileM + m);
        t2 += __ldcg(Q + 1 * kTileM + m);
        t3 += __ldcg(Q + 2 * kTileM + m);
        tS += __ldcg(Q + 3 * kTileM + m);
        tG += __ldcg(Q + 4 * kTileM + m);
      }
    }
  }
  if (h == 0 && m < nrows) {
    const float s1 = t1, s2 = t2, s3 = t3;
    float S = tS, G = tG;
    float fs;
    if (obj == kObjAckley) {
      const float r = sqrtf(s1 / (float)d);
      const float e1 = expf(-0.2f * r), e2 = expf(s2 / (float)d);
      fs = 20.f + 2.718281828f - 20.f * e1 - e2;
      S = 20.f + 2.718281828f + 20.f * e1 + expf(S / (float)d);
      G = (r > 0.f ? 4.f * e1 * s3 / ((float)d * r) : 3.0e38f) + 6.283185307f * e2;
    } else {
      if (obj != kObjRastrigin) S = s1;
      fs = s1;
    }
    const int i = row0 + m;
    // error bound of fs: split products (relative to |M||y|) through the
    // derivative bound G, plus FP32 rounding of the terms and their sum
    const float tau = 2.f * R.band_u * G * R.rownorm * pf_yn + (float)d * 0x1.0p-21f * S + 1e-30f;
    if (mode == 1) {
      fout[i] = (double)fs;
    } else if (mode == 2) {
      R.f[0][i] = (double)fs;
      R.fx[0][i] = 0;
      R.tau[i] = tau;
    } else {
      // decided in FP32; the margins cover the rounding of the FP64 values
      const float fif = (float)pf_fi;
      const float tif = pf_fx ? 0.f : pf_tau;
      const float mrg = 0x1.0p-22f * fabsf(fif);
      const float bp = (float)s_bestprev;
      const bool sure_reject = fs - tau > fif + tif + mrg;
      const bool sure_accept = fs + tau < fif - tif - mrg;
      const bool ambiguous = !sure_reject && !sure_accept;
      const bool may_be_best = R.band_all && fs - tau <= bp + 0x1.0p-22f * fabsf(bp);
      const bool near = fs - tau <= R.near_thr || fif - tif <= R.near_thr;
      // only a trial the split bound cannot place on one side of the stop target
          // needs FP64 for the stop rule: surely below (or above) decides it as well
          const bool may_stop = R.target > 0.0 && fs - tau < (float)R.target * 1.001f &&
                                !(fs + tau < (float)R.target * 0.999f);
      s_ftrial[m] = (double)fs;
      if ((ambiguous && (R.band_all || near)) || may_be_best || may_stop || !(fs == fs) || !(fif == fif)) {
        // the split values cannot decide (or the trial may become the best):
        // FP64 decision in k_band_fp64
        const uint32_t e = atomicAdd(R.band_cnt, 1u);
        R.band[e] = BandEntry{it.x, i, pf_fx ? 0 : 1, 0};
        atomicAdd(&st->band_n, 1);
        atomicAdd(&st->band_left, 1);
        s_flag[m] = 4;
        atomicAdd(&s_nlist, 1);
      } else {
        // decided on the split values (an undecidable comparison far from the
        // optimum goes to the smaller split value, ties to the trial)
        const bool acc = sure_accept || (ambiguous && fs <= fif);
        s_flag[m] = acc ? 1 : 0;
        s_fnew[m] = acc ? (double)fs : pf_fi;
        s_taunew[m] = acc ? tau : tif;
      }
    }
  }
  __syncthreads();
  if (mode != 0) return;

  // ---- write back fitness, flags, debug; list the accepted rows
  Best bb;
  bb.init();
  if (tid < nrows) {
    const int mm = tid, i = row0 + mm;
    const uint8_t fl = s_flag[mm];
    if (!(fl & 4)) {  // rows sent to the FP64 band are finished by k_band_fp64
      const bool acc = fl & 1;
      R.f[0][i] = s_fnew[mm];
      if (acc) {
        R.fx[0][i] = 0;
        R.tau[i] = s_taunew[mm];
        s_acc[atomicAdd(&s_nacc, 1)] = mm;
        if (R.jde) {
          // jDE: the accepted trial's F_i and CR_i replace the target's (in place)
          double Fi, CRi;
          jde_params(R, (uint32_t)i, s_gen + 1, R.jF[0], R.jCR[0], Fi, CRi);
          R.jF[0][i] = Fi;
          R.jCR[0][i] = CRi;
        }
      }
      if (R.dbg_ftrial) {
        R.dbg_ftrial[i] = s_ftrial[mm];
        R.dbg_accept[i] = acc ? 1 : 0;
        R.dbg_fp64[i] = 0;
      }
      bb.offer(s_fnew[mm], i);
    }
  }
  if (tid == 0) {
    atomicAdd(&R.stats[0], (unsigned long long)s_nlist);
    atomicAdd(&R.stats[1], (unsigned long long)nrows);
  }
  __syncthreads();
  // accepted trials replace their targets in place
  {
    const int na = s_nacc;
    const int dp2 = R.dp / 2;
    for (int e = warp; e < na; e += kFitThreads / 32) {
      const int i = row0 + s_acc[e];
      const double2* src = reinterpret_cast<const double2*>(R.T + (size_t)i * R.dp);
      double2* dst = reinterpret_cast<double2*>(R.X[0] + (size_t)i * R.dp);
      for (int j = lane; j < dp2; j += 32) dst[j] = src[j];
    }
  }
  // ---- best partial of the tile, then the last CTA of the run finishes the generation
  bb.warp_reduce();
  if (lane == 0) {
    s_bf[warp] = bb.f;
    s_bk[warp] = bb.k;
    s_bi[warp] = bb.i;
  }
  __syncthreads();
  if (tid == 0) {
    bb.init();
    for (int w = 0; w < kFitThreads / 32; ++w) bb.take(s_bf[w], s_bk[w], s_bi[w]);
    // the band kernel that follows reduces the partials of every tile
    R.part[it.y].f = bb.f;
    R.part[it.y].idx = bb.i;
  }
}

// ------------------------------------------------------------------ FP64 band kernel
// Work item (entry e, vector v, chunk c): v = 0 is the trial T[i], v = 1 the
// target X[i]; chunk c covers output coordinates [cw c, cw c + cw) plus the
// next one (for Rosenbrock).  The CTA stages the chunk's rows of M and the
// vector y = (x - o) s in shared memory with one round of coalesced loads,
// forms z_j = sum_k M[j][k] y_k (a warp per output, lanes over k) and the FP64
// objective terms of the chunk; partial sums go to band_part.  The CTA
// completing the last chunk of an entry decides the selection in FP64, the one
// completing the last entry of a run finishes that run's generation.
__global__ void __launch_bounds__(256) k_band_fp64(const RunDesc* __restrict__ runs, int nruns,
                                                   const BandEntry* __restrict__ band,
                                                   const uint32_t* __restrict__ band_cnt, int nch_max) {
  extern __shared__ __align__(16) double s_dyn[];
  __shared__ double s_z[33];
  __shared__ int s_last, s_acc, s_fin, s_stop, s_bn;
  __shared__ long long s_gen;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  pdl_launch_dependents();
  pdl_wait();
  const uint32_t n = *(volatile const uint32_t*)band_cnt;
  // runs that sent no row to the band finish their generation here
  for (int r = blockIdx.x; r < nruns; r += gridDim.x) {
    const RunDesc& R = runs[r];
    if (tid == 0) {
      s_stop = *(volatile int32_t*)&R.st->stop;
      s_bn = *(volatile int32_t*)&R.st->band_n;
      s_gen = *(volatile int64_t*)&R.st->gen;
    }
    __syncthreads();
    if (!s_stop && s_bn == 0) finish_generation(R, s_gen + 1, R.ntiles_tc, R.part, R.X[0]);
    __syncthreads();
  }
  const long long total = (long long)n * 2 * nch_max;
  for (long long idx = blockIdx.x; idx < total; idx += gridDim.x) {
    const int e = (int)(idx / (2 * nch_max));
    const int v = (int)((idx / nch_max) % 2);
    const int c = (int)(idx % nch_max);
    const BandEntry be = band[e];
    const RunDesc& R = runs[be.run];
    if (c >= R.nch || (v == 1 && !be.need_target)) continue;
    const int d = R.d, i = be.row, cw = R.band_cw;
    const int j0 = c * cw;
    const int nout = min(cw + 1, d - j0);  // outputs of this chunk, with the next coordinate
    double* s_y = s_dyn;
    double* s_m = s_dyn + R.dp;
    const double* x = (v == 0 ? R.T : R.X[0]) + (size_t)i * R.dp;
    for (int k = tid; k < d; k += blockDim.x) s_y[k] = shifted(x[k], R.o[k], R);
    if (R.rotate)
      for (int q = tid; q < nout * d; q += blockDim.x) s_m[q] = __ldg(R.Mrow + (size_t)j0 * d + q);
    __syncthreads();
    for (int jl = warp; jl < nout; jl += 8) {
      double acc = 0.0;
      if (R.rotate) {
        // two independent chains per lane, then the fixed xor tree
        const double* mr = s_m + (size_t)jl * d;
        double acc1 = 0.0;
        for (int k = lane; k < d; k += 64) {
          acc = fma(mr[k], s_y[k], acc);
          if (k + 32 < d) acc1 = fma(mr[k + 32], s_y[k + 32], acc1);
        }
        acc = warp_sum(acc + acc1);
      } else {
        acc = s_y[j0 + jl];
      }
      if (lane == 0) s_z[jl] = acc;
    }
    __syncthreads();
    if (warp == 0) {
      const int j = j0 + lane;
      double t1 = 0.0, t2 = 0.0;
      if (lane < cw && j < d) {
        const double z = s_z[lane];
        if (R.obj == kObjSphere) {
          t1 = z * z;
        } else if (R.obj == kObjRastrigin) {
          t1 = z * z - 10.0 * cos2pi_f64(z) + 10.0;
        } else if (R.obj == kObjAckley) {
          t1 = z * z;
          t2 = cos2pi_f64(z);
        } else if (R.obj == kObjRosenbrock && j + 1 < d) {
          const double t0 = z + 1.0, tn = s_z[lane + 1] + 1.0;
          const double a = tn - t0 * t0, b = t0 - 1.0;
          t1 = 100.0 * a * a + b * b;
        }
      }
      t1 = warp_sum(t1);
      t2 = warp_sum(t2);
      if (lane == 0) {
        R.band_part[((size_t)e * 2 + v) * nch_max + c] = make_double2(t1, t2);
        __threadfence();
        const uint32_t need = (uint32_t)((1 + be.need_target) * R.nch);
        s_last = (atomicAdd(&R.band_tk[e], 1u) == need - 1u);
      }
    }
    __syncthreads();
    if (s_last) {
      if (warp == 0) {
        __threadfence();
        // sum the chunk partials of each vector in chunk order (lanes, then a fixed tree)
        double f2[2] = {0.0, 0.0};
#pragma unroll
        for (int vv = 0; vv < 2; ++vv) {
          if (vv == 1 && !be.need_target) break;
          double s1 = 0.0, s2 = 0.0;
          for (int cc = lane; cc < R.nch; cc += 32) {
            const double2 p = __ldcg(&R.band_part[((size_t)e * 2 + vv) * nch_max + cc]);
            s1 += p.x;
            s2 += p.y;
          }
          s1 = warp_sum(s1);
          s2 = warp_sum(s2);
          f2[vv] = R.obj == kObjAckley ? 20.0 + 2.718281828459045 - 20.0 * exp(-0.2 * sqrt(s1 / d)) - exp(s2 / d) : s1;
        }
        if (lane == 0) {
          const double ft = f2[0];
          const double fi = be.need_target ? f2[1] : R.f[0][i];
          const bool acc = fit_key(ft) <= fit_key(fi) && fit_key(ft) != 0x7FFFFFFFFFFFFFFFLL;  // NaN ranks last
          R.f[0][i] = acc ? ft : fi;
          R.fx[0][i] = 1;
          R.tau[i] = 0.f;
          if (acc && R.jde) {
            // jDE: the accepted trial's F_i and CR_i replace the target's (in place)
            double Fi, CRi;
            jde_params(R, (uint32_t)i, *(volatile int64_t*)&R.st->gen + 1, R.jF[0], R.jCR[0], Fi, CRi);
            R.jF[0][i] = Fi;
            R.jCR[0][i] = CRi;
          }
          if (R.dbg_ftrial) {
            R.dbg_ftrial[i] = ft;
            R.dbg_accept[i] = acc ? 1 : 0;
            R.dbg_fp64[i] = 1;
          }
          R.band_tk[e] = 0;
          s_acc = acc;
        }
      }
      __syncthreads();
      if (s_acc) {
        const double2* src = reinterpret_cast<const double2*>(R.T + (size_t)i * R.dp);
        double2* dst = reinterpret_cast<double2*>(R.X[0] + (size_t)i * R.dp);
        for (int j = tid; j < R.dp / 2; j += blockDim.x) dst[j] = src[j];
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        s_fin = (atomicSub(&R.st->band_left, 1) == 1);
      }
      __syncthreads();
      if (s_fin) {
        __threadfence();
        const int64_t g = *(volatile int64_t*)&R.st->gen + 1;
        finish_generation(R, g, R.ntiles_tc, R.part, R.X[0], band, (int)n, be.run, R.f[0]);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ host side
static size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static uint16_t host_bf16_rn(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  return (uint16_t)(u >> 16);
}
static float host_bf16_to_f(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}
static float host_tf32_rna(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) != 0x7F800000u) {
    u += 0x1000u;  // round half away from zero on the 13 dropped bits
    u &= 0xFFFFE000u;
  }
  float f;
  memcpy(&f, &u, 4);
  return f;
}

// K chunk of the fitness kernel's pipeline: the whole K in one stage when it
// fits, else two stages of at most kStageBudget; divided by kc_div (an
// autotuner choice that leaves the product order, hence the results, alone).
static int plan_kc(const RunDesc& R, int esz, int kc_div) {
  int kc;
  if (kc_div == 1 && (size_t)2 * (kTileM + R.ntn) * R.kpad * esz <= kSingleStageMax) {
    kc = R.kpad;
  } else {
    kc = (int)(kStageBudget / (2 * (kTileM + R.ntn) * esz)) / 16 * 16;
    kc = std::max(16, std::min(kc, R.kpad));
    kc = std::max(16, kc / kc_div / 16 * 16);
  }
  return kc;
}

// Work items of the trial kernel for one run: CTAs of `warps` warps, each
// warp 32 / lpt targets.
static int trial_groups(const RunDesc& R, int warps) {
  const int per = warps * (32 / R.lpt);
  return (R.np + per - 1) / per;
}

// Stages of the K pipeline: one when the whole K of one N tile is one chunk,
// else `stages` (at least 2) as far as kFitSmemMax allows.
static int plan_stages(const RunDesc& R, int esz, int stages) {
  if (R.kc >= R.kpad && R.nn == 1) return 1;
  const size_t stage = 2 * (size_t)(R.kc * esz / 16) * 16 * 128 + 2 * (size_t)(R.kc * esz / 16) * (R.ntn / 8) * 128;
  int S = std::max(2, std::min(stages, kMaxStages));
  while (S > 2 && (size_t)S * stage > kFitSmemMax) --S;
  return S;
}

static size_t plan_smem(const RunDesc& R, int esz) {
  const size_t stage = 2 * (size_t)(R.kc * esz / 16) * 16 * 128 + 2 * (size_t)(R.kc * esz / 16) * (R.ntn / 8) * 128;
  return (size_t)R.nstage * stage;
}

// B operand: N tiles of M's rows (n = output coordinate), each tile two
// parts (high, low) in the canonical K-major layout with ntn / 8 row groups.
static void pack_b(const de_config& c, const RunDesc& R, std::vector<uint8_t>& out) {
  const int d = c.d, esz = R.esz, ntn = R.ntn, kpad = R.kpad;
  const size_t part = (size_t)ntn * kpad * esz;
  out.assign((size_t)R.nn * 2 * part, 0);
  const int RG = ntn / 8, per = 16 / esz;
  for (int n = 0; n < d; ++n)
    for (int k = 0; k < d; ++k) {
      const double mv = c.rot ? c.rot[(size_t)n * d + k] : (n == k ? 1.0 : 0.0);
      const float mf = (float)mv;
      const int nt = n / ntn, nl = n % ntn;
      const size_t off = (size_t)nt * 2 * part + (((size_t)(k / per) * RG + nl / 8) * 128) + (nl % 8) * 16 +
                         (k % per) * esz;
      if (esz == 2) {
        const uint16_t hi = host_bf16_rn(mf);
        const uint16_t lo = host_bf16_rn(mf - host_bf16_to_f(hi));
        memcpy(&out[off], &hi, 2);
        memcpy(&out[off + part], &lo, 2);
      } else {
        const float hi = host_tf32_rna(mf);
        const float lo = host_tf32_rna(mf - hi);
        memcpy(&out[off], &hi, 4);
        memcpy(&out[off + part], &lo, 4);
      }
    }
}

de_status tc_plan_build(TcPlan& p, std::vector<RunDesc>& runs, const de_config* cfgs, int prec, cudaStream_t s,
                        std::string& err) {
  p.prec = prec;
  p.var = false;
  for (const auto& R : runs) p.var = p.var || R.strategy != 0 || R.jde;
  const int esz = prec == DE_PREC_BF16X3 ? 2 : 4;
  size_t bytes = 0;
  std::vector<size_t> offA(runs.size()), offB(runs.size()), offY(runs.size()), offT(runs.size()), offS(runs.size());
  std::vector<size_t> offP(runs.size(), 0), offK(runs.size(), 0);
  p.nsplit = 1;
  std::vector<int2> trial_items, fit_items;
  size_t smem = 0;
  p.fit_offset.assign(runs.size(), 0);
  for (size_t r = 0; r < runs.size(); ++r) {
    RunDesc& R = runs[r];
    R.esz = esz;
    R.kpad = (int)round_up(R.d, 16);
    // lanes per target of the trial kernel: the fewest lanes (a power of two)
    // whose 4 coordinates each cover the padded row, at most a warp
    R.lpt = 1;
    while (R.lpt < 32 && 4 * R.lpt < R.kpad) R.lpt *= 2;
    R.ntn = R.d <= 256 ? (int)round_up(R.d, 16) : 256;
    R.nn = (R.d + R.ntn - 1) / R.ntn;
    R.npad = R.nn * R.ntn;
    if (R.obj == kObjRosenbrock && R.nn > 1) {
      err = "split precision supports Rosenbrock only for d <= 256";
      return DE_ERR_UNSUPPORTED;
    }
    R.kc = plan_kc(R, esz, 1);
    R.nstage = plan_stages(R, esz, 2);
    R.ntiles_tc = (R.np + kTileM - 1) / kTileM;
    R.a_tile_bytes = 2 * kTileM * R.kpad * esz;
    R.b_tile_bytes = 2 * R.ntn * R.kpad * esz;
    // one split product yh mh + yh ml + yl mh misses y m by at most 3 u^2 |y m|
    // (u = 2^-8 for bf16, 2^-11 for tf32: the dropped yl ml and the two
    // residuals); FP32 accumulation of kpad products adds kpad 2^-24
    R.band_u = (float)((esz == 2 ? 3.0 * std::ldexp(1.0, -16) : 3.0 * std::ldexp(1.0, -22)) +
                       R.kpad * std::ldexp(1.0, -24));
    R.band_cw = std::max(1, std::min(8, (int)(kBandSmem / (8 * (size_t)R.d)) - 1));
    R.nch = (R.d + R.band_cw - 1) / R.band_cw;
    // near the optimum: where the split bound (about 4 u f) reaches an eighth
    // of the stopping accuracy, comparisons are redone in FP64.  The accuracy
    // is the target, capped at the paper's 1e-8 (Sec. 7.3.4): a larger target
    // (a run stopped at some other error) must not make every value "near";
    // its stop decision is exact on its own (only trials the split bound
    // cannot place on one side of the target are redone in FP64)
    R.near_thr = R.target > 0.0 ? (float)(std::min(R.target, 1e-8) / (8.0 * R.band_u)) : 0.f;
    smem = std::max(smem, plan_smem(R, esz));
    bytes = round_up(bytes, 1024);
    offA[r] = bytes;
    bytes += (size_t)R.ntiles_tc * R.a_tile_bytes;
    bytes = round_up(bytes, 1024);
    offB[r] = bytes;
    bytes += (size_t)R.nn * R.b_tile_bytes;
    bytes = round_up(bytes, 256);
    offY[r] = bytes;
    bytes += (size_t)R.ntiles_tc * kTileM * sizeof(float);
    bytes = round_up(bytes, 256);
    offT[r] = bytes;
    bytes += (size_t)R.np * sizeof(float);
    bytes = round_up(bytes, 256);
    offS[r] = bytes;
    bytes += 2 * sizeof(unsigned long long);
    if (R.nn > 1) {
      // per-row partial sums of each N tile and the per-tile tickets
      bytes = round_up(bytes, 256);
      offP[r] = bytes;
      bytes += (size_t)R.ntiles_tc * R.nn * 5 * kTileM * sizeof(float);
      bytes = round_up(bytes, 256);
      offK[r] = bytes;
      bytes += (size_t)R.ntiles_tc * sizeof(uint32_t);
      p.nsplit = std::max(p.nsplit, R.nn);
    }

    p.fit_offset[r] = (int)fit_items.size();
    for (int t = 0; t < R.ntiles_tc; ++t) fit_items.push_back(make_int2((int)r, t));
  }
  p.smem_fit = smem;
  p.nruns = (int)runs.size();
  // trial kernel: about one CTA per SM, at most 8 targets (warps) per CTA
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  {
    long long tot = 0;
    for (auto& R : runs) tot += R.np;
    p.trial_rows = (int)std::max(1LL, std::min(8LL, (tot + nsm - 1) / nsm));
    for (size_t r = 0; r < runs.size(); ++r)
      for (int gI = 0; gI < trial_groups(runs[r], p.trial_rows); ++gI)
        trial_items.push_back(make_int2((int)r, gI));
  }
  // FP64 band list shared by all runs of the handle
  size_t cap = 0;
  int nch_max = 1, dmax = 1;
  for (auto& R : runs) {
    cap += (size_t)R.np;
    nch_max = std::max(nch_max, R.nch);
    dmax = std::max(dmax, R.d);
  }
  bytes = round_up(bytes, 256);
  const size_t off_band = bytes;
  bytes += cap * sizeof(BandEntry);
  bytes = round_up(bytes, 256);
  const size_t off_bcnt = bytes;
  bytes += 256;
  const size_t off_bpart = bytes;
  bytes += cap * 2 * (size_t)nch_max * sizeof(double2);
  bytes = round_up(bytes, 256);
  const size_t off_btk = bytes;
  bytes += cap * sizeof(uint32_t);
  bytes = round_up(bytes, 256);
  const size_t off_ctl = bytes;
  bytes += round_up(sizeof(PersistCtl), 256);
  p.nch_max = nch_max;
  p.smem_band = 0;
  for (auto& R : runs)
    p.smem_band = std::max(p.smem_band, (size_t)(R.dp + (R.band_cw + 1) * R.d) * sizeof(double));
  p.grid_band = 2 * nsm;
  cudaError_t e = cudaMalloc(&p.arena, bytes);
  if (e != cudaSuccess) {
    err = std::string("cudaMalloc(split operands): ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DE_ERR_OOM : DE_ERR_CUDA;
  }
  e = cudaMemsetAsync(p.arena, 0, bytes, s);
  std::vector<uint8_t> bbuf;
  for (size_t r = 0; r < runs.size() && e == cudaSuccess; ++r) {
    RunDesc& R = runs[r];
    uint8_t* base = (uint8_t*)p.arena;
    R.A = base + offA[r];
    R.B = base + offB[r];
    R.ynorm = (float*)(base + offY[r]);
    R.tau = (float*)(base + offT[r]);
    R.stats = (unsigned long long*)(base + offS[r]);
    R.npart = R.nn > 1 ? (float*)(base + offP[r]) : nullptr;
    R.nticket = R.nn > 1 ? (uint32_t*)(base + offK[r]) : nullptr;
    R.band = (BandEntry*)(base + off_band);
    R.band_cnt = (uint32_t*)(base + off_bcnt);
    R.band_part = (double2*)(base + off_bpart);
    R.band_tk = (uint32_t*)(base + off_btk);
    R.nch_max = nch_max;
    pack_b(cfgs[r], R, bbuf);
    e = cudaMemcpyAsync((void*)R.B, bbuf.data(), bbuf.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // bbuf is reused
  }
  if (e == cudaSuccess) e = cudaMalloc(&p.d_trial_items, trial_items.size() * sizeof(int2));
  if (e == cudaSuccess) e = cudaMalloc(&p.d_fit_items, fit_items.size() * sizeof(int2));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p.d_trial_items, trial_items.data(), trial_items.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p.d_fit_items, fit_items.data(), fit_items.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  p.nitems_trial = (int)trial_items.size();
  p.nitems_fit = (int)fit_items.size();
  p.d_band = (BandEntry*)((uint8_t*)p.arena + off_band);
  p.d_ctl = (PersistCtl*)((uint8_t*)p.arena + off_ctl);
  {
    // the persistent cluster kernel runs a single run whose clusters all fit at once
    const char* env = getenv("DE_GB300_PERSIST");
    if (!(env && env[0] == '0') && e == cudaSuccess) persist_plan(p.persist, runs[0], (int)runs.size(), prec);
    // ... and the persistent batch kernel a batch of runs of at most 128
    // coordinates (DE_GB300_PERSIST_BATCH=0 disables it)
    const char* envb = getenv("DE_GB300_PERSIST_BATCH");
    if (!(env && env[0] == '0') && !(envb && envb[0] == '0') && e == cudaSuccess && runs.size() >= 2)
      pbatch_plan(p.pbatch, runs, prec);
    cudaGetLastError();
  }
  p.d_band_cnt = (uint32_t*)((uint8_t*)p.arena + off_bcnt);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_band_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(p.smem_band, 1));
  if (e == cudaSuccess) {
    if (esz == 2) {
      e = cudaFuncSetAttribute(k_fit_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    } else {
      e = cudaFuncSetAttribute(k_fit_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
  }
  if (e != cudaSuccess) {
    err = std::string("split-precision plan: ") + cudaGetErrorString(e);
    return DE_ERR_CUDA;
  }
  return DE_OK;
}

de_status tc_set_geometry(TcPlan& p, std::vector<RunDesc>& runs, int trial_rows, int kc_div, int stages,
                          cudaStream_t s, std::string& err) {
  const int esz = p.prec == DE_PREC_BF16X3 ? 2 : 4;
  size_t smem = 0;
  for (auto& R : runs) {
    R.kc = plan_kc(R, esz, kc_div);
    R.nstage = plan_stages(R, esz, stages);
    smem = std::max(smem, plan_smem(R, esz));
  }
  std::vector<int2> items;
  for (size_t r = 0; r < runs.size(); ++r)
    for (int gI = 0; gI < trial_groups(runs[r], trial_rows); ++gI) items.push_back(make_int2((int)r, gI));
  cudaError_t e = cudaSuccess;
  if (items.size() != (size_t)p.nitems_trial) {
    if (p.d_trial_items) cudaFree(p.d_trial_items);
    p.d_trial_items = nullptr;
    e = cudaMalloc(&p.d_trial_items, items.size() * sizeof(int2));
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p.d_trial_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    e = esz == 2 ? cudaFuncSetAttribute(k_fit_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                 : cudaFuncSetAttribute(k_fit_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  if (e != cudaSuccess) {
    err = std::string("split-precision geometry: ") + cudaGetErrorString(e);
    return DE_ERR_CUDA;
  }
  p.nitems_trial = (int)items.size();
  p.trial_rows = trial_rows;
  p.smem_fit = smem;
  return DE_OK;
}

void tc_plan_free(TcPlan& p) {
  pbatch_free(p.pbatch);
  if (p.arena) cudaFree(p.arena);
  if (p.d_trial_items) cudaFree(p.d_trial_items);
  if (p.d_fit_items) cudaFree(p.d_fit_items);
  p.arena = nullptr;
  p.d_trial_items = nullptr;
  p.d_fit_items = nullptr;
}

// Launch with programmatic stream serialization: the kernel may begin while
// its predecessor on the stream finishes (it waits with griddepcontrol.wait).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, int block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

void tc_generation_launch(const TcPlan& p, const RunDesc* runs, cudaStream_t s) {
  const int tb = 32 * p.trial_rows;
  const dim3 gt(p.nitems_trial);
  const int2* ti = p.d_trial_items;
  if (p.prec == DE_PREC_BF16X3) {
    if (p.var && p.trial_occ) launch_pdl(k_trial_split<2, true, true>, gt, tb, 0, s, runs, ti);
    else if (p.var) launch_pdl(k_trial_split<2, true, false>, gt, tb, 0, s, runs, ti);
    else if (p.trial_occ) launch_pdl(k_trial_split<2, false, true>, gt, tb, 0, s, runs, ti);
    else launch_pdl(k_trial_split<2, false, false>, gt, tb, 0, s, runs, ti);
    launch_pdl(k_fit_tc<2>, dim3(p.nitems_fit, p.nsplit), kFitThreads, p.smem_fit, s, runs,
               (const int2*)p.d_fit_items, 0, (double*)nullptr, 0);
  } else {
    if (p.var && p.trial_occ) launch_pdl(k_trial_split<4, true, true>, gt, tb, 0, s, runs, ti);
    else if (p.var) launch_pdl(k_trial_split<4, true, false>, gt, tb, 0, s, runs, ti);
    else if (p.trial_occ) launch_pdl(k_trial_split<4, false, true>, gt, tb, 0, s, runs, ti);
    else launch_pdl(k_trial_split<4, false, false>, gt, tb, 0, s, runs, ti);
    launch_pdl(k_fit_tc<4>, dim3(p.nitems_fit, p.nsplit), kFitThreads, p.smem_fit, s, runs,
               (const int2*)p.d_fit_items, 0, (double*)nullptr, 0);
  }
  launch_pdl(k_band_fp64, dim3(p.grid_band), 256, p.smem_band, s, runs, p.nruns, (const BandEntry*)p.d_band,
             (const uint32_t*)p.d_band_cnt, p.nch_max);
}

void tc_init_eval_launch(const TcPlan& p, const RunDesc* runs, int run, const RunDesc& R, cudaStream_t s) {
  const int2* items = p.d_fit_items + p.fit_offset[run];
  if (p.prec == DE_PREC_BF16X3) {
    k_prep_rows<2><<<(R.np + 7) / 8, 256, 0, s>>>(runs, run, R.X[0], R.dp, R.np);
    k_fit_tc<2><<<R.ntiles_tc, kFitThreads, p.smem_fit, s>>>(runs, items, 2, (double*)nullptr, R.np);
  } else {
    k_prep_rows<4><<<(R.np + 7) / 8, 256, 0, s>>>(runs, run, R.X[0], R.dp, R.np);
    k_fit_tc<4><<<R.ntiles_tc, kFitThreads, p.smem_fit, s>>>(runs, items, 2, (double*)nullptr, R.np);
  }
}

de_status tc_eval_launch(const TcPlan& p, const RunDesc* runs, int run, const RunDesc& R, const double* x, int64_t ld,
                         int n, double* f, cudaStream_t s, std::string& err) {
  // the run's operand buffer holds ntiles_tc tiles: evaluate in batches of that many rows
  const int cap = R.ntiles_tc * kTileM;
  for (int r0 = 0; r0 < n; r0 += cap) {
    const int nb = std::min(cap, n - r0);
    const int tiles = (nb + kTileM - 1) / kTileM;
    const int2* items = p.d_fit_items + p.fit_offset[run];
    if (p.prec == DE_PREC_BF16X3) {
      k_prep_rows<2><<<(nb + 7) / 8, 256, 0, s>>>(runs, run, x + (size_t)r0 * ld, ld, nb);
      k_fit_tc<2><<<tiles, kFitThreads, p.smem_fit, s>>>(runs, items, 1, f + r0, nb);
    } else {
      k_prep_rows<4><<<(nb + 7) / 8, 256, 0, s>>>(runs, run, x + (size_t)r0 * ld, ld, nb);
      k_fit_tc<4><<<tiles, kFitThreads, p.smem_fit, s>>>(runs, items, 1, f + r0, nb);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      err = std::string("split-precision eval: ") + cudaGetErrorString(e);
      return DE_ERR_CUDA;
    }
  }
  return DE_OK;
}

de_status tc_eval_rows(const RunDesc* desc, const int2* items, int tiles, int esz, size_t smem, const double* x,
                       int64_t ld, int n, double* f, cudaStream_t s, std::string& err) {
  cudaFuncAttributes fa{};
  cudaError_t e = esz == 2 ? cudaFuncGetAttributes(&fa, k_fit_tc<2>) : cudaFuncGetAttributes(&fa, k_fit_tc<4>);
  if (e == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < smem) {
    e = esz == 2 ? cudaFuncSetAttribute(k_fit_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                 : cudaFuncSetAttribute(k_fit_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  if (e == cudaSuccess) {
    if (esz == 2) {
      k_prep_rows<2><<<(n + 7) / 8, 256, 0, s>>>(desc, 0, x, ld, n);
      k_fit_tc<2><<<tiles, kFitThreads, smem, s>>>(desc, items, 1, f, n);
    } else {
      k_prep_rows<4><<<(n + 7) / 8, 256, 0, s>>>(desc, 0, x, ld, n);
      k_fit_tc<4><<<tiles, kFitThreads, smem, s>>>(desc, items, 1, f, n);
    }
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    err = std::string("split-precision eval: ") + cudaGetErrorString(e);
    return DE_ERR_CUDA;
  }
  return DE_OK;
}

}  // namespace de
