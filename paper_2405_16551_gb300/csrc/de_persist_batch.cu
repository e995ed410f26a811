// de_persist_batch.cu -- the split-precision generation loop of a batch of
// independent runs (uneven NP, D and objective) as one cooperative persistent
// kernel, one CTA per SM.
//
// The batch is cut into work items: the 128-target tiles of every run, in run
// order.  CTA c owns a fixed, contiguous slice of items for the whole launch
// (slices balanced by an estimate of each item's time) and, for every
// generation, processes its items in order.  One item is one DE generation of
// its targets (Eq. 2, Eq. 3, bound repair, the objective of Sec. 7.3.1 and
// greedy selection, Sec. 2), the work of the three-kernel path's trial and
// fitness tiles done in one place:
//
//   trials     the whole CTA, R.lpt lanes per target: FP64 trial rows to the
//              next generation's rows, their shifted vectors rounded to FP32
//              and split into high and low parts straight into the A operand
//              in shared memory (the 128 targets are the products' M
//              dimension);
//   products   z = M y as Y M^T, three split passes accumulated in FP32 in
//              tensor memory; the run's split M (the B operand, N = its padded
//              D) is copied into shared memory by one bulk asynchronous copy
//              when the CTA's run changes, while that item's trials are built;
//   epilogue   the objective terms from TMEM (two threads per target, one per
//              column half), the split error bound and the selection decisions
//              it allows; the targets it cannot decide are re-evaluated in
//              FP64 by the whole CTA;
//   rows       rejected trials' rows overwritten by their targets, fitness
//              values and the tile's best partial.
//
// There is no grid barrier.  Each run has an arrival counter: an item adds
// one after its rows, fitness and partial are written (release order).  Before
// a CTA builds trials of generation g of run r it waits (bounded) until the
// counter shows every tile of r done with generation g - 1, then reduces r's
// tile partials itself (the same order in every CTA) into the best record and
// the stop rule of Sec. 7.3.4; the CTA that owns tile 0 of r publishes them.
// Items of a stopped run are skipped.  Every CTA processes generation g - 1 of
// all its items before generation g, and the launch is cooperative (every CTA
// resident), so the waits always end.  The population, fitness and FP64 flags
// are double buffered by generation parity.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "de_cta_tile.cuh"
#include "de_device.cuh"
#include "de_kernels.h"
#include "de_tcgen05.cuh"

namespace de {

constexpr int kPbThreads = 256;
constexpr int kPbSliceRuns = 64;           // runs one CTA's slice may touch
constexpr long long kPbSpin = 1LL << 22;   // polls of a run's arrival counter (each a round trip to L2: seconds in all)

struct PbLayout {
  uint32_t a, b, y, red, total;
};

// shared memory of a CTA for runs of at most kpad_max padded K (= padded N)
// and dp_max row length: A (128 target rows, two parts), B (the split M, two
// parts), two FP64 vectors for the FP64 decisions, their reduction slots
__host__ __device__ inline PbLayout pb_layout(int kpad_max, int dp_max, int esz) {
  PbLayout L;
  L.a = 0;
  L.b = 2u * (uint32_t)kTileM * (uint32_t)(kpad_max * esz);  // a multiple of 4096
  L.y = L.b + 2u * (uint32_t)kpad_max * (uint32_t)(kpad_max * esz);
  L.red = L.y + (uint32_t)(2 * dp_max) * 8u;
  L.total = L.red + 16u * 8u;
  return L;
}

template <int ESZ>
__global__ void __launch_bounds__(kPbThreads, 1)
    k_persist_batch(const RunDesc* __restrict__ runs, const int4* __restrict__ items, const int2* __restrict__ slices,
                    PersistCtl* ctl, unsigned* __restrict__ cnt, long long gens, int kpad_max, int dp_max,
                    uint32_t ncols) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cta = (int)blockIdx.x;
  const int2 sl = slices[cta];
  // failure-detection test (off unless set by the launcher): this CTA leaves
  // out the arrival of its first item's first generation, and the waits give
  // up after test_spin polls
  const bool test_skip = ctl->test_skip == cta + 1;
  const long long spin_limit = ctl->test_spin > 0 ? ctl->test_spin : kPbSpin;
  const int run_lo = sl.x < sl.y ? items[sl.x].x : 0;
  const int nsr = sl.x < sl.y ? items[sl.y - 1].x - run_lo + 1 : 0;  // runs of the slice (<= kPbSliceRuns)

  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ RunDesc sR;
  __shared__ __align__(8) uint64_t s_bar[2];  // [0] products done, [1] split M copied
  __shared__ uint32_t s_tmem;
  __shared__ float s_part[5][kTileM];
  __shared__ double s_fi[kTileM], s_fnew[kTileM], s_ftrial[kTileM];
  __shared__ float s_taunew[kTileM], s_yn[kTileM];
  __shared__ uint8_t s_fx0[kTileM], s_fxnew[kTileM];
  __shared__ uint8_t s_flag[kTileM];  // bit 0 accept, 1 decided in FP64, 2 pending FP64
  __shared__ int s_blist[kTileM];
  __shared__ double s_bf[kPbThreads / 32];
  __shared__ long long s_bk[kPbThreads / 32];
  __shared__ int s_bi[kPbThreads / 32];
  __shared__ int s_nb, s_abort, s_issued, s_mfail;
  // per run of the slice: stopped, generation at launch, last generation
  // observed complete (loop index), owner of tile 0, best f of the last
  // complete generation (FP32, for the FP64-decision policy)
  __shared__ int s_rstop[kPbSliceRuns], s_rdone[kPbSliceRuns], s_rpub[kPbSliceRuns];
  __shared__ long long s_rgen0[kPbSliceRuns];
  __shared__ float s_rbest[kPbSliceRuns];
  static_assert(sizeof(RunDesc) % 8 == 0, "descriptor copied in 8-byte words");

  const PbLayout L = pb_layout(kpad_max, dp_max, ESZ);
  uint8_t* sA = smem + L.a;
  double* sY = reinterpret_cast<double*>(smem + L.y);
  double* s_red = reinterpret_cast<double*>(smem + L.red);
  const uint32_t bar_mma = smem_u32(&s_bar[0]), bar_b = smem_u32(&s_bar[1]);
  const uint32_t fmt = ESZ == 2 ? 1u : 2u;

  // ---------------------------------------------------------------- set-up
  if (tid == 0) {
    mbar_init(bar_mma, 1);
    mbar_init(bar_b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
    s_mfail = 0;
  }
  for (int q = tid; q < nsr; q += blockDim.x) {
    const RunDesc& Rq = runs[run_lo + q];
    s_rstop[q] = *(volatile int32_t*)&Rq.st->stop;
    s_rgen0[q] = *(volatile int64_t*)&Rq.st->gen;
    s_rdone[q] = 0;
    s_rbest[q] = to_f32_rn(*(volatile double*)&Rq.st->best_f);
    s_rpub[q] = 0;
  }
  for (int it = sl.x + tid; it < sl.y; it += blockDim.x)
    if (items[it].y == 0) s_rpub[items[it].x - run_lo] = 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  int cur_run = -1;
  uint32_t mma_phase = 0, b_phase = 0;
  bool b_wait = false;  // (thread 0) a copy of the split M is in flight
  bool abort = false;

  // the stop rule of run r (slice index q) after its generation g, from the
  // tile partials of g: warp 0 reduces, lane 0 decides and, for the owner of
  // tile 0, publishes
  auto reduce_run = [&](const RunDesc& R, int q, int64_t g) {
    const int nt = R.ntiles_tc;
    Best b;
    b.init();
    const BestPartial* pp = R.part + (size_t)(g & 1) * nt;
    for (int t = lane; t < nt; t += 32) b.offer(__ldcg(&pp[t].f), __ldcg(&pp[t].idx));
    b.warp_reduce();
    if (lane == 0) {
      const int64_t evals = (int64_t)R.np * (1 + g);  // the initial population counts as NP evaluations
      int sp = 0;
      if (R.target > 0.0 && b.i >= 0 && b.f < R.target) sp = 1;
      else if (R.max_evals > 0 && evals >= R.max_evals) sp = 2;
      else if (g >= R.max_gens) sp = 3;
      s_rstop[q] = sp;
      s_rbest[q] = to_f32_rn(b.f);
      if (s_rpub[q]) {
        RunState* st = R.st;
        st->best_f = b.f;
        st->best_idx = b.i;
        st->gen = g;
        st->evals = evals;
        st->stop = sp;
        if (b.i < 0) atomicOr(&st->err, kErrNonFinite);
      }
    }
  };

  // wait (warp 0, bounded) until every tile of run r finished generation
  // number `k` of this launch (k >= 1)
  auto wait_run = [&](const RunDesc& R, int r, int k) -> bool {
    const unsigned target = (unsigned)k * (unsigned)R.ntiles_tc;
    for (long long p = 0; p < spin_limit; ++p) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt + r) : "memory");
      if (v >= target) return true;
      // the abort flag every 16th poll (a read after every poll doubles
      // the round trips per poll)
      if ((p & 15) == 15 && *(volatile int*)&ctl->abort) return false;
    }
    if (lane == 0) {
      atomicExch(&ctl->abort, 1);
      atomicOr(&R.st->err, kErrTimeout);
    }
    return false;
  };

  for (long long itg = 0; itg < gens && !abort; ++itg) {
    for (int it = sl.x; it < sl.y; ++it) {
      const int4 w = items[it];  // run, tile, first row, rows
      const int r = w.x, q = r - run_lo;
      if (s_rstop[q]) continue;  // uniform: written before the last barrier
      if (r != cur_run) {
        // the run's descriptor; its split M follows asynchronously (the
        // products of the previous item, which read the old one, are done)
        __syncthreads();
        for (int k = tid; k < (int)(sizeof(RunDesc) / 8); k += blockDim.x)
          reinterpret_cast<uint64_t*>(&sR)[k] = reinterpret_cast<const uint64_t*>(runs + r)[k];
        __syncthreads();
        if (tid == 0) {
          bool ok = true;
          if (b_wait) {  // the previous copy (of a run whose items were all skipped) lands first
            ok = mbar_wait(bar_b, b_phase);
            if (ok) {
              b_phase ^= 1u;
              b_wait = false;
            } else {
              atomicOr(&sR.st->err, kErrTimeout);
              atomicExch(&ctl->abort, 1);
              s_abort = 1;
            }
          }
          if (ok) {
            mbar_expect_tx(bar_b, (uint32_t)sR.b_tile_bytes);
            bulk_g2s(smem_u32(smem + L.b), sR.B, (uint32_t)sR.b_tile_bytes, bar_b);
            b_wait = true;
          }
        }
        cur_run = r;
      }
      const RunDesc& R = sR;
      // generation itg of run r needs every tile of its previous generation
      if (itg > 0 && s_rdone[q] < (int)itg) {
        if (warp == 0) {
          const bool ok = wait_run(R, r, (int)itg);
          if (__all_sync(0xffffffffu, ok)) reduce_run(R, q, s_rgen0[q] + itg);
          else if (lane == 0) s_abort = 1;
        }
        if (tid == 0) s_rdone[q] = (int)itg;
      }
      if (tid == 0) {
        s_nb = 0;
        if (*(volatile int*)&ctl->abort) s_abort = 1;
      }
      __syncthreads();
      if (s_abort) break;
      if (s_rstop[q]) continue;

      const int tile = w.y, row0 = w.z, nrows = w.w;
      const int d = R.d, dp = R.dp, obj = R.obj;
      const int64_t g = s_rgen0[q] + itg + 1;
      const int cur = (int)((g - 1) & 1), nxt = cur ^ 1;
      const double* __restrict__ X = R.X[cur];
      double* __restrict__ Xn = R.X[nxt];
      const uint32_t a_part = (uint32_t)(R.a_tile_bytes / 2), b_part = (uint32_t)(R.b_tile_bytes / 2);

      // the selection inputs of row m (TMEM lane), fetched while the trials
      // are built; column half h of the epilogue
      const int m = 32 * (warp & 3) + lane, h = warp >> 2;
      double pf_fi = 0.0;
      float pf_tau = 0.f;
      uint8_t pf_fx = 1;
      if (h == 0 && m < nrows) {
        const int i = row0 + m;
        pf_fi = __ldcg(&R.f[cur][i]);
        pf_fx = __ldcg(&R.fx[cur][i]);
        pf_tau = __ldcg(&R.tau[i]);
      }

      // ---- 1. trials, R.lpt lanes per target (one 4-coordinate chunk per
      // lane covers the padded row: d <= 128), round rd of warp w holding
      // targets (8 rd + w) tpw ..; the trial rows go straight to the next
      // generation's rows (a rejected trial is overwritten by its target in
      // step 6).  The loads of round rd + 1 are in flight while round rd is
      // computed (two register sets).
      {
        const int lpt = R.lpt, tpw = 32 / lpt, sub = lane & (lpt - 1), j0 = 4 * sub;
        const int per_round = (kPbThreads / 32) * tpw;
        const int rounds = (nrows + per_round - 1) / per_round;
        struct Unit {
          TrialSetup s;
          ChunkIn c;
          int m;
          bool v;
        };
        auto prep = [&](int rd, Unit& U) {
          if (rd >= rounds) return;
          const int mm = (rd * (kPbThreads / 32) + warp) * tpw + lane / lpt;
          U.v = mm < nrows;
          U.m = U.v ? mm : nrows - 1;  // idle segments repeat a valid target without writing
          U.s = trial_setup(R, (uint32_t)(row0 + U.m), g, sub, 0u, U.v);
          if (j0 < d) trial_load(R, X, U.s, (uint32_t)(row0 + U.m), g, j0, U.c);
        };
        auto finish = [&](int rd, const Unit& U) {
          if (rd >= rounds) return;  // uniform
          const int i = row0 + U.m;
          double t[4] = {0.0, 0.0, 0.0, 0.0};
          uint32_t bits = 0;
          if (j0 < d) {
            bits = trial_compute(R, U.s, j0, U.c, t);
            if (U.v) {
              double* row = Xn + (size_t)i * dp + j0;
              *reinterpret_cast<double2*>(row) = make_double2(t[0], t[1]);
              *reinterpret_cast<double2*>(row + 2) = make_double2(t[2], t[3]);
            }
          }
          float yn2 = 0.f;
          if (j0 < R.kpad) {
            float y[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              y[e] = (j0 + e < d) ? to_f32_rn(shifted(t[e], __ldg(R.o + j0 + e), R)) : 0.f;
              yn2 += y[e] * y[e];
            }
            if (U.v) store_split4<ESZ>(sA, a_part, U.m, j0, y);
          }
          if (R.dbg_trial) trial_debug(R, (uint32_t)i, j0, lane, bits, t, lpt, U.v);
          for (int o = lpt >> 1; o > 0; o >>= 1) yn2 += __shfl_xor_sync(0xffffffffu, yn2, o);
          if (U.v && sub == 0) s_yn[U.m] = sqrtf(yn2);
        };
        Unit ua, ub;
        prep(0, ua);
        prep(1, ub);
        for (int rd = 0; rd < rounds; rd += 2) {
          finish(rd, ua);
          prep(rd + 2, ua);
          finish(rd + 1, ub);
          prep(rd + 3, ub);
        }
      }
      // generic-proxy writes of A become visible to the tensor cores' async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();

      // ---- 2. split products Z = Y M^T (thread 0 issues all three passes)
      if (tid == 0) {
        bool ok = !s_abort;
        if (ok && b_wait) {
          ok = mbar_wait(bar_b, b_phase);
          if (ok) {
            b_phase ^= 1u;
            b_wait = false;
          }
        }
        if (ok) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int ksteps = R.kpad * ESZ / 32;
          const uint32_t a0 = smem_u32(sA), b0 = smem_u32(smem + L.b), bk = (uint32_t)(R.ntn / 8) * 128u;
          const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(R.ntn >> 3) << 17) |
                                 ((uint32_t)(kTileM >> 4) << 24);
          for (int ks = 0; ks < ksteps; ++ks) {
#pragma unroll
            for (int pass = 0; pass < 3; ++pass) {
              const uint32_t a = a0 + (pass == 2 ? a_part : 0u) + (uint32_t)ks * 2u * 2048u;
              const uint32_t b = b0 + (pass == 1 ? b_part : 0u) + (uint32_t)ks * 2u * bk;
              mma_split<ESZ>(tmem, smem_desc(a, 2048u, 128u), smem_desc(b, bk, 128u), idesc,
                             (ks > 0 || pass > 0) ? 1u : 0u);
            }
          }
          mma_commit(bar_mma);
        } else {
          atomicOr(&R.st->err, kErrTimeout);
          atomicExch(&ctl->abort, 1);
          s_abort = 1;
        }
        s_issued = ok ? 1 : 0;
      }
      __syncthreads();

      // ---- 3. epilogue: objective terms of row m, column half h, from TMEM
      const bool issued = s_issued != 0;
      bool have = false;
      if (issued) {
        have = mbar_wait(bar_mma, mma_phase);
        if (!have && lane == 0) {
          atomicOr(&R.st->err, kErrTimeout);
          atomicExch(&ctl->abort, 1);
          s_abort = 1;
          s_mfail = 1 + (int)mma_phase;
        }
        mma_phase ^= 1u;
      }
      have = __all_sync(0xffffffffu, have);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      EpiAcc acc_{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const int half = R.ntn / 2, cb = h * half;
      const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
      if (have) {
        for (int c = 0; c < half; c += 32) {
          float v[32];
          const int wc = min(32, half - c);  // a multiple of 8
          const uint32_t ta = tmem + lane_base + (uint32_t)(cb + c);
          if (wc == 32) {
            tmem_ld_cols32(ta, v);
          } else if (wc == 24) {
            tmem_ld_cols16(ta, v);
            tmem_ld8(ta + 16u, v + 16);
          } else if (wc == 16) {
            tmem_ld_cols16(ta, v);
          } else {
            tmem_ld8(ta, v);
          }
          epi_dispatch(obj, v, wc, cb + c, d, c == 0, acc_);
        }
        if (obj == kObjRosenbrock && h == 0 && half < d) {
          // the term of the last column of this half needs the next column
          const float tn = tmem_ld1(tmem + lane_base + (uint32_t)half) + 1.f;
          const float aa = tn - acc_.prev_t * acc_.prev_t, bb = acc_.prev_t - 1.f;
          acc_.a1 += fmaf(100.f * aa, aa, bb * bb);
          acc_.aG += 400.f * fabsf(acc_.prev_t) * fabsf(aa) + 2.f * fabsf(bb) + 200.f * fabsf(aa);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      if (h == 1) {
        s_part[0][m] = acc_.a1;
        s_part[1][m] = acc_.a2;
        s_part[2][m] = acc_.a3;
        s_part[3][m] = acc_.aS;
        s_part[4][m] = acc_.aG;
      }
      __syncthreads();

      // ---- 4. the decisions the split error bound allows (Sec. 2, selection)
      if (h == 0 && m < nrows) {
        const float s1 = acc_.a1 + s_part[0][m], s2 = acc_.a2 + s_part[1][m], s3 = acc_.a3 + s_part[2][m];
        float S = acc_.aS + s_part[3][m], G = acc_.aG + s_part[4][m];
        float fs;
        if (obj == kObjAckley) {
          const float rq = sqrtf(s1 / (float)d);
          const float e1 = expf(-0.2f * rq), e2 = expf(s2 / (float)d);
          fs = 20.f + 2.718281828f - 20.f * e1 - e2;
          S = 20.f + 2.718281828f + 20.f * e1 + expf(S / (float)d);
          G = (rq > 0.f ? 4.f * e1 * s3 / ((float)d * rq) : 3.0e38f) + 6.283185307f * e2;
        } else {
          if (obj != kObjRastrigin) S = s1;
          fs = s1;
        }
        // error bound of fs: split products (relative to |M||y|) through the
        // derivative bound G, plus FP32 rounding of the terms and their sum
        const float tau = 2.f * R.band_u * G * R.rownorm * s_yn[m] + (float)d * 0x1.0p-21f * S + 1e-30f;
        const float fif = to_f32_rn(pf_fi);
        const float tif = pf_fx ? 0.f : pf_tau;
        const float mrg = 0x1.0p-22f * fabsf(fif);
        const float bp = s_rbest[q];
        const bool sure_reject = fs - tau > fif + tif + mrg;
        const bool sure_accept = fs + tau < fif - tif - mrg;
        const bool ambiguous = !sure_reject && !sure_accept;
        const bool may_be_best = R.band_all && fs - tau <= bp + 0x1.0p-22f * fabsf(bp);
        const bool near = fs - tau <= R.near_thr || fif - tif <= R.near_thr;
        // only a trial the split bound cannot place on one side of the stop
        // target needs FP64 for the stop rule
        const bool may_stop = R.target > 0.0 && fs - tau < (float)R.target * 1.001f &&
                              !(fs + tau < (float)R.target * 0.999f);
        const double fsd = f64_of_f32(fs);
        s_ftrial[m] = fsd;
        s_fi[m] = pf_fi;
        s_fx0[m] = pf_fx;
        if (!have) {
          s_flag[m] = 0;  // the launch is abandoned; keep the target
          s_fnew[m] = pf_fi;
          s_fxnew[m] = pf_fx;
          s_taunew[m] = pf_tau;
        } else if ((ambiguous && (R.band_all || near)) || may_be_best || may_stop || !(fs == fs) || !(fif == fif)) {
          s_blist[atomicAdd(&s_nb, 1)] = m;
          s_flag[m] = 4;
        } else {
          // decided on the split values (an undecidable comparison far from the
          // optimum goes to the smaller split value, ties to the trial)
          const bool acc = sure_accept || (ambiguous && fs <= fif);
          s_flag[m] = acc ? 1 : 0;
          s_fnew[m] = acc ? fsd : pf_fi;
          s_fxnew[m] = acc ? 0 : pf_fx;
          s_taunew[m] = acc ? tau : pf_tau;
        }
      }
      __syncthreads();

      // ---- 5. FP64 decisions of the listed targets, by the whole CTA, in
      // list order (the order does not change any value)
      const int nb = s_nb;
      for (int b = 0; b < nb; ++b) {
        const int lm = s_blist[b], i = row0 + lm;
        const bool need_t = !s_fx0[lm];
        for (int j = tid; j < d; j += blockDim.x) {
          const double oj = __ldg(R.o + j);
          sY[j] = shifted(__ldcg(Xn + (size_t)i * dp + j), oj, R);
          if (need_t) sY[dp + j] = shifted(__ldcg(X + (size_t)i * dp + j), oj, R);
        }
        __syncthreads();
        const double ft = cta_fitness_fp64(R, sY, s_red);
        const double fi = need_t ? cta_fitness_fp64(R, sY + dp, s_red) : s_fi[lm];
        if (tid == 0) {
          const bool acc = fit_key(ft) <= fit_key(fi) && fit_key(ft) != 0x7FFFFFFFFFFFFFFFLL;  // NaN ranks last
          s_ftrial[lm] = ft;
          s_fnew[lm] = acc ? ft : fi;
          s_fxnew[lm] = 1;
          s_taunew[lm] = 0.f;
          s_flag[lm] = (acc ? 1 : 0) | 2;
        }
        __syncthreads();
      }

      // ---- 6. next-generation fitness, rows, debug capture, best partial
      Best bb;
      bb.init();
      if (tid < nrows) {
        const int i = row0 + tid;
        const uint8_t fl = s_flag[tid];
        R.f[nxt][i] = s_fnew[tid];
        R.fx[nxt][i] = s_fxnew[tid];
        R.tau[i] = s_taunew[tid];
        if (R.dbg_ftrial) {
          R.dbg_ftrial[i] = s_ftrial[tid];
          R.dbg_accept[i] = fl & 1;
          R.dbg_fp64[i] = (fl >> 1) & 1;
        }
        bb.offer(s_fnew[tid], i);
      }
      {
        // a rejected trial's row becomes its target's again: warp w copies
        // rows w, w + 8, .. (dp / 2 <= 64 double2 each, two per lane), the
        // loads of eight rows issued before their stores
        const int dp2 = dp / 2;
        for (int e0 = warp; e0 < nrows; e0 += 8 * (kPbThreads / 32)) {
          double2 v[8][2];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int e = e0 + k * (kPbThreads / 32);
            const bool cp = e < nrows && !(s_flag[e] & 1);
            const double2* src = reinterpret_cast<const double2*>(X + (size_t)(row0 + e) * dp);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh)
              if (cp && lane + 32 * hh < dp2) v[k][hh] = __ldcg(src + lane + 32 * hh);
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int e = e0 + k * (kPbThreads / 32);
            const bool cp = e < nrows && !(s_flag[e] & 1);
            double2* dst = reinterpret_cast<double2*>(Xn + (size_t)(row0 + e) * dp);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh)
              if (cp && lane + 32 * hh < dp2) dst[lane + 32 * hh] = v[k][hh];
          }
        }
      }
      bb.warp_reduce();
      if (lane == 0) {
        s_bf[warp] = bb.f;
        s_bk[warp] = bb.k;
        s_bi[warp] = bb.i;
      }
      __syncthreads();
      if (tid == 0) {
        bb.init();
        for (int k = 0; k < kPbThreads / 32; ++k) bb.take(s_bf[k], s_bk[k], s_bi[k]);
        BestPartial* pp = R.part + (size_t)(g & 1) * R.ntiles_tc + tile;
        pp->f = bb.f;
        pp->idx = bb.i;
        atomicAdd(&R.stats[0], (unsigned long long)nb);
        atomicAdd(&R.stats[1], (unsigned long long)nrows);
        // release: the item's rows, fitness and partial (ordered before by the
        // CTA barrier) are visible to every CTA that observes the count
        if (!(test_skip && itg == 0 && it == sl.x))
          asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(cnt + r), "r"(1u) : "memory");
      }
    }
    __syncthreads();
    abort = s_abort != 0;
  }

  // ---------------------------------------------------------------- teardown
  // the owner of tile 0 of each run that is still running publishes the
  // best record and stop rule of its last generation
  if (!abort && gens > 0 && warp == 0) {
    for (int q = 0; q < nsr; ++q) {
      if (!s_rpub[q] || s_rstop[q] || s_rdone[q] == (int)gens) continue;
      const RunDesc& R = runs[run_lo + q];
      if (!__all_sync(0xffffffffu, wait_run(R, run_lo + q, (int)gens))) break;
      reduce_run(R, q, s_rgen0[q] + gens);
    }
  }
  // copies and products still in flight land before the CTA leaves and frees TMEM
  if (tid == 0) {
    if (b_wait) mbar_wait(bar_b, b_phase);
    if (s_mfail) mbar_wait(bar_mma, (uint32_t)(s_mfail - 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ------------------------------------------------------------------ host side
static const void* pb_kernel(int prec) {
  return prec == DE_PREC_BF16X3 ? (const void*)k_persist_batch<2> : (const void*)k_persist_batch<4>;
}

// Estimated time of one item (arbitrary units): a fixed part (wait, products,
// barriers, release), trial rounds of R.lpt lanes per target, the rows written
// and the epilogue columns.  Used only to balance the slices.
static long long item_cost(const RunDesc& R, int nrows) {
  const long long rounds = ((long long)nrows * R.lpt + kPbThreads - 1) / kPbThreads;
  return 400 + 100 * rounds + (long long)nrows * R.dp / 64 + 4 * R.ntn;
}

bool pbatch_plan(PbPlan& pp, const std::vector<RunDesc>& runs, int prec) {
  pp.ok = false;
  const int nruns = (int)runs.size();
  if (nruns < 2) return false;
  int kpad_max = 16, dp_max = 4;
  for (const RunDesc& R : runs) {
    // one N tile (N = the padded D), the whole split M resident in shared
    // memory (the three-kernel path's K chunking does not apply)
    if (R.nn != 1 || R.d > 128 || R.ntn != R.kpad || R.strategy != 0 || R.jde || R.obj > kObjAckley) return false;
    kpad_max = std::max(kpad_max, R.kpad);
    dp_max = std::max(dp_max, R.dp);
  }
  const int esz = prec == DE_PREC_BF16X3 ? 2 : 4;
  const size_t smem = pb_layout(kpad_max, dp_max, esz).total;
  const void* k = pb_kernel(prec);
  int per_sm = 0, dev = 0, nsm = 0, optin = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (smem + fa.sharedSizeBytes > (size_t)optin) return false;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kPbThreads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return false;
  }
  uint32_t ncols = 32;
  while ((int)ncols < kpad_max) ncols *= 2;
  // items: the 128-target tiles of every run, in run order
  std::vector<int4> items;
  std::vector<long long> cost;
  for (int r = 0; r < nruns; ++r)
    for (int t = 0, row = 0; row < runs[r].np; ++t, row += kTileM) {
      const int n = std::min(kTileM, runs[r].np - row);
      items.push_back(make_int4(r, t, row, n));
      cost.push_back(item_cost(runs[r], n));
    }
  const int nitems = (int)items.size();
  const int nct = std::min(per_sm * nsm, nitems);
  // contiguous slices of nearly equal estimated time: CTA c takes the items
  // whose cost midpoint falls in [W c / nct, W (c + 1) / nct)
  long long W = 0;
  for (long long c : cost) W += c;
  std::vector<int2> slices(nct);
  {
    int lo = 0;
    long long acc = 0;
    for (int c = 0; c < nct; ++c) {
      int hi = lo;
      const long long lim = W * (c + 1) / nct;
      while (hi < nitems && (c == nct - 1 || acc + cost[hi] / 2 < lim)) acc += cost[hi++];
      slices[c] = make_int2(lo, hi);
      if (hi > lo && items[hi - 1].x - items[lo].x + 1 > kPbSliceRuns) return false;
      lo = hi;
    }
  }
  if (cudaMalloc(&pp.d_items, items.size() * sizeof(int4)) != cudaSuccess ||
      cudaMalloc(&pp.d_slices, slices.size() * sizeof(int2)) != cudaSuccess ||
      cudaMalloc(&pp.d_cnt, (size_t)nruns * sizeof(unsigned)) != cudaSuccess ||
      cudaMemcpy(pp.d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(pp.d_slices, slices.data(), slices.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    pbatch_free(pp);
    return false;
  }
  pp.nct = nct;
  pp.nruns = nruns;
  pp.smem = smem;
  pp.prec = prec;
  pp.kpad_max = kpad_max;
  pp.dp_max = dp_max;
  pp.ncols = ncols;
  pp.ok = true;
  return true;
}

void pbatch_free(PbPlan& pp) {
  if (pp.d_items) cudaFree(pp.d_items);
  if (pp.d_slices) cudaFree(pp.d_slices);
  if (pp.d_cnt) cudaFree(pp.d_cnt);
  pp.d_items = nullptr;
  pp.d_slices = nullptr;
  pp.d_cnt = nullptr;
  pp.ok = false;
}

cudaError_t pbatch_launch(const PbPlan& pp, const RunDesc* runs, PersistCtl* ctl, long long gens, cudaStream_t s,
                          int test_skip) {
  cudaError_t e = persist_ctl_reset(ctl, test_skip, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(pp.d_cnt, 0, (size_t)pp.nruns * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const int4* items = pp.d_items;
  const int2* slices = pp.d_slices;
  unsigned* cnt = pp.d_cnt;
  int kpad_max = pp.kpad_max, dp_max = pp.dp_max;
  uint32_t ncols = pp.ncols;
  void* args[] = {(void*)&runs, (void*)&items, (void*)&slices, (void*)&ctl, (void*)&cnt, (void*)&gens,
                  (void*)&kpad_max, (void*)&dp_max, (void*)&ncols};
  return cudaLaunchCooperativeKernel(pb_kernel(pp.prec), dim3((unsigned)pp.nct), dim3(kPbThreads), args, pp.smem, s);
}

}  // namespace de
