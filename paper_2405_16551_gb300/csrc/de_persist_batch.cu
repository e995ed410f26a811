// de_persist_batch.cu -- the split-precision generation loop of a batch of
// independent runs (uneven NP, D and objective) as one cooperative persistent
// kernel with CTA-local tensor-core products.
//
// The batch is cut into work items: tiles of at most 8 consecutive targets of
// one run, in run order.  CTA c owns a fixed, contiguous slice of items for
// the whole launch and, for every generation, processes its items in order.
// One item is one DE generation of its targets (Eq. 2, Eq. 3, bound repair,
// the objective of Sec. 7.3.1 and greedy selection, Sec. 2), computed the way
// k_persist_cta computes it: one target per warp, the split y of the tile as
// the 16-row B operand, the run's split M (loaded into shared memory when the
// run changes) as the 128-row A operand, three split passes issued by three
// warps, the FP32 objective by 16 threads per target, the rows the split
// error bound cannot decide re-evaluated in FP64 by the whole CTA.
//
// There is no grid barrier.  Each run has an arrival counter: an item adds
// one after its rows, fitness and best partial are written (release order).
// Before a CTA builds trials of generation g of run r it waits (bounded)
// until the counter shows every tile of r done with generation g - 1, then
// reduces r's tile partials itself (the same order in every CTA) into the best
// record and the stop rule of Sec. 7.3.4; the CTA that owns tile 0 of r
// publishes them.  Items of a stopped run are skipped.  Every CTA processes
// generation g - 1 of all its items before generation g, and the launch is
// cooperative (every CTA resident), so the waits always end.  The population,
// fitness and FP64 flags are double buffered by generation parity.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "de_cta_tile.cuh"
#include "de_device.cuh"
#include "de_kernels.h"
#include "de_tcgen05.cuh"

namespace de {

constexpr int kPbRows = 8;                 // targets per item: one per warp
constexpr int kPbSliceRuns = 64;           // runs one CTA's slice may touch
constexpr long long kPbSpin = 1LL << 22;   // polls of a run's arrival counter (with back-off)

struct PbLayout {
  uint32_t yop, mop, z, y, red, total;
};

// shared memory of a CTA for runs of at most kpad_max padded K and dp_max
// padded row length
__host__ __device__ inline PbLayout pb_layout(int kpad_max, int dp_max, int esz) {
  PbLayout L;
  const uint32_t y_part = (uint32_t)(kpad_max * esz / 16) * 256u, m_part = (uint32_t)(kpad_max * esz / 16) * 2048u;
  L.yop = 0;
  L.mop = (2u * y_part + 1023u) / 1024u * 1024u;
  L.z = L.mop + 2u * m_part;
  L.y = L.z + (uint32_t)kPbRows * (uint32_t)(kpad_max + 4) * 4u;
  L.y = (L.y + 15u) / 16u * 16u;
  L.red = L.y + (uint32_t)(2 * dp_max) * 8u;
  L.total = L.red + 2u * 256u * 8u;
  return L;
}

template <int ESZ>
__global__ void __launch_bounds__(256, 2)
    k_persist_batch(const RunDesc* __restrict__ runs, const int4* __restrict__ items, const int2* __restrict__ slices,
                    PersistCtl* ctl, unsigned* __restrict__ cnt, long long gens, int kpad_max, int dp_max) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cta = (int)blockIdx.x;
  const int2 sl = slices[cta];
  const int run_lo = sl.x < sl.y ? items[sl.x].x : 0;
  const int nsr = sl.x < sl.y ? items[sl.y - 1].x - run_lo + 1 : 0;  // runs of the slice (<= kPbSliceRuns)

  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ RunDesc sR;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_tmem;
  __shared__ double s_f[kPbRows], s_ft[kPbRows];
  __shared__ float s_tau[kPbRows], s_yn[kPbRows];
  __shared__ uint8_t s_fx[kPbRows], s_flag[kPbRows];  // flag bit 0 accept, 1 decided in FP64, 2 pending FP64
  __shared__ long long s_key[kPbRows];
  __shared__ int s_blist[kPbRows];
  __shared__ int s_nb, s_abort, s_have, s_mfail;
  // per run of the slice: stopped, generation at launch, last generation
  // observed complete (loop index), owner of tile 0, best f of the last
  // complete generation (FP32, for the FP64-band policy)
  __shared__ int s_rstop[kPbSliceRuns], s_rdone[kPbSliceRuns], s_rpub[kPbSliceRuns];
  __shared__ long long s_rgen0[kPbSliceRuns];
  __shared__ float s_rbest[kPbSliceRuns];
  static_assert(sizeof(RunDesc) % 8 == 0, "descriptor copied in 8-byte words");

  const PbLayout L = pb_layout(kpad_max, dp_max, ESZ);
  uint8_t* sYop = smem + L.yop;
  uint8_t* sMop = smem + L.mop;
  float* zbuf = reinterpret_cast<float*>(smem + L.z);
  double* sY = reinterpret_cast<double*>(smem + L.y);
  double* s_red = reinterpret_cast<double*>(smem + L.red);
  const uint32_t bar_mma = smem_u32(&s_bar);
  const uint32_t ncols = 64u;  // three accumulators of 128 lanes x 16 columns
  const uint32_t fmt = ESZ == 2 ? 1u : 2u;
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kCtaRowsMax >> 3) << 17) |
                         ((uint32_t)(kTileM >> 4) << 24);

  // ---------------------------------------------------------------- set-up
  if (tid == 0) {
    mbar_init(bar_mma, 3);  // one commit per issuing warp
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
  // the y operand starts at zero (rows past a tile's targets stay zero or
  // stale; their products land in columns nobody reads)
  for (uint32_t q = tid * 16u; q < L.mop; q += blockDim.x * 16u) *reinterpret_cast<uint4*>(smem + q) = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  int cur_run = -1;
  double tr[4], tx[4], osh[4];
  uint32_t mma_phase = 0;
  bool abort = false;

  // the stop rule of run r (slice index q) after its generation g, from the
  // tile partials of g: warp 0 reduces, lane 0 decides and, for the owner of
  // tile 0, publishes
  auto reduce_run = [&](const RunDesc& R, int q, int64_t g) {
    const int nt = (R.np + kPbRows - 1) / kPbRows;
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
    const int nt = (R.np + kPbRows - 1) / kPbRows;
    const unsigned target = (unsigned)k * (unsigned)nt;
    for (long long p = 0; p < kPbSpin; ++p) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt + r) : "memory");
      if (v >= target) return true;
      if (*(volatile int*)&ctl->abort) return false;
      __nanosleep(64);
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
        // the run's descriptor, shift and split M
        __syncthreads();
        for (int k = tid; k < (int)(sizeof(RunDesc) / 8); k += blockDim.x)
          reinterpret_cast<uint64_t*>(&sR)[k] = reinterpret_cast<const uint64_t*>(runs + r)[k];
        __syncthreads();
        cta_load_m<ESZ>(sR, sMop, cta_m_part(sR));
#pragma unroll
        for (int e = 0; e < 4; ++e) osh[e] = 4 * lane + e < sR.d ? sR.o[4 * lane + e] : 0.0;
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
        s_have = 1;
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
      const uint32_t y_part = cta_y_part(R), m_part = cta_m_part(R);
      const int zs = cta_zstride(R);
      if (tid < nrows) {
        const int i = row0 + tid;
        s_f[tid] = R.f[cur][i];
        s_fx[tid] = R.fx[cur][i];
        s_tau[tid] = R.tau[i];
      }

      // ---- 1. trials (one target per warp) -> registers and the y operand
      if (warp < nrows) {
        const int i = row0 + warp;
        const int j0 = 4 * lane;
        const TrialSetup ts = trial_setup(R, (uint32_t)i, g, lane);
        ChunkIn cin;
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        uint32_t bits = 0;
        if (j0 < d) {
          trial_load(R, X, ts, (uint32_t)i, g, j0, cin);
          bits = trial_compute(R, ts, j0, cin, t);
#pragma unroll
          for (int e = 0; e < 4; ++e) tx[e] = cin.xi[e];
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) tr[e] = t[e];
        float yn2 = 0.f;
        if (j0 < R.kpad) {
          float y[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            y[e] = (j0 + e < d) ? to_f32_rn(shifted(t[e], osh[e], R)) : 0.f;
            yn2 += y[e] * y[e];
          }
          cta_store_split4<ESZ>(sYop, y_part, warp, j0, y);
        }
        if (R.dbg_trial) trial_debug(R, (uint32_t)i, j0, lane, bits, t);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) yn2 += __shfl_xor_sync(0xffffffffu, yn2, o);
        if (lane == 0) s_yn[warp] = sqrtf(yn2);
      }
      // generic-proxy writes of the operands become visible to the tensor
      // cores' async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();

      // ---- 2. split products: warps 0, 1, 2 issue one pass each
      if (warp < 3 && lane == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int ksteps = R.kpad * ESZ / 32;
        const int pass = warp;
        const uint64_t dm = smem_desc(smem_u32(sMop) + (pass == 1 ? m_part : 0u), 2048u, 128u);
        const uint64_t dy = smem_desc(smem_u32(sYop) + (pass == 2 ? y_part : 0u), 256u, 128u);
        for (int ks = 0; ks < ksteps; ++ks)
          mma_split<ESZ>(tmem + 16u * (uint32_t)pass, dm + (uint64_t)(ks * 256), dy + (uint64_t)(ks * 32), idesc,
                         ks > 0 ? 1u : 0u);
        mma_commit(bar_mma);
      }
      // ---- 3a. warps 0..3 copy the accumulators' columns 0..7 (targets) of
      // lanes 32 w .. 32 w + 31 (coordinates) to shared memory as rows of z
      if (warp < 4) {
        const bool ok = mbar_wait(bar_mma, mma_phase);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (__all_sync(0xffffffffu, ok)) {
          float v[8], w1[8], w2[8];
          const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16);
          tmem_ld8(ta, v);
          tmem_ld8(ta + 16u, w1);
          tmem_ld8(ta + 32u, w2);
          const int j = 32 * warp + lane;
          if (j < d) {
#pragma unroll
            for (int e = 0; e < 8; ++e)
              if (e < nrows) zbuf[(size_t)e * zs + j] = (v[e] + w1[e]) + w2[e];
          }
        } else if (lane == 0) {
          atomicOr(&R.st->err, kErrTimeout);
          atomicExch(&ctl->abort, 1);
          s_abort = 1;
          s_have = 0;
          s_mfail = 1 + (int)mma_phase;
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      }
      mma_phase ^= 1u;
      __syncthreads();

      // ---- 3b. FP32 objective (16 threads per target) and the decisions the
      // split error bound allows
      const bool have = s_have != 0;
      {
        const int rr = tid >> 4, sub = tid & 15;
        const bool valid = rr < nrows;
        EpiAcc acc_{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (valid && have) epi_strided_dispatch(obj, zbuf + (size_t)rr * zs, sub, d, acc_);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          acc_.a1 += __shfl_xor_sync(0xffffffffu, acc_.a1, o);
          acc_.aS += __shfl_xor_sync(0xffffffffu, acc_.aS, o);
          acc_.aG += __shfl_xor_sync(0xffffffffu, acc_.aG, o);
        }
        if (obj == kObjAckley) {
#pragma unroll
          for (int o = 8; o > 0; o >>= 1) {
            acc_.a2 += __shfl_xor_sync(0xffffffffu, acc_.a2, o);
            acc_.a3 += __shfl_xor_sync(0xffffffffu, acc_.a3, o);
          }
        }
        if (sub == 0 && valid) {
          uint8_t flag = 0;
          if (have) {
            const float s1 = acc_.a1, s2 = acc_.a2, s3 = acc_.a3;
            float S = acc_.aS, G = acc_.aG;
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
            const float tau = 2.f * R.band_u * G * R.rownorm * s_yn[rr] + (float)d * 0x1.0p-21f * S + 1e-30f;
            const float fif = to_f32_rn(s_f[rr]);
            const float tif = s_fx[rr] ? 0.f : s_tau[rr];
            const float mrg = 0x1.0p-22f * fabsf(fif);
            const float bp = s_rbest[q];
            const bool sure_reject = fs - tau > fif + tif + mrg;
            const bool sure_accept = fs + tau < fif - tif - mrg;
            const bool ambiguous = !sure_reject && !sure_accept;
            const bool may_be_best = R.band_all && fs - tau <= bp + 0x1.0p-22f * fabsf(bp);
            const bool near = fs - tau <= R.near_thr || fif - tif <= R.near_thr;
            // only a trial the split bound cannot place on one side of the
            // stop target needs FP64 for the stop rule
            const bool may_stop = R.target > 0.0 && fs - tau < (float)R.target * 1.001f &&
                                  !(fs + tau < (float)R.target * 0.999f);
            const double fsd = f64_of_f32(fs);
            s_ft[rr] = fsd;
            if ((ambiguous && (R.band_all || near)) || may_be_best || may_stop || !(fs == fs) || !(fif == fif)) {
              s_blist[atomicAdd(&s_nb, 1)] = rr;
              flag = 4;
            } else if (sure_accept || (ambiguous && fs <= fif)) {
              flag = 1;
              s_f[rr] = fsd;
              s_fx[rr] = 0;
              s_tau[rr] = tau;
            }
          }
          s_flag[rr] = flag;
        }
      }
      __syncthreads();

      // ---- 3c. FP64 decisions of the listed targets, by the whole CTA
      const int nb = s_nb;
      for (int b = 0; b < nb; ++b) {
        const int lr = s_blist[b];
        const bool need_t = !s_fx[lr];
        if (lr == warp) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int j = 4 * lane + e;
            if (j >= d) continue;
            sY[j] = shifted(tr[e], osh[e], R);
            if (need_t) sY[dp + j] = shifted(tx[e], osh[e], R);
          }
        }
        __syncthreads();
        const double ft = cta_fitness_fp64(R, sY, s_red);
        const double fi = need_t ? cta_fitness_fp64(R, sY + dp, s_red) : s_f[lr];
        if (tid == 0) {
          const bool acc = fit_key(ft) <= fit_key(fi) && fit_key(ft) != 0x7FFFFFFFFFFFFFFFLL;  // NaN ranks last
          s_ft[lr] = ft;
          s_f[lr] = acc ? ft : fi;
          s_fx[lr] = 1;
          s_tau[lr] = 0.f;
          s_flag[lr] = (acc ? 1 : 0) | 2;
        }
        __syncthreads();
      }

      // ---- 4. next-generation rows, fitness, debug capture, best partial
      if (warp < nrows) {
        const int i = row0 + warp;
        const bool acc = s_flag[warp] & 1;
        const int j0 = 4 * lane;
        if (j0 < d) {
          double* dst = Xn + (size_t)i * dp + j0;
          const double* src = acc ? tr : tx;
          *reinterpret_cast<double2*>(dst) = make_double2(src[0], src[1]);
          *reinterpret_cast<double2*>(dst + 2) = make_double2(src[2], src[3]);
        }
      }
      if (tid < nrows) {
        const int i = row0 + tid;
        R.f[nxt][i] = s_f[tid];
        R.fx[nxt][i] = s_fx[tid];
        R.tau[i] = s_tau[tid];
        s_key[tid] = fit_key(s_f[tid]);
        if (R.dbg_ftrial) {
          R.dbg_ftrial[i] = s_ft[tid];
          R.dbg_accept[i] = s_flag[tid] & 1;
          R.dbg_fp64[i] = (s_flag[tid] >> 1) & 1;
        }
      }
      __syncthreads();
      if (tid == 0) {
        // the tile's best (lowest key, then lowest index; NaN never)
        long long bk = 0x7FFFFFFFFFFFFFFFLL;
        int bi = -1;
        for (int k = 0; k < nrows; ++k)
          if (s_key[k] != 0x7FFFFFFFFFFFFFFFLL && (bi < 0 || s_key[k] < bk)) {
            bk = s_key[k];
            bi = k;
          }
        const int nt = (R.np + kPbRows - 1) / kPbRows;
        BestPartial* pp = R.part + (size_t)(g & 1) * nt + tile;
        pp->f = bi >= 0 ? s_f[bi] : CUDART_INF;
        pp->idx = bi >= 0 ? row0 + bi : -1;
        atomicAdd(&R.stats[0], (unsigned long long)nb);
        atomicAdd(&R.stats[1], (unsigned long long)nrows);
        // release: the item's rows, fitness and partial (ordered before by the
        // CTA barrier) are visible to every CTA that observes the count
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
  // products still in flight after a failed wait must land before TMEM is freed
  if (tid == 0 && s_mfail) mbar_wait(bar_mma, (uint32_t)(s_mfail - 1));
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ------------------------------------------------------------------ host side
static const void* pb_kernel(int prec) {
  return prec == DE_PREC_BF16X3 ? (const void*)k_persist_batch<2> : (const void*)k_persist_batch<4>;
}

bool pbatch_plan(PbPlan& pp, const std::vector<RunDesc>& runs, int prec) {
  pp.ok = false;
  const int nruns = (int)runs.size();
  if (nruns < 2) return false;
  int kpad_max = 16, dp_max = 4;
  for (const RunDesc& R : runs) {
    // (the three-kernel path's K chunking does not apply: the whole split M
    // is copied into shared memory)
    if (R.nn != 1 || R.d > 128 || R.ntn > 128 || R.strategy != 0 || R.jde || R.obj > kObjAckley)
      return false;
    kpad_max = std::max(kpad_max, R.kpad);
    dp_max = std::max(dp_max, R.dp);
  }
  const size_t smem = pb_layout(kpad_max, dp_max, prec == DE_PREC_BF16X3 ? 2 : 4).total;
  if (smem > 220 * 1024) return false;
  const void* k = pb_kernel(prec);
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return false;
  }
  // items: tiles of at most kPbRows targets, in run order
  std::vector<int4> items;
  for (int r = 0; r < nruns; ++r)
    for (int t = 0, row = 0; row < runs[r].np; ++t, row += kPbRows)
      items.push_back(make_int4(r, t, row, std::min(kPbRows, runs[r].np - row)));
  const int nitems = (int)items.size();
  const int nct = std::min(per_sm * nsm, nitems);
  // contiguous slices of nearly equal item counts
  std::vector<int2> slices(nct);
  for (int c = 0; c < nct; ++c) {
    const int lo = (int)((long long)nitems * c / nct), hi = (int)((long long)nitems * (c + 1) / nct);
    slices[c] = make_int2(lo, hi);
    if (hi > lo && items[hi - 1].x - items[lo].x + 1 > kPbSliceRuns) return false;
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

cudaError_t pbatch_launch(const PbPlan& pp, const RunDesc* runs, PersistCtl* ctl, long long gens, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(PersistCtl), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(pp.d_cnt, 0, (size_t)pp.nruns * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const int4* items = pp.d_items;
  const int2* slices = pp.d_slices;
  unsigned* cnt = pp.d_cnt;
  int kpad_max = pp.kpad_max, dp_max = pp.dp_max;
  void* args[] = {(void*)&runs, (void*)&items, (void*)&slices, (void*)&ctl, (void*)&cnt, (void*)&gens,
                  (void*)&kpad_max, (void*)&dp_max};
  return cudaLaunchCooperativeKernel(pb_kernel(pp.prec), dim3((unsigned)pp.nct), dim3(256), args, pp.smem, s);
}

}  // namespace de
