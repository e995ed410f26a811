// de_persist_cta.cu -- the split-precision generation loop as one cooperative
// persistent kernel in which every CTA runs the tensor-core products of its
// own targets.
//
// CTA t owns `rows` (at most 16) consecutive targets for the whole launch and
// keeps the split M (the B operand) resident in shared memory.  One
// generation:
//
//   1. every warp builds the trials of its targets (Eq. 2, Eq. 3, bound
//      repair; FP64, one target per warp at a time, the same routines as the
//      other paths), keeps the trial and target rows in registers and writes
//      the split rows of y = (t - o) s into the CTA's own A operand;
//   2. one thread issues the three split products on tcgen05 with the roles
//      of the operands exchanged: A is M (128 rows, one per output
//      coordinate z_j, zero past D; resident for the whole launch), B the
//      16-row y tile (N = 16), so that TMEM lane j, column r holds z_j of
//      target r and the tensor work scales with 16 targets, not 128;
//   3. the eight warps copy the accumulator (lanes 32 (w mod 4) .., columns
//      8 (w / 4) ..) to shared memory as rows of z; every target is then evaluated in
//      FP32 by 16 threads (strided columns, fixed xor tree: the order of the
//      cluster kernel, so both give the same values) and its selection is
//      decided where the split error bound allows.  The other targets (and
//      trials that could stop the run) are re-evaluated in FP64 by the whole
//      CTA, with M^T read at L2;
//   4. the CTA writes its next-generation rows to the other population buffer
//      (double buffering: no CTA overwrites a row another CTA still reads as
//      a donor), its best partial, and arrives at a grid barrier (bounded
//      spin on a global counter).  After the barrier every CTA reduces all
//      partials in the same order, so every CTA takes the same best record
//      and stop decision (Sec. 7.3.4).
//
// There is no cluster and no distributed shared memory: the grid barrier is
// the only synchronisation between CTAs.  The launch is cooperative, so every
// CTA is resident.  Every wait is bounded; on expiry the kernel records
// kErrTimeout, the CTAs agree on an abort through a global flag and leave at
// the same point of the loop with the population of the last complete
// generation.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "de_cta_tile.cuh"
#include "de_device.cuh"
#include "de_kernels.h"
#include "de_tcgen05.cuh"

namespace de {

constexpr long long kCtaGridSpin = 1LL << 22;     // polls of the grid barrier (each a round trip to L2: seconds in all)

struct CtaLayout {
  uint32_t yop, mop, z, y, red, total;
};

__host__ __device__ inline CtaLayout cta_layout(const RunDesc& R) {
  CtaLayout L;
  L.yop = 0;
  L.mop = (2u * cta_y_part(R) + 1023u) / 1024u * 1024u;
  L.z = L.mop + 2u * cta_m_part(R);
  L.y = L.z + (uint32_t)(kCtaRowsMax * cta_zstride(R)) * 4u;  // 16-byte aligned: zstride is a multiple of 4
  L.y = (L.y + 15u) / 16u * 16u;
  L.red = L.y + (uint32_t)(2 * R.dp) * 8u;  // FP64 y of a band row's trial and target
  L.total = L.red + 2u * 256u * 8u;         // FP64 terms of the band evaluation
  return L;
}

// VAR: the run uses a strategy variant or jDE (a separate instance, so that
// plain DE/rand/1/bin keeps its register allocation)
template <int ESZ, bool VAR>
__global__ void __launch_bounds__(256, 1)
    k_persist_cta(const RunDesc* __restrict__ runs, int run, PersistCtl* ctl, long long gens, int rows) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cta = (int)blockIdx.x, nct = (int)gridDim.x;
  // failure-detection test (off unless set by the launcher): this CTA leaves
  // out its first grid-barrier arrival and the barrier gives up after test_spin polls
  const bool test_skip = ctl->test_skip == cta + 1;
  const long long spin_limit = ctl->test_spin > 0 ? ctl->test_spin : kCtaGridSpin;
  // the run descriptor lives in shared memory for the whole launch
  __shared__ RunDesc sR;
  static_assert(sizeof(RunDesc) % 8 == 0, "descriptor copied in 8-byte words");
  for (int q = tid; q < (int)(sizeof(RunDesc) / 8); q += blockDim.x)
    reinterpret_cast<uint64_t*>(&sR)[q] = reinterpret_cast<const uint64_t*>(runs + run)[q];
  __syncthreads();
  const RunDesc& R = sR;
  RunState* st = R.st;
  const int d = R.d, dp = R.dp, np = R.np, obj = R.obj;
  const int row0 = cta * rows;
  const bool has_target = R.target > 0.0;
  const float target_f = (float)R.target * 1.001f, target_lo = (float)R.target * 0.999f;

  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ double s_f[kCtaRowsMax], s_ft[kCtaRowsMax];
  __shared__ float s_tau[kCtaRowsMax], s_yn[kCtaRowsMax];
  __shared__ uint8_t s_fx[kCtaRowsMax], s_flag[kCtaRowsMax];  // flag bit 0 accept, 1 decided in FP64, 2 pending FP64
  __shared__ int s_blist[kCtaRowsMax];
  __shared__ int s_nb, s_stop, s_abort, s_bidx, s_have, s_mfail;
  __shared__ long long s_gen;
  __shared__ double s_best;
  __shared__ float s_bestf;                 // s_best rounded to FP32 (the decisions run in FP32)
  __shared__ long long s_key[kCtaRowsMax];  // ordered key of s_f (best-partial scan)
  __shared__ unsigned long long s_nband_total;

  const CtaLayout L = cta_layout(R);
  const uint32_t y_part = cta_y_part(R), m_part = cta_m_part(R);
  uint8_t* sYop = smem + L.yop;  // B operand: split y of this CTA's targets
  uint8_t* sMop = smem + L.mop;  // A operand: split M
  const int zs = cta_zstride(R);
  float* zbuf = reinterpret_cast<float*>(smem + L.z);
  double* sY = reinterpret_cast<double*>(smem + L.y);  // [2][dp]: FP64 y of a band row's trial and target
  double* s_red = reinterpret_cast<double*>(smem + L.red);

  const uint32_t bar_mma = smem_u32(&s_bar[1]);
  // three accumulators of 128 lanes x 16 columns, one per split pass: warps
  // 0, 1 and 2 issue the passes at the same time (one thread issues a product
  // only every several tens of cycles); z is their sum in pass order.  The
  // split M, the A operand of every product of the launch, lives in tensor
  // memory from column kColA on (high part, then low part), so that a product
  // reads only its 512-byte B operand from shared memory instead of also the
  // 4 KB of A, which bounded the products at about 45 cycles each.
  constexpr uint32_t kColA = 64u, kColPart = ESZ == 2 ? 64u : 128u;
  constexpr uint32_t ncols = ESZ == 2 ? 256u : 512u;
  const uint32_t fmt = ESZ == 2 ? 1u : 2u;
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kCtaRowsMax >> 3) << 17) |
                         ((uint32_t)(kTileM >> 4) << 24);

  // ---------------------------------------------------------------- set-up
  if (tid == 0) {
    mbar_init(bar_mma, 3);  // one commit per issuing warp
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_gen = *(volatile int64_t*)&st->gen;
    s_stop = *(volatile int32_t*)&st->stop;
    s_best = *(volatile double*)&st->best_f;
    s_bestf = to_f32_rn(s_best);
    s_bidx = max(*(volatile int32_t*)&st->best_idx, 0);  // DE/best/1 base (row 0 when none is finite)
    s_abort = 0;
    s_mfail = 0;
    s_nband_total = 0;
    if (cta == 0) ctl->gen0 = s_gen;  // generation counter at launch, for the trial count
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // the y operand starts at zero (rows past this CTA's targets stay zero)
  for (uint32_t q = tid * 16u; q < L.mop; q += blockDim.x * 16u) *reinterpret_cast<uint4*>(smem + q) = make_uint4(0u, 0u, 0u, 0u);
  // the split M as the A operand: 128 rows (rows past ntn zero)
  cta_load_m<ESZ>(R, sMop, m_part);
  {
    const int cur0 = (int)(*(volatile int64_t*)&st->gen & 1);
    if (tid < kCtaRowsMax) {
      const int i = row0 + tid;
      const bool mine = tid < rows && i < np;
      s_f[tid] = mine ? R.f[cur0][i] : CUDART_INF;
      s_fx[tid] = mine ? R.fx[cur0][i] : 1;
      s_tau[tid] = mine ? R.tau[i] : 0.f;
      s_yn[tid] = 0.f;
      s_key[tid] = fit_key(s_f[tid]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  const uint32_t tmem = s_tmem;
  {
    // split M into tensor memory: row r of A (lane r) from the shared-memory
    // copy, one 16-byte k-group (4 columns) per store; warps w and w + 4
    // share lanes 32 (w mod 4) .. + 31 and take alternate k-groups
    const int q4 = warp & 3, r = 32 * q4 + lane;
    const int nkg = R.kpad * ESZ / 16;
    for (int part = 0; part < 2; ++part)
      for (int kg = warp >> 2; kg < nkg; kg += 2) {
        const uint4 v = *reinterpret_cast<const uint4*>(sMop + (uint32_t)part * m_part + (uint32_t)kg * 2048u +
                                                        (uint32_t)(r >> 3) * 128u + (uint32_t)(r & 7) * 16u);
        const uint32_t ta = tmem + ((uint32_t)(32 * q4) << 16) + kColA + (uint32_t)part * kColPart + 4u * (uint32_t)kg;
        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(ta), "r"(v.x), "r"(v.y),
                     "r"(v.z), "r"(v.w)
                     : "memory");
      }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }

  // Targets of this warp: local rows (warp - shift) + 8 q.  With at most 7
  // targets per CTA (plain DE/rand/1/bin) warp 0 has none: it reduces the
  // previous generation's best partials while the other warps build trials.
  const int shift = (!VAR && rows <= 7) ? 1 : 0;
  // per-warp registers: trial and current rows of this warp's targets, and the
  // lane's coordinates of the shift
  double tr[2][4], tx[2][4], osh[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int j = 4 * lane + e;
    osh[e] = j < d ? R.o[j] : 0.0;
  }
  long long gen = s_gen;
  bool abort = s_abort != 0;
  bool reduce_pending = false;  // partials of generation gen still to reduce
  bool rows_in_regs = false;    // tx holds the current rows (after the first generation of a launch)
  bool have_next = false;       // nts / nu hold the draws of generation gen + 1
  TrialSetup nts[2];            // plain DE: r1, r2, r3, j_rand of the next generation
  U32x4 nu[2];                  // ... and the lane's crossover block
  unsigned nbar = 0;            // grid barriers passed in this launch
  uint32_t mma_phase = 0;

  for (long long itg = 0;; ++itg) {
    const int64_t g = gen + 1;
    const int cur = (int)(gen & 1), nxt = cur ^ 1;
    const double* __restrict__ X = R.X[cur];
    double* __restrict__ Xn = R.X[nxt];
    const double* jFc = VAR && R.jde ? R.jF[cur] : nullptr;
    const double* jCRc = VAR && R.jde ? R.jCR[cur] : nullptr;
    const bool more = itg < gens && !abort;

    // ---- 0. best record and stop rule of generation gen, whose partials are
    // complete (the grid barrier passed): warp 0, the same order in every CTA
    if (reduce_pending && warp == 0) {
      Best b;
      b.init();
      const BestPartial* pp = R.part + (size_t)(gen & 1) * nct;
      for (int t = lane; t < nct; t += 32) b.offer(__ldcg(&pp[t].f), __ldcg(&pp[t].idx));
      b.warp_reduce();
      if (lane == 0) {
        const double bf = b.f;
        const int bi = b.i;
        const int64_t evals = (int64_t)np * (1 + gen);  // the initial population counts as NP evaluations
        int sp = 0;
        if (R.target > 0.0 && bi >= 0 && bf < R.target) sp = 1;
        else if (R.max_evals > 0 && evals >= R.max_evals) sp = 2;
        else if (gen >= R.max_gens) sp = 3;
        s_stop = sp;
        s_best = bf;
        s_bestf = to_f32_rn(bf);
        if (bi >= 0) s_bidx = bi;
        s_gen = gen;
        if (cta == 0) {
          // one writer of the run state; evals are published at the end
          st->best_f = bf;
          st->best_idx = bi;
          st->gen = gen;
          st->stop = sp;
          if (bi < 0) atomicOr(&st->err, kErrNonFinite);
        }
      }
    }
    reduce_pending = false;
    // the variants need the best record before their trials (DE/best/1
    // base), and a debug capture must not record trials of a generation that
    // the stop rule cancels: both take the stop decision first
    const bool ordered = VAR || R.dbg_trial != nullptr;
    if (ordered || !more) __syncthreads();
    if (!more) break;
    if (ordered && s_stop) break;
    if (tid == 0) {
      s_nb = 0;
      s_have = 1;  // cleared by warp 0 or 4 when its wait for the products gives up
    }

    // ---- 1. trials of this CTA's targets -> registers and the A operand;
    // the loads of both of a warp's targets are issued before either is used
    {
      TrialSetup ts[2];
      ChunkIn cin[2];
      TrialVar tv[2];
      bool valid[2];
      const int j0 = 4 * lane;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int lr = warp - shift + 8 * q;
        const int i = row0 + lr;
        valid[q] = warp >= shift && lr < rows && i < np;
        if (!valid[q]) continue;
        if constexpr (VAR) {
          ts[q] = trial_setup_var(R, (uint32_t)i, g, lane, s_bidx, jFc, jCRc, tv[q]);
          if (j0 < d) trial_load(R, X, ts[q], (uint32_t)i, g, j0, cin[q]);
        } else {
          // the draws were made while this CTA waited at the last grid barrier
          ts[q] = have_next ? nts[q] : trial_setup(R, (uint32_t)i, g, lane, 0u, false);
          if (R.dbg_idx && lane == 0) {
            R.dbg_idx[3 * i + 0] = (int32_t)ts[q].r1;
            R.dbg_idx[3 * i + 1] = (int32_t)ts[q].r2;
            R.dbg_idx[3 * i + 2] = (int32_t)ts[q].r3;
            R.dbg_jrand[i] = (int32_t)ts[q].jr;
          }
          if (j0 < d) {
            cin[q].u = have_next ? nu[q]
                                 : draw_block(R.seed, kPurposeStep, R.run_id, 0u, (uint32_t)g, (uint32_t)i, 1u + lane);
            const double* rows3[3] = {X + (size_t)ts[q].r1 * dp + j0, X + (size_t)ts[q].r2 * dp + j0,
                                      X + (size_t)ts[q].r3 * dp + j0};
            double* dst[3] = {cin[q].x1, cin[q].x2, cin[q].x3};
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              const double2 a = __ldcg(reinterpret_cast<const double2*>(rows3[r]));
              const double2 b2 = __ldcg(reinterpret_cast<const double2*>(rows3[r] + 2));
              dst[r][0] = a.x;
              dst[r][1] = a.y;
              dst[r][2] = b2.x;
              dst[r][3] = b2.y;
            }
            if (rows_in_regs) {
              // the target is the row this warp wrote in the last generation
#pragma unroll
              for (int e = 0; e < 4; ++e) cin[q].xi[e] = tx[q][e];
            } else {
              const double2 a = __ldcg(reinterpret_cast<const double2*>(X + (size_t)i * dp + j0));
              const double2 b2 = __ldcg(reinterpret_cast<const double2*>(X + (size_t)i * dp + j0 + 2));
              cin[q].xi[0] = a.x;
              cin[q].xi[1] = a.y;
              cin[q].xi[2] = b2.x;
              cin[q].xi[3] = b2.y;
            }
          }
        }
      }
      // compiled twice, for a unit domain scale (no multiplication on the
      // FP64 pipe) and any other
      auto build = [&](auto unit) {
      constexpr bool UNIT = decltype(unit)::value;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (!valid[q]) continue;
        const int lr = warp - shift + 8 * q;
        const int i = row0 + lr;
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        uint32_t bits = 0;
        if (j0 < d) {
          if constexpr (VAR) bits = trial_compute(R, ts[q], j0, cin[q], t, tv[q].F, tv[q].thr, tv[q].L);
          else bits = trial_compute(R, ts[q], j0, cin[q], t);
#pragma unroll
          for (int e = 0; e < 4; ++e) tx[q][e] = cin[q].xi[e];
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) tr[q][e] = t[e];
        float yn2 = 0.f;
        if (j0 < R.kpad) {
          float y[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            y[e] = (j0 + e < d) ? to_f32_rn(shifted_as<UNIT>(t[e], osh[e], R.scale)) : 0.f;
            yn2 += y[e] * y[e];
          }
          cta_store_split4<ESZ>(sYop, y_part, lr, j0, y);
        }
        if (R.dbg_trial) trial_debug(R, (uint32_t)i, j0, lane, bits, t);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) yn2 += __shfl_xor_sync(0xffffffffu, yn2, o);
        if (lane == 0) s_yn[lr] = sqrtf(yn2);
      }
      };
      if (R.unit_scale) build(std::true_type{});
      else build(std::false_type{});
    }
    // generic-proxy writes of A become visible to the tensor cores' async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // otherwise the stop rule of generation gen was reduced meanwhile; a
    // stopped run leaves before anything of generation g is written
    if (!ordered && s_stop) break;
    const float bp = s_bestf;

    // ---- 2. split products on tcgen05: z = Mh yh + Ml yh + Mh yl, M as the
    // 128-row A operand and the targets' y as the 16-row B operand
    if (warp < 3 && lane == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int ksteps = R.kpad * ESZ / 32;
      const int pass = warp;
      // descriptors of the operands' first K step; a byte offset enters the
      // 14-bit address field (16-byte units) and never carries out of it
      // A in tensor memory: a K step (two k-groups) is 8 columns
      const uint32_t ta = tmem + kColA + (pass == 1 ? kColPart : 0u);
      const uint64_t dy = smem_desc(smem_u32(sYop) + (pass == 2 ? y_part : 0u), 256u, 128u);
      for (int ks = 0; ks < ksteps; ++ks)
        mma_split_ta<ESZ>(tmem + 16u * (uint32_t)pass, ta + 8u * (uint32_t)ks, dy + (uint64_t)(ks * 32), idesc,
                          ks > 0 ? 1u : 0u);
      mma_commit(bar_mma);
    }
    // ---- 3a. every warp copies one block of the accumulator (TMEM lanes
    // 32 (w mod 4) .. + 31 = coordinates j, columns 8 (w / 4) .. + 7 = targets)
    // to shared memory as rows of z
    {
      const bool ok = mbar_wait(bar_mma, mma_phase);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const bool have_w = __all_sync(0xffffffffu, ok);
      if (have_w) {
        float v[8], w1[8], w2[8];
        const int q = warp & 3, cb = (warp >> 2) * 8;
        const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)cb;
        tmem_ld8(ta, v);
        tmem_ld8(ta + 16u, w1);
        tmem_ld8(ta + 32u, w2);
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (v[e] + w1[e]) + w2[e];
        const int j = 32 * q + lane;
        if (j < d) {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (cb + e < rows) zbuf[(size_t)(cb + e) * zs + j] = v[e];
        }
      } else if (lane == 0) {
        atomicOr(&st->err, kErrTimeout);
        atomicExch(&ctl->abort, 1);
        s_abort = 1;
        s_have = 0;
        s_mfail = 1 + (int)mma_phase;  // the phase whose products may still be in flight, plus one
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    mma_phase ^= 1u;
    __syncthreads();

    // ---- 3b. FP32 objective of every target (16 threads per row) and the
    // selections the split error bound decides
    const bool have = s_have != 0;
    {
      const int rr = tid >> 4, sub = tid & 15;
      const int i = row0 + rr;
      const bool valid = rr < rows && i < np;
      EpiAcc acc_{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (valid && have) epi_strided_dispatch(obj, zbuf + (size_t)rr * zs, sub, d, acc_);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        acc_.a1 += __shfl_xor_sync(0xffffffffu, acc_.a1, o);
        acc_.aS += __shfl_xor_sync(0xffffffffu, acc_.aS, o);
        acc_.aG += __shfl_xor_sync(0xffffffffu, acc_.aG, o);
      }
      if (obj == kObjAckley) {  // the other objectives leave these two at zero
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          acc_.a2 += __shfl_xor_sync(0xffffffffu, acc_.a2, o);
          acc_.a3 += __shfl_xor_sync(0xffffffffu, acc_.a3, o);
        }
      }
      if (sub == 0) {
        uint8_t flag = 0;
        if (valid && have) {
          const float s1 = acc_.a1, s2 = acc_.a2, s3 = acc_.a3;
          float S = acc_.aS, G = acc_.aG;
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
          // FP32 throughout; the FP64 values are converted on the integer
          // pipe (the FP64 pipe is the trial construction's bottleneck)
          const float tau = 2.f * R.band_u * G * R.rownorm * s_yn[rr] + (float)d * 0x1.0p-21f * S + 1e-30f;
          const float fif = to_f32_rn(s_f[rr]);
          const float tif = s_fx[rr] ? 0.f : s_tau[rr];
          const float mrg = 0x1.0p-22f * fabsf(fif);
          const bool sure_reject = fs - tau > fif + tif + mrg;
          const bool sure_accept = fs + tau < fif - tif - mrg;
          const bool ambiguous = !sure_reject && !sure_accept;
          const bool may_be_best = R.band_all && fs - tau <= bp + 0x1.0p-22f * fabsf(bp);
          const bool near = fs - tau <= R.near_thr || fif - tif <= R.near_thr;
          // only a trial the split bound cannot place on one side of the stop
          // target needs FP64 for the stop rule: surely below (or above)
          // decides it as well
          const bool may_stop = has_target && fs - tau < target_f && !(fs + tau < target_lo);
          const double fsd = f64_of_f32(fs);
          s_ft[rr] = fsd;
          if ((ambiguous && (R.band_all || near)) || may_be_best || may_stop || !(fs == fs) || !(fif == fif)) {
            s_blist[atomicAdd(&s_nb, 1)] = rr;
            flag = 4;
          } else if (sure_accept || (ambiguous && fs <= fif)) {
            // decided on the split values (an undecidable comparison far from
            // the optimum goes to the smaller split value, ties to the trial)
            flag = 1;
            s_f[rr] = fsd;
            s_key[rr] = fit_key(fsd);
            s_fx[rr] = 0;
            s_tau[rr] = tau;
          }
        }
        s_flag[rr] = flag;
      }
    }
    __syncthreads();

    // ---- 3c. FP64 decisions of the listed targets (listing order), by the
    // whole CTA; the owning warp publishes the FP64 y vectors
    const int nb = s_nb;
    for (int b = 0; b < nb; ++b) {
      const int lr = s_blist[b];
      const bool need_t = !s_fx[lr];
      if ((lr & 7) + shift == warp) {
        const int q = lr >> 3;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 4 * lane + e;
          if (j >= d) continue;
          sY[j] = shifted(q ? tr[1][e] : tr[0][e], osh[e], R);
          if (need_t) sY[dp + j] = shifted(q ? tx[1][e] : tx[0][e], osh[e], R);
        }
      }
      __syncthreads();
      const double ft = cta_fitness_fp64(R, sY, s_red);
      const double fi = need_t ? cta_fitness_fp64(R, sY + dp, s_red) : s_f[lr];
      if (tid == 0) {
        const bool acc = fit_key(ft) <= fit_key(fi) && fit_key(ft) != 0x7FFFFFFFFFFFFFFFLL;  // NaN ranks last
        s_ft[lr] = ft;
        s_f[lr] = acc ? ft : fi;
        s_key[lr] = fit_key(acc ? ft : fi);
        s_fx[lr] = 1;
        s_tau[lr] = 0.f;
        s_flag[lr] = (acc ? 1 : 0) | 2;
      }
      __syncthreads();
    }
    if (tid == 0) s_nband_total += (unsigned long long)nb;  // published once, at the end of the launch

    // ---- 4. next-generation rows (they stay in registers as the next
    // targets), debug capture, best partial
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int lr = warp - shift + 8 * q;
      const int i = row0 + lr;
      if (warp < shift || lr >= rows || i >= np) continue;
      const bool acc = s_flag[lr] & 1;
      if (VAR && R.jde && lane == 0) {
        // jDE: an accepted trial passes its F_i and CR_i on
        double Fi = __ldcg(jFc + i), CRi = __ldcg(jCRc + i);
        if (acc) jde_params(R, (uint32_t)i, g, jFc, jCRc, Fi, CRi);
        R.jF[nxt][i] = Fi;
        R.jCR[nxt][i] = CRi;
      }
      if (acc) {
#pragma unroll
        for (int e = 0; e < 4; ++e) tx[q][e] = tr[q][e];
      }
      const int j0 = 4 * lane;
      if (j0 < d) {
        double* dst = Xn + (size_t)i * dp + j0;
        *reinterpret_cast<double2*>(dst) = make_double2(tx[q][0], tx[q][1]);
        *reinterpret_cast<double2*>(dst + 2) = make_double2(tx[q][2], tx[q][3]);
      }
    }
    rows_in_regs = true;
    if (tid == 0) {
      // the CTA's best (lowest key, then lowest index; NaN never): a scan of
      // at most 16 precomputed keys
      long long bk = 0x7FFFFFFFFFFFFFFFLL;
      int bi = -1;
      for (int r = 0; r < rows && row0 + r < np; ++r)
        if (s_key[r] != 0x7FFFFFFFFFFFFFFFLL && (bi < 0 || s_key[r] < bk)) {
          bk = s_key[r];
          bi = r;
        }
      BestPartial* pp = R.part + (size_t)(g & 1) * nct + cta;
      pp->f = bi >= 0 ? s_f[bi] : CUDART_INF;
      pp->idx = bi >= 0 ? row0 + bi : -1;
    }
    if (R.dbg_ftrial && warp == 0 && lane < rows && row0 + lane < np) {
      const int i = row0 + lane;
      R.dbg_ftrial[i] = s_ft[lane];
      R.dbg_accept[i] = s_flag[lane] & 1;
      R.dbg_fp64[i] = (s_flag[lane] >> 1) & 1;
    }
    __syncthreads();  // every row and the partial are written

    // ---- 5. grid barrier on one arrival counter.  Warp 0 arrives and polls
    // the count with one load in flight and no pause; the other warps draw
    // the next generation's indices, j_rand and crossover blocks meanwhile
    // (they depend on (seed, generation, target) only).  Measured: reading
    // the abort flag after every poll doubled the round trips per poll (it
    // is read every 16th), more polling warps crowd the counter's L2 slice,
    // which also takes the arrivals, and relaxed polls with one acquire fence
    // after them cost more than acquire polls.
    if (warp == 0 && s_abort == 0) {
      if (lane == 0 && !(test_skip && nbar == 0)) {
        // release: this CTA's rows and partial (ordered before by the CTA
        // barrier) are visible to every CTA that observes the count
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(&ctl->sbar[0]), "r"(1u) : "memory");
      }
      const unsigned target = (nbar + 1u) * (unsigned)nct;
      bool ok = false;
      for (long long k = 0; k < spin_limit; ++k) {
        unsigned v = 0u;
        if (lane == 0) asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&ctl->sbar[0]) : "memory");
        if (__shfl_sync(0xffffffffu, v, 0) >= target) {
          ok = true;
          break;
        }
        if ((k & 15) == 15 && *(volatile int*)&ctl->abort) break;
      }
      if (!ok && lane == 0) {
        if (!*(volatile int*)&ctl->abort) {
          atomicExch(&ctl->abort, 1);
          atomicOr(&st->err, kErrTimeout);
        }
        s_abort = 1;
      }
    }
    if (!VAR) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int lr = warp - shift + 8 * q;
        const int i = row0 + lr;
        if (warp < shift || lr >= rows || i >= np) continue;
        nts[q] = trial_setup(R, (uint32_t)i, g + 1, lane, 0u, false);
        nu[q] = draw_block(R.seed, kPurposeStep, R.run_id, 0u, (uint32_t)(g + 1), (uint32_t)i, 1u + lane);
      }
    }
    have_next = !VAR;
    ++nbar;
    __syncthreads();
    abort = s_abort != 0;
    if (abort) break;
    gen = g;
    reduce_pending = true;
  }

  // ---------------------------------------------------------------- teardown
  if (tid == 0) atomicAdd(&R.stats[0], s_nband_total);
  {
    const int curf = (int)(gen & 1);
    if (tid < rows && row0 + tid < np) {
      const int i = row0 + tid;
      R.f[curf][i] = s_f[tid];
      R.fx[curf][i] = s_fx[tid];
      R.tau[i] = s_tau[tid];
    }
  }
  // copies and products still in flight after a failed wait must land
  // before the CTA leaves and frees its tensor memory (bounded waits)
  if (tid == 0 && s_mfail) mbar_wait(bar_mma, (uint32_t)(s_mfail - 1));
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ------------------------------------------------------------------ host side
template <int ESZ, bool VAR>
static const void* cta_kernel() {
  return (const void*)k_persist_cta<ESZ, VAR>;
}

static const void* cta_kernel(int prec, bool var) {
  if (prec == DE_PREC_BF16X3) return var ? cta_kernel<2, true>() : cta_kernel<2, false>();
  return var ? cta_kernel<4, true>() : cta_kernel<4, false>();
}

bool persist_cta_plan(PersistPlan& pp, const RunDesc& R, int nruns, int prec) {
  pp.cta_ok = false;
  // one run, one N tile of at most 128 columns, rows of at most 128
  // coordinates (one 4-coordinate chunk per lane); the whole split M is
  // copied into shared memory (the three-kernel path's K chunking does not apply)
  if (nruns != 1 || R.nn != 1 || R.d > 128 || R.ntn > 128) return false;
  const size_t smem = cta_layout(R).total;
  if (smem > 220 * 1024) return false;
  const bool var = R.strategy != 0 || R.jde;
  const void* k = cta_kernel(prec, var);
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return false;
  }
  // tensor memory: 256 columns a CTA (BF16x3: accumulators and the split M)
  // or 512 (TF32x3) of the SM's 512, so at most 2 or 1 resident CTAs
  per_sm = std::min(per_sm, prec == DE_PREC_BF16X3 ? 2 : 1);
  pp.cta_cap = per_sm * nsm;
  pp.cta_smem = smem;
  // first choice: the fewest targets per CTA that keep every CTA resident
  int rows = std::max(1, (R.np + pp.cta_cap - 1) / pp.cta_cap);
  if (rows > kCtaRowsMax) return false;
  if (const char* env = getenv("DE_GB300_PERSIST_CTA_ROWS")) {
    const int v = atoi(env);
    if (v >= 1 && v <= kCtaRowsMax) rows = v;
  }
  if (!persist_cta_set_rows(pp, R, rows)) return false;
  pp.cta_ok = true;
  pp.prec = prec;
  pp.var = var;
  return true;
}

bool persist_cta_set_rows(PersistPlan& pp, const RunDesc& R, int rows) {
  if (rows < 1 || rows > kCtaRowsMax) return false;
  const int ntiles = (R.np + rows - 1) / rows;
  if (ntiles > pp.cta_cap) return false;
  pp.cta_rows = rows;
  pp.cta_ntiles = ntiles;
  return true;
}

cudaError_t persist_cta_launch(const PersistPlan& pp, const RunDesc* runs, PersistCtl* ctl, long long gens,
                               cudaStream_t s, int test_skip) {
  cudaError_t e = persist_ctl_reset(ctl, test_skip, s);
  if (e != cudaSuccess) return e;
  int run = 0, rows = pp.cta_rows;
  void* args[] = {(void*)&runs, (void*)&run, (void*)&ctl, (void*)&gens, (void*)&rows};
  e = cudaLaunchCooperativeKernel(cta_kernel(pp.prec, pp.var), dim3((unsigned)pp.cta_ntiles), dim3(256), args,
                                  pp.cta_smem, s);
  if (e != cudaSuccess) return e;
  k_persist_close_launch(runs, ctl, s);
  return cudaGetLastError();
}

}  // namespace de
