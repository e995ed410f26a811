// de_persist.cu -- the split-precision generation loop as one persistent
// kernel built on thread-block clusters.
//
// A cluster of C CTAs (one per SM) owns one 128-row tile of the population;
// the cluster's CTA 0 (the leader) holds the tile's tensor-core operands in
// shared memory, its accumulator in tensor memory, and the FP64 fitness state
// of its 128 targets.  One generation:
//
//   1. every CTA of the cluster builds 128 / C trials (Eq. 2, Eq. 3, bound
//      repair; FP64, warp per target, as in the other paths), keeps the trial
//      and target rows in registers, and writes the split operand rows and
//      |y| straight into the leader's shared memory (distributed shared
//      memory);
//   2. cluster barrier; the leader runs the three split products on tcgen05
//      (M is resident in its shared memory for the whole launch) and sends
//      each accumulator row from TMEM to the CTA that owns the target;
//      after a second cluster barrier every CTA evaluates the objective terms
//      of its rows in FP32 and decides every selection the split-precision
//      bound allows, on the leader's tile state;
//   3. rows it cannot decide (and trials that could become the best) are
//      re-evaluated in FP64: their owners publish y to the leader, the other
//      CTAs of the cluster each compute a block of z = M y and its objective
//      terms, and the leader sums the partials in a fixed order and decides;
//   4. every CTA writes its targets' next-generation rows (trial or target,
//      from registers) to the other population buffer (double buffering: no
//      cluster can overwrite a row another cluster still reads as a donor);
//   5. the leaders meet at a grid-wide barrier (bounded spin on a global
//      counter), reduce the per-tile best partials (double buffered by
//      generation parity) into the best record and evaluate the stop rule of
//      Sec. 7.3.4; every CTA takes the same decision.
//
// All clusters must be resident at once: the host launches this path only
// when the occupancy query says they are, and every wait is bounded (on
// expiry the kernel records kErrTimeout, the leaders agree on an abort through
// a global flag, and every CTA leaves at the same point of the loop).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cstdlib>
#include <cstring>

#include "de_device.cuh"
#include "de_kernels.h"
#include "de_tcgen05.cuh"

namespace cg = cooperative_groups;

namespace de {

constexpr int kPBandMax = 4;              // band rows per exchange round
constexpr int kPC = 8;                    // CTAs per cluster
constexpr int kPMaxC = 16;                // largest cluster
constexpr long long kGridSpin = 1LL << 22;  // polls of the grid barrier (each a round trip to L2: seconds in all)

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Arrival of one CTA at the grid barrier: its writes before the call are
// released to every CTA that sees the count.
__device__ __forceinline__ void grid_arrive(PersistCtl* ctl) {
  __threadfence();
  atomicAdd(&ctl->bar, 1u);
}

// Wait until `target` CTAs have arrived at the grid barrier (called by a
// whole warp: every lane reads the same counter in the same instruction, so
// all of them leave the loop together); at most `spin` polls, each a round
// trip to L2 with no pause (the abort flag is read every 16th: a read after
// every poll doubled the round trips per poll).
__device__ bool grid_wait(PersistCtl* ctl, unsigned target, long long spin) {
  for (long long k = 0; k < spin; ++k) {
    if (ld_acquire_u32(&ctl->bar) >= target) return true;
    if ((k & 15) == 15 && *(volatile int*)&ctl->abort) return false;
  }
  atomicExch(&ctl->abort, 1);
  return false;
}

// Row stride (floats) of the accumulator rows a CTA receives: at least the
// N extent, and 4 mod 8 so that the leader's 16-byte stores of 32 rows at a
// time spread over all banks.
__host__ __device__ inline int persist_zstride(const RunDesc& R) { return R.ntn + ((12 - R.ntn % 8) % 8); }

// Byte offset of those rows in the kernel's dynamic shared memory.  The
// leader keeps them in its A operand (free once the products are complete;
// the other CTAs write the next operands only after the generation's last
// cluster barrier), the other CTAs after their own layout (rows of M, band
// vectors, reduction scratch).
__host__ __device__ inline size_t persist_z_offset(const RunDesc& R, int C, bool leader) {
  if (leader) return (size_t)R.b_tile_bytes;
  const int cwp = (R.d + C - 2) / (C - 1);
  const size_t member = ((size_t)(cwp + 1) * R.d + (size_t)2 * kPBandMax * R.dp + 16 * 17 + 17) * sizeof(double);
  return (member + 15) / 16 * 16;
}

// NCH: 128-coordinate chunks per row (1 for d <= 128, 2 for d <= 256);
// VAR: the run uses a strategy variant or jDE (a separate instance, so that
// plain DE/rand/1/bin keeps its register allocation)
template <int ESZ, int NCH, bool VAR>
__global__ void __launch_bounds__(256, 1)
    k_persist(const RunDesc* __restrict__ runs, int run, PersistCtl* ctl, long long gens, int prows) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int crank = (int)cluster.block_rank();
  const bool leader = crank == 0;
  const int tile = (int)blockIdx.x / C;
  const int nclusters = (int)gridDim.x / C;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // failure-detection test (off unless set by the launcher): this CTA leaves
  // out its first grid-barrier arrival and the waits give up after test_spin polls
  const bool test_skip = ctl->test_skip == (int)blockIdx.x + 1;
  const long long spin_limit = ctl->test_spin > 0 ? ctl->test_spin : kGridSpin;
  // the run descriptor lives in shared memory for the whole launch: its fields
  // are read in every phase, after barriers that would force global reloads
  __shared__ RunDesc sR;
  static_assert(sizeof(RunDesc) % 8 == 0, "descriptor copied in 8-byte words");
  for (int q = tid; q < (int)(sizeof(RunDesc) / 8); q += blockDim.x)
    reinterpret_cast<uint64_t*>(&sR)[q] = reinterpret_cast<const uint64_t*>(runs + run)[q];
  __syncthreads();
  const RunDesc& R = sR;
  RunState* st = R.st;
  const int d = R.d, dp = R.dp, np = R.np, obj = R.obj;
  // prows targets per cluster (a multiple of C, at most 128; rows past prows
  // of the MMA tile stay zero); CTA r holds rows r rpm .. r rpm + rpm - 1 and
  // warp w of it rows w and w + 8 of those
  const int kPRows = prows;
  const int row0 = tile * kPRows;
  const int rpm = kPRows / C;  // rows per CTA, at most 16

  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ uint32_t s_tmem;
  // leader: tile state
  __shared__ double s_f[kTileM];
  __shared__ double s_ft[kTileM];
  __shared__ float s_tau[kTileM];
  __shared__ float s_yn[kTileM];
  __shared__ uint8_t s_fx[kTileM];
  __shared__ uint8_t s_flag[kTileM];  // bit 0 accept, bit 1 decided in FP64, bit 2 pending FP64
  __shared__ int s_blist[kTileM];
  __shared__ double s_bpart[2 * kPBandMax][kPMaxC][2];
  __shared__ int s_nb, s_stop, s_abort, s_bidx, s_have;
  __shared__ long long s_gen;
  __shared__ double s_best;
  __shared__ double s_bf[8];
  __shared__ long long s_bk[8];
  __shared__ int s_bi[8];
  __shared__ unsigned long long s_nband_total;

  const uint32_t a_part = (uint32_t)(R.a_tile_bytes / 2), b_part = (uint32_t)(R.b_tile_bytes / 2);
  uint8_t* sB = smem;
  uint8_t* sA = smem + 2 * b_part;
  double* sY = reinterpret_cast<double*>(sA + 2 * a_part);  // leader: band vectors [2 kPBandMax][dp]
  double* sM = reinterpret_cast<double*>(smem);            // other CTAs: their rows of M
  const int cwp = (d + C - 2) / (C - 1);                    // band columns per non-leader CTA (<= 15)
  double* sYm = sM + (size_t)(cwp + 1) * d;                 // other CTAs: band vectors [2 kPBandMax][dp]
  double (*s_red)[17] = reinterpret_cast<double (*)[17]>(sYm + (size_t)2 * kPBandMax * dp);  // [16][17]
  double* s_zb = reinterpret_cast<double*>(s_red + 16);     // 17 outputs of the band block

  // views of the leader's shared memory
  uint8_t* lA = cluster.map_shared_rank(sA, 0);
  float* l_yn = cluster.map_shared_rank(s_yn, 0);
  double* lY = cluster.map_shared_rank(sY, 0);
  int* l_nb = cluster.map_shared_rank(&s_nb, 0);
  int* l_blist = cluster.map_shared_rank(s_blist, 0);
  uint8_t* l_flag = cluster.map_shared_rank(s_flag, 0);
  uint8_t* l_fx = cluster.map_shared_rank(s_fx, 0);
  double* l_bpart = cluster.map_shared_rank(&s_bpart[0][0][0], 0);
  int* l_stop = cluster.map_shared_rank(&s_stop, 0);
  int* l_abort = cluster.map_shared_rank(&s_abort, 0);
  double* l_best = cluster.map_shared_rank(&s_best, 0);
  int* l_bidx = cluster.map_shared_rank(&s_bidx, 0);
  long long* l_gen = cluster.map_shared_rank(&s_gen, 0);
  double* l_f = cluster.map_shared_rank(s_f, 0);
  double* l_ft = cluster.map_shared_rank(s_ft, 0);
  float* l_tau = cluster.map_shared_rank(s_tau, 0);
  int* l_have = cluster.map_shared_rank(&s_have, 0);
  // every CTA: the FP32 accumulator rows of its targets (written by the
  // leader), after both layouts above
  const int zs = persist_zstride(R);
  const size_t zoff_lead = persist_z_offset(R, C, true), zoff_member = persist_z_offset(R, C, false);
  float* zbuf = reinterpret_cast<float*>(smem + (leader ? zoff_lead : zoff_member));

  const uint32_t bar_b = smem_u32(&s_bar[0]), bar_mma = smem_u32(&s_bar[1]);
  const uint32_t ncols = R.ntn <= 32 ? 32u : (R.ntn <= 64 ? 64u : (R.ntn <= 128 ? 128u : 256u));
  const uint32_t fmt = ESZ == 2 ? 1u : 2u;
  const uint32_t idesc =
      (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(R.ntn >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
  const uint32_t bk = (uint32_t)(R.ntn / 8) * 128u;

  // ---------------------------------------------------------------- set-up
  if (leader) {
    if (tid == 0) {
      mbar_init(bar_b, 1);
      mbar_init(bar_mma, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      s_gen = *(volatile int64_t*)&st->gen;
      s_stop = *(volatile int32_t*)&st->stop;
      s_best = *(volatile double*)&st->best_f;
      s_bidx = max(*(volatile int32_t*)&st->best_idx, 0);  // DE/best/1 base (row 0 when none is finite)
      s_abort = 0;
      s_nband_total = 0;
      if (blockIdx.x == 0) ctl->gen0 = s_gen;  // generation counter at launch, for the trial count
    }
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                   "r"(ncols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // rows of the tile past the population end start at zero in the operand
    // (their products are never read; the leader's accumulator rows later
    // reuse the start of this region)
    for (uint32_t q = tid * 16u; q < 2u * a_part; q += blockDim.x * 16u)
      *reinterpret_cast<uint4*>(sA + q) = make_uint4(0u, 0u, 0u, 0u);
    const int cur0 = (int)(*(volatile int64_t*)&st->gen & 1);
    for (int m = tid; m < kTileM; m += blockDim.x) {
      const int i = row0 + m;
      const bool mine = m < kPRows && i < np;
      s_f[m] = mine ? R.f[cur0][i] : CUDART_INF;
      s_fx[m] = mine ? R.fx[cur0][i] : 1;
      s_tau[m] = mine ? R.tau[i] : 0.f;
      s_yn[m] = 0.f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      // M split stays resident for the whole launch
      mbar_expect_tx(bar_b, 2 * b_part);
      bulk_g2s(smem_u32(sB), R.B, b_part, bar_b);
      bulk_g2s(smem_u32(sB) + b_part, R.B + b_part, b_part, bar_b);
      if (!mbar_wait(bar_b, 0u)) {
        atomicOr(&st->err, kErrTimeout);
        s_abort = 1;
      }
    }
  } else if (R.rotate) {
    // this CTA's rows of M for the FP64 band products
    const int j0 = (crank - 1) * cwp;
    const int nr = max(0, min(cwp + 1, d - j0));
    for (int q = tid; q < nr * d; q += blockDim.x) sM[q] = R.Mrow[(size_t)j0 * d + q];
  }
  cluster.sync();
  const uint32_t tmem = leader ? s_tmem : 0u;

  // per-warp registers: trial and target rows of this warp's targets, and the
  // lane's coordinates of the shift
  double tr[2][NCH][4], tx[2][NCH][4], osh[NCH][4];
#pragma unroll
  for (int c = 0; c < NCH; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = 128 * c + 4 * lane + e;
      osh[c][e] = j < d ? R.o[j] : 0.0;
    }
  long long gen = *l_gen;
  int stop = *l_stop;
  double best_prev = *l_best;
  int best_idx = *l_bidx;
  bool abort = *l_abort != 0;

  for (long long itg = 0; itg < gens && !stop && !abort; ++itg) {
    const int64_t g = gen + 1;
    const int cur = (int)(gen & 1), nxt = cur ^ 1;
    const double* __restrict__ X = R.X[cur];
    double* __restrict__ Xn = R.X[nxt];
    const double* jFc = VAR && R.jde ? R.jF[cur] : nullptr;
    const double* jCRc = VAR && R.jde ? R.jCR[cur] : nullptr;

    // ---- 1. trials of this CTA's rows -> registers and the leader's operand tile;
    // all loads of the warp's rows are issued before any of them is used
    constexpr int QB = NCH == 1 ? 2 : 1;  // rows whose loads are in flight together
#pragma unroll
    for (int qb = 0; qb < 2; qb += QB) {
      TrialSetup ts[2];
      ChunkIn cin[2][NCH];
      TrialVar tv[2];
      bool valid[2] = {false, false};
#pragma unroll
      for (int q = qb; q < qb + QB; ++q) {
        const int i = row0 + crank * rpm + warp + 8 * q;
        valid[q] = warp + 8 * q < rpm && i < np;
        if (valid[q]) {
          if constexpr (VAR) ts[q] = trial_setup_var(R, (uint32_t)i, g, lane, best_idx, jFc, jCRc, tv[q]);
          else ts[q] = trial_setup(R, (uint32_t)i, g, lane);
#pragma unroll
          for (int c = 0; c < NCH; ++c) {
            const int j0 = 128 * c + 4 * lane;
            if (j0 < d) trial_load(R, X, ts[q], (uint32_t)i, g, j0, cin[q][c]);
          }
        }
      }
      // compiled twice, for a unit domain scale (no multiplication on the
      // FP64 pipe) and any other
      auto build = [&](auto unit) {
      constexpr bool UNIT = decltype(unit)::value;
#pragma unroll
      for (int q = qb; q < qb + QB; ++q) {
        if (!valid[q]) continue;
        const int lr = crank * rpm + warp + 8 * q;
        const int i = row0 + lr;
        float yn2 = 0.f;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          const int j0 = 128 * c + 4 * lane;
          double t[4] = {0.0, 0.0, 0.0, 0.0};
          uint32_t bits = 0;
          if (j0 < d) {
            if constexpr (VAR) bits = trial_compute(R, ts[q], j0, cin[q][c], t, tv[q].F, tv[q].thr, tv[q].L);
            else bits = trial_compute(R, ts[q], j0, cin[q][c], t);
#pragma unroll
            for (int e = 0; e < 4; ++e) tx[q][c][e] = cin[q][c].xi[e];
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) tr[q][c][e] = t[e];
          if (j0 < R.kpad) {
            float y[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              y[e] = (j0 + e < d) ? to_f32_rn(shifted_as<UNIT>(t[e], osh[c][e], R.scale)) : 0.f;
              yn2 += y[e] * y[e];
            }
            store_split4<ESZ>(lA, a_part, lr, j0, y);
          }
          if (R.dbg_trial) trial_debug(R, (uint32_t)i, j0, lane, bits, t);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) yn2 += __shfl_xor_sync(0xffffffffu, yn2, o);
        if (lane == 0) l_yn[lr] = sqrtf(yn2);
      }
      };
      if (R.unit_scale) build(std::true_type{});
      else build(std::false_type{});
    }
    cluster.sync();  // operands complete

    // ---- 2. leader: split products; each accumulator row goes to the CTA
    // that owns the target (distributed shared memory)
    if (leader) {
      if (tid == 0) {
        s_nb = 0;
        asm volatile("fence.proxy.async;" ::: "memory");
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int ksteps = R.kpad * ESZ / 32;
        const uint32_t aa = smem_u32(sA), bb = smem_u32(sB);
        for (int ks = 0; ks < ksteps; ++ks) {
#pragma unroll
          for (int pass = 0; pass < 3; ++pass) {
            const uint32_t a = aa + (pass == 2 ? a_part : 0u) + (uint32_t)ks * 2u * 2048u;
            const uint32_t b = bb + (pass == 1 ? b_part : 0u) + (uint32_t)ks * 2u * bk;
            mma_split<ESZ>(tmem, smem_desc(a, 2048u, 128u), smem_desc(b, bk, 128u), idesc,
                           (ks > 0 || pass > 0) ? 1u : 0u);
          }
        }
        mma_commit(bar_mma);
      }
      __syncthreads();
      // every thread's bounded wait must have seen the products complete;
      // otherwise no row is delivered and every target goes to the FP64 band
      const bool have = __syncthreads_and(mbar_wait(bar_mma, (uint32_t)(itg & 1)) ? 1 : 0) != 0;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int m = 32 * (warp & 3) + lane;
      const int half = R.ntn / 2;
      const int cb = (warp >> 2) * half;
      const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
      const bool rows_here = (warp & 3) * 32 < kPRows;  // TMEM lanes of this warp hold targets
      if (have && rows_here) {
        const bool mine = m < kPRows && row0 + m < np;
        const int owner = mine ? m / rpm : 0;
        float* dst = cluster.map_shared_rank(reinterpret_cast<float*>(smem + (owner == 0 ? zoff_lead : zoff_member)),
                                             owner) +
                     (size_t)(m % rpm) * zs + cb;
        for (int c = 0; c < half; c += 32) {
          float v[32];
          const int w = min(32, half - c);
          const uint32_t ta = tmem + lane_base + (uint32_t)(cb + c);
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
          if (mine) {
#pragma unroll
            for (int e = 0; e < 32; e += 4)
              if (e < w) *reinterpret_cast<float4*>(dst + c + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
          }
        }
      } else if (!have && tid == 0) {
        atomicOr(&st->err, kErrTimeout);
        s_abort = 1;
      }
      if (tid == 0) s_have = have ? 1 : 0;
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    cluster.sync();  // accumulator rows delivered

    // ---- 2b. every CTA, for its own targets: the FP32 objective from the
    // accumulator row (16 threads per row, columns strided, then a fixed xor
    // tree) and the selection, on the leader's tile state
    {
      const int rr = tid >> 4, sub = tid & 15;
      const int lr = crank * rpm + rr;
      const int i = row0 + lr;
      const bool valid = rr < rpm && i < np;
      const bool have = *l_have != 0;
      EpiAcc acc_{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (valid && have) epi_strided_dispatch(obj, zbuf + (size_t)rr * zs, sub, d, acc_);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        acc_.a1 += __shfl_xor_sync(0xffffffffu, acc_.a1, o);
        acc_.a2 += __shfl_xor_sync(0xffffffffu, acc_.a2, o);
        acc_.a3 += __shfl_xor_sync(0xffffffffu, acc_.a3, o);
        acc_.aS += __shfl_xor_sync(0xffffffffu, acc_.aS, o);
        acc_.aG += __shfl_xor_sync(0xffffffffu, acc_.aG, o);
      }
      if (sub == 0 && rr < rpm) {
        uint8_t flag = 0;
        if (valid) {
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
          const float tau = 2.f * R.band_u * G * R.rownorm * l_yn[lr] + (float)d * 0x1.0p-21f * S + 1e-30f;
          const double fi = l_f[lr];
          const float fif = (float)fi;
          const float tif = l_fx[lr] ? 0.f : l_tau[lr];
          const float mrg = 0x1.0p-22f * fabsf(fif);
          const float bp = (float)best_prev;
          const bool sure_reject = fs - tau > fif + tif + mrg;
          const bool sure_accept = fs + tau < fif - tif - mrg;
          const bool ambiguous = !sure_reject && !sure_accept;
          const bool may_be_best = R.band_all && fs - tau <= bp + 0x1.0p-22f * fabsf(bp);
          const bool near = fs - tau <= R.near_thr || fif - tif <= R.near_thr;
          // only a trial the split bound cannot place on one side of the stop target
          // needs FP64 for the stop rule: surely below (or above) decides it as well
          const bool may_stop = R.target > 0.0 && fs - tau < (float)R.target * 1.001f &&
                                !(fs + tau < (float)R.target * 0.999f);
          l_ft[lr] = (double)fs;
          if ((ambiguous && (R.band_all || near)) || may_be_best || may_stop || !(fs == fs) || !(fif == fif) || !have) {
            l_blist[atomicAdd(l_nb, 1)] = lr;
            flag = 4;
          } else if (sure_accept || (ambiguous && fs <= fif)) {
            // decided on the split values (an undecidable comparison far from
            // the optimum goes to the smaller split value, ties to the trial)
            flag = 1;
            l_f[lr] = (double)fs;
            l_fx[lr] = 0;
            l_tau[lr] = tau;
          }
        }
        l_flag[lr] = flag;
      }
    }
    cluster.sync();  // decisions and the band list are visible

    // ---- 3. FP64 decisions of the listed rows, spread over the cluster
    const int nb = *l_nb;
    for (int b0 = 0; b0 < nb; b0 += kPBandMax) {
      const int nbb = min(kPBandMax, nb - b0);
      // owners write y of the trial (slot 2e) and of the target (slot 2e + 1)
      // into every other CTA's shared memory
      for (int e = 0; e < nbb; ++e) {
        const int lr = l_blist[b0 + e];
        if (lr / rpm != crank) continue;
        const int lw = lr % rpm;
        if ((lw & 7) != warp) continue;
        const int q = lw >> 3;
        const bool need_t = !l_fx[lr];
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          const int j0 = 128 * c + 4 * lane;
          if (j0 >= d) continue;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (j0 + k >= d) continue;
            const double yt = shifted(q ? tr[1][c][k] : tr[0][c][k], osh[c][k], R);
            const double yx = shifted(q ? tx[1][c][k] : tx[0][c][k], osh[c][k], R);
            for (int r = 1; r < C; ++r) {
              double* dst = cluster.map_shared_rank(sYm, r);
              dst[(size_t)(2 * e) * dp + j0 + k] = yt;
              if (need_t) dst[(size_t)(2 * e + 1) * dp + j0 + k] = yx;
            }
          }
        }
      }
      cluster.sync();
      if (!leader) {
        // this CTA's block of outputs z_j, j in [j0, j0 + nout); thread t takes
        // output t & 15 over k slice t >> 4, two accumulator chains
        const int j0 = (crank - 1) * cwp;
        const int nout = max(0, min(cwp + 1, d - j0));
        const int jl = tid & 15, ks = tid >> 4;
        const int kper = (d + 15) / 16;
        for (int v = 0; v < 2 * nbb; ++v) {
          const int lr = l_blist[b0 + v / 2];
          if ((v & 1) && l_fx[lr]) continue;
          const double* yv = sYm + (size_t)v * dp;
          double p0 = 0.0, p1 = 0.0;
          if (jl < nout) {
            const int ka = ks * kper, kb = min(d, ka + kper);
            if (R.rotate) {
              const double* mr = sM + (size_t)jl * d;
              int k = ka;
              for (; k + 1 < kb; k += 2) {
                p0 = fma(mr[k], yv[k], p0);
                p1 = fma(mr[k + 1], yv[k + 1], p1);
              }
              if (k < kb) p0 = fma(mr[k], yv[k], p0);
            } else if (ks == 0) {
              p0 = yv[j0 + jl];
            }
          }
          s_red[ks][jl] = p0 + p1;
          __syncthreads();
          if (tid < 16) {
            // fixed pairwise tree over the 16 k slices
            double r8[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) r8[q] = s_red[2 * q][tid] + s_red[2 * q + 1][tid];
#pragma unroll
            for (int q = 0; q < 4; ++q) r8[q] = r8[2 * q] + r8[2 * q + 1];
            s_zb[tid] = (r8[0] + r8[1]) + (r8[2] + r8[3]);
          }
          __syncthreads();
          if (warp == 0) {
            double t1 = 0.0, t2 = 0.0;
            const int j = j0 + lane;
            if (lane < min(cwp, nout)) {
              const double z = s_zb[lane];
              if (obj == kObjSphere) {
                t1 = z * z;
              } else if (obj == kObjRastrigin) {
                t1 = z * z - 10.0 * cos2pi_f64(z) + 10.0;
              } else if (obj == kObjAckley) {
                t1 = z * z;
                t2 = cos2pi_f64(z);
              } else if (obj == kObjRosenbrock && j + 1 < d) {
                const double t0 = z + 1.0, tn = s_zb[lane + 1] + 1.0;
                const double a = tn - t0 * t0, b = t0 - 1.0;
                t1 = 100.0 * a * a + b * b;
              }
            }
            t1 = warp_sum(t1);
            t2 = warp_sum(t2);
            if (lane == 0) {
              l_bpart[(v * kPMaxC + crank) * 2 + 0] = t1;
              l_bpart[(v * kPMaxC + crank) * 2 + 1] = t2;
            }
          }
          __syncthreads();
        }
      }
      cluster.sync();
      if (leader && tid < nbb) {
        const int lr = s_blist[b0 + tid];
        auto combine = [&](int v) {
          double s1 = 0.0, s2 = 0.0;
          for (int r = 1; r < C; ++r) {
            s1 += s_bpart[v][r][0];
            s2 += s_bpart[v][r][1];
          }
          return obj == kObjAckley ? 20.0 + 2.718281828459045 - 20.0 * exp(-0.2 * sqrt(s1 / d)) - exp(s2 / d) : s1;
        };
        const double ft = combine(2 * tid);
        const double fi = s_fx[lr] ? s_f[lr] : combine(2 * tid + 1);
        const bool acc = fit_key(ft) <= fit_key(fi) && fit_key(ft) != 0x7FFFFFFFFFFFFFFFLL;
        s_ft[lr] = ft;
        s_f[lr] = acc ? ft : fi;
        s_fx[lr] = 1;
        s_tau[lr] = 0.f;
        s_flag[lr] = (acc ? 1 : 0) | 2;
      }
    }

    // ---- 4. leader: best partial and debug; everyone: next-generation rows
    if (leader) {
      __syncthreads();
      Best b;
      b.init();
      if (tid < kPRows && row0 + tid < np) {
        const int i = row0 + tid;
        b.offer(s_f[tid], i);
        if (R.dbg_ftrial) {
          R.dbg_ftrial[i] = s_ft[tid];
          R.dbg_accept[i] = s_flag[tid] & 1;
          R.dbg_fp64[i] = (s_flag[tid] >> 1) & 1;
        }
      }
      b.warp_reduce();
      if (lane == 0) {
        s_bf[warp] = b.f;
        s_bk[warp] = b.k;
        s_bi[warp] = b.i;
      }
      __syncthreads();
      if (tid == 0) {
        b.init();
        for (int w = 0; w < 8; ++w) b.take(s_bf[w], s_bk[w], s_bi[w]);
        BestPartial* pp = R.part + (size_t)(g & 1) * nclusters + tile;
        pp->f = b.f;
        pp->idx = b.i;
        s_nband_total += (unsigned long long)s_nb;  // published once, at the end of the launch
      }
    }
    // the FP64 band changes decisions after the last cluster barrier; without
    // band rows the members already see the final flags
    if (nb > 0) cluster.sync();  // final decisions visible
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (warp + 8 * q >= rpm) break;
      const int lr = crank * rpm + warp + 8 * q;
      const int i = row0 + lr;
      if (i >= np) continue;
      const bool acc = l_flag[lr] & 1;
      if (VAR && R.jde && lane == 0) {
        // jDE: an accepted trial passes its F_i and CR_i on
        double Fi = __ldcg(jFc + i), CRi = __ldcg(jCRc + i);
        if (acc) jde_params(R, (uint32_t)i, g, jFc, jCRc, Fi, CRi);
        R.jF[nxt][i] = Fi;
        R.jCR[nxt][i] = CRi;
      }
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        const int j0 = 128 * c + 4 * lane;
        if (j0 >= d) continue;
        double* dst = Xn + (size_t)i * dp + j0;
        if (acc) {
          *reinterpret_cast<double2*>(dst) = make_double2(tr[q][c][0], tr[q][c][1]);
          *reinterpret_cast<double2*>(dst + 2) = make_double2(tr[q][c][2], tr[q][c][3]);
        } else {
          *reinterpret_cast<double2*>(dst) = make_double2(tx[q][c][0], tx[q][c][1]);
          *reinterpret_cast<double2*>(dst + 2) = make_double2(tx[q][c][2], tx[q][c][3]);
        }
      }
    }
    // every CTA arrives at the grid barrier once its rows are written; the
    // leader waits for all of them
    __syncthreads();
    if (!leader && tid == 0 && !(test_skip && itg == 0)) grid_arrive(ctl);

    // ---- 5. grid barrier (thread 0 of each leader); best record and stop
    // rule (the leader's warp 0 reduces the clusters' partials)
    if (leader && warp == 0) {
      if (!s_abort) {
        // the whole warp polls (one load per poll, no divergent spin)
        if (lane == 0 && !(test_skip && itg == 0)) grid_arrive(ctl);
        __syncwarp();
        if (!grid_wait(ctl, (unsigned)(itg + 1) * (unsigned)(nclusters * C), spin_limit) && lane == 0) {
          atomicOr(&st->err, kErrTimeout);
          s_abort = 1;
        }
        __syncwarp();
      }
      if (!s_abort) {
        Best b;
        b.init();
        const BestPartial* pp = R.part + (size_t)(g & 1) * nclusters;
        for (int t = lane; t < nclusters; t += 32) b.offer(__ldcg(&pp[t].f), __ldcg(&pp[t].idx));
        b.warp_reduce();
        if (lane == 0) {
          const double bf = b.f;
          const int bi = b.i;
          const int64_t evals = (int64_t)np * (1 + g);  // the initial population counts as NP evaluations
          int sp = 0;
          if (R.target > 0.0 && bi >= 0 && bf < R.target) sp = 1;
          else if (R.max_evals > 0 && evals >= R.max_evals) sp = 2;
          else if (g >= R.max_gens) sp = 3;
          s_stop = sp;
          s_best = bf;
          if (bi >= 0) s_bidx = bi;
          s_gen = g;
          if (tile == 0) {
            // one writer of the run state; evals are published at the end
            st->best_f = bf;
            st->best_idx = bi;
            st->gen = g;
            st->stop = sp;
          }
        }
      }
    }
    cluster.sync();  // barrier passed: next generation's donors are complete
    gen = *l_gen;
    stop = *l_stop;
    best_prev = *l_best;
    best_idx = *l_bidx;
    abort = *l_abort != 0;
  }

  // no CTA may leave while another still reads its shared memory
  cluster.sync();

  // ---------------------------------------------------------------- teardown
  if (leader) {
    if (tid == 0) atomicAdd(&R.stats[0], s_nband_total);
    const int curf = (int)(gen & 1);
    for (int m = tid; m < kPRows; m += blockDim.x) {
      const int i = row0 + m;
      if (i < np) {
        R.f[curf][i] = s_f[m];
        R.fx[curf][i] = s_fx[m];
        R.tau[i] = s_tau[m];
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
  }
}

// Evaluation counter, trial counter and tickets after a launch (one thread).
__global__ void k_persist_close(const RunDesc* __restrict__ runs, int run, const PersistCtl* ctl) {
  const RunDesc& R = runs[run];
  RunState* st = R.st;
  R.stats[1] += (unsigned long long)R.np * (unsigned long long)(st->gen - ctl->gen0);
  st->evals = (int64_t)R.np * (1 + st->gen);
  st->ticket = 0;
  st->band_n = 0;
  st->band_left = 0;
}

void k_persist_close_launch(const RunDesc* runs, const PersistCtl* ctl, cudaStream_t s) {
  k_persist_close<<<1, 1, 0, s>>>(runs, 0, ctl);
}

// ------------------------------------------------------------------ host side
size_t persist_smem(const RunDesc& R, int C) {
  const size_t lead = (size_t)R.a_tile_bytes + R.b_tile_bytes + (size_t)2 * kPBandMax * R.dp * sizeof(double);
  const size_t member = persist_z_offset(R, C, false) + (size_t)16 * persist_zstride(R) * sizeof(float);
  return std::max(lead, member);
}

static bool persist_cluster_plan(PersistPlan& pp, const RunDesc& R, int nruns, int prec);

// Both persistent forms; the CTA-local one is the first choice where it
// applies (the autotuner may pick the cluster form instead).  The
// environment variable DE_GB300_PERSIST_MODE=cluster / cta keeps one form.
bool persist_plan(PersistPlan& pp, const RunDesc& R, int nruns, int prec) {
  const char* env = getenv("DE_GB300_PERSIST_MODE");
  const bool want_cl = !(env && strcmp(env, "cta") == 0), want_cta = !(env && strcmp(env, "cluster") == 0);
  pp.cl_ok = want_cl && persist_cluster_plan(pp, R, nruns, prec);
  pp.cta_ok = want_cta && persist_cta_plan(pp, R, nruns, prec);
  pp.prec = prec;
  pp.var = R.strategy != 0 || R.jde;
  pp.mode = pp.cta_ok ? 1 : 0;
  pp.ok = pp.cl_ok || pp.cta_ok;
  return pp.ok;
}

static bool persist_cluster_plan(PersistPlan& pp, const RunDesc& R, int nruns, int prec) {
  // one run, one N tile, whole K resident, rows of at most 128 coordinates
  // (the trial and target rows of a warp then stay in registers)
  if (nruns != 1 || R.nn != 1 || R.kc != R.kpad || R.d > 128) return false;
  const int C = kPC;
  // the FP64 band gives each of the C - 1 member CTAs a block of cwp + 1
  // outputs (the last one Rosenbrock's neighbour term), computed by 16
  // threads: cwp <= 15, so d <= 15 (C - 1) = 105
  if ((R.d + C - 2) / (C - 1) > 15) return false;
  const size_t smem = persist_smem(R, C);
  if (smem > 220 * 1024) return false;
  // first choice: tiles of 128 rows (smaller populations take one tile of
  // their own size, a multiple of C); the split autotuner then times smaller
  // tiles (fewer trials per CTA, more clusters at the grid barrier)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  auto query = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
  };
  const bool var = R.strategy != 0 || R.jde;
  const cudaError_t e = prec == DE_PREC_BF16X3 ? (var ? query(k_persist<2, 1, true>) : query(k_persist<2, 1, false>))
                                               : (var ? query(k_persist<4, 1, true>) : query(k_persist<4, 1, false>));
  if (e != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return false;
  }
  pp.C = C;
  pp.maxcl = nclusters;
  int prows = std::min(kTileM, (R.np + C - 1) / C * C);
  if (const char* env = getenv("DE_GB300_PERSIST_ROWS")) {
    const int v = atoi(env);
    if (v >= C && v <= kTileM && v % C == 0) prows = v;
  }
  if (!persist_set_rows(pp, R, prows)) return false;
  pp.smem = smem;
  pp.prec = prec;
  pp.nch = 1;
  pp.var = var;
  return true;
}

bool persist_set_rows(PersistPlan& pp, const RunDesc& R, int prows) {
  if (pp.C < 1 || prows < pp.C || prows > kTileM || prows % pp.C != 0) return false;
  const int ntiles = (R.np + prows - 1) / prows;
  if (ntiles > pp.maxcl) return false;
  pp.prows = prows;
  pp.ntiles = ntiles;
  return true;
}

cudaError_t persist_ctl_reset(PersistCtl* ctl, int test_skip, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(PersistCtl), s);
  if (e != cudaSuccess || test_skip <= 0) return e;
  // about 4096 polls instead of 2^22: the test's wait runs out in milliseconds
  const int skip = test_skip;
  const long long spin = 4096;
  e = cudaMemcpyAsync(&ctl->test_skip, &skip, sizeof skip, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl->test_spin, &spin, sizeof spin, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // skip and spin live on this stack frame
  return e;
}

cudaError_t persist_launch(const PersistPlan& pp, const RunDesc* runs, PersistCtl* ctl, long long gens,
                           cudaStream_t s, int test_skip) {
  if (pp.mode == 1) return persist_cta_launch(pp, runs, ctl, gens, s, test_skip);
  cudaError_t e = persist_ctl_reset(ctl, test_skip, s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(pp.ntiles * pp.C));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = pp.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)pp.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (pp.prec == DE_PREC_BF16X3) {
    if (pp.var) e = cudaLaunchKernelEx(&cfg, k_persist<2, 1, true>, runs, 0, ctl, gens, pp.prows);
    else e = cudaLaunchKernelEx(&cfg, k_persist<2, 1, false>, runs, 0, ctl, gens, pp.prows);
  } else {
    if (pp.var) e = cudaLaunchKernelEx(&cfg, k_persist<4, 1, true>, runs, 0, ctl, gens, pp.prows);
    else e = cudaLaunchKernelEx(&cfg, k_persist<4, 1, false>, runs, 0, ctl, gens, pp.prows);
  }
  if (e != cudaSuccess) return e;
  k_persist_close<<<1, 1, 0, s>>>(runs, 0, ctl);
  return cudaGetLastError();
}

}  // namespace de
