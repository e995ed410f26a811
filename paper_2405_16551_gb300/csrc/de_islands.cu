// de_islands.cu -- the island (multi-population) model of DE (Sec. 3.2; on
// the GPU the multi-population model of Sec. 5.4): the runs of a batch are
// islands that evolve independently and exchange migrants on a ring.
//
// Synchronous migration (Sec. 5.4: the generation kernels end and a
// migration kernel runs), after every generation g with g % interval == 0:
//   k_island_select  one CTA per island: the island's nmig best individuals
//                    (ascending f, lower index first, NaN last) are copied
//                    to a staging area, and its nmig worst slots (descending
//                    f, NaN first, higher index first) are recorded;
//   k_island_apply   one CTA per island: island k writes island k-1's
//                    migrants (ring) into its worst slots (the q-th best
//                    into the q-th worst), with their fitness (and jDE
//                    parameters), then recomputes its best record;
//   k_island_group   one CTA: the model stops as a whole once any island's
//                    best is below the target (every island gets stop
//                    reason "target"), and the migration is marked done.
// Staging between two kernels makes the exchange independent of the order in
// which CTAs run: every migrant is read before any island is written.  The
// three kernels run after every generation and return at once when no
// migration is due, so a CUDA graph of generations can hold them.
//
// Asynchronous migration (Sec. 3.2 names both strategies; in the GPU form of
// Sec. 5.4 the asynchronous one migrates inside the generation kernel, so an
// island may receive migrants of an island that is ahead of it or behind it,
// and runs cannot be repeated).  Here the staleness is fixed to one migration
// interval, through a mailbox of two slots:
//   k_island_async   one CTA per island, one kernel: at migration point g the
//                    island posts its nmig best to slot (g / interval) & 1 and
//                    takes, into its nmig worst, the migrants its ring
//                    predecessor posted at the previous migration point (from
//                    the other slot; none at the first point).  No CTA reads a
//                    slot that a CTA of the same launch writes, so the islands
//                    need no ordering among themselves and the results do not
//                    depend on it;
//   k_island_group   as above, and it records the post.
#include <cuda_runtime.h>

#include "de_common.cuh"
#include "de_device.cuh"
#include "de_internal.cuh"
#include "de_island_dev.cuh"
#include "de_kernels.h"

namespace de {

// a migration is due after generation gen
__device__ __forceinline__ bool island_due(const IslandCtl* ctl, int64_t gen) {
  return ctl->interval > 0 && gen > 0 && gen % ctl->interval == 0 && gen > ctl->mig_gen;
}

__global__ void __launch_bounds__(256) k_island_select(const RunDesc* __restrict__ runs, const IslandCtl* ctl,
                                                       IslandStage stage) {
  const int k = blockIdx.x;
  const RunDesc& R = runs[k];
  const int64_t gen = *(volatile int64_t*)&R.st->gen;
  if (!island_due(ctl, gen)) return;
  const int cur = (int)(gen & 1), nmig = ctl->nmig;
  const double* f = R.f[cur];
  __shared__ int best[kIslandMaxMigrants], worst[kIslandMaxMigrants];
  for (int q = 0; q < nmig; ++q) {
    const int b = island_pick(f, R.np, best, q, false);
    if (threadIdx.x == 0) best[q] = b;
    __syncthreads();
  }
  for (int q = 0; q < nmig; ++q) {
    const int w = island_pick(f, R.np, worst, q, true);
    if (threadIdx.x == 0) worst[q] = w;
    __syncthreads();
  }
  for (int q = 0; q < nmig; ++q) {
    const size_t s = (size_t)k * nmig + q;
    const double* src = R.X[cur] + (size_t)best[q] * R.dp;
    for (int j = threadIdx.x; j < R.dp; j += blockDim.x) stage.x[s * stage.dp + j] = src[j];
    if (threadIdx.x == 0) {
      stage.f[s] = f[best[q]];
      stage.fx[s] = R.fx[cur][best[q]];
      if (R.jde) {
        stage.F[s] = R.jF[cur][best[q]];
        stage.CR[s] = R.jCR[cur][best[q]];
      }
      stage.widx[s] = worst[q];
    }
  }
}

__global__ void __launch_bounds__(256) k_island_apply(const RunDesc* __restrict__ runs, const IslandCtl* ctl,
                                                      IslandStage stage) {
  const int k = blockIdx.x, m = ctl->m;
  const RunDesc& R = runs[k];
  const int64_t gen = *(volatile int64_t*)&R.st->gen;
  if (!island_due(ctl, gen)) return;
  const int cur = (int)(gen & 1), nmig = ctl->nmig;
  const int from = (k + m - 1) % m;
  for (int q = 0; q < nmig; ++q) {
    const size_t s = (size_t)from * nmig + q;
    const int w = stage.widx[(size_t)k * nmig + q];
    double* dst = R.X[cur] + (size_t)w * R.dp;
    for (int j = threadIdx.x; j < R.dp; j += blockDim.x) dst[j] = stage.x[s * stage.dp + j];
    if (threadIdx.x == 0) {
      R.f[cur][w] = stage.f[s];
      R.fx[cur][w] = stage.fx[s];
      if (R.jde) {
        R.jF[cur][w] = stage.F[s];
        R.jCR[cur][w] = stage.CR[s];
      }
    }
  }
  __syncthreads();
  island_best_record(R, cur);
}

__global__ void __launch_bounds__(256) k_island_async(const RunDesc* __restrict__ runs, const IslandCtl* ctl,
                                                      IslandStage stage) {
  const int k = blockIdx.x;
  const RunDesc& R = runs[k];
  const int64_t gen = *(volatile int64_t*)&R.st->gen;
  if (!island_due(ctl, gen)) return;
  const int64_t ep = gen / ctl->interval;
  const size_t wslot = (size_t)(ep & 1) * stage.slot, rslot = (size_t)((ep & 1) ^ 1) * stage.slot;
  // the previous migration point posted (not so after a reset or a population change)
  const bool take = ctl->post_gen >= 0 && ctl->post_gen == gen - ctl->interval;
  island_exchange(R, k, ctl->m, ctl->nmig, (int)(gen & 1), stage, true, wslot, take, rslot);
}

// posted: this launch follows k_island_async (a due migration posted)
__global__ void __launch_bounds__(256) k_island_group(const RunDesc* __restrict__ runs, IslandCtl* ctl, int posted) {
  const int m = ctl->m;
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const RunDesc& R = runs[k];
    const RunState* st = R.st;
    if (st->stop == 1 || (R.target > 0.0 && st->best_idx >= 0 && st->best_f < R.target)) atomicOr(&any, 1);
  }
  __syncthreads();
  if (any)
    for (int k = threadIdx.x; k < m; k += blockDim.x) runs[k].st->stop = 1;
  if (threadIdx.x == 0) {
    const int64_t gen = runs[0].st->gen;
    if (island_due(ctl, gen)) {
      ctl->mig_gen = gen;
      if (posted) ctl->post_gen = gen;
    }
  }
}

void k_island_launch(const RunDesc* runs, IslandCtl* ctl, const IslandStage& stage, int m, bool migrate,
                     bool async, cudaStream_t s) {
  if (migrate && async) {
    k_island_async<<<m, 256, 0, s>>>(runs, ctl, stage);
  } else if (migrate) {
    k_island_select<<<m, 256, 0, s>>>(runs, ctl, stage);
    k_island_apply<<<m, 256, 0, s>>>(runs, ctl, stage);
  }
  k_island_group<<<1, 256, 0, s>>>(runs, ctl, migrate && async ? 1 : 0);
}

}  // namespace de
