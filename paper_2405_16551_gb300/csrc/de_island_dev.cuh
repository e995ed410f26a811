// de_island_dev.cuh -- device routines of the island model (Sec. 3.2; on the
// GPU the multi-population model of Sec. 5.4) shared by the migration kernels
// between generations (de_islands.cu) and the cooperative persistent FP64
// kernel (de_fp64.cu), which migrates inside its generation loop.
#pragma once
#include <cuda_runtime.h>

#include "de_device.cuh"
#include "de_internal.cuh"
#include "de_kernels.h"

namespace de {

// CTA-wide arg-extremum of (key, index) over i in [0, np) minus the `ntaken`
// indices already chosen; worst = largest (key, index), else smallest.
static __device__ int island_pick(const double* __restrict__ f, int np, const int* taken, int ntaken, bool worst) {
  __shared__ long long sk[32];
  __shared__ int si[32];
  long long bk = worst ? (long long)0x8000000000000000LL : 0x7FFFFFFFFFFFFFFFLL;
  int bi = -1;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    bool t = false;
    for (int q = 0; q < ntaken; ++q) t |= taken[q] == i;
    if (t) continue;
    const long long k = fit_key(f[i]);
    const bool take = bi < 0 || (worst ? (k > bk || (k == bk && i > bi)) : (k < bk || (k == bk && i < bi)));
    if (take) {
      bk = k;
      bi = i;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    const bool take = oi >= 0 && (bi < 0 || (worst ? (ok > bk || (ok == bk && oi > bi)) : (ok < bk || (ok == bk && oi < bi))));
    if (take) {
      bk = ok;
      bi = oi;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sk[warp] = bk;
    si[warp] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      const long long ok = sk[w];
      const int oi = si[w];
      const bool take = oi >= 0 && (bi < 0 || (worst ? (ok > bk || (ok == bk && oi > bi)) : (ok < bk || (ok == bk && oi < bi))));
      if (take) {
        bk = ok;
        bi = oi;
      }
    }
    si[0] = bi;
  }
  __syncthreads();
  const int r = si[0];
  __syncthreads();
  return r;
}

// the island's best record after an exchange (the whole CTA)
static __device__ void island_best_record(const RunDesc& R, int cur) {
  __shared__ double sf[32];
  __shared__ long long sk[32];
  __shared__ int si[32];
  Best b;
  b.init();
  for (int i = threadIdx.x; i < R.np; i += blockDim.x) b.offer(R.f[cur][i], i);
  b.warp_reduce();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sf[warp] = b.f;
    sk[warp] = b.k;
    si[warp] = b.i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    b.init();
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b.take(sf[w], sk[w], si[w]);
    if (b.i >= 0) {
      R.st->best_f = b.f;
      R.st->best_idx = b.i;
    }
  }
}

// One island's exchange at a migration point (the whole CTA; the population
// of the point is X[cur], f[cur]).  post: its nmig best (ascending f, lower
// index first, NaN last) go to mailbox entries wslot + k nmig + q.  take: the
// entries rslot + (k - 1 mod m) nmig + q, posted by its ring predecessor,
// replace its nmig worst (the q-th into the q-th worst, with fitness and jDE
// parameters), and the island's best record is recomputed.  Best and worst
// are chosen before any row changes; they are disjoint rows (nmig <= np / 2,
// and both orders are total).
static __device__ void island_exchange(const RunDesc& R, int k, int m, int nmig, int cur, const IslandStage& stage,
                                       bool post, size_t wslot, bool take, size_t rslot) {
  const double* f = R.f[cur];
  __shared__ int best[kIslandMaxMigrants], worst[kIslandMaxMigrants];
  for (int q = 0; q < nmig && post; ++q) {
    const int b = island_pick(f, R.np, best, q, false);
    if (threadIdx.x == 0) best[q] = b;
    __syncthreads();
  }
  for (int q = 0; q < nmig && take; ++q) {
    const int w = island_pick(f, R.np, worst, q, true);
    if (threadIdx.x == 0) worst[q] = w;
    __syncthreads();
  }
  for (int q = 0; q < nmig && post; ++q) {
    const size_t s = wslot + (size_t)k * nmig + q;
    const double* src = R.X[cur] + (size_t)best[q] * R.dp;
    for (int j = threadIdx.x; j < R.dp; j += blockDim.x) stage.x[s * stage.dp + j] = src[j];
    if (threadIdx.x == 0) {
      stage.f[s] = f[best[q]];
      stage.fx[s] = R.fx[cur][best[q]];
      if (R.jde) {
        stage.F[s] = R.jF[cur][best[q]];
        stage.CR[s] = R.jCR[cur][best[q]];
      }
    }
  }
  if (!take) return;
  const int from = (k + m - 1) % m;
  for (int q = 0; q < nmig; ++q) {
    const size_t s = rslot + (size_t)from * nmig + q;
    const int w = worst[q];
    double* dst = R.X[cur] + (size_t)w * R.dp;
    for (int j = threadIdx.x; j < R.dp; j += blockDim.x) dst[j] = __ldcg(stage.x + s * stage.dp + j);
    if (threadIdx.x == 0) {
      R.f[cur][w] = __ldcg(stage.f + s);
      R.fx[cur][w] = __ldcg(stage.fx + s);
      if (R.jde) {
        R.jF[cur][w] = __ldcg(stage.F + s);
        R.jCR[cur][w] = __ldcg(stage.CR + s);
      }
    }
  }
  __syncthreads();
  island_best_record(R, cur);
}

}  // namespace de
