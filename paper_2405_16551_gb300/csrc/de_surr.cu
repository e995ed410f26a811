// de_surr.cu -- surrogate-assisted DE generations.
//
// The paper has no surrogate (its Abstract motivates costly objectives).  In
// this workload every target draws k candidate trials, one per candidate
// stream of the STEP draws (stream 0 is the plain DE/rand/1/bin trial of
// Eq. 2 / Eq. 3).  The surrogate network predicts each candidate's fitness;
// only the candidate with the lowest prediction is evaluated with the true
// objective.  Greedy selection (Sec. 2) then runs as in plain DE.  Each
// evaluated trial and its true fitness enter an archive, and the network is
// retrained on it.  With one candidate the generation is plain DE.
//
//   k_surr_trials    candidate trials (a warp per candidate)
//   k_surr_choose    argmin of the predictions per target (ties: lowest
//                    candidate), copy of the chosen trial
//   (k_eval_rows)    true evaluation of the chosen trials
//   k_surr_select    greedy selection, archive append, best record, stop test
//   k_surr_targets   training targets: standardised log f of the window
#include <cuda_runtime.h>
#include <math.h>
#include <math_constants.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "de_common.cuh"
#include "de_device.cuh"
#include "de_internal.cuh"
#include "de_kernels.h"
#include "de_surr.h"

namespace de {

__global__ void k_surr_trials(const RunDesc* __restrict__ runs, int run, double* __restrict__ out, int k) {
  const RunDesc& R = runs[run];
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= (long long)R.np * k) return;
  const RunState* st = R.st;
  if (*(volatile const int32_t*)&st->stop) return;
  const int64_t gen = *(volatile const int64_t*)&st->gen;
  const int64_t g = gen + 1;
  const double* X = R.X[R.dbuf ? (int)(gen & 1) : 0];
  const uint32_t i = (uint32_t)(w / k), c = (uint32_t)(w % k);
  const TrialSetup s = trial_setup(R, i, g, lane, c, false);
  double* row = out + (size_t)w * R.dp;
  for (int j0 = 4 * lane; j0 < R.d; j0 += 128) {
    double t[4];
    trial_chunk(R, X, s, i, g, j0, t, c);
    *reinterpret_cast<double2*>(row + j0) = make_double2(t[0], t[1]);
    *reinterpret_cast<double2*>(row + j0 + 2) = make_double2(t[2], t[3]);
  }
}

__global__ void k_surr_choose(const RunDesc* __restrict__ runs, int run, const double* __restrict__ C, int k,
                              const float* __restrict__ yhat, double* __restrict__ T, float* __restrict__ ysel,
                              int32_t* __restrict__ csel) {
  const RunDesc& R = runs[run];
  const int lane = threadIdx.x & 31;
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (i >= R.np) return;
  if (*(volatile const int32_t*)&R.st->stop) return;
  float v = CUDART_INF_F;
  int ci = lane;
  if (lane < k) {
    v = yhat[(size_t)i * k + lane];
    if (!(v == v)) v = CUDART_INF_F;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oc = __shfl_xor_sync(0xffffffffu, ci, o);
    if (ov < v || (ov == v && oc < ci)) {
      v = ov;
      ci = oc;
    }
  }
  const double* src = C + ((size_t)i * k + ci) * R.dp;
  for (int j = lane; j < R.dp; j += 32) T[(size_t)i * R.dp + j] = src[j];
  if (lane == 0) {
    ysel[i] = yhat[(size_t)i * k + ci];
    csel[i] = ci;
  }
}

// A warp per target, 8 targets per CTA; the last CTA (ticket) reduces the
// per-CTA best partials in CTA order and takes the stop decision.
__global__ void __launch_bounds__(256) k_surr_select(const RunDesc* __restrict__ runs, int run,
                                                     const double* __restrict__ T, const double* __restrict__ ft,
                                                     const int32_t* __restrict__ csel, double* __restrict__ arch_x,
                                                     double* __restrict__ arch_f, long long head, int cap) {
  __shared__ double s_bf[8];
  __shared__ long long s_bk[8];
  __shared__ int s_bi[8];
  __shared__ int s_stop, s_last;
  __shared__ long long s_gen;
  const RunDesc& R = runs[run];
  RunState* st = R.st;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    s_stop = *(volatile int32_t*)&st->stop;
    s_gen = *(volatile int64_t*)&st->gen;
  }
  __syncthreads();
  if (s_stop) return;
  const int64_t g = s_gen + 1;
  const int cur = (int)(s_gen & 1), nxt = cur ^ 1;
  const int dp = R.dp, d = R.d;
  Best bb;
  bb.init();
  const int i = blockIdx.x * 8 + warp;
  if (i < R.np) {
    const double fi = R.f[cur][i], t = ft[i];
    const bool acc = fit_key(t) <= fit_key(fi) && fit_key(t) != 0x7FFFFFFFFFFFFFFFLL;  // t <= fi, NaN never
    const double* src = acc ? T + (size_t)i * dp : R.X[cur] + (size_t)i * dp;
    double* dst = R.X[nxt] + (size_t)i * dp;
    const size_t slot = (size_t)((head + i) % cap);
    for (int j = lane; j < dp; j += 32) {
      dst[j] = src[j];
      arch_x[slot * dp + j] = T[(size_t)i * dp + j];
    }
    if (R.dbg_trial)
      for (int j = lane; j < d; j += 32) R.dbg_trial[(size_t)i * d + j] = T[(size_t)i * dp + j];
    const double fnew = acc ? t : fi;
    if (lane == 0) {
      R.f[nxt][i] = fnew;
      R.fx[nxt][i] = 1;
      arch_f[slot] = t;
      if (R.dbg_ftrial) {
        R.dbg_ftrial[i] = t;
        R.dbg_accept[i] = acc ? 1 : 0;
        R.dbg_fp64[i] = 1;
        if (R.dbg_cand) R.dbg_cand[i] = csel[i];
      }
    }
    bb.offer(fnew, i);
  }
  if (lane == 0) {
    s_bf[warp] = bb.f;
    s_bk[warp] = bb.k;
    s_bi[warp] = bb.i;
  }
  __syncthreads();
  if (tid == 0) {
    bb.init();
    for (int w = 0; w < 8; ++w) bb.take(s_bf[w], s_bk[w], s_bi[w]);
    R.part[blockIdx.x].f = bb.f;
    R.part[blockIdx.x].idx = bb.i;
    __threadfence();
    const uint32_t tk = atomicAdd(&st->ticket, 1u);
    s_last = (tk == gridDim.x - 1u);
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    finish_generation(R, g, (int)gridDim.x, R.part, R.X[nxt]);
  }
}

__global__ void k_surr_targets(const double* __restrict__ f, float* __restrict__ t, long long base, int n, int cap,
                               double mu, double inv_sd) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const size_t slot = (size_t)((base + e) % cap);
    const double v = f[slot];
    t[slot] = isfinite(v) ? (float)((log(fmax(v, 0.0) + 1e-30) - mu) * inv_sd) : 0.f;
  }
}

// ------------------------------------------------------------------ host side
// Spearman rank correlation (average ranks for ties).
static double spearman(const std::vector<float>& a, const std::vector<double>& b) {
  const size_t n = a.size();
  if (n < 3) return 0.0;
  auto ranks = [n](auto const& v) {
    std::vector<size_t> o(n);
    std::iota(o.begin(), o.end(), 0);
    std::sort(o.begin(), o.end(), [&](size_t x, size_t y) { return v[x] < v[y]; });
    std::vector<double> r(n);
    for (size_t s = 0; s < n;) {
      size_t e = s;
      while (e + 1 < n && !(v[o[s]] < v[o[e + 1]])) ++e;
      const double avg = 0.5 * (double)(s + e);
      for (size_t q = s; q <= e; ++q) r[o[q]] = avg;
      s = e + 1;
    }
    return r;
  };
  std::vector<double> fa(n);
  std::vector<double> fb(n);
  for (size_t e = 0; e < n; ++e) {
    fa[e] = std::isfinite(a[e]) ? (double)a[e] : 1e300;
    fb[e] = std::isfinite(b[e]) ? b[e] : 1e300;
  }
  const std::vector<double> ra = ranks(fa), rb = ranks(fb);
  const double ma = std::accumulate(ra.begin(), ra.end(), 0.0) / n, mb = std::accumulate(rb.begin(), rb.end(), 0.0) / n;
  double sab = 0, saa = 0, sbb = 0;
  for (size_t e = 0; e < n; ++e) {
    sab += (ra[e] - ma) * (rb[e] - mb);
    saa += (ra[e] - ma) * (ra[e] - ma);
    sbb += (rb[e] - mb) * (rb[e] - mb);
  }
  return (saa > 0 && sbb > 0) ? sab / std::sqrt(saa * sbb) : 0.0;
}

de_status surr_create(Surrogate*& S, int k, int steps, uint64_t seed, const RunDesc& R, cudaStream_t s,
                      std::string& err) {
  S = new Surrogate();
  S->k = k;
  if (steps > 0) S->steps = steps;
  S->since_train = S->retrain - S->warmup;  // first training after the warm-up generations
  const size_t np = R.np, dp = R.dp, cap = S->cap;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) / 256 * 256;
    const size_t o = off;
    off += bytes;
    return o;
  };
  const size_t oC = take(np * k * dp * sizeof(double)), oT = take(np * dp * sizeof(double));
  const size_t oF = take(np * sizeof(double)), oY = take(np * k * sizeof(float)), oYs = take(np * sizeof(float));
  const size_t oCs = take(np * sizeof(int32_t)), oAx = take(cap * dp * sizeof(double));
  const size_t oAf = take(cap * sizeof(double)), oAt = take(cap * sizeof(float));
  cudaError_t e = cudaMalloc(&S->arena, off);
  if (e != cudaSuccess) {
    err = std::string("surrogate buffers: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DE_ERR_OOM : DE_ERR_CUDA;
  }
  e = cudaMemsetAsync(S->arena, 0, off, s);
  if (e != cudaSuccess) {
    err = std::string("surrogate buffers: ") + cudaGetErrorString(e);
    return DE_ERR_CUDA;
  }
  uint8_t* A = (uint8_t*)S->arena;
  S->C = (double*)(A + oC);
  S->T = (double*)(A + oT);
  S->ftrial = (double*)(A + oF);
  S->yhat = (float*)(A + oY);
  S->yhat_sel = (float*)(A + oYs);
  S->cand_sel = (int32_t*)(A + oCs);
  S->arch_x = (double*)(A + oAx);
  S->arch_f = (double*)(A + oAf);
  S->arch_t = (float*)(A + oAt);
  S->h_f.resize(np);
  S->h_y.resize(np);
  const de_status st = mlp_create(seed ^ 0x53555252ull, s, &S->mlp);
  if (st != DE_OK) {
    err = "surrogate network could not be created";
    return st;
  }
  return DE_OK;
}

void surr_destroy(Surrogate* S) {
  if (!S) return;
  if (S->mlp) mlp_destroy(S->mlp);
  if (S->arena) cudaFree(S->arena);
  delete S;
}

de_status surr_reset(Surrogate& S, cudaStream_t s, std::string& err) {
  (void)s;
  S.head = S.count = S.gens = S.trainings = S.screened = 0;
  S.since_train = S.retrain - S.warmup;
  S.k_eff = 1;
  S.trained = false;
  S.last_rho = NAN;
  const de_status st = mlp_reset(S.mlp);
  if (st != DE_OK) err = "surrogate network reset failed";
  return st;
}

static de_status surr_train(Surrogate& S, const RunDesc& R, cudaStream_t s, std::string& err) {
  const int n = (int)std::min<long long>(S.count, S.window);
  if (n < 2) return DE_OK;
  const long long base = ((S.head - n) % S.cap + S.cap) % S.cap;
  // window fitness to the host (one or two segments of the ring)
  S.h_win.resize(n);
  const long long first = std::min<long long>(n, S.cap - base);
  cudaError_t e = cudaMemcpyAsync(S.h_win.data(), S.arch_f + base, first * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && first < n)
    e = cudaMemcpyAsync(S.h_win.data() + first, S.arch_f, (n - first) * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    err = std::string("surrogate window: ") + cudaGetErrorString(e);
    return DE_ERR_CUDA;
  }
  double sum = 0, sum2 = 0;
  long long cnt = 0;
  for (double v : S.h_win)
    if (std::isfinite(v)) {
      const double l = std::log(std::max(v, 0.0) + 1e-30);
      sum += l;
      sum2 += l * l;
      ++cnt;
    }
  if (cnt < 2) return DE_OK;
  const double mu = sum / cnt, var = std::max(sum2 / cnt - mu * mu, 1e-24);
  k_surr_targets<<<64, 256, 0, s>>>(S.arch_f, S.arch_t, base, n, S.cap, mu, 1.0 / std::sqrt(var));
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("surrogate targets: ") + cudaGetErrorString(e);
    return DE_ERR_CUDA;
  }
  const de_status st = mlp_train_rows(S.mlp, S.arch_x, R.dp, S.arch_t, n, (int)base, S.cap, S.steps, S.lr);
  if (st != DE_OK) {
    err = "surrogate training failed";
    return st;
  }
  S.trained = true;
  S.since_train = 0;
  ++S.trainings;
  return DE_OK;
}

de_status surr_generation(Surrogate& S, const RunDesc* d_run, const RunDesc& R, cudaStream_t s, std::string& err) {
  const int np = R.np, dp = R.dp, k = S.k_eff;
  const MlpDev& P = mlp_dev(S.mlp);
  bool predicted = false;
  if (k > 1) {
    const long long threads = (long long)np * k * 32;
    k_surr_trials<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(d_run, 0, S.C, k);
    mlp_forward_launch(P, S.C, dp, np * k, S.yhat, s);
    k_surr_choose<<<(unsigned)((np * 32LL + 255) / 256), 256, 0, s>>>(d_run, 0, S.C, k, S.yhat, S.T, S.yhat_sel,
                                                                      S.cand_sel);
    predicted = true;
    ++S.screened;
  } else {
    k_surr_trials<<<(unsigned)((np * 32LL + 255) / 256), 256, 0, s>>>(d_run, 0, S.T, 1);
    cudaMemsetAsync(S.cand_sel, 0, np * sizeof(int32_t), s);
    if (S.trained) {
      mlp_forward_launch(P, S.T, dp, np, S.yhat_sel, s);
      predicted = true;
    }
  }
  k_eval_rows_launch(d_run, 0, R, S.T, dp, np, S.ftrial, nullptr, s);
  k_surr_select<<<(np + 7) / 8, 256, 0, s>>>(d_run, 0, S.T, S.ftrial, S.cand_sel, S.arch_x, S.arch_f, S.head, S.cap);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(S.h_f.data(), S.ftrial, np * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && predicted)
    e = cudaMemcpyAsync(S.h_y.data(), S.yhat_sel, np * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    err = std::string("surrogate generation: ") + cudaGetErrorString(e);
    return DE_ERR_CUDA;
  }
  S.head = (S.head + np) % S.cap;
  S.count = std::min<long long>(S.count + np, S.cap);
  ++S.gens;
  ++S.since_train;
  if (predicted) {
    S.last_rho = spearman(S.h_y, S.h_f);
    S.k_eff = S.last_rho >= S.rho_min ? S.k : 1;
  }
  if (S.since_train >= S.retrain) return surr_train(S, R, s, err);
  return DE_OK;
}

}  // namespace de
