// de_api.cu -- the C ABI of include/de.h: handle, device memory, launches,
// CUDA graphs, autotuning, checkpoints.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "de.h"
#include "de_common.cuh"
#include "de_device.cuh"
#include "de_internal.cuh"
#include "de_kernels.h"
#include "de_surr.h"

using namespace de;

struct de_handle {
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
  int device = 0;
  int nruns = 0;
  int prec = DE_PREC_FP64;
  bool dbuf = true;         // generation g in X[g & 1] (FP64 and persistent split paths)
  std::vector<de_config> cfg;
  std::vector<RunDesc> run;  // host copy of the descriptors
  RunDesc* d_run = nullptr;
  int4* d_items = nullptr;  // FP64 generation kernel work list: (run, tile, first row, rows)
  int nitems = 0;
  int rows = 8;             // rows per tile of the FP64 generation kernel
  int threads = 256;
  size_t smem_gen = 0;
  TcPlan tc;                // split-precision plan (de_tc.cu)
  char* arena = nullptr;
  size_t arena_bytes = 0;
  RunState* h_state = nullptr;  // pinned mirror of the device states
  cudaGraphExec_t graph = nullptr;
  int graph_gens = 0;
  Surrogate* surr = nullptr;  // surrogate-assisted generations (surrogate_k >= 2)
  bool variants = false;      // some run uses a strategy variant or jDE
  bool suite = false;         // some run uses an objective of the proposed benchmark (5..20)
  bool fp64_persist = false;  // FP64: every generation of a call in one cooperative launch
  bool fp64_cluster = false;  // ... launched as one thread-block cluster (one run of at most 8 tiles)
  PersistCtl* d_ctl64 = nullptr;
  // island model (de_init_islands): the runs are islands on a migration ring
  bool islands = false;
  IslandCtl* d_isl = nullptr;
  IslandStage stage{};
  void* isl_mem = nullptr;
  IslandCtl isl{};
  // failure-detection test (DE_GB300_TEST_GRID_TIMEOUT=k at de_init): CTA
  // k - 1 of every cooperative FP64 launch leaves out its first grid-barrier
  // arrival, and the barrier gives up after a few thousand polls
  int test_grid_skip = 0;
  // split precision, several runs: every generation of a call in one
  // cooperative launch of the persistent batch kernel (kernel path 5)
  bool pbatch_on = false;
  // per run: a hash of the problem (objective, F, CR, bounds, scale, seed,
  // run_id, precision, strategy, jDE, FP64 band policy, shift, rotation and
  // permutation), written to checkpoints and checked by de_load
  std::vector<uint64_t> fingerprint;
  std::string err;
};

// Buffer holding the population of generation `gen`: the FP64 kernel writes
// generation g + 1 into the other buffer; the split-precision kernels update
// buffer 0 in place.
static int cur_buf(const de_handle* h, int64_t gen) { return h->dbuf ? (int)(gen & 1) : 0; }

static thread_local std::string g_err;

namespace de {
// The thread's last error message, as de_last_error(NULL) returns it (for
// entry points outside this file).
void set_last_error(const std::string& m) { g_err = m; }
}  // namespace de
static const char* kVersion = "de_gb300 1.0 sm_103a";

// ---------------------------------------------------------------- helpers
static de_status fail(de_handle* h, de_status s, const std::string& msg) {
  if (h) h->err = msg;
  g_err = msg;
  return s;
}

#define DE_CUDA(h, call)                                                                          \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return fail((h), e_ == cudaErrorMemoryAllocation ? DE_ERR_OOM : DE_ERR_CUDA,                \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                            \
  } while (0)

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }



// ---------------------------------------------------------------- benchmark suite
// Functions of the proposed benchmark (Table 2) built from several basic
// functions: hybrid parts (share of the coordinates in percent) or
// composition components (sigma, lambda, bias).
struct SuiteSpec {
  int kind;  // 0 basic, 1 hybrid, 2 composition
  int n;
  int fn[5];
  int pct[5];
  double sigma[5], lambda[5], bias[5];
};

static SuiteSpec suite_spec(int obj) {
  switch (obj) {
    case DE_OBJ_HYBRID1:
      return {1, 3, {DE_OBJ_BENT_CIGAR, DE_OBJ_HGBAT, DE_OBJ_RASTRIGIN}, {30, 30, 40}, {}, {}, {}};
    case DE_OBJ_HYBRID2:
      return {1, 4, {DE_OBJ_SCHAFFER_F6, DE_OBJ_HGBAT, DE_OBJ_ROSENBROCK, DE_OBJ_SCHWEFEL}, {20, 20, 30, 30}, {}, {}, {}};
    case DE_OBJ_HYBRID3:
      return {1, 5,
              {DE_OBJ_KATSUURA, DE_OBJ_HAPPYCAT, DE_OBJ_GRIEWANK_ROSENBROCK, DE_OBJ_SCHWEFEL, DE_OBJ_ACKLEY},
              {30, 20, 20, 10, 20}, {}, {}, {}};
    case DE_OBJ_COMPOSITION1:
      return {2, 3, {DE_OBJ_RASTRIGIN, DE_OBJ_GRIEWANK, DE_OBJ_SCHWEFEL}, {}, {10, 20, 30}, {1, 10, 1}, {0, 100, 200}};
    case DE_OBJ_COMPOSITION2:
      return {2, 4, {DE_OBJ_ACKLEY, DE_OBJ_ELLIPTIC, DE_OBJ_GRIEWANK, DE_OBJ_RASTRIGIN}, {}, {10, 20, 30, 40},
              {10, 1e-6, 10, 1}, {0, 100, 200, 300}};
    case DE_OBJ_COMPOSITION3:
      return {2, 5, {DE_OBJ_SCHAFFER_F6, DE_OBJ_SCHWEFEL, DE_OBJ_GRIEWANK, DE_OBJ_ROSENBROCK, DE_OBJ_RASTRIGIN}, {},
              {10, 20, 20, 30, 40}, {0.005, 1, 10, 1, 10}, {0, 100, 200, 300, 400}};
    default:
      return {0, 1, {obj}, {100}, {}, {}, {}};
  }
}

// [-100, 100] mapped onto a basic function's customary domain inside hybrid
// and composition functions
static double suite_domain_scale(int fn) {
  switch (fn) {
    case DE_OBJ_RASTRIGIN: return 5.12 / 100.0;
    case DE_OBJ_ROSENBROCK: return 2.048 / 100.0;
    case DE_OBJ_SCHWEFEL: return 1000.0 / 100.0;
    case DE_OBJ_GRIEWANK: return 600.0 / 100.0;
    case DE_OBJ_HGBAT:
    case DE_OBJ_HAPPYCAT:
    case DE_OBJ_KATSUURA:
    case DE_OBJ_GRIEWANK_ROSENBROCK: return 5.0 / 100.0;
    default: return 1.0;
  }
}

// Hybrid split: parts 0..n-2 take ceil(p d) coordinates (integer arithmetic
// on the percentages), the last the rest; false when a part would be empty.
static bool suite_segments(const SuiteSpec& sp, int d, int32_t seg[6]) {
  seg[0] = 0;
  int used = 0;
  for (int q = 0; q + 1 < sp.n; ++q) {
    used += (sp.pct[q] * d + 99) / 100;
    seg[q + 1] = used;
  }
  seg[sp.n] = d;
  for (int q = 0; q < sp.n; ++q)
    if (seg[q + 1] - seg[q] < 1) return false;
  return true;
}

// (shift, rotation) pairs a config carries: n for a composition function
static int suite_pairs(int obj) {
  const SuiteSpec sp = suite_spec(obj);
  return sp.kind == 2 ? sp.n : 1;
}

static de_status validate(const de_config& c, int idx, std::string& why) {
  char b[256];
  auto bad = [&](const char* what) {
    snprintf(b, sizeof b, "config %d: %s", idx, what);
    why = b;
    return DE_ERR_INVALID_ARG;
  };
  if (c.np < 4 || c.np > (1 << 20)) return bad("np must be in [4, 2^20] (three distinct donors besides the target)");
  if (c.d < 1 || c.d > 4096) return bad("d must be in [1, 4096]");
  if (!(c.f >= 0.0 && c.f <= 2.0)) return bad("F must be in [0, 2]");
  if (!(c.cr >= 0.0 && c.cr <= 1.0)) return bad("CR must be in [0, 1]");
  if (!std::isfinite(c.lo) || !std::isfinite(c.hi) || !(c.lo < c.hi)) return bad("bounds must be finite with lo < hi");
  if (c.objective < DE_OBJ_SPHERE || c.objective > DE_OBJ_COMPOSITION3) return bad("objective out of range");
  if (c.objective >= DE_OBJ_ZAKHAROV) {
    if (c.precision != DE_PREC_FP64) return bad("the benchmark suite's objectives run in FP64 only");
    const SuiteSpec sp = suite_spec(c.objective);
    int32_t seg[6];
    if (sp.kind == 1 && !suite_segments(sp, c.d, seg)) return bad("d is too small for this hybrid function's parts");
    if (sp.kind == 2 && c.scale != 1.0)
      return bad("composition functions take scale 1 (each component has its own domain scale)");
  }
  if (c.perm) {
    if (suite_spec(c.objective).kind != 1) return bad("perm applies to the hybrid functions only");
    std::vector<char> seen(c.d, 0);
    for (int j = 0; j < c.d; ++j) {
      if (c.perm[j] < 0 || c.perm[j] >= c.d || seen[c.perm[j]]) return bad("perm is not a permutation of 0..d-1");
      seen[c.perm[j]] = 1;
    }
  }
  if (c.objective == DE_OBJ_ODE) {
    if (c.d != 20) return bad("the ODE objective has d = 20 (stiffness and damping of 10 oscillators)");
    if (c.precision != DE_PREC_FP64) return bad("the ODE objective runs in FP64 only");
    if (c.rot) return bad("the ODE objective takes no rotation");
  }
  if (!std::isfinite(c.scale) || c.scale == 0.0) return bad("scale must be finite and nonzero");
  if (c.run_id >= (1u << 20)) return bad("run_id must be < 2^20");
  if (c.precision < DE_PREC_FP64 || c.precision > DE_PREC_TF32X3) return bad("precision out of range");
  if (c.max_evals < 0 || c.max_generations < 0) return bad("max_evals and max_generations must be >= 0");
  if (c.fp64_band != DE_BAND_NEAR && c.fp64_band != DE_BAND_ALL) return bad("fp64_band out of range");
  if (c.surrogate_k < 0 || c.surrogate_k > 32) return bad("surrogate_k must be in [0, 32]");
  if (c.surrogate_steps < 0 || c.surrogate_steps > 100000) return bad("surrogate_steps must be in [0, 100000]");
  if (c.strategy < DE_RAND1BIN || c.strategy > DE_RAND1EXP) return bad("strategy out of range");
  if (c.surrogate_k >= 2) {
    if (c.precision != DE_PREC_FP64) return bad("surrogate-assisted generations run in FP64 only");
    if (c.d != 20) return bad("the surrogate network takes d = 20");
  }
  if (!std::isfinite(c.target_error) && !(c.target_error < 0)) return bad("target_error must be finite");
  const int pairs = (c.objective >= DE_OBJ_SPHERE && c.objective <= DE_OBJ_COMPOSITION3) ? suite_pairs(c.objective) : 1;
  if (c.shift)
    for (size_t j = 0; j < (size_t)pairs * c.d; ++j)
      if (!std::isfinite(c.shift[j])) return bad("shift has a non-finite entry");
  if (c.rot)
    for (size_t k = 0; k < (size_t)pairs * c.d * c.d; ++k)
      if (!std::isfinite(c.rot[k])) return bad("rotation has a non-finite entry");
  return DE_OK;
}

// Shared memory of one FP64 generation CTA for `rows` rows of stride dp
// (trial, shifted, rotated and second-term buffers).
// A composition function's tile keeps every component's shifted and rotated
// rows: trials plus 2 ncomp buffers.
static size_t gen_smem(int rows, int dp, int ncomp = 1) {
  return (size_t)std::max(4, 1 + 2 * ncomp) * rows * dp * sizeof(double);
}

// Split every run into tiles of at most h->rows targets, of near-equal size.
static de_status build_items(de_handle* h) {
  std::vector<int4> items;
  size_t smem = 0;
  for (int r = 0; r < h->nruns; ++r) {
    RunDesc& R = h->run[r];
    int rows = std::max(1, std::min(h->rows, 8));
    while (rows > 1 && gen_smem(rows, R.dp, suite_comps(R)) > 200 * 1024) --rows;
    const int nt = (R.np + rows - 1) / rows;
    R.rows = (R.np + nt - 1) / nt;  // the largest tile after even splitting
    R.ntiles = nt;
    smem = std::max(smem, gen_smem(R.rows, R.dp, suite_comps(R)));
    for (int t = 0; t < nt; ++t) {
      const int a = (int)((long long)t * R.np / nt), b = (int)((long long)(t + 1) * R.np / nt);
      items.push_back(make_int4(r, t, a, b - a));
    }
  }
  h->smem_gen = smem;
  h->nitems = (int)items.size();
  if (h->d_items) cudaFree(h->d_items);
  h->d_items = nullptr;
  DE_CUDA(h, cudaMalloc(&h->d_items, items.size() * sizeof(int4)));
  DE_CUDA(h, cudaMemcpyAsync(h->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice,
                             h->stream));
  return DE_OK;
}

static de_status upload_desc(de_handle* h) {
  DE_CUDA(h, cudaMemcpyAsync(h->d_run, h->run.data(), h->run.size() * sizeof(RunDesc), cudaMemcpyHostToDevice,
                             h->stream));
  return DE_OK;
}

static void drop_graph(de_handle* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  h->graph_gens = 0;
}

// Island model: forget the last migration (and the mailbox of asynchronous
// migration) and apply the model's group stop to the current state (after
// (re)initialisation, a population change or a restore).
static de_status islands_resync(de_handle* h) {
  if (!h->islands) return DE_OK;
  h->isl.mig_gen = -1;
  h->isl.post_gen = -1;
  DE_CUDA(h, cudaMemcpyAsync(h->d_isl, &h->isl, sizeof(IslandCtl), cudaMemcpyHostToDevice, h->stream));
  k_island_launch(h->d_run, h->d_isl, h->stage, h->nruns, false, false, h->stream);
  DE_CUDA(h, cudaGetLastError());
  return DE_OK;
}

// Enqueue one generation of every run (the kernels skip stopped runs).
static de_status launch_generation(de_handle* h, cudaStream_t s) {
  if (h->prec == DE_PREC_FP64) {
    k_gen_fp64_launch(h->d_run, h->d_items, h->nitems, h->threads, h->smem_gen, h->variants, h->suite, s);
    if (h->islands) k_island_launch(h->d_run, h->d_isl, h->stage, h->nruns, true, h->isl.async != 0, s);
  } else {
    tc_generation_launch(h->tc, h->d_run, s);
  }
  DE_CUDA(h, cudaGetLastError());
  return DE_OK;
}
static de_status launch_generation(de_handle* h) { return launch_generation(h, h->stream); }

static de_status read_states(de_handle* h);

static de_status enqueue_generations(de_handle* h, int64_t n) {
  if (h->surr) {
    // host-driven: each generation ends with the surrogate's screening decision
    for (int64_t k = 0; k < n; ++k) {
      de_status s = read_states(h);
      if (s != DE_OK) return s;
      if (h->h_state[0].stop) break;
      s = surr_generation(*h->surr, h->d_run, h->run[0], h->stream, h->err);
      if (s != DE_OK) return fail(h, s, h->err);
    }
    return DE_OK;
  }
  if (h->fp64_persist) {
    // one cooperative (or one-cluster) launch runs up to 2^20 generations (or
    // stops early)
    for (int64_t left = n; left > 0; left -= (int64_t)1 << 20) {
      const long long g = std::min<int64_t>(left, (int64_t)1 << 20);
      if (h->fp64_cluster)
        DE_CUDA(h, k_gen_fp64_cluster_launch(h->d_run, h->d_items, h->nitems, h->threads, h->smem_gen, h->variants,
                                             h->suite, h->d_ctl64, g, h->stream));
      else
        DE_CUDA(h, k_gen_fp64_persist_launch(h->d_run, h->d_items, h->nitems, h->nruns, h->threads, h->smem_gen,
                                             h->variants, h->suite, h->d_ctl64, g, h->stream, h->test_grid_skip,
                                             h->islands ? h->d_isl : nullptr, h->islands ? &h->stage : nullptr));
    }
    return DE_OK;
  }
  if (h->prec != DE_PREC_FP64 && h->pbatch_on) {
    // one launch of the persistent batch kernel runs up to 2^20 generations
    // of every run (a run's arrival count stays below 2^32)
    for (int64_t left = n; left > 0; left -= (int64_t)1 << 20)
      DE_CUDA(h, pbatch_launch(h->tc.pbatch, h->d_run, h->tc.d_ctl, std::min<int64_t>(left, (int64_t)1 << 20),
                               h->stream, h->test_grid_skip));
    return DE_OK;
  }
  if (h->prec != DE_PREC_FP64 && h->tc.persist.ok) {
    // one persistent launch runs up to 2^20 generations (or stops early); the
    // launch's grid-barrier count stays below 2^32
    for (int64_t left = n; left > 0; left -= (int64_t)1 << 20)
      DE_CUDA(h, persist_launch(h->tc.persist, h->d_run, h->tc.d_ctl, std::min<int64_t>(left, (int64_t)1 << 20),
                                h->stream, h->test_grid_skip));
    return DE_OK;
  }
  const int kChunk = 64;
  if (n >= kChunk) {
    if (!h->graph || h->graph_gens != kChunk) {
      drop_graph(h);
      // capture on the handle's private stream (the caller's stream may be the
      // legacy default stream, which cannot be captured); nothing runs during
      // capture, and the graph is then launched on the caller's stream
      if (!h->cap_stream) DE_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
      cudaGraph_t g = nullptr;
      DE_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      de_status s = DE_OK;
      for (int k = 0; k < kChunk && s == DE_OK; ++k) s = launch_generation(h, h->cap_stream);
      cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
      if (s != DE_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e != cudaSuccess) return fail(h, DE_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&h->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(h, DE_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      h->graph_gens = kChunk;
    }
    while (n >= kChunk) {
      DE_CUDA(h, cudaGraphLaunch(h->graph, h->stream));
      n -= kChunk;
    }
  }
  for (int64_t k = 0; k < n; ++k) {
    de_status s = launch_generation(h);
    if (s != DE_OK) return s;
  }
  return DE_OK;
}

static de_status read_states(de_handle* h) {
  // the states of all runs are one contiguous block starting at run 0's
  DE_CUDA(h, cudaMemcpyAsync(h->h_state, h->run[0].st, h->nruns * sizeof(RunState), cudaMemcpyDeviceToHost,
                             h->stream));
  DE_CUDA(h, cudaStreamSynchronize(h->stream));
  return DE_OK;
}

static de_status check_device_errors(de_handle* h) {
  for (int r = 0; r < h->nruns; ++r) {
    if (h->h_state[r].err & kErrTimeout) return fail(h, DE_ERR_TIMEOUT, "a device-side wait timed out (run " + std::to_string(r) + ")");
    if (h->h_state[r].err & kErrNonFinite)
      return fail(h, DE_ERR_NONFINITE, "every fitness of run " + std::to_string(r) + " is NaN");
  }
  return DE_OK;
}

// (Re)initialise run r's population from the INIT stream and evaluate it.
static de_status init_run(de_handle* h, int r) {
  RunDesc& R = h->run[r];
  RunState st{};
  st.best_idx = -1;
  st.evals = R.np;  // the initial population counts as NP evaluations
  DE_CUDA(h, cudaMemcpyAsync(R.st, &st, sizeof st, cudaMemcpyHostToDevice, h->stream));
  DE_CUDA(h, cudaMemsetAsync(R.X[0], 0, (size_t)R.np * R.dp * sizeof(double), h->stream));
  if (R.obj == DE_OBJ_ODE) k_ode_reference_launch(h->d_run, r, const_cast<double*>(R.ode_ref), h->stream);
  k_init_population_launch(h->d_run, r, R.np, R.dp, h->stream);
  if (R.jde) k_jde_init_launch(h->d_run, r, R.np, h->stream);
  if (h->prec == DE_PREC_FP64) {
    k_eval_rows_launch(h->d_run, r, R, R.X[0], R.dp, R.np, R.f[0], R.fx[0], h->stream);
  } else {
    // split precisions evaluate the initial population in their own precision
    // (values with error bounds, like accepted trials); the best record is
    // made FP64 when a caller reads it
    tc_init_eval_launch(h->tc, h->d_run, r, R, h->stream);
  }
  k_best_init_launch(h->d_run, r, h->stream);
  DE_CUDA(h, cudaGetLastError());
  return DE_OK;
}

// Split precisions keep some fitness values in split precision; the best
// record handed to a caller is made FP64 here (the best row is evaluated in
// FP64 when its stored value is not).
static de_status exact_best(de_handle* h, int r) {
  if (h->prec == DE_PREC_FP64) return DE_OK;
  RunState& st = h->h_state[r];
  if (st.best_idx < 0) return DE_OK;
  const RunDesc& R = h->run[r];
  const int cur = cur_buf(h, st.gen);
  uint8_t fx = 1;
  DE_CUDA(h, cudaMemcpyAsync(&fx, R.fx[cur] + st.best_idx, 1, cudaMemcpyDeviceToHost, h->stream));
  DE_CUDA(h, cudaStreamSynchronize(h->stream));
  if (fx) return DE_OK;
  double* fb = R.f[cur] + st.best_idx;
  k_eval_rows_launch(h->d_run, r, R, R.X[cur] + (size_t)st.best_idx * R.dp, R.dp, 1, fb,
                     R.fx[cur] + st.best_idx, h->stream);
  DE_CUDA(h, cudaGetLastError());
  DE_CUDA(h, cudaMemcpyAsync(&st.best_f, fb, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  DE_CUDA(h, cudaStreamSynchronize(h->stream));
  DE_CUDA(h, cudaMemcpyAsync(&R.st->best_f, &st.best_f, sizeof(double), cudaMemcpyHostToDevice, h->stream));
  DE_CUDA(h, cudaStreamSynchronize(h->stream));
  return DE_OK;
}

// ---------------------------------------------------------------- autotuner
// Picks the rows per tile of the FP64 generation kernel by timing candidates
// on the handle's own problem; results are cached in a text file keyed by
// the problem shape.  The choice never changes results (tiling does not
// enter the arithmetic of a trial), only speed.
static std::string tune_cache_path() {
  const char* p = getenv("DE_GB300_TUNE_CACHE");
  if (p && *p) return p;
  const char* home = getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/de_gb300_tune.txt";
}

static std::string tune_key(const de_handle* h) {
  long long sum_np = 0, sum_d = 0;
  for (auto& R : h->run) {
    sum_np += R.np;
    sum_d += (long long)R.np * R.d;
  }
  char b[256];
  snprintf(b, sizeof b, "gen_fp64v4 runs=%d np0=%d d0=%d obj0=%d rot0=%d sumnp=%lld sumnd=%lld", h->nruns, h->run[0].np,
           h->run[0].d, h->run[0].obj, h->run[0].rotate, sum_np, sum_d);
  return b;
}

// The cache file's entries, parsed once per change of the file (path, size
// and modification time): a de_init then costs one stat, not a read and a
// parse of the whole file.  The last line of a key wins.
struct TuneCache {
  std::mutex mu;
  std::string path;
  long long size = -1, mtime_ns = -1;
  std::map<std::string, int> entries;
};
static TuneCache g_tune;

static void tune_refresh(const std::string& path) {
  struct stat sb;
  if (stat(path.c_str(), &sb) != 0) {
    g_tune.path = path;
    g_tune.size = g_tune.mtime_ns = -1;
    g_tune.entries.clear();
    return;
  }
  const long long mt = (long long)sb.st_mtim.tv_sec * 1000000000LL + sb.st_mtim.tv_nsec;
  if (path == g_tune.path && (long long)sb.st_size == g_tune.size && mt == g_tune.mtime_ns) return;
  g_tune.path = path;
  g_tune.size = (long long)sb.st_size;
  g_tune.mtime_ns = mt;
  g_tune.entries.clear();
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return;
  char line[512];
  while (fgets(line, sizeof line, f)) {
    char* bar = strchr(line, '|');
    if (!bar) continue;
    *bar = 0;
    g_tune.entries[line] = atoi(bar + 1);
  }
  fclose(f);
}

static bool tune_lookup(const std::string& key, int& rows) {
  std::lock_guard<std::mutex> lk(g_tune.mu);
  tune_refresh(tune_cache_path());
  const auto it = g_tune.entries.find(key);
  if (it == g_tune.entries.end() || it->second <= 0) return false;
  rows = it->second;
  return true;
}

static void tune_store(const std::string& key, int rows) {
  std::lock_guard<std::mutex> lk(g_tune.mu);
  std::string p = tune_cache_path();
  const size_t slash = p.find_last_of('/');
  if (slash != std::string::npos && slash > 0) mkdir(p.substr(0, slash).c_str(), 0755);
  FILE* f = fopen(p.c_str(), "a");
  if (!f) return;
  fprintf(f, "%s|%d\n", key.c_str(), rows);
  fclose(f);
  g_tune.size = g_tune.mtime_ns = -1;  // re-read on the next lookup (other processes may append too)
}

static int heuristic_rows(const de_handle* h, int nsm) {
  long long np_total = 0;
  for (auto& R : h->run) np_total += R.np;
  // about one CTA per SM, at most 8 rows (one warp per target)
  return (int)std::max(1LL, std::min(8LL, (np_total + nsm - 1) / nsm));
}

// The cooperative persistent FP64 kernel applies to runs without a surrogate
// or islands whose tiles all fit on the device at once (the grid barrier's
// count, tiles x 2^20 generations per launch, stays below 2^32);
// DE_GB300_FP64_PERSIST=0 disables it, =1 forces it where it applies.
static bool fp64_persist_ok(const de_handle* h) {
  if (h->prec != DE_PREC_FP64 || h->surr || (h->islands && h->suite) || !h->d_ctl64 || h->nitems >= 4096) return false;
  if (const char* e = getenv("DE_GB300_FP64_PERSIST"))
    if (e[0] == '0') return false;
  return h->nitems <= k_gen_fp64_persist_capacity(h->threads, h->smem_gen, h->variants, h->suite, h->islands);
}

// ... and as one thread-block cluster: one run of at most 8 tiles.
static bool fp64_cluster_ok(const de_handle* h) {
  return h->nruns == 1 && fp64_persist_ok(h) &&
         k_gen_fp64_cluster_fits(h->nitems, h->threads, h->smem_gen, h->variants, h->suite);
}

static de_status autotune_fp64(de_handle* h, int nsm) {
  const char* env = getenv("DE_GB300_AUTOTUNE");
  const bool enabled = !(env && env[0] == '0');
  h->rows = heuristic_rows(h, nsm);
  if (!enabled) return DE_OK;
  const std::string key = tune_key(h);
  int cached = 0;
  if (tune_lookup(key, cached)) {
    // value: rows per tile, plus 100 x the mode that won (0: one kernel per
    // generation, 1: cooperative persistent kernel, 2: the same as one cluster)
    h->rows = cached % 100;
    h->fp64_persist = cached >= 100;
    h->fp64_cluster = cached >= 200;
    return DE_OK;
  }
  // candidates are timed on the freshly initialised problem, which is then
  // initialised again (initialisation is a pure function of the seed)
  cudaEvent_t e0, e1;
  DE_CUDA(h, cudaEventCreate(&e0));
  DE_CUDA(h, cudaEventCreate(&e1));
  float best_ms = 1e30f;
  int best_rows = h->rows, best_mode = 0;
  std::vector<RunDesc> saved = h->run;
  for (auto& R : h->run) {
    R.target = 0.0;  // no stop rule while timing
    R.max_evals = 0;
    R.max_gens = INT64_MAX / 4;
  }
  de_status st_all = DE_OK;
  for (int rows : {1, 2, 3, 4, 5, 6, 7, 8}) {
    h->rows = rows;
    st_all = build_items(h);
    if (st_all == DE_OK) st_all = upload_desc(h);
    if (st_all != DE_OK) break;
    k_configure(h->smem_gen);
    for (int r = 0; r < h->nruns; ++r) {
      int32_t zero = 0;
      DE_CUDA(h, cudaMemcpyAsync(&h->run[r].st->stop, &zero, sizeof zero, cudaMemcpyHostToDevice, h->stream));
    }
    for (int k = 0; k < 2; ++k) launch_generation(h);
    DE_CUDA(h, cudaEventRecord(e0, h->stream));
    const int reps = 5;
    for (int k = 0; k < reps; ++k) launch_generation(h);
    DE_CUDA(h, cudaEventRecord(e1, h->stream));
    DE_CUDA(h, cudaEventSynchronize(e1));
    float ms = 0.f;
    DE_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms * 0.97f) {
      best_ms = ms;
      best_rows = rows;
      best_mode = 0;
    }
    // the same tiles in one cooperative launch, and as one cluster
    for (int mode = 1; mode <= 2 && st_all == DE_OK; ++mode) {
      if (mode == 1 ? !fp64_persist_ok(h) : !fp64_cluster_ok(h)) continue;
      for (int r = 0; r < h->nruns; ++r) {
        int32_t zero = 0;
        DE_CUDA(h, cudaMemcpyAsync(&h->run[r].st->stop, &zero, sizeof zero, cudaMemcpyHostToDevice, h->stream));
      }
      h->fp64_persist = true;
      h->fp64_cluster = mode == 2;
      st_all = enqueue_generations(h, 2);
      if (st_all == DE_OK) {
        DE_CUDA(h, cudaEventRecord(e0, h->stream));
        st_all = enqueue_generations(h, reps);
        DE_CUDA(h, cudaEventRecord(e1, h->stream));
        DE_CUDA(h, cudaEventSynchronize(e1));
        DE_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
      }
      h->fp64_persist = false;
      h->fp64_cluster = false;
      if (st_all == DE_OK && ms < best_ms * 0.97f) {
        best_ms = ms;
        best_rows = rows;
        best_mode = mode;
      }
    }
    if (st_all != DE_OK) break;
  }
  for (int r = 0; r < h->nruns; ++r) {
    // keep the tile fields, restore the stop rule
    saved[r].rows = h->run[r].rows;
    saved[r].ntiles = h->run[r].ntiles;
  }
  h->run = saved;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st_all != DE_OK) return st_all;
  h->rows = best_rows;
  h->fp64_persist = best_mode >= 1;
  h->fp64_cluster = best_mode == 2;
  tune_store(key, best_rows + 100 * best_mode);
  return DE_OK;
}

// Split precisions, three-kernel path: targets per trial CTA and the K chunk
// of the fitness kernel, timed on the handle's own problem and cached like
// the FP64 choice (neither changes results).  The persistent cluster kernel
// takes its geometry from occupancy and is not tuned here.
static std::string tune_key_split(const de_handle* h) {
  long long sum_np = 0, sum_d = 0;
  for (auto& R : h->run) {
    sum_np += R.np;
    sum_d += (long long)R.np * R.d;
  }
  char b[256];
  snprintf(b, sizeof b, "split_v4 prec=%d runs=%d np0=%d d0=%d obj0=%d sumnp=%lld sumnd=%lld", h->prec, h->nruns,
           h->run[0].np, h->run[0].d, h->run[0].obj, sum_np, sum_d);
  return b;
}

static de_status autotune_split(de_handle* h) {
  const char* env = getenv("DE_GB300_AUTOTUNE");
  if ((env && env[0] == '0') || h->tc.persist.ok) return DE_OK;
  const std::string key = tune_key_split(h);
  // cached value: 1000 x trial-kernel instance (1: held to 85 registers) + 100
  // x targets per trial CTA + 10 x K-chunk divisor + pipeline stages
  int code = 0;
  if (tune_lookup(key, code)) {
    h->tc.trial_occ = code / 1000;
    de_status s = tc_set_geometry(h->tc, h->run, (code / 100) % 10, (code / 10) % 10, code % 10, h->stream, h->err);
    if (s == DE_OK) s = upload_desc(h);
    return s;
  }
  cudaEvent_t e0, e1;
  DE_CUDA(h, cudaEventCreate(&e0));
  DE_CUDA(h, cudaEventCreate(&e1));
  std::vector<RunDesc> saved = h->run;
  for (auto& R : h->run) {
    R.target = 0.0;  // no stop rule while timing
    R.max_evals = 0;
    R.max_gens = INT64_MAX / 4;
  }
  float best_ms = 1e30f;
  int best = 0;
  de_status st_all = DE_OK;
  for (int oc = 0; oc < 2 && st_all == DE_OK; ++oc)
  for (int tr : {2, 4, 8}) {
    h->tc.trial_occ = oc;
    for (int kd : {1, 2, 4})
      for (int ns : {2, 4}) {
      st_all = tc_set_geometry(h->tc, h->run, tr, kd, ns, h->stream, h->err);
      if (st_all == DE_OK) st_all = upload_desc(h);
      if (st_all != DE_OK) break;
      for (int r = 0; r < h->nruns; ++r) {
        int32_t zero = 0;
        DE_CUDA(h, cudaMemcpyAsync(&h->run[r].st->stop, &zero, sizeof zero, cudaMemcpyHostToDevice, h->stream));
      }
      launch_generation(h);
      DE_CUDA(h, cudaEventRecord(e0, h->stream));
      for (int k = 0; k < 6; ++k) launch_generation(h);
      DE_CUDA(h, cudaEventRecord(e1, h->stream));
      DE_CUDA(h, cudaEventSynchronize(e1));
      float ms = 0.f;
      DE_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms * 0.97f) {
        best_ms = ms;
        best = oc * 1000 + tr * 100 + kd * 10 + ns;
      }
      }
    if (st_all != DE_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (size_t r = 0; r < saved.size(); ++r) {
    saved[r].kc = h->run[r].kc;
    saved[r].nstage = h->run[r].nstage;
  }
  h->run = saved;
  if (st_all != DE_OK) return st_all;
  h->tc.trial_occ = best / 1000;
  de_status s = tc_set_geometry(h->tc, h->run, (best / 100) % 10, (best / 10) % 10, best % 10, h->stream, h->err);
  if (s == DE_OK) s = upload_desc(h);
  if (s == DE_OK) tune_store(key, best);
  return s;
}

// The persistent split-precision form and its tile: the cluster kernel with
// rows per cluster timed from 128 down (multiples of the cluster size), and
// the CTA-local kernel with targets per CTA timed from the fewest that keep
// every CTA resident up to 16.  Both are timed on the handle's own problem and
// the faster is cached like the other choices (value: 1000 x form + rows); the
// choice never changes results.  DE_GB300_PERSIST_ROWS /
// DE_GB300_PERSIST_CTA_ROWS fix the tile instead.
static std::string tune_key_persist(const de_handle* h) {
  const RunDesc& R = h->run[0];
  char b[256];
  // the debug capture and the band policy change the kernel's timing (the
  // capture orders the stop decision before the trials)
  snprintf(b, sizeof b, "persist_v3 prec=%d np=%d d=%d obj=%d rot=%d var=%d cl=%d cta=%d dbg=%d band=%d", h->prec,
           R.np, R.d, R.obj, R.rotate, h->tc.persist.var ? 1 : 0, h->tc.persist.cl_ok ? 1 : 0,
           h->tc.persist.cta_ok ? 1 : 0, R.dbg_trial ? 1 : 0, R.band_all);
  return b;
}

static bool persist_choose(PersistPlan& pp, const RunDesc& R, int mode, int rows) {
  if (mode == 1) {
    if (!pp.cta_ok || !persist_cta_set_rows(pp, R, rows)) return false;
  } else {
    if (!pp.cl_ok || !persist_set_rows(pp, R, rows)) return false;
  }
  pp.mode = mode;
  return true;
}

static de_status autotune_persist(de_handle* h) {
  const char* env = getenv("DE_GB300_AUTOTUNE");
  PersistPlan& pp = h->tc.persist;
  if ((env && env[0] == '0') || !pp.ok || getenv("DE_GB300_PERSIST_ROWS") || getenv("DE_GB300_PERSIST_CTA_ROWS"))
    return DE_OK;
  const std::string key = tune_key_persist(h);
  int cached = 0;
  if (tune_lookup(key, cached) && persist_choose(pp, h->run[0], cached / 1000, cached % 1000)) return DE_OK;
  // candidates: (form, rows)
  std::vector<std::pair<int, int>> cand;
  if (pp.cl_ok)
    for (int rows = pp.prows; rows >= pp.C; rows -= pp.C) cand.push_back({0, rows});
  if (pp.cta_ok) {
    const int first = pp.cta_rows;
    for (int rows : {first, first + 1, first + 2, 8, 10, 12, 16})
      if (rows >= first && rows <= 16 &&
          std::find(cand.begin(), cand.end(), std::make_pair(1, rows)) == cand.end())
        cand.push_back({1, rows});
  }
  const PersistPlan keep = pp;
  cudaEvent_t e0, e1;
  DE_CUDA(h, cudaEventCreate(&e0));
  DE_CUDA(h, cudaEventCreate(&e1));
  std::vector<RunDesc> saved = h->run;
  for (auto& R : h->run) {
    R.target = 0.0;  // no stop rule while timing
    R.max_evals = 0;
    R.max_gens = INT64_MAX / 4;
  }
  de_status st_all = upload_desc(h);
  float best_ms = 1e30f;
  std::pair<int, int> best = {keep.mode, keep.mode == 1 ? keep.cta_rows : keep.prows};
  for (const auto& c : cand) {
    if (st_all != DE_OK) break;
    if (!persist_choose(pp, h->run[0], c.first, c.second)) continue;
    int32_t zero = 0;
    DE_CUDA(h, cudaMemcpyAsync(&h->run[0].st->stop, &zero, sizeof zero, cudaMemcpyHostToDevice, h->stream));
    st_all = enqueue_generations(h, 4);
    float ms = 1e30f;
    for (int rep = 0; rep < 2 && st_all == DE_OK; ++rep) {
      DE_CUDA(h, cudaEventRecord(e0, h->stream));
      st_all = enqueue_generations(h, 24);
      DE_CUDA(h, cudaEventRecord(e1, h->stream));
      DE_CUDA(h, cudaEventSynchronize(e1));
      float t = 0.f;
      DE_CUDA(h, cudaEventElapsedTime(&t, e0, e1));
      ms = std::min(ms, t);
    }
    if (st_all == DE_OK && ms < best_ms * 0.98f) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->run = saved;
  pp = keep;
  persist_choose(pp, h->run[0], best.first, best.second);
  if (st_all != DE_OK) return st_all;
  const de_status s = upload_desc(h);
  if (s == DE_OK) tune_store(key, 1000 * best.first + best.second);
  return s;
}

// Batches in split precision: the persistent batch kernel (kernel path 5,
// double-buffered population) against the three-kernel path in CUDA graphs
// (path 1, population updated in place), timed on the handle's own problem
// after the three-kernel geometry is tuned; the faster is kept and cached.
// DE_GB300_PERSIST_BATCH=1 forces path 5 where it applies, =0 disables it.
static void set_dbuf(de_handle* h, bool on) {
  h->dbuf = on;
  for (auto& R : h->run) R.dbuf = on ? 1 : 0;
}

static de_status choose_pbatch(de_handle* h) {
  if (!h->tc.pbatch.ok) return DE_OK;
  const char* force = getenv("DE_GB300_PERSIST_BATCH");
  const char* env = getenv("DE_GB300_AUTOTUNE");
  bool on = false;
  if (force && force[0] == '1') {
    on = true;
  } else if (!(env && env[0] == '0')) {
    const std::string key = "pbatch_v2 " + tune_key_split(h);
    int cached = 0;
    if (tune_lookup(key, cached)) {
      on = cached == 1;
    } else {
      cudaEvent_t e0, e1;
      DE_CUDA(h, cudaEventCreate(&e0));
      DE_CUDA(h, cudaEventCreate(&e1));
      std::vector<RunDesc> saved = h->run;
      for (auto& R : h->run) {
        R.target = 0.0;  // no stop rule while timing
        R.max_evals = 0;
        R.max_gens = INT64_MAX / 4;
      }
      auto time_gens = [&](bool pb, float& ms_per_gen) -> de_status {
        set_dbuf(h, pb);
        h->pbatch_on = pb;
        de_status s = upload_desc(h);
        for (int r = 0; r < h->nruns && s == DE_OK; ++r) {
          int32_t zero = 0;
          DE_CUDA(h, cudaMemcpyAsync(&h->run[r].st->stop, &zero, sizeof zero, cudaMemcpyHostToDevice, h->stream));
        }
        const int G = 12;
        if (s == DE_OK) s = enqueue_generations(h, 2);
        DE_CUDA(h, cudaEventRecord(e0, h->stream));
        if (s == DE_OK) s = enqueue_generations(h, G);
        DE_CUDA(h, cudaEventRecord(e1, h->stream));
        DE_CUDA(h, cudaEventSynchronize(e1));
        float ms = 0.f;
        DE_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
        ms_per_gen = ms / G;
        return s;
      };
      float ms_graph = 0.f, ms_pb = 0.f;
      de_status s = time_gens(false, ms_graph);
      if (s == DE_OK) s = time_gens(true, ms_pb);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      h->run = saved;
      if (s != DE_OK) return s;
      on = ms_pb < ms_graph * 0.98f;
      tune_store(key, on ? 1 : 2);
    }
  }
  h->pbatch_on = on;
  set_dbuf(h, on);
  return upload_desc(h);
}

// ---------------------------------------------------------------- C ABI
extern "C" {

const char* de_version(void) { return kVersion; }

const char* de_status_string(de_status s) {
  switch (s) {
    case DE_OK: return "DE_OK";
    case DE_ERR_INVALID_ARG: return "DE_ERR_INVALID_ARG";
    case DE_ERR_CUDA: return "DE_ERR_CUDA";
    case DE_ERR_OOM: return "DE_ERR_OOM";
    case DE_ERR_TIMEOUT: return "DE_ERR_TIMEOUT";
    case DE_ERR_NONFINITE: return "DE_ERR_NONFINITE";
    case DE_ERR_STATE: return "DE_ERR_STATE";
    case DE_ERR_IO: return "DE_ERR_IO";
    case DE_ERR_UNSUPPORTED: return "DE_ERR_UNSUPPORTED";
  }
  return "DE_ERR_UNKNOWN";
}

const char* de_last_error(de_handle* h) { return h ? h->err.c_str() : g_err.c_str(); }

de_status de_destroy(de_handle* h) {
  if (!h) return DE_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graph(h);
  surr_destroy(h->surr);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  tc_plan_free(h->tc);
  if (h->d_items) cudaFree(h->d_items);
  if (h->d_run) cudaFree(h->d_run);
  if (h->d_ctl64) cudaFree(h->d_ctl64);
  if (h->isl_mem) cudaFree(h->isl_mem);
  if (h->arena) cudaFree(h->arena);
  if (h->h_state) cudaFreeHost(h->h_state);
  delete h;
  return DE_OK;
}

// 64-bit FNV-1a over 8-byte words (the problem data can be 4096^2 doubles).
static uint64_t fnv_words(uint64_t h, const void* data, size_t bytes) {
  const uint8_t* p = (const uint8_t*)data;
  for (size_t i = 0; i < bytes; i += 8) {
    uint64_t w = 0;
    memcpy(&w, p + i, std::min<size_t>(8, bytes - i));
    h = (h ^ w) * 0x100000001B3ull;
  }
  return h;
}

// Identity of a run's problem for checkpoints: everything that fixes its
// trajectory except the stopping limits (a resumed run may get a new budget).
static uint64_t problem_fingerprint(const de_config& c) {
  uint64_t h = 0xCBF29CE484222325ull;
  const int32_t ints[8] = {c.np, c.d, c.objective, c.precision, c.strategy, c.jde ? 1 : 0, c.fp64_band,
                           (int32_t)c.run_id};
  const double reals[6] = {c.f, c.cr, c.lo, c.hi, c.scale, 0.0};
  h = fnv_words(h, ints, sizeof ints);
  h = fnv_words(h, reals, sizeof reals);
  h = fnv_words(h, &c.seed, sizeof c.seed);
  const int pairs = (c.objective >= DE_OBJ_SPHERE && c.objective <= DE_OBJ_COMPOSITION3) ? suite_pairs(c.objective) : 1;
  const uint64_t none = 0x9E3779B97F4A7C15ull;
  h = c.shift ? fnv_words(h, c.shift, (size_t)pairs * c.d * sizeof(double)) : fnv_words(h, &none, 8);
  h = c.rot ? fnv_words(h, c.rot, (size_t)pairs * c.d * c.d * sizeof(double)) : fnv_words(h, &none, 8);
  h = c.perm ? fnv_words(h, c.perm, (size_t)c.d * sizeof(int32_t)) : fnv_words(h, &none, 8);
  return h;
}

de_status de_init_batch(const de_config* cfgs, int32_t nruns, void* cuda_stream, de_handle** out) {
  g_err.clear();
  if (!out) return fail(nullptr, DE_ERR_INVALID_ARG, "out is NULL");
  if (!cfgs || nruns < 1) return fail(nullptr, DE_ERR_INVALID_ARG, "need at least one config");
  for (int r = 0; r < nruns; ++r) {
    std::string why;
    if (validate(cfgs[r], r, why) != DE_OK) return fail(nullptr, DE_ERR_INVALID_ARG, why);
    if (cfgs[r].precision != cfgs[0].precision)
      return fail(nullptr, DE_ERR_INVALID_ARG, "all runs of a batch must share the precision");
    if (cfgs[r].surrogate_k >= 2 && nruns != 1)
      return fail(nullptr, DE_ERR_INVALID_ARG, "surrogate-assisted generations take one run per handle");
    if ((cfgs[r].strategy != DE_RAND1BIN || cfgs[r].jde) && cfgs[r].surrogate_k >= 2)
      return fail(nullptr, DE_ERR_UNSUPPORTED,
                  "the best/1/bin and rand/1/exp strategies and jDE run without a surrogate");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, DE_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  // three attributes (cudaGetDeviceProperties fills the whole structure and
  // costs a good part of a de_init)
  int cc_major = 0, cc_minor = 0, nsm = 0;
  e = cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(nullptr, DE_ERR_CUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
  if (!(cc_major == 10 && cc_minor == 3))
    return fail(nullptr, DE_ERR_UNSUPPORTED, "this library is built for compute capability 10.3 (sm_103a)");

  de_handle* h = new de_handle();
  h->stream = (cudaStream_t)cuda_stream;
  h->device = dev;
  h->nruns = nruns;
  h->prec = cfgs[0].precision;
  for (int r = 0; r < nruns; ++r) {
    h->variants = h->variants || cfgs[r].strategy != DE_RAND1BIN || cfgs[r].jde;
    h->suite = h->suite || cfgs[r].objective >= DE_OBJ_ZAKHAROV;
  }
  h->cfg.assign(cfgs, cfgs + nruns);
  for (int r = 0; r < nruns; ++r) h->fingerprint.push_back(problem_fingerprint(cfgs[r]));
  for (auto& c : h->cfg) {
    c.shift = nullptr;
    c.rot = nullptr;
    c.perm = nullptr;
  }
  h->run.resize(nruns);

  // ---- arena layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = align_up(off, 256);
    size_t o = off;
    off += std::max<size_t>(bytes, 1);
    return o;
  };
  struct Offs {
    size_t X0, X1, f0, f1, fx0, fx1, o, MT, Mr, st, part, T, ref, jF0, jF1, jC0, jC1, perm;
    size_t dbg_idx, dbg_jrand, dbg_mask, dbg_trial, dbg_ftrial, dbg_accept, dbg_fp64, dbg_cand;
  };
  std::vector<Offs> offs(nruns);
  const size_t states_off = take((size_t)nruns * sizeof(RunState));  // one contiguous block
  for (int r = 0; r < nruns; ++r) {
    const de_config& c = cfgs[r];
    const int dp = (c.d + 3) / 4 * 4;
    const size_t pop = (size_t)c.np * dp * sizeof(double);
    Offs& O = offs[r];
    O.X0 = take(pop);
    O.X1 = take(pop);
    O.f0 = take(c.np * sizeof(double));
    O.f1 = take(c.np * sizeof(double));
    O.fx0 = take(c.np);
    O.fx1 = take(c.np);
    const int pairs = suite_pairs(c.objective);
    O.o = take((size_t)pairs * dp * sizeof(double));
    O.MT = c.rot ? take((size_t)pairs * c.d * c.d * sizeof(double)) : 0;
    O.perm = suite_spec(c.objective).kind == 1 ? take((size_t)c.d * sizeof(int32_t)) : 0;
    O.Mr = (c.rot && c.precision != DE_PREC_FP64) ? take((size_t)c.d * c.d * sizeof(double)) : 0;
    O.st = states_off + (size_t)r * sizeof(RunState);
    O.part = take((size_t)2 * c.np * sizeof(BestPartial));  // double buffered by generation parity
    const bool split = c.precision != DE_PREC_FP64;
    O.T = split ? take(pop) : 0;
    O.ref = c.objective == DE_OBJ_ODE ? take((size_t)kOdeSteps * kOdeN * sizeof(double)) : 0;
    if (c.jde) {
      O.jF0 = take(c.np * sizeof(double));
      O.jF1 = take(c.np * sizeof(double));
      O.jC0 = take(c.np * sizeof(double));
      O.jC1 = take(c.np * sizeof(double));
    }
    if (c.debug_capture) {
      const int nw = (c.d + 31) / 32;
      O.dbg_idx = take((size_t)c.np * 3 * sizeof(int32_t));
      O.dbg_jrand = take((size_t)c.np * sizeof(int32_t));
      O.dbg_mask = take((size_t)c.np * nw * sizeof(uint32_t));
      O.dbg_trial = take((size_t)c.np * c.d * sizeof(double));
      O.dbg_ftrial = take((size_t)c.np * sizeof(double));
      O.dbg_accept = take((size_t)c.np);
      O.dbg_fp64 = take((size_t)c.np);
      O.dbg_cand = take((size_t)c.np * sizeof(int32_t));
    }
  }
  h->arena_bytes = align_up(off, 256);
  e = cudaMalloc(&h->arena, h->arena_bytes);
  if (e != cudaSuccess) {
    std::string m = std::string("cudaMalloc(") + std::to_string(h->arena_bytes) + "): " + cudaGetErrorString(e);
    de_destroy(h);
    return fail(nullptr, e == cudaErrorMemoryAllocation ? DE_ERR_OOM : DE_ERR_CUDA, m);
  }
  auto fin = [&](de_status s) {
    if (s != DE_OK) {
      std::string m = h->err;
      de_destroy(h);
      g_err = m;
      return s;
    }
    *out = h;
    return DE_OK;
  };
#define TRY(x)                      \
  do {                              \
    de_status s_ = (x);             \
    if (s_ != DE_OK) return fin(s_); \
  } while (0)
  cudaError_t ce = cudaMallocHost(&h->h_state, nruns * sizeof(RunState));
  if (ce != cudaSuccess) return fin(fail(h, DE_ERR_OOM, "cudaMallocHost failed"));
  ce = cudaMalloc(&h->d_run, nruns * sizeof(RunDesc));
  if (ce != cudaSuccess) return fin(fail(h, DE_ERR_OOM, "cudaMalloc(run table) failed"));
  ce = cudaMemsetAsync(h->arena, 0, h->arena_bytes, h->stream);
  if (ce != cudaSuccess) return fin(fail(h, DE_ERR_CUDA, std::string("memset: ") + cudaGetErrorString(ce)));

  std::vector<double> tmp;
  for (int r = 0; r < nruns; ++r) {
    const de_config& c = cfgs[r];
    const Offs& O = offs[r];
    RunDesc& R = h->run[r];
    memset(&R, 0, sizeof R);
    R.np = c.np;
    R.d = c.d;
    R.dp = (c.d + 3) / 4 * 4;
    R.obj = c.objective;
    R.F = c.f;
    R.CR = c.cr;
    R.lo = c.lo;
    R.hi = c.hi;
    R.scale = c.scale;
    R.lo_key = ordered_key(c.lo);
    R.lo_half = 0.5 * c.lo;
    R.hi_half = 0.5 * c.hi;
    R.hi_key = ordered_key(c.hi);
    R.lo_hk = hi_key32(c.lo);
    R.hi_hk = hi_key32(c.hi);
    R.unit_scale = c.scale == 1.0;
    R.cr_thr = cr_threshold(c.cr);
    R.seed = c.seed;
    R.run_id = c.run_id;
    R.rotate = c.rot != nullptr;
    R.target = c.target_error;
    R.max_evals = c.max_evals;
    R.max_gens = c.max_generations;
    R.prec = c.precision;
    R.nw = (c.d + 31) / 32;
    R.band_all = c.fp64_band == DE_BAND_ALL;
    char* A = h->arena;
    R.X[0] = (double*)(A + O.X0);
    R.X[1] = (double*)(A + O.X1);
    R.f[0] = (double*)(A + O.f0);
    R.f[1] = (double*)(A + O.f1);
    R.fx[0] = (uint8_t*)(A + O.fx0);
    R.fx[1] = (uint8_t*)(A + O.fx1);
    R.o = (const double*)(A + O.o);
    R.MT = R.rotate ? (const double*)(A + O.MT) : nullptr;
    R.Mrow = (R.rotate && c.precision != DE_PREC_FP64) ? (const double*)(A + O.Mr) : nullptr;
    R.st = (RunState*)(A + O.st);
    R.part = (BestPartial*)(A + O.part);
    if (c.precision != DE_PREC_FP64) {
      R.T = (double*)(A + O.T);
    }
    if (c.objective == DE_OBJ_ODE) R.ode_ref = (const double*)(A + O.ref);
    R.strategy = c.strategy;
    R.jde = c.jde ? 1 : 0;
    {
      const SuiteSpec sp = suite_spec(c.objective);
      R.nc = sp.n;
      for (int q = 0; q < sp.n; ++q) {
        R.sfn[q] = sp.fn[q];
        R.sscale[q] = suite_domain_scale(sp.fn[q]);
        R.ssigma[q] = sp.sigma[q];
        R.slambda[q] = sp.lambda[q];
        R.sbias[q] = sp.bias[q];
      }
      if (sp.kind == 1) {
        suite_segments(sp, c.d, R.seg);
        R.perm = (const int32_t*)(A + O.perm);
      }
      for (int q = 0; q < sp.n; ++q) {
        const int n = sp.kind == 1 ? R.seg[q + 1] - R.seg[q] : c.d;
        R.skex[q] = 10.0 / std::pow((double)n, 1.2);
      }
    }
    if (c.jde) {
      R.jF[0] = (double*)(A + O.jF0);
      R.jF[1] = (double*)(A + O.jF1);
      R.jCR[0] = (double*)(A + O.jC0);
      R.jCR[1] = (double*)(A + O.jC1);
    }
    if (c.debug_capture) {
      R.dbg_idx = (int32_t*)(A + O.dbg_idx);
      R.dbg_jrand = (int32_t*)(A + O.dbg_jrand);
      R.dbg_mask = (uint32_t*)(A + O.dbg_mask);
      R.dbg_trial = (double*)(A + O.dbg_trial);
      R.dbg_ftrial = (double*)(A + O.dbg_ftrial);
      R.dbg_accept = (uint8_t*)(A + O.dbg_accept);
      R.dbg_fp64 = (uint8_t*)(A + O.dbg_fp64);
      R.dbg_cand = (int32_t*)(A + O.dbg_cand);
    }
    const int pairs = suite_pairs(c.objective);
    if (c.shift) {
      ce = cudaMemcpy2DAsync((void*)R.o, R.dp * sizeof(double), c.shift, c.d * sizeof(double), c.d * sizeof(double),
                             pairs, cudaMemcpyHostToDevice, h->stream);
      if (ce != cudaSuccess) return fin(fail(h, DE_ERR_CUDA, std::string("copy shift: ") + cudaGetErrorString(ce)));
    }
    if (R.perm) {
      std::vector<int32_t> pm(c.d);
      for (int j = 0; j < c.d; ++j) pm[j] = c.perm ? c.perm[j] : j;
      ce = cudaMemcpyAsync((void*)R.perm, pm.data(), c.d * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);  // pm goes out of scope
      if (ce != cudaSuccess) return fin(fail(h, DE_ERR_CUDA, std::string("copy perm: ") + cudaGetErrorString(ce)));
    }
    if (c.rot) {
      // every component's M, transposed
      tmp.resize((size_t)pairs * c.d * c.d);
      for (int q = 0; q < pairs; ++q) {
        const double* Mq = c.rot + (size_t)q * c.d * c.d;
        double* Tq = tmp.data() + (size_t)q * c.d * c.d;
        for (int j = 0; j < c.d; ++j)
          for (int k = 0; k < c.d; ++k) Tq[(size_t)k * c.d + j] = Mq[(size_t)j * c.d + k];
      }
      ce = cudaMemcpyAsync((void*)R.MT, tmp.data(), tmp.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream);
      if (ce == cudaSuccess && R.Mrow)
        ce = cudaMemcpyAsync((void*)R.Mrow, c.rot, (size_t)c.d * c.d * sizeof(double), cudaMemcpyHostToDevice,
                             h->stream);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);  // tmp is reused
      if (ce != cudaSuccess) return fin(fail(h, DE_ERR_CUDA, std::string("copy rotation: ") + cudaGetErrorString(ce)));
      double rn = 0.0;
      for (int j = 0; j < c.d; ++j) {
        double s = 0.0;
        for (int k = 0; k < c.d; ++k) s += c.rot[(size_t)j * c.d + k] * c.rot[(size_t)j * c.d + k];
        rn = std::max(rn, std::sqrt(s));
      }
      R.rownorm = (float)rn;
    } else {
      R.rownorm = 1.0f;
    }
  }
  if (h->prec != DE_PREC_FP64) {
    TRY(tc_plan_build(h->tc, h->run, cfgs, h->prec, h->stream, h->err));
    h->dbuf = h->tc.persist.ok;
  }
  for (auto& R : h->run) R.dbuf = h->dbuf ? 1 : 0;
  TRY(build_items(h));
  TRY(upload_desc(h));
  k_configure(h->smem_gen);
  for (int r = 0; r < nruns; ++r) TRY(init_run(h, r));
  if (h->prec == DE_PREC_FP64 && cfgs[0].surrogate_k < 2) {
    ce = cudaMalloc(&h->d_ctl64, sizeof(PersistCtl));
    if (ce != cudaSuccess) return fin(fail(h, DE_ERR_OOM, "cudaMalloc(persistent control) failed"));
    TRY(autotune_fp64(h, nsm));
    TRY(build_items(h));
    TRY(upload_desc(h));
    k_configure(h->smem_gen);
    if (const char* e = getenv("DE_GB300_FP64_PERSIST")) {
      // forced on where it applies: 1 cooperative launch, 2 one cluster
      if (e[0] == '1' || e[0] == '2') h->fp64_persist = true;
      h->fp64_cluster = e[0] == '2';
    }
    if (h->fp64_cluster && !fp64_cluster_ok(h)) h->fp64_cluster = false;
    if (h->fp64_persist && !fp64_persist_ok(h)) h->fp64_persist = h->fp64_cluster = false;
    // the failure-detection test applies to the generations after set-up
    // (not to the autotuner's timing launches)
    if (const char* v = getenv("DE_GB300_TEST_GRID_TIMEOUT")) h->test_grid_skip = std::max(0, atoi(v));
    for (int r = 0; r < nruns; ++r) TRY(init_run(h, r));
  } else if (h->prec != DE_PREC_FP64) {
    if (h->tc.persist.ok) {
      TRY(autotune_persist(h));
    } else {
      TRY(autotune_split(h));
      TRY(choose_pbatch(h));
    }
    // the failure-detection test applies to the generations after set-up
    if (const char* v = getenv("DE_GB300_TEST_GRID_TIMEOUT")) h->test_grid_skip = std::max(0, atoi(v));
    for (int r = 0; r < nruns; ++r) {
      TRY(init_run(h, r));
      // the counters start after the timing generations
      if (h->run[r].stats) {
        ce = cudaMemsetAsync(h->run[r].stats, 0, 2 * sizeof(unsigned long long), h->stream);
        if (ce != cudaSuccess) return fin(fail(h, DE_ERR_CUDA, std::string("init: ") + cudaGetErrorString(ce)));
      }
    }
  }
  if (cfgs[0].surrogate_k >= 2) {
    const de_status ss = surr_create(h->surr, cfgs[0].surrogate_k, cfgs[0].surrogate_steps,
                                     cfgs[0].seed ^ ((uint64_t)cfgs[0].run_id << 32), h->run[0], h->stream, h->err);
    if (ss != DE_OK) return fin(fail(h, ss, h->err));
  }
  ce = cudaStreamSynchronize(h->stream);
  if (ce != cudaSuccess) return fin(fail(h, DE_ERR_CUDA, std::string("init: ") + cudaGetErrorString(ce)));
#undef TRY
  return fin(DE_OK);
}

de_status de_init(const de_config* cfg, void* cuda_stream, de_handle** out) {
  if (!cfg) return fail(nullptr, DE_ERR_INVALID_ARG, "cfg is NULL");
  return de_init_batch(cfg, 1, cuda_stream, out);
}

de_status de_reset(de_handle* h, int32_t run) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (run < -1 || run >= h->nruns) return fail(h, DE_ERR_INVALID_ARG, "run out of range");
  h->err.clear();
  for (int r = (run < 0 ? 0 : run); r < (run < 0 ? h->nruns : run + 1); ++r) {
    de_status s = init_run(h, r);
    if (s != DE_OK) return s;
  }
  if (h->surr) {
    const de_status s = surr_reset(*h->surr, h->stream, h->err);
    if (s != DE_OK) return fail(h, s, h->err);
  }
  return islands_resync(h);
}

de_status de_init_islands(const de_config* cfg, int32_t nislands, int32_t interval, int32_t migrants,
                          void* cuda_stream, de_handle** out) {
  return de_init_islands_ex(cfg, nislands, interval, migrants, DE_MIGRATE_SYNC, cuda_stream, out);
}

de_status de_init_islands_ex(const de_config* cfg, int32_t nislands, int32_t interval, int32_t migrants,
                             int32_t migration, void* cuda_stream, de_handle** out) {
  g_err.clear();
  if (!cfg || !out) return fail(nullptr, DE_ERR_INVALID_ARG, "cfg or out is NULL");
  if (migration != DE_MIGRATE_SYNC && migration != DE_MIGRATE_ASYNC)
    return fail(nullptr, DE_ERR_INVALID_ARG, "migration must be DE_MIGRATE_SYNC or DE_MIGRATE_ASYNC");
  if (nislands < 2 || nislands > 4096) return fail(nullptr, DE_ERR_INVALID_ARG, "nislands must be in [2, 4096]");
  if (interval < 1) return fail(nullptr, DE_ERR_INVALID_ARG, "interval must be >= 1");
  if (migrants < 1 || migrants > kIslandMaxMigrants || 2 * migrants > cfg->np)
    return fail(nullptr, DE_ERR_INVALID_ARG, "migrants must be in [1, min(32, np / 2)]");
  if ((uint64_t)cfg->run_id + (uint64_t)nislands > (1u << 20))
    return fail(nullptr, DE_ERR_INVALID_ARG, "run_id + nislands must be <= 2^20");
  if (cfg->precision != DE_PREC_FP64 || cfg->surrogate_k >= 2)
    return fail(nullptr, DE_ERR_UNSUPPORTED, "the island model runs on the FP64 path without a surrogate");
  std::vector<de_config> cfgs(nislands, *cfg);
  for (int k = 0; k < nislands; ++k) cfgs[k].run_id = cfg->run_id + (uint32_t)k;
  de_handle* h = nullptr;
  de_status st = de_init_batch(cfgs.data(), nislands, cuda_stream, &h);
  if (st != DE_OK) return st;
  const int dp = h->run[0].dp;
  // two mailbox slots of nislands x migrants (synchronous migration uses the first)
  const size_t n = 2 * (size_t)nislands * migrants;
  const size_t bytes = n * (dp * sizeof(double) + 3 * sizeof(double) + sizeof(int32_t) + 1) + 1024;
  cudaError_t e = cudaMalloc(&h->isl_mem, bytes + sizeof(IslandCtl));
  if (e != cudaSuccess) {
    de_destroy(h);
    return fail(nullptr, DE_ERR_OOM, "cudaMalloc(island staging) failed");
  }
  char* p = (char*)h->isl_mem;
  h->d_isl = (IslandCtl*)p;
  p += 256;
  h->stage.x = (double*)p;
  p += n * dp * sizeof(double);
  h->stage.f = (double*)p;
  p += n * sizeof(double);
  h->stage.F = (double*)p;
  p += n * sizeof(double);
  h->stage.CR = (double*)p;
  p += n * sizeof(double);
  h->stage.widx = (int32_t*)p;
  p += n * sizeof(int32_t);
  h->stage.fx = (uint8_t*)p;
  h->stage.dp = dp;
  h->stage.slot = nislands * migrants;
  h->isl = IslandCtl{nislands, interval, migrants, migration == DE_MIGRATE_ASYNC ? 1 : 0, -1, -1};
  h->islands = true;
  // the cooperative FP64 kernel migrates inside its generation loop (not
  // for the benchmark suite's objectives, and never as one cluster: islands
  // are at least two runs); otherwise migration runs between generations
  h->fp64_cluster = false;
  h->fp64_persist = h->fp64_persist && fp64_persist_ok(h);
  drop_graph(h);
  st = islands_resync(h);
  if (st == DE_OK) {
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) st = fail(h, DE_ERR_CUDA, std::string("islands: ") + cudaGetErrorString(e));
  }
  if (st != DE_OK) {
    std::string m = h->err;
    de_destroy(h);
    g_err = m;
    return st;
  }
  *out = h;
  return DE_OK;
}

de_status de_step(de_handle* h, int64_t generations) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (generations < 0) return fail(h, DE_ERR_INVALID_ARG, "generations must be >= 0");
  h->err.clear();
  return enqueue_generations(h, generations);
}

de_status de_run(de_handle* h, de_result* out) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  h->err.clear();
  auto t0 = std::chrono::steady_clock::now();
  de_status s = read_states(h);
  if (s != DE_OK) return s;
  int64_t chunk = 64;
  for (;;) {
    bool all = true;
    int64_t left = 0;
    for (int r = 0; r < h->nruns; ++r)
      if (!h->h_state[r].stop) {
        all = false;
        left = std::max<int64_t>(left, h->run[r].max_gens - h->h_state[r].gen);
      }
    if (all) break;
    // the persistent kernels stop the run themselves: one launch
    const bool persistent = h->fp64_persist || (h->prec != DE_PREC_FP64 && (h->tc.persist.ok || h->pbatch_on));
    s = enqueue_generations(h, std::max<int64_t>(1, persistent ? left : std::min<int64_t>(chunk, left)));
    if (s != DE_OK) return s;
    s = read_states(h);
    if (s != DE_OK) return s;
    s = check_device_errors(h);
    if (s != DE_OK) return s;
    chunk = std::min<int64_t>(chunk * 2, 1024);
  }
  for (int r = 0; r < h->nruns && out; ++r) {
    s = exact_best(h, r);
    if (s != DE_OK) return s;
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (out)
    for (int r = 0; r < h->nruns; ++r) {
      out[r].best_f = h->h_state[r].best_f;
      out[r].best_index = h->h_state[r].best_idx;
      out[r].stop_reason = h->h_state[r].stop;
      out[r].generations = h->h_state[r].gen;
      out[r].evals = h->h_state[r].evals;
      out[r].seconds = secs;
    }
  return DE_OK;
}

de_status de_eval(de_handle* h, int32_t run, const double* x_dev, int64_t ld, int32_t n, double* f_dev) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (run < 0 || run >= h->nruns) return fail(h, DE_ERR_INVALID_ARG, "run out of range");
  const RunDesc& R = h->run[run];
  if (n < 0) return fail(h, DE_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return DE_OK;
  if (!x_dev || !f_dev) return fail(h, DE_ERR_INVALID_ARG, "x_dev and f_dev must be device pointers");
  if (ld < R.d) return fail(h, DE_ERR_INVALID_ARG, "ld must be >= d");
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, x_dev) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail(h, DE_ERR_INVALID_ARG, "x_dev is not device memory");
  }
  if (cudaPointerGetAttributes(&a, f_dev) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail(h, DE_ERR_INVALID_ARG, "f_dev is not device memory");
  }
  if (h->prec == DE_PREC_FP64) {
    k_eval_rows_launch(h->d_run, run, R, x_dev, ld, n, f_dev, nullptr, h->stream);
  } else {
    de_status s = tc_eval_launch(h->tc, h->d_run, run, R, x_dev, ld, n, f_dev, h->stream, h->err);
    if (s != DE_OK) return s;
  }
  DE_CUDA(h, cudaGetLastError());
  return DE_OK;
}

de_status de_get_shape(de_handle* h, int32_t run, int32_t* np, int32_t* d, int32_t* nruns) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (nruns) *nruns = h->nruns;
  if (run < 0 || run >= h->nruns) return np || d ? fail(h, DE_ERR_INVALID_ARG, "run out of range") : DE_OK;
  if (np) *np = h->run[run].np;
  if (d) *d = h->run[run].d;
  return DE_OK;
}

de_status de_get_population(de_handle* h, int32_t run, double* x_host, double* f_host) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (run < 0 || run >= h->nruns) return fail(h, DE_ERR_INVALID_ARG, "run out of range");
  de_status s = read_states(h);
  if (s != DE_OK) return s;
  const RunDesc& R = h->run[run];
  const int cur = cur_buf(h, h->h_state[run].gen);
  if (x_host)
    DE_CUDA(h, cudaMemcpy2DAsync(x_host, R.d * sizeof(double), R.X[cur], R.dp * sizeof(double), R.d * sizeof(double),
                                 R.np, cudaMemcpyDeviceToHost, h->stream));
  if (f_host)
    DE_CUDA(h, cudaMemcpyAsync(f_host, R.f[cur], R.np * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  DE_CUDA(h, cudaStreamSynchronize(h->stream));
  return DE_OK;
}

de_status de_set_population(de_handle* h, int32_t run, const double* x_host, const double* f_host) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (run < 0 || run >= h->nruns) return fail(h, DE_ERR_INVALID_ARG, "run out of range");
  if (!x_host) return fail(h, DE_ERR_INVALID_ARG, "x_host is NULL");
  const RunDesc& R = h->run[run];
  for (size_t k = 0; k < (size_t)R.np * R.d; ++k)
    if (!std::isfinite(x_host[k])) return fail(h, DE_ERR_NONFINITE, "population has a non-finite entry");
  de_status s = read_states(h);
  if (s != DE_OK) return s;
  const int cur = cur_buf(h, h->h_state[run].gen);
  DE_CUDA(h, cudaMemsetAsync(R.X[cur], 0, (size_t)R.np * R.dp * sizeof(double), h->stream));
  DE_CUDA(h, cudaMemcpy2DAsync(R.X[cur], R.dp * sizeof(double), x_host, R.d * sizeof(double), R.d * sizeof(double),
                               R.np, cudaMemcpyHostToDevice, h->stream));
  if (f_host) {
    DE_CUDA(h, cudaMemcpyAsync(R.f[cur], f_host, R.np * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    DE_CUDA(h, cudaMemsetAsync(R.fx[cur], 1, R.np, h->stream));
  } else {
    k_eval_rows_launch(h->d_run, run, R, R.X[cur], R.dp, R.np, R.f[cur], R.fx[cur], h->stream);
  }
  k_best_init_launch(h->d_run, run, h->stream);
  DE_CUDA(h, cudaGetLastError());
  s = islands_resync(h);
  if (s != DE_OK) return s;
  DE_CUDA(h, cudaStreamSynchronize(h->stream));
  return DE_OK;
}

de_status de_set_generation(de_handle* h, int32_t run, int64_t generation) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (run < 0 || run >= h->nruns) return fail(h, DE_ERR_INVALID_ARG, "run out of range");
  if (generation < 0 || generation >= (int64_t)UINT32_MAX)
    return fail(h, DE_ERR_INVALID_ARG, "generation must be in [0, 2^32 - 1)");
  de_status s = read_states(h);
  if (s != DE_OK) return s;
  const RunDesc& R = h->run[run];
  const int cur = cur_buf(h, h->h_state[run].gen), want = cur_buf(h, generation);
  if (cur != want) {
    DE_CUDA(h, cudaMemcpyAsync(R.X[want], R.X[cur], (size_t)R.np * R.dp * sizeof(double), cudaMemcpyDeviceToDevice,
                               h->stream));
    DE_CUDA(h, cudaMemcpyAsync(R.f[want], R.f[cur], R.np * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    DE_CUDA(h, cudaMemcpyAsync(R.fx[want], R.fx[cur], R.np, cudaMemcpyDeviceToDevice, h->stream));
    if (R.jde) {
      DE_CUDA(h, cudaMemcpyAsync(R.jF[want], R.jF[cur], R.np * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
      DE_CUDA(h, cudaMemcpyAsync(R.jCR[want], R.jCR[cur], R.np * sizeof(double), cudaMemcpyDeviceToDevice,
                                 h->stream));
    }
  }
  DE_CUDA(h, cudaMemcpyAsync(&R.st->gen, &generation, sizeof generation, cudaMemcpyHostToDevice, h->stream));
  int64_t ev = (int64_t)R.np * (1 + generation);
  DE_CUDA(h, cudaMemcpyAsync(&R.st->evals, &ev, sizeof ev, cudaMemcpyHostToDevice, h->stream));
  k_best_init_launch(h->d_run, run, h->stream);
  DE_CUDA(h, cudaGetLastError());
  s = islands_resync(h);
  if (s != DE_OK) return s;
  DE_CUDA(h, cudaStreamSynchronize(h->stream));
  return DE_OK;
}

de_status de_get_adaptive(de_handle* h, int32_t run, double* f_host, double* cr_host) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (run < 0 || run >= h->nruns) return fail(h, DE_ERR_INVALID_ARG, "run out of range");
  const RunDesc& R = h->run[run];
  if (!R.jde) return fail(h, DE_ERR_STATE, "the run does not use jDE");
  de_status s = read_states(h);
  if (s != DE_OK) return s;
  const int cur = cur_buf(h, h->h_state[run].gen);
  if (f_host)
    DE_CUDA(h, cudaMemcpyAsync(f_host, R.jF[cur], R.np * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (cr_host)
    DE_CUDA(h, cudaMemcpyAsync(cr_host, R.jCR[cur], R.np * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  DE_CUDA(h, cudaStreamSynchronize(h->stream));
  return DE_OK;
}

de_status de_set_adaptive(de_handle* h, int32_t run, const double* f_host, const double* cr_host) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (run < 0 || run >= h->nruns) return fail(h, DE_ERR_INVALID_ARG, "run out of range");
  const RunDesc& R = h->run[run];
  if (!R.jde) return fail(h, DE_ERR_STATE, "the run does not use jDE");
  for (int i = 0; i < R.np; ++i) {
    if (f_host && !(f_host[i] >= 0.0 && f_host[i] <= 2.0)) return fail(h, DE_ERR_INVALID_ARG, "F_i must be in [0, 2]");
    if (cr_host && !(cr_host[i] >= 0.0 && cr_host[i] <= 1.0))
      return fail(h, DE_ERR_INVALID_ARG, "CR_i must be in [0, 1]");
  }
  de_status s = read_states(h);
  if (s != DE_OK) return s;
  const int cur = cur_buf(h, h->h_state[run].gen);
  if (f_host)
    DE_CUDA(h, cudaMemcpyAsync(R.jF[cur], f_host, R.np * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  if (cr_host)
    DE_CUDA(h, cudaMemcpyAsync(R.jCR[cur], cr_host, R.np * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  DE_CUDA(h, cudaStreamSynchronize(h->stream));
  return DE_OK;
}

de_status de_get_best(de_handle* h, int32_t run, double* best_f, int32_t* best_index, double* best_x,
                      int64_t* generations, int64_t* evals, int32_t* stop_reason) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (run < 0 || run >= h->nruns) return fail(h, DE_ERR_INVALID_ARG, "run out of range");
  const RunDesc& R = h->run[run];
  de_status s = read_states(h);
  if (s != DE_OK) return s;
  s = exact_best(h, run);
  if (s != DE_OK) return s;
  const RunState& st = h->h_state[run];
  if (best_x) {
    // the best individual's vector, read from the current population
    if (st.best_idx < 0) return fail(h, DE_ERR_NONFINITE, "no finite fitness in the population");
    const double* row = R.X[cur_buf(h, st.gen)] + (size_t)st.best_idx * R.dp;
    DE_CUDA(h, cudaMemcpyAsync(best_x, row, R.d * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    DE_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  if (best_f) *best_f = st.best_f;
  if (best_index) *best_index = st.best_idx;
  if (generations) *generations = st.gen;
  if (evals) *evals = st.evals;
  if (stop_reason) *stop_reason = st.stop;
  return DE_OK;
}

de_status de_get_debug(de_handle* h, int32_t run, const de_debug* out) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (run < 0 || run >= h->nruns) return fail(h, DE_ERR_INVALID_ARG, "run out of range");
  if (!out) return fail(h, DE_ERR_INVALID_ARG, "out is NULL");
  const RunDesc& R = h->run[run];
  if (!R.dbg_trial) return fail(h, DE_ERR_STATE, "debug capture was not enabled for this run");
  auto cp = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    if (!dst) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream);
  };
  DE_CUDA(h, cp(out->idx, R.dbg_idx, (size_t)R.np * 3 * sizeof(int32_t)));
  DE_CUDA(h, cp(out->jrand, R.dbg_jrand, (size_t)R.np * sizeof(int32_t)));
  DE_CUDA(h, cp(out->mask, R.dbg_mask, (size_t)R.np * R.nw * sizeof(uint32_t)));
  DE_CUDA(h, cp(out->trial, R.dbg_trial, (size_t)R.np * R.d * sizeof(double)));
  DE_CUDA(h, cp(out->f_trial, R.dbg_ftrial, (size_t)R.np * sizeof(double)));
  DE_CUDA(h, cp(out->accept, R.dbg_accept, (size_t)R.np));
  DE_CUDA(h, cp(out->fp64_checked, R.dbg_fp64, (size_t)R.np));
  DE_CUDA(h, cp(out->cand, R.dbg_cand, (size_t)R.np * sizeof(int32_t)));
  DE_CUDA(h, cudaStreamSynchronize(h->stream));
  return DE_OK;
}

de_status de_get_surrogate_stats(de_handle* h, int64_t* trainings, int64_t* screened_generations, double* last_rho,
                                 int32_t* k_now) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (!h->surr) return fail(h, DE_ERR_STATE, "the handle has no surrogate (surrogate_k < 2)");
  if (trainings) *trainings = h->surr->trainings;
  if (screened_generations) *screened_generations = h->surr->screened;
  if (last_rho) *last_rho = h->surr->last_rho;
  if (k_now) *k_now = h->surr->k_eff;
  return DE_OK;
}

de_status de_get_plan(de_handle* h, int32_t* kernel_path, int32_t* cluster_size) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  const bool persist = h->prec != DE_PREC_FP64 && h->tc.persist.ok;
  if (kernel_path)
    *kernel_path = h->prec == DE_PREC_FP64 ? (h->fp64_persist ? 3 : 0)
                   : h->pbatch_on         ? 5
                                           : (persist ? (h->tc.persist.mode == 1 ? 4 : 2) : 1);
  if (cluster_size)
    *cluster_size = persist ? (h->tc.persist.mode == 1 ? 0 : h->tc.persist.C)
                            : (h->prec == DE_PREC_FP64 && h->fp64_cluster ? h->nitems : 0);
  return DE_OK;
}

de_status de_get_stats(de_handle* h, int32_t run, int64_t* fp64_reevals, int64_t* trials) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (run < 0 || run >= h->nruns) return fail(h, DE_ERR_INVALID_ARG, "run out of range");
  unsigned long long v[2] = {0, 0};
  if (h->run[run].stats) {
    DE_CUDA(h, cudaMemcpyAsync(v, h->run[run].stats, sizeof v, cudaMemcpyDeviceToHost, h->stream));
    DE_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  if (fp64_reevals) *fp64_reevals = (int64_t)v[0];
  if (trials) *trials = (int64_t)v[1];
  return DE_OK;
}

// ---------------------------------------------------------------- checkpoints
static uint32_t crc32_update(uint32_t crc, const void* data, size_t n) {
  // reflected CRC-32 (polynomial 0x04C11DB7, reversed form 0xEDB88320), bitwise
  const uint8_t* p = (const uint8_t*)data;
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) {
    crc ^= p[i];
    for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
  }
  return ~crc;
}

struct CkptHeader {
  char magic[8];
  uint32_t version;
  int32_t nruns;
  uint64_t payload_bytes;
  uint32_t crc;
  uint32_t pad;
};

de_status de_save(de_handle* h, const char* path) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (!path) return fail(h, DE_ERR_INVALID_ARG, "path is NULL");
  if (h->surr) return fail(h, DE_ERR_UNSUPPORTED, "checkpoints do not cover the surrogate's archive and network");
  de_status s = read_states(h);
  if (s != DE_OK) return s;
  std::vector<char> payload;
  auto put = [&](const void* p, size_t n) {
    const char* c = (const char*)p;
    payload.insert(payload.end(), c, c + n);
  };
  for (int r = 0; r < h->nruns; ++r) {
    const RunDesc& R = h->run[r];
    const int cur = cur_buf(h, h->h_state[r].gen);
    int32_t shape[5] = {R.np, R.d, R.prec, R.strategy, R.jde};
    put(shape, sizeof shape);
    put(&h->fingerprint[r], sizeof(uint64_t));
    put(&h->h_state[r], sizeof(RunState));
    std::vector<double> x((size_t)R.np * R.dp), f(R.np);
    std::vector<uint8_t> fx(R.np);
    DE_CUDA(h, cudaMemcpyAsync(x.data(), R.X[cur], x.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    DE_CUDA(h, cudaMemcpyAsync(f.data(), R.f[cur], f.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    DE_CUDA(h, cudaMemcpyAsync(fx.data(), R.fx[cur], fx.size(), cudaMemcpyDeviceToHost, h->stream));
    DE_CUDA(h, cudaStreamSynchronize(h->stream));
    put(x.data(), x.size() * sizeof(double));
    put(f.data(), f.size() * sizeof(double));
    put(fx.data(), fx.size());
    if (R.tau) {
      std::vector<float> tau(R.np);
      DE_CUDA(h, cudaMemcpy(tau.data(), R.tau, tau.size() * sizeof(float), cudaMemcpyDeviceToHost));
      put(tau.data(), tau.size() * sizeof(float));
    }
    if (R.jde) {
      std::vector<double> a(2 * (size_t)R.np);
      DE_CUDA(h, cudaMemcpyAsync(a.data(), R.jF[cur], R.np * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      DE_CUDA(h, cudaMemcpyAsync(a.data() + R.np, R.jCR[cur], R.np * sizeof(double), cudaMemcpyDeviceToHost,
                                 h->stream));
      DE_CUDA(h, cudaStreamSynchronize(h->stream));
      put(a.data(), a.size() * sizeof(double));
    }
  }
  CkptHeader hd{};
  memcpy(hd.magic, "DEGB300", 8);
  hd.version = 4;
  hd.nruns = h->nruns;
  hd.payload_bytes = payload.size();
  hd.crc = crc32_update(0, payload.data(), payload.size());
  FILE* fp = fopen(path, "wb");
  if (!fp) return fail(h, DE_ERR_IO, std::string("cannot open ") + path + " for writing");
  bool ok = fwrite(&hd, sizeof hd, 1, fp) == 1 && fwrite(payload.data(), 1, payload.size(), fp) == payload.size();
  ok = (fclose(fp) == 0) && ok;
  if (!ok) return fail(h, DE_ERR_IO, std::string("write failed: ") + path);
  return DE_OK;
}

de_status de_load(de_handle* h, const char* path) {
  if (!h) return fail(nullptr, DE_ERR_INVALID_ARG, "handle is NULL");
  if (!path) return fail(h, DE_ERR_INVALID_ARG, "path is NULL");
  if (h->surr) return fail(h, DE_ERR_UNSUPPORTED, "checkpoints do not cover the surrogate's archive and network");
  FILE* fp = fopen(path, "rb");
  if (!fp) return fail(h, DE_ERR_IO, std::string("cannot open ") + path);
  CkptHeader hd{};
  std::vector<char> payload;
  bool ok = fread(&hd, sizeof hd, 1, fp) == 1 && memcmp(hd.magic, "DEGB300", 8) == 0 && hd.version == 4 &&
            hd.payload_bytes < (1ull << 40);
  if (ok) {
    payload.resize(hd.payload_bytes);
    ok = fread(payload.data(), 1, payload.size(), fp) == payload.size();
  }
  fclose(fp);
  if (!ok) return fail(h, DE_ERR_IO, std::string("not a readable checkpoint: ") + path);
  if (crc32_update(0, payload.data(), payload.size()) != hd.crc) return fail(h, DE_ERR_IO, "checkpoint CRC mismatch");
  if (hd.nruns != h->nruns) return fail(h, DE_ERR_STATE, "checkpoint has a different number of runs");
  size_t off = 0;
  auto get = [&](void* p, size_t n) {
    if (off + n > payload.size()) return false;
    memcpy(p, payload.data() + off, n);
    off += n;
    return true;
  };
  // every run is parsed and checked on the host before anything reaches the
  // device, so that a rejected file leaves the handle as it was
  struct RunCkpt {
    RunState st;
    std::vector<double> x, f, adapt;
    std::vector<uint8_t> fx;
    std::vector<float> tau;
  };
  std::vector<RunCkpt> rc(h->nruns);
  for (int r = 0; r < h->nruns; ++r) {
    const RunDesc& R = h->run[r];
    RunCkpt& c = rc[r];
    int32_t shape[5];
    uint64_t fp = 0;
    if (!get(shape, sizeof shape) || !get(&fp, sizeof fp) || !get(&c.st, sizeof c.st))
      return fail(h, DE_ERR_IO, "checkpoint truncated");
    if (shape[0] != R.np || shape[1] != R.d || shape[2] != R.prec || shape[3] != R.strategy || shape[4] != R.jde)
      return fail(h, DE_ERR_STATE, "checkpoint shape of run " + std::to_string(r) + " differs from the handle's");
    if (fp != h->fingerprint[r])
      return fail(h, DE_ERR_STATE, "checkpoint of run " + std::to_string(r) +
                                       " was written for another problem (objective, F, CR, bounds, seed, shift or "
                                       "rotation differ)");
    c.x.resize((size_t)R.np * R.dp);
    c.f.resize(R.np);
    c.fx.resize(R.np);
    if (!get(c.x.data(), c.x.size() * sizeof(double)) || !get(c.f.data(), c.f.size() * sizeof(double)) ||
        !get(c.fx.data(), c.fx.size()))
      return fail(h, DE_ERR_IO, "checkpoint truncated");
    if (R.tau) {
      c.tau.resize(R.np);
      if (!get(c.tau.data(), c.tau.size() * sizeof(float))) return fail(h, DE_ERR_IO, "checkpoint truncated");
    }
    if (R.jde) {
      c.adapt.resize(2 * (size_t)R.np);
      if (!get(c.adapt.data(), c.adapt.size() * sizeof(double))) return fail(h, DE_ERR_IO, "checkpoint truncated");
    }
  }
  if (off != payload.size()) return fail(h, DE_ERR_IO, "checkpoint has trailing bytes");
  for (int r = 0; r < h->nruns; ++r) {
    const RunDesc& R = h->run[r];
    RunCkpt& c = rc[r];
    const int cur = cur_buf(h, c.st.gen);
    if (R.tau)
      DE_CUDA(h, cudaMemcpyAsync(R.tau, c.tau.data(), c.tau.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    if (R.jde) {
      DE_CUDA(h, cudaMemcpyAsync(R.jF[cur], c.adapt.data(), R.np * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      DE_CUDA(h, cudaMemcpyAsync(R.jCR[cur], c.adapt.data() + R.np, R.np * sizeof(double), cudaMemcpyHostToDevice,
                                 h->stream));
    }
    c.st.ticket = 0;
    c.st.band_n = 0;
    c.st.band_left = 0;
    DE_CUDA(h, cudaMemcpyAsync(R.X[cur], c.x.data(), c.x.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    DE_CUDA(h, cudaMemcpyAsync(R.f[cur], c.f.data(), c.f.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    DE_CUDA(h, cudaMemcpyAsync(R.fx[cur], c.fx.data(), c.fx.size(), cudaMemcpyHostToDevice, h->stream));
    DE_CUDA(h, cudaMemcpyAsync(R.st, &c.st, sizeof c.st, cudaMemcpyHostToDevice, h->stream));
  }
  DE_CUDA(h, cudaStreamSynchronize(h->stream));
  const de_status s = islands_resync(h);
  if (s != DE_OK) return s;
  DE_CUDA(h, cudaStreamSynchronize(h->stream));
  return DE_OK;
}

de_status de_eval_noalloc(int32_t precision, int32_t objective, int32_t d, double scale, const double* shift_dev,
                          const double* rot_dev, const double* x_dev, int64_t ld, int32_t n, double* f_dev,
                          void* cuda_stream) {
  if (precision == DE_PREC_FP64)
    return fail(nullptr, DE_ERR_UNSUPPORTED, "de_eval_noalloc: FP64 evaluation uses no scratch; call de_eval");
  if (precision != DE_PREC_BF16X3 && precision != DE_PREC_TF32X3)
    return fail(nullptr, DE_ERR_INVALID_ARG, "de_eval_noalloc: precision out of range");
  if (objective < DE_OBJ_SPHERE || objective > DE_OBJ_ACKLEY)
    return fail(nullptr, DE_ERR_INVALID_ARG, "de_eval_noalloc: objective out of range");
  if (d < 1 || d > 4096) return fail(nullptr, DE_ERR_INVALID_ARG, "de_eval_noalloc: d must be in [1, 4096]");
  if (objective == DE_OBJ_ROSENBROCK && d > 256)
    return fail(nullptr, DE_ERR_UNSUPPORTED, "de_eval_noalloc: split precision supports Rosenbrock only for d <= 256");
  if (!std::isfinite(scale) || scale == 0.0)
    return fail(nullptr, DE_ERR_INVALID_ARG, "de_eval_noalloc: scale must be finite and nonzero");
  if (n < 0) return fail(nullptr, DE_ERR_INVALID_ARG, "de_eval_noalloc: n must be >= 0");
  if (n == 0) return DE_OK;
  if (ld < d) return fail(nullptr, DE_ERR_INVALID_ARG, "de_eval_noalloc: ld must be >= d");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, DE_ERR_CUDA, "de_eval_noalloc: no current CUDA device");
  }
  const void* ptrs[4] = {x_dev, f_dev, shift_dev, rot_dev};
  const char* names[4] = {"x_dev", "f_dev", "shift_dev", "rot_dev"};
  for (int q = 0; q < 4; ++q) {
    if (!ptrs[q]) {
      if (q < 2) return fail(nullptr, DE_ERR_INVALID_ARG, std::string("de_eval_noalloc: ") + names[q] + " is NULL");
      continue;
    }
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, ptrs[q]) != cudaSuccess || a.type != cudaMemoryTypeDevice || a.device != dev) {
      cudaGetLastError();
      return fail(nullptr, DE_ERR_INVALID_ARG,
                  std::string("de_eval_noalloc: ") + names[q] + " is not device memory of the current device");
    }
  }
  std::string err;
  const de_status s = noalloc_eval(precision, objective, d, scale, shift_dev, rot_dev, x_dev, ld, n, f_dev,
                                   (cudaStream_t)cuda_stream, err);
  if (s != DE_OK) return fail(nullptr, s, err);
  return DE_OK;
}

}  // extern "C"
