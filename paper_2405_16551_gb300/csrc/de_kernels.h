// de_kernels.h -- host-side launchers of the kernels (called by de_api.cu).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "de.h"
#include "de_internal.cuh"

namespace de {

void set_last_error(const std::string& m);

// grid-barrier state of a persistent launch
struct PersistCtl {
  unsigned int bar;  // grid barrier arrivals of the current launch
  int abort;         // set when a bounded wait expired
  long long gen0;    // generation counter when the launch began
  unsigned int stopped[3];  // runs stopped per iteration mod 3 (batched FP64 launch)
  // failure-detection test of the cooperative FP64 kernel (0 = off): CTA
  // test_skip - 1 leaves out its first grid-barrier arrival, and the barrier
  // gives up after test_spin polls, so that the bounded wait runs out
  int test_skip;
  long long test_spin;
  // island model in the cooperative FP64 kernel: tiles whose best is below
  // the target, per iteration mod 3 (the model's common stop)
  unsigned int below[3];
  // grid-barrier arrivals of the CTA-local split kernel in sbar[0] (the rest
  // of the 128 bytes keeps other fields off its line)
  unsigned int sbar[32];
};
// zero the control block of a persistent launch; test_skip > 0 also arms the
// failure-detection test (test_skip, and test_spin = 4096 polls)
cudaError_t persist_ctl_reset(PersistCtl* ctl, int test_skip, cudaStream_t s);
// FP64 path (de_fp64.cu)
void k_configure(size_t smem_gen);
// var: some run uses a strategy variant or jDE; suite: some run uses an
// objective of the proposed benchmark (5..20)
void k_gen_fp64_launch(const RunDesc* runs, const int4* items, int nitems, int threads, size_t smem, bool var,
                       bool suite, cudaStream_t s);
// the generation loop of FP64 runs in one cooperative launch (every item
// co-resident: nitems <= k_gen_fp64_persist_capacity; gens <= 2^20)
// test_skip > 0: the grid-barrier failure test (PersistCtl::test_skip)
// isl (NULL without islands): the runs are islands (de_init_islands_ex) whose
// migrations and common stop run inside the launch
struct IslandCtl;
struct IslandStage;
cudaError_t k_gen_fp64_persist_launch(const RunDesc* runs, const int4* items, int nitems, int nruns, int threads,
                                      size_t smem, bool var, bool suite, PersistCtl* ctl, long long gens,
                                      cudaStream_t s, int test_skip = 0, IslandCtl* isl = nullptr,
                                      const IslandStage* stage = nullptr);
// CTAs of the cooperative FP64 kernel that fit at once (isl: the island instance)
int k_gen_fp64_persist_capacity(int threads, size_t smem, bool var, bool suite, bool isl = false);
// the same loop as one thread-block cluster of nitems CTAs (one run,
// nitems <= 8), the cluster barrier between generations
cudaError_t k_gen_fp64_cluster_launch(const RunDesc* runs, const int4* items, int nitems, int threads, size_t smem,
                                      bool var, bool suite, PersistCtl* ctl, long long gens, cudaStream_t s);
bool k_gen_fp64_cluster_fits(int nitems, int threads, size_t smem, bool var, bool suite);
void k_init_population_launch(const RunDesc* runs, int run, int np, int dp, cudaStream_t s);
// f (and, when fx is not NULL, the FP64 flags) of n rows of x; Rh is the
// host copy of run `run`'s descriptor
void k_eval_rows_launch(const RunDesc* runs, int run, const RunDesc& Rh, const double* x, int64_t ld, int n,
                        double* f, uint8_t* fx, cudaStream_t s);
inline int suite_comps(const RunDesc& R) { return R.obj >= DE_OBJ_COMPOSITION1 ? R.nc : 1; }
void k_best_init_launch(const RunDesc* runs, int run, cudaStream_t s);
void k_jde_init_launch(const RunDesc* runs, int run, int np, cudaStream_t s);
void k_ode_reference_launch(const RunDesc* runs, int run, double* ref, cudaStream_t s);

// island model (de_islands.cu)
constexpr int kIslandMaxMigrants = 32;
struct IslandCtl {
  int32_t m;         // islands (the runs of the handle)
  int32_t interval;  // generations between migrations
  int32_t nmig;      // migrants per island and migration
  int32_t async;     // 1: asynchronous migration through the mailbox
  int64_t mig_gen;   // generation of the last migration (-1: none)
  int64_t post_gen;  // asynchronous: generation of the mailbox's last post (-1: none)
};
// Two slots of m x nmig migrants: synchronous migration stages through slot 0
// between its select and apply kernels; asynchronous migration posts to slot
// (g / interval) & 1 at migration point g and reads the other one.
struct IslandStage {
  double* x;          // rows of dp doubles
  double* f;
  uint8_t* fx;
  double* F;          // jDE parameters
  double* CR;
  int32_t* widx;      // the receiving island's worst slots (synchronous)
  int32_t dp;
  int32_t slot;       // migrants per slot (m x nmig)
};
// migrate: also run the exchange kernels (else only the group stop test);
// async: the asynchronous exchange kernel instead of the synchronous pair
void k_island_launch(const RunDesc* runs, IslandCtl* ctl, const IslandStage& stage, int m, bool migrate,
                     bool async, cudaStream_t s);

// persistent cluster path (de_persist.cu)
struct PersistPlan {
  bool ok = false;   // some persistent form applies (mode says which runs)
  int mode = 0;      // 0: thread-block clusters (k_persist); 1: CTA-local products (k_persist_cta)
  bool cl_ok = false;  // the cluster form applies
  int C = 0, ntiles = 0, prec = 0, nch = 1, prows = 128;
  int maxcl = 0;  // clusters that fit on the device at once
  bool var = false;  // the run uses a strategy variant or jDE
  size_t smem = 0;
  // CTA-local form: targets per CTA, CTAs, resident-CTA capacity, shared memory
  bool cta_ok = false;
  int cta_rows = 0, cta_ntiles = 0, cta_cap = 0;
  size_t cta_smem = 0;
};

// the persistent batch kernel (de_persist_batch.cu): work items are the runs'
// 128-target tiles, a fixed contiguous slice of items per CTA, per-run
// arrival counters
struct PbPlan {
  bool ok = false;
  int nct = 0, nruns = 0, prec = 0, kpad_max = 0, dp_max = 0;
  uint32_t ncols = 32;       // tensor-memory columns of a CTA
  size_t smem = 0;
  int4* d_items = nullptr;   // (run, 128-row tile, first row, rows)
  int2* d_slices = nullptr;  // per CTA: [first item, last item + 1)
  unsigned* d_cnt = nullptr; // per run: items done in this launch
};
bool pbatch_plan(PbPlan& pp, const std::vector<RunDesc>& runs, int prec);
void pbatch_free(PbPlan& pp);
cudaError_t pbatch_launch(const PbPlan& pp, const RunDesc* runs, PersistCtl* ctl, long long gens, cudaStream_t s,
                          int test_skip = 0);

// split-precision tensor-core path (de_tc.cu)
struct TcPlan {
  int prec = 0;
  int nitems_trial = 0;   // warps-per-row work items of the trial kernel
  int nitems_fit = 0;     // 128-row tiles over all runs
  int2* d_trial_items = nullptr;
  int2* d_fit_items = nullptr;
  void* arena = nullptr;  // operand copies of M, the A tiles, |y|, tau, stats
  size_t smem_fit = 0;
  std::vector<int> fit_offset;  // first fit item of each run
  BandEntry* d_band = nullptr;  // FP64 band list (all runs)
  uint32_t* d_band_cnt = nullptr;
  int nch_max = 1;
  size_t smem_band = 0;
  int grid_band = 0;
  int trial_rows = 8;          // targets (warps) per trial CTA
  int trial_occ = 0;           // 1: the trial kernel instance held to 85 registers (more warps per SM)
  int nsplit = 1;              // N tiles spread over CTAs of the fitness kernel (the largest N-tile count)
  int nruns = 0;
  bool var = false;            // some run uses a strategy variant or jDE
  PersistPlan persist;         // the persistent cluster kernel, when it applies
  PbPlan pbatch;               // the persistent batch kernel, when it applies
  PersistCtl* d_ctl = nullptr;
};
bool persist_plan(PersistPlan& pp, const RunDesc& R, int nruns, int prec);
// rows per cluster of a planned persistent launch (a multiple of C, at most
// 128, with every tile resident); false leaves the plan unchanged
bool persist_set_rows(PersistPlan& pp, const RunDesc& R, int prows);
cudaError_t persist_launch(const PersistPlan& pp, const RunDesc* runs, PersistCtl* ctl, long long gens,
                           cudaStream_t s, int test_skip = 0);
// the CTA-local persistent form (de_persist_cta.cu): one run of at most 128
// coordinates, at most 16 targets per CTA, every CTA resident
bool persist_cta_plan(PersistPlan& pp, const RunDesc& R, int nruns, int prec);
bool persist_cta_set_rows(PersistPlan& pp, const RunDesc& R, int rows);
cudaError_t persist_cta_launch(const PersistPlan& pp, const RunDesc* runs, PersistCtl* ctl, long long gens,
                               cudaStream_t s, int test_skip = 0);
// counters after a persistent launch of run 0 (evaluations, trials, tickets)
void k_persist_close_launch(const RunDesc* runs, const PersistCtl* ctl, cudaStream_t s);

de_status tc_plan_build(TcPlan& p, std::vector<RunDesc>& runs, const de_config* cfgs, int prec, cudaStream_t s,
                        std::string& err);
void tc_plan_free(TcPlan& p);
// Launch geometry that leaves the results unchanged (autotuner): targets per
// trial CTA, a divisor of the fitness kernel's default K chunk, and the
// stages of its K pipeline.
de_status tc_set_geometry(TcPlan& p, std::vector<RunDesc>& runs, int trial_rows, int kc_div, int stages,
                          cudaStream_t s, std::string& err);
void tc_generation_launch(const TcPlan& p, const RunDesc* runs, cudaStream_t s);
// Split-precision evaluation of run `run`'s population X[0] into f[0] (fx = 0,
// tau set): the initial evaluation of split-precision runs.
void tc_init_eval_launch(const TcPlan& p, const RunDesc* runs, int run, const RunDesc& R, cudaStream_t s);
de_status tc_eval_launch(const TcPlan& p, const RunDesc* runs, int run, const RunDesc& R, const double* x, int64_t ld,
                         int n, double* f, cudaStream_t s, std::string& err);
// Evaluation of n caller rows with a device descriptor and work list that
// the caller placed (all tiles of one launch); raises k_fit_tc's dynamic
// shared-memory limit to `smem` when it is lower, never lowers it.
de_status tc_eval_rows(const RunDesc* desc, const int2* items, int tiles, int esz, size_t smem, const double* x,
                       int64_t ld, int n, double* f, cudaStream_t s, std::string& err);

// no-allocation evaluation (de_noalloc.cu)
de_status noalloc_eval(int prec, int obj, int d, double scale, const double* o, const double* M, const double* x,
                       int64_t ld, int n, double* f, cudaStream_t s, std::string& err);

}  // namespace de
