// de_internal.cuh -- device data layout shared by the kernels and the runtime.
//
// HBM layout of one run (all device buffers 256-byte aligned):
//   X[2]     np x dp doubles, row-major, dp = d rounded up to 4 (32-byte rows);
//            X[g & 1] is the generation-g population, X[(g + 1) & 1] the next
//            one (synchronous replacement, double buffered)
//   f[2]     np doubles, fitness of X[0] / X[1]
//   fx[2]    np bytes, 1 when f[.] was computed in FP64 (split precisions)
//   o        dp doubles (shift, zero padded); nc x dp for a composition function
//   MT       d x d doubles, MT[k d + j] = M[j][k] (transposed: a warp reading
//            consecutive j for one k is one coalesced row); nc of them for a
//            composition function
//   perm     d int32 (hybrid functions)
//   Bsplit   tensor-core operand copies of M (split precisions only)
//   state    one RunState (generation, evaluations, best record, stop flag)
//   part     one BestPartial per row tile of the generation kernel
//   jF, jCR  [2] np doubles each (jDE only), the control parameters of X[0] / X[1]
// A batch of runs is a table of RunDesc in device memory plus a flat list of
// (run, tile) work items; one launch covers every tile of every run.
#pragma once
#include <stdint.h>

namespace de {

struct RunState {
  int64_t gen;         // generations completed
  int64_t evals;       // objective evaluations, np (1 + gen)
  double best_f;       // FP64 best fitness
  int32_t best_idx;    // its index, -1 before the first evaluation
  int32_t stop;        // de_stop_reason, 0 while running
  uint32_t ticket;     // CTAs of the current generation that finished
  int32_t err;         // device-side error bits (kErr*)
  int32_t band_n;      // rows of this generation sent to the FP64 band (split precisions)
  int32_t band_left;   // of those, rows still waiting for their FP64 decision
};

// One row whose selection is decided in FP64 (split precisions).
struct BandEntry {
  int32_t run;
  int32_t row;
  int32_t need_target;  // 1 when the target's stored fitness is not FP64
  int32_t pad;
};

struct BestPartial {
  double f;
  int32_t idx;
  int32_t pad;
};

constexpr int32_t kErrTimeout = 1;
constexpr int32_t kErrNonFinite = 2;

struct RunDesc {
  // problem
  int32_t np, d, dp, obj;
  double F, CR, lo, hi, scale;
  long long lo_key, hi_key;  // ordered integer keys of lo and hi
  double lo_half, hi_half;   // lo / 2 and hi / 2 (bound repair as one fma)
  int32_t unit_scale;        // scale == 1: the shift needs no multiplication
  int32_t lo_hk, hi_hk;      // ordered keys of the high words of lo and hi (hi_key32)
  int32_t pad0;
  uint64_t cr_thr;
  uint64_t seed;
  uint32_t run_id;
  int32_t rotate;
  double target;
  int64_t max_evals, max_gens;
  int32_t prec;
  int32_t nw;    // ceil(d / 32)
  int32_t dbuf;  // 1: generation g lives in X[g & 1]; 0: the split kernels update X[0] in place
  int32_t pad1;
  int32_t strategy;  // de_strategy (FP64 path): 0 rand/1/bin, 1 best/1/bin, 2 rand/1/exp
  int32_t jde;       // 1: per-individual F and CR in jF / jCR (jDE)
  double* jF[2];     // jDE: np values of F_i for X[0] / X[1]
  double* jCR[2];    // jDE: np values of CR_i
  // benchmark suite (objectives 5..20, FP64 path): parts of a hybrid
  // function or components of a composition function
  int32_t nc;              // parts / components (1 for a basic function)
  int32_t sfn[5];          // basic function of each
  int32_t seg[6];          // hybrid: first permuted position of each part, seg[nc] = d
  double sscale[5];        // domain scale of each
  double skex[5];          // Katsuura's exponent 10 / n^1.2 of each (n: its length)
  double slambda[5], ssigma[5], sbias[5];  // composition: height, coverage, bias
  const int32_t* perm;     // hybrid: d positions of the permutation
  // buffers
  double* X[2];
  double* f[2];
  uint8_t* fx[2];
  const double* o;
  const double* MT;
  const double* Mrow;  // d x d, row-major M (z_j = sum_k M[j][k] y_k), split path FP64 band
  const double* ode_ref;  // ODE objective: kOdeSteps x 10 positions of the hidden parameter vector o
  RunState* st;
  BestPartial* part;
  int32_t ntiles;     // tiles of the FP64 generation kernel
  int32_t rows;       // rows per tile of the FP64 generation kernel
  // split-precision path
  double* T;          // np x dp trial rows
  float* ynorm;       // ntiles_tc * 128, |y|_2 of each trial (error bound of the split GEMM)
  float* tau;         // np, error bound of a split-precision f[i] (0 when f[i] is FP64)
  unsigned long long* stats;  // [0] FP64 re-evaluations, [1] trials evaluated
  uint8_t* A;         // tensor-core A operand, ntiles_tc tiles of a_tile_bytes
  const uint8_t* B;   // tensor-core B operand (M split), nn tiles of b_tile_bytes
  int32_t kpad, npad; // padded K (= input dim) and N (= output dim) of the GEMM
  int32_t ntiles_tc;  // 128-row tiles
  int32_t kc;         // K elements staged per pipeline step
  int32_t nstage;     // stages of the fitness kernel's K pipeline (1: whole K resident)
  int32_t lpt;        // lanes per target in the split trial kernel (power of two, <= 32)
  int32_t ntn;        // N tile width (columns of one accumulator), <= 256
  int32_t nn;         // number of N tiles
  int32_t esz;        // operand element bytes: 2 (bf16) or 4 (tf32)
  int32_t a_tile_bytes, b_tile_bytes;
  int32_t nch;        // column chunks of the FP64 band kernel
  int32_t band_cw;    // columns per chunk (<= 32)
  BandEntry* band;    // shared list of FP64-decided rows (all runs of the handle)
  uint32_t* band_cnt; // its length this generation
  double2* band_part; // per entry: [2 vectors][nch_max] partial sums (s1, s2)
  uint32_t* band_tk;  // per entry: chunk tickets
  int32_t nch_max;    // chunks per vector slot in band_part
  float rownorm;      // max_j |M_j|_2
  float band_u;       // unit error of one split product sum, relative to sum_k |M_jk y_k|
  int32_t band_all;   // 1: every undecidable comparison and every possible new best go to FP64
  float near_thr;     // fitness below which an undecidable comparison goes to FP64
  float* npart;       // several N tiles: per tile, N tile and row the 5 partial epilogue sums
  uint32_t* nticket;  // several N tiles: CTAs of each row tile that have written their partial sums
  // debug capture (all NULL unless enabled)
  int32_t* dbg_idx;
  int32_t* dbg_jrand;
  uint32_t* dbg_mask;
  double* dbg_trial;
  double* dbg_ftrial;
  uint8_t* dbg_accept;
  uint8_t* dbg_fp64;
  int32_t* dbg_cand;  // candidate stream of the evaluated trial (surrogate generations)
};

}  // namespace de
