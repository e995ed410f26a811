/*
 * de.h -- C ABI of the GB300 (sm_103a) DE/rand/1/bin library, libde_gb300.so.
 *
 * The method is differential evolution as stated in "GPU Based Differential
 * Evolution: New Insights and Comparative Study" (arXiv 2405.16551):
 *   - a population of NP individuals, each a D-dimensional real vector,
 *     initialised uniformly inside the bounds and evaluated (Sec. 2);
 *   - per target i, the DE/rand/1 mutant y_i = x_r1 + F (x_r2 - x_r3) with
 *     r1, r2, r3 mutually distinct and different from i (Sec. 2, Eq. 2);
 *   - binomial crossover: trial coordinate j is the mutant's when
 *     rand_j <= CR or j = j_rand, else the target's (Sec. 2, Eq. 3);
 *   - greedy selection: the trial replaces the target when its objective is
 *     no worse (Sec. 2, Selection; Sec. 6.2.5);
 *   - objectives are minimised over [-100, 100]^D after a shift y = x - o and
 *     a rotation z = M y (Sec. 7.3.1); runs stop at error 1e-8 or at the
 *     function-evaluation budget (Sec. 7.3.4).
 *
 * Conventions (every entry point):
 *   - The return value is a de_status.  No C++ exception crosses this
 *     boundary and the library never aborts, traps or exits the process.
 *     On any status other than DE_OK, de_last_error(h) (or
 *     de_last_error(NULL) when no handle exists) gives a one-line message.
 *   - Output pointers are written only when the call returns DE_OK.
 *   - A handle owns all device memory it allocates.  It issues all of its
 *     work on the CUDA stream given to de_init / de_init_batch (NULL = the
 *     legacy default stream).  Calls that return host data synchronise that
 *     stream; de_step and de_eval only enqueue work.
 *   - A handle may be used by one host thread at a time.
 *   - Host arrays are dense row-major; "host" and "device" below say which
 *     address space a pointer must be in.
 *   - Population rows are stored on the device with a padded row stride
 *     (D rounded up to a multiple of 4 doubles); the host-facing calls below
 *     take and return dense rows of D values.
 *   - Random numbers come from Philox4x32-10 (Salmon et al., SC'11) keyed by
 *     the seed, with the counter built from (draw block, individual,
 *     generation, run_id and purpose), so results do not depend on launch
 *     shapes and a CPU program can draw the same numbers.
 */
#ifndef DE_GB300_H
#define DE_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DE_API __attribute__((visibility("default")))
#else
#define DE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DE_OK = 0,
    DE_ERR_INVALID_ARG = 1, /* a size, pointer or parameter is out of range */
    DE_ERR_CUDA = 2,        /* a CUDA runtime call failed (message has the CUDA error) */
    DE_ERR_OOM = 3,         /* device or host allocation failed */
    DE_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    DE_ERR_NONFINITE = 5,   /* a non-finite value where a finite one is required */
    DE_ERR_STATE = 6,       /* the call does not fit the handle's state */
    DE_ERR_IO = 7,          /* checkpoint file could not be read or written, or is corrupt */
    DE_ERR_UNSUPPORTED = 8  /* the device or configuration is not supported */
} de_status;

/* Objectives (Sec. 7.3.1 stand-ins; minimum 0 at x = o):
 *   SPHERE      sum z_j^2
 *   RASTRIGIN   sum (z_j^2 - 10 cos(2 pi z_j) + 10)
 *   ROSENBROCK  sum_{j<D-1} 100 (t_{j+1} - t_j^2)^2 + (t_j - 1)^2,  t = z + 1
 *   ACKLEY      20 + e - 20 exp(-0.2 sqrt(sum z_j^2 / D)) - exp(sum cos(2 pi z_j) / D)
 *   ODE         fit of a 10-oscillator damped chain (D = 20, FP64, no rotation).
 *               The paper defines no such problem (it motivates costly
 *               objectives in its Abstract); the workload is a reading.  Ten
 *               unit masses in a chain: springs k_i to ground, dampers c_i,
 *               unit springs between neighbours, walls at both ends, with
 *               k_i = 0.5 + 4.5 (x_i + 100)/200 and
 *               c_i = 0.01 + 0.49 (x_{10+i} + 100)/200.
 *               Integrated by RK4 with dt = 1e-3 for 2000 steps from
 *               q(0) = e_1, p(0) = 0.
 *               f = mean over steps and masses of (q - q_o)^2, where q_o is
 *               the trajectory of the hidden parameter vector, passed as
 *               the shift o; f(o) = 0 exactly.
 *
 * The benchmark the paper proposes for GPU DEs (Sec. 7.3, Table 2; FP64
 * only).  Basic functions of z (same shift / scale / rotation as above; each
 * is 0 at z = 0; n the dimension, i = 1..n):
 *   ZAKHAROV    sum z_i^2 + (sum 0.5 i z_i)^2 + (sum 0.5 i z_i)^4
 *   SCHWEFEL    modified Schwefel: 418.9828872724338 n - sum g(z_i + 420.9687462275036),
 *               g(t) = t sin sqrt|t| on [-500, 500]; beyond, with m = fmod(|t|, 500),
 *               g = +-(500 - m) sin sqrt(500 - m) - (|t| - 500)^2 / (10^4 n)
 *   BENT_CIGAR  z_1^2 + 10^6 sum_{i>=2} z_i^2
 *   HGBAT       |a^2 - b^2|^(1/2) + (0.5 a + b)/n + 0.5,  a = sum x_i^2, b = sum x_i, x = z - 1
 *   SCHAFFER_F6 expanded: sum over the cyclic pairs (z_i, z_{i+1}) of
 *               0.5 + (sin^2 sqrt(s) - 0.5) / (1 + 0.001 s)^2, s = u^2 + v^2
 *   KATSUURA    (10/n^2) prod_i (1 + i sum_{j=1}^{32} |2^j z_i - round(2^j z_i)| / 2^j)^(10/n^1.2) - 10/n^2
 *   HAPPYCAT    |a - n|^(1/4) + (0.5 a + b)/n + 0.5 (a, b as HGBAT)
 *   GRIEWANK_ROSENBROCK  expanded: sum over the cyclic pairs of G(100 (u^2 - v)^2 + (u - 1)^2),
 *               (u, v) = (z_i + 1, z_{i+1} + 1), G(r) = r^2/4000 - cos r + 1
 *   ELLIPTIC    sum (10^6)^((i-1)/(n-1)) z_i^2
 *   GRIEWANK    sum z_i^2 / 4000 - prod cos(z_i / sqrt i) + 1
 * Hybrid functions (Sec. 7.3.2): z = M ((x - o) scale) is permuted by
 * de_config.perm (NULL: identity) and split into parts of ceil(p_k d)
 * coordinates (the last part takes the rest); part k, multiplied by its
 * function's domain scale, is evaluated by that function as an
 * n_k-dimensional one, and f is the sum.
 *   HYBRID1  Bent Cigar, HGBat, Rastrigin;                   p = 0.3, 0.3, 0.4
 *   HYBRID2  Schaffer F6, HGBat, Rosenbrock, Schwefel;       p = 0.2, 0.2, 0.3, 0.3
 *   HYBRID3  Katsuura, HappyCat, Griewank-Rosenbrock, Schwefel, Ackley; p = 0.3, 0.2, 0.2, 0.1, 0.2
 * Composition functions (Sec. 7.3.3): n components, each with its own shift
 * o_c and rotation M_c (de_config.shift holds n*d values, de_config.rot n
 * row-major d*d matrices):
 *   f = sum_c omega_c (lambda_c g_c(M_c ((x - o_c) s_c)) + bias_c),
 *   omega_c = w_c / sum w,  w_c = exp(-D_c / (2 d sigma_c^2)) / sqrt(D_c),  D_c = |x - o_c|^2
 * (omega_c = 1 for the first c with x = o_c).  s_c is the component's domain
 * scale; de_config.scale must be 1.
 *   COMPOSITION1  Rastrigin, Griewank, Schwefel; sigma 10, 20, 30; lambda 1, 10, 1; bias 0, 100, 200
 *   COMPOSITION2  Ackley, Elliptic, Griewank, Rastrigin; sigma 10, 20, 30, 40;
 *                 lambda 10, 1e-6, 10, 1; bias 0, 100, 200, 300
 *   COMPOSITION3  Schaffer F6, Schwefel, Griewank, Rosenbrock, Rastrigin; sigma 10, 20, 20, 30, 40;
 *                 lambda 0.005, 1, 10, 1, 10; bias 0, 100, 200, 300, 400
 * Domain scales inside hybrid and composition functions: Rastrigin 5.12/100,
 * Rosenbrock 2.048/100, Schwefel 1000/100, Griewank 600/100, HGBat,
 * HappyCat, Katsuura and Griewank-Rosenbrock 5/100, the others 1.  The
 * stand-alone basic functions take de_config.scale instead. */
typedef enum {
    DE_OBJ_SPHERE = 0,
    DE_OBJ_RASTRIGIN = 1,
    DE_OBJ_ROSENBROCK = 2,
    DE_OBJ_ACKLEY = 3,
    DE_OBJ_ODE = 4,
    DE_OBJ_ZAKHAROV = 5,
    DE_OBJ_SCHWEFEL = 6,
    DE_OBJ_BENT_CIGAR = 7,
    DE_OBJ_HGBAT = 8,
    DE_OBJ_SCHAFFER_F6 = 9,
    DE_OBJ_KATSUURA = 10,
    DE_OBJ_HAPPYCAT = 11,
    DE_OBJ_GRIEWANK_ROSENBROCK = 12,
    DE_OBJ_ELLIPTIC = 13,
    DE_OBJ_GRIEWANK = 14,
    DE_OBJ_HYBRID1 = 15,
    DE_OBJ_HYBRID2 = 16,
    DE_OBJ_HYBRID3 = 17,
    DE_OBJ_COMPOSITION1 = 18,
    DE_OBJ_COMPOSITION2 = 19,
    DE_OBJ_COMPOSITION3 = 20
} de_objective;

/* Arithmetic of the rotation z = M y and of the objective terms.
 *   FP64     DFMA on CUDA cores, FP64 terms.
 *   BF16X3   tcgen05 tensor cores: y and M split into bf16 high and low parts,
 *            z = yh Mh + yh Ml + yl Mh accumulated in FP32 (TMEM); FP32 terms.
 *            About 16 bits of y and M take part (2^-16 relative per product).
 *   TF32X3   the same with tf32 parts (22 bits, 2^-22 per product).
 * The split forms are the library's FP32-class arithmetic: there is no plain
 * FP32 form, because the rotation is a dense contraction that runs on the
 * tensor cores.  In BF16X3/TF32X3 the selection comparison is redone in FP64
 * as de_fp64_band says, and the best-so-far record returned by de_get_best /
 * de_run is the FP64 fitness of the best individual. */
typedef enum {
    DE_PREC_FP64 = 0,
    DE_PREC_BF16X3 = 1,
    DE_PREC_TF32X3 = 2
} de_precision;

typedef enum {
    DE_STOP_NONE = 0,        /* still running */
    DE_STOP_TARGET = 1,      /* best f < target_error (f* = 0) */
    DE_STOP_EVALS = 2,       /* evaluations >= max_evals */
    DE_STOP_GENERATIONS = 3  /* generations == max_generations */
} de_stop_reason;

/* One run's configuration.  Ranges are checked by de_init. */
typedef struct {
    int32_t np;               /* population size, 4 <= np <= 2^20 (Eq. 2 needs 3 donors besides i) */
    int32_t d;                /* dimension, 1 <= d <= 4096 (ODE: d == 20) */
    double f;                 /* differential weight F, 0 <= F <= 2 (Eq. 2) */
    double cr;                /* crossover rate C_R, 0 <= CR <= 1 (Eq. 3) */
    double lo, hi;            /* box bounds, finite, lo < hi; the paper's range is [-100, 100] */
    int32_t objective;        /* de_objective */
    double scale;             /* y = (x - o) * scale; 1.0 keeps the search range (Sec. 7.3.1) */
    const double* shift;      /* host, d values of o (composition functions: n*d, one row per
                                 component), or NULL for o = 0; copied by de_init.  The problem
                                 data of Sec. 7.3.1 is the caller's: it is passed, not drawn
                                 by the library, so that any other program (a CPU reference,
                                 another run) can be given the very same arrays */
    const double* rot;        /* host, d*d row-major M (z = M y; composition functions: n such
                                 matrices), or NULL for no rotation; copied */
    uint64_t seed;            /* Philox key */
    uint32_t run_id;          /* Philox stream id, < 2^20; distinct runs of one seed differ here */
    int32_t precision;        /* de_precision */
    double target_error;      /* stop once best f < target_error (Sec. 7.3.4 uses 1e-8); <= 0 disables */
    int64_t max_evals;        /* stop once evaluations >= max_evals, counting the initial NP; 0 = none */
    int64_t max_generations;  /* stop after this many generations (de_run); >= 0 */
    int32_t debug_capture;    /* nonzero: keep indices, masks, trials, f_trial and flags of the last generation */
    int32_t fp64_band;        /* split precisions: de_fp64_band, when a selection is redone in FP64 */
    int32_t surrogate_k;      /* 0 or 1: plain DE.  2..32: surrogate-assisted generations with this many
                                 candidate trials per target (FP64, d == 20, one run per handle; see
                                 de_get_surrogate_stats) */
    int32_t surrogate_steps;  /* Adam steps per retraining of the surrogate; 0 = 25 */
    int32_t strategy;         /* de_strategy: base vector and crossover of the trial (Sec. 2); not with a
                                 surrogate */
    int32_t jde;              /* nonzero: jDE self-adaptive F and CR per individual (Sec. 2, the adaptive
                                 variant); f and cr are the initial values; not with a surrogate */
    const int32_t* perm;      /* host, d indices: the permutation of a hybrid function (position k of the
                                 permuted vector is z[perm[k]]), or NULL for the identity; must be NULL
                                 for other objectives; copied by de_init */
} de_config;

/* Trial-construction strategies (Sec. 2 names the variants by base vector,
 * number of difference vectors and crossover):
 *   DE_RAND1BIN  base x_r1, one difference x_r2 - x_r3, binomial crossover (Eq. 2, Eq. 3)
 *   DE_BEST1BIN  base x_best (the lowest-index best of the current population; row 0 when no
 *                fitness is finite), difference x_r1 - x_r2 of the first two drawn donors,
 *                binomial crossover
 *   DE_RAND1EXP  base x_r1, difference x_r2 - x_r3, exponential crossover: coordinates
 *                j_rand, j_rand + 1, ... (cyclic) for a block of length L, where L - 1 is the
 *                number of leading crossover draws rand_0, rand_1, ... at or below the CR
 *                threshold (at most d - 1); the other coordinates come from the target
 * jDE (de_config.jde) applies to every strategy: before the trial of target i
 * is built, with probability 0.1 each (draws 1 and 3 of the JDE stream of
 * (i, g) below floor(0.1 * 2^32)), F_i becomes 0.1 + 0.9 u_0 and CR_i becomes
 * u_2 (u_k = draw k / 2^32); otherwise the stored values are used.  The
 * trial uses F_i and CR_i; the stored values become the trial's when the
 * trial is accepted. */
typedef enum {
    DE_RAND1BIN = 0,
    DE_BEST1BIN = 1,
    DE_RAND1EXP = 2
} de_strategy;

/* When the split precisions redo a selection comparison in FP64.
 *   DE_BAND_NEAR (default)  the split values cannot decide it within their
 *                           error bound and one of the two values is near the
 *                           optimum (below min(target_error, 1e-8) / (8 u), u
 *                           the unit error of the split product), or the
 *                           trial's error bound straddles the stop target
 *                           (the stop rule of Sec. 7.3.4 is then decided in
 *                           FP64; a trial surely below or above the target
 *                           decides it on its split value); elsewhere the split values
 *                           decide, and a decision may then differ from the
 *                           FP64 one only inside the split error bound
 *   DE_BAND_ALL             every comparison the split values cannot decide,
 *                           and every trial that could become the best: the
 *                           run takes the FP64 decisions everywhere (up to
 *                           FP64 rounding) at the cost of more FP64 work */
typedef enum {
    DE_BAND_NEAR = 0,
    DE_BAND_ALL = 1
} de_fp64_band;

/* Result of de_run for one run. */
typedef struct {
    double best_f;            /* FP64 fitness of the best individual */
    int32_t best_index;       /* its index (lowest index on ties) */
    int32_t stop_reason;      /* de_stop_reason */
    int64_t generations;      /* generations run so far */
    int64_t evals;            /* objective evaluations so far, NP (1 + generations) */
    double seconds;           /* wall time of the de_run call */
} de_result;

/* Host buffers for de_get_debug, each sized for the run's np and d
 * (nw = ceil(d / 32)); any pointer may be NULL to skip that field. */
typedef struct {
    int32_t* idx;             /* np*3: r1, r2, r3 per target */
    int32_t* jrand;           /* np */
    uint32_t* mask;           /* np*nw: bit j%32 of word j/32 set when coordinate j was crossed */
    double* trial;            /* np*d: trial vectors after bound repair */
    double* f_trial;          /* np: fitness of each trial (FP64 when the FP64 band re-evaluated it) */
    uint8_t* accept;          /* np: 1 when the trial replaced the target */
    uint8_t* fp64_checked;    /* np: 1 when the selection was decided on FP64 fitness values */
    int32_t* cand;            /* np: candidate stream of the evaluated trial (0 outside surrogate mode);
                                 surrogate generations do not fill idx, jrand and mask */
} de_debug;

typedef struct de_handle de_handle;

/* Version string of the library ("de_gb300 <major>.<minor> sm_103a"). */
DE_API const char* de_version(void);

/* Create a handle for one run: validate cfg, allocate device buffers on the
 * stream, copy shift and rotation, initialise the population (Sec. 2:
 * x_ij = lo + (hi - lo) u_ij with u_ij from the INIT stream) and evaluate it.
 * cuda_stream: a cudaStream_t or NULL.  *out receives the handle.
 * Errors: DE_ERR_INVALID_ARG (cfg out of range, out == NULL), DE_ERR_OOM,
 * DE_ERR_CUDA, DE_ERR_UNSUPPORTED (not a compute-capability 10.3 device). */
DE_API de_status de_init(const de_config* cfg, void* cuda_stream, de_handle** out);

/* Create a handle for nruns independent runs (each with its own np, d,
 * objective, shift, rotation, seed and run_id) that advance together: one
 * generation of the handle is one generation of every run that has not
 * stopped, in a single set of launches.  Runs must share precision.
 * Errors as de_init; DE_ERR_INVALID_ARG when nruns < 1 or any cfg is invalid. */
DE_API de_status de_init_batch(const de_config* cfgs, int32_t nruns, void* cuda_stream, de_handle** out);

/* The island model (Sec. 3.2; on the GPU, the multi-population model of
 * Sec. 5.4, which the paper leaves to future work for DE): nislands copies
 * of *cfg, island k with run_id = cfg->run_id + k, evolve as the runs of one
 * batch.  Synchronous migration on a ring after every generation g with
 * g % interval == 0: the `migrants` best individuals of island k (ascending
 * f, lower index first, NaN last) replace the `migrants` worst of island
 * (k + 1) % nislands (descending f, NaN first, higher index first), the q-th
 * best into the q-th worst, all taken before any is written; a migrant keeps
 * its fitness (and its jDE parameters).  The model stops as a whole: when any
 * island's best is below target_error every island stops with reason
 * DE_STOP_TARGET; the evaluation and generation limits apply per island
 * (the islands advance together).  Results come per island from de_run
 * (nruns = nislands) and de_get_best.
 * Errors: DE_ERR_INVALID_ARG (nislands outside [2, 4096], interval < 1,
 * migrants outside [1, min(32, np / 2)], run_id + nislands > 2^20, or cfg
 * invalid), DE_ERR_UNSUPPORTED (split precision or a surrogate), DE_ERR_OOM,
 * DE_ERR_CUDA. */
DE_API de_status de_init_islands(const de_config* cfg, int32_t nislands, int32_t interval, int32_t migrants,
                                 void* cuda_stream, de_handle** out);

/* Migration strategies of the island model (Sec. 3.2 names synchronous and
 * asynchronous migration). */
typedef enum {
  DE_MIGRATE_SYNC = 0,  /* as de_init_islands */
  DE_MIGRATE_ASYNC = 1  /* one interval late, through a mailbox (below) */
} de_migration;

/* de_init_islands with a migration strategy.  DE_MIGRATE_ASYNC: in the GPU
 * form of Sec. 5.4 asynchronous migration happens inside the generation
 * kernel, so an island may receive migrants of an island that is ahead of it
 * or behind it and runs cannot be repeated; here the staleness is fixed to one
 * interval.  At every migration point (generation g, g % interval == 0) island
 * k posts its `migrants` best (the order above) to a device mailbox and takes,
 * into its `migrants` worst, the migrants island k - 1 posted at the previous
 * migration point (none at the first point after de_init, de_reset,
 * de_set_population or de_load, which empty the mailbox).  One kernel per
 * migration, no ordering among the islands, reproducible results.  Same
 * errors as de_init_islands, plus DE_ERR_INVALID_ARG for another `migration`
 * value. */
DE_API de_status de_init_islands_ex(const de_config* cfg, int32_t nislands, int32_t interval, int32_t migrants,
                                    int32_t migration, void* cuda_stream, de_handle** out);

/* Re-initialise run `run` (or every run when run == -1) as de_init did
 * (Sec. 2, initialisation): population from the INIT stream, evaluation,
 * counters and best record reset.  Enqueued on the handle's stream;
 * allocates nothing. */
DE_API de_status de_reset(de_handle* h, int32_t run);

/* Enqueue `generations` generations (>= 0) on the handle's stream, with no
 * stop test other than the per-run stop flags the device sets itself.
 * One generation is the loop of Sec. 2: per target the mutant of Eq. 2, the
 * crossover of Eq. 3, bound repair, the objective of Sec. 7.3.1 and greedy
 * selection (Sec. 2, Selection; Sec. 6.2.5), then the best-so-far record and
 * the stopping rule of Sec. 7.3.4.  Generation g builds every trial from the
 * generation g-1 population (synchronous replacement, as the kernel-per-
 * operation GPU designs of Sec. 5.3 and Sec. 6.1 do).  A trial whose
 * objective is NaN never replaces its target, and any trial replaces a
 * target whose objective is NaN (NaN ranks below every number).
 * Returns once the work is enqueued; a device-side error shows at the next
 * synchronising call (DE_ERR_TIMEOUT, DE_ERR_NONFINITE). */
DE_API de_status de_step(de_handle* h, int64_t generations);

/* Run until every run has stopped under the stopping rule of Sec. 7.3.4
 * (best f below target_error, or the evaluation budget max_evals, counting
 * the initial population) or after max_generations, checking the stop flags
 * between launches.  out: host array of nruns results (may be NULL).
 * Synchronises.
 * Errors: DE_ERR_TIMEOUT (a bounded device-side wait gave up; the run's
 * population is then undefined until de_reset), DE_ERR_NONFINITE (every
 * fitness of a run is NaN), DE_ERR_CUDA. */
DE_API de_status de_run(de_handle* h, de_result* out);

/* Evaluate n rows with run `run`'s objective, shift, rotation and precision:
 * the function evaluation of Sec. 6.2.2 on the objectives of Sec. 7.3.1
 * (y = (x - o) scale, z = M y, then the basic, hybrid or composition
 * function).  x_dev: device, n rows of d doubles with row stride ld (>= d)
 * doubles.  f_dev: device, n doubles.  Both caller-owned; enqueued on the
 * stream.  In a split precision, a row whose bounded device-side wait gave up
 * (it should not on a healthy device) comes back as NaN. */
DE_API de_status de_eval(de_handle* h, int32_t run, const double* x_dev, int64_t ld, int32_t n, double* f_dev);

/* ---- evaluation without a handle and without allocation ----------------
 * The paper has no counterpart to this call; it serves deployment only.
 *
 * Evaluates n rows of the shifted, rotated objective in a split precision
 * (BF16X3 or TF32X3).  The same kernels run as in de_eval on a handle with
 * the same objective, d, scale, shift, rotation and precision, so the results
 * are bit-identical.  This call needs no handle and allocates nothing on any
 * call: no cudaMalloc, cudaFree, pinned host memory or library allocator.
 * It is for callers that cannot allocate device memory at the point where
 * they evaluate.  One case is a process whose device memory is already held
 * by its own caching allocator or fixed arena, where another allocation could
 * fail or fragment it.  Another is a loop running beside other streams'
 * work, where cudaFree synchronises the whole device and cudaMalloc may.
 * (de_init allocates a population arena, operand copies and band lists.)
 *
 * Scratch: one 16 MiB array in the library's device memory on each device.
 * It holds the descriptor, the split copy of M, |y| per row and the
 * tensor-core operand tiles.  Nothing in it needs to start at zero, because
 * each call writes every part it uses before reading it.  Rows past n in the
 * last 128-row tile are computed on but never reach f_dev.
 *
 * Limit: the scratch bounds d and n per call.  A call needs about 1 KiB,
 * plus 2 e npad kpad bytes for M, plus 256 e kpad + 520 bytes per 128 rows,
 * where:
 *   e = 2 for BF16X3, 4 for TF32X3;
 *   kpad = d rounded up to 16;
 *   npad = kpad for d <= 256, else d rounded up to 256.
 * The largest d is 1920 (BF16X3) / 1280 (TF32X3); a larger d returns
 * DE_ERR_INVALID_ARG naming that limit.  The largest n per call
 * (BF16X3 / TF32X3):
 *   d = 10: 246,400 / 126,976     d = 30: 126,976 / 64,384
 *   d = 100: 36,992 / 18,432      d = 1000: 3,072 / 1,024
 * A larger n returns DE_ERR_INVALID_ARG, naming the largest n for that d and
 * precision, and launches nothing.
 * A bounded device-side wait that gives up (it should not on a healthy
 * device) cannot be reported by the call, which has returned by then: the
 * rows of the affected 128-row tiles come back as NaN.
 *
 * First call: the first call on each device looks up the scratch's address
 * (cudaGetSymbolAddress), with that device current.  This may also load the
 * library's device code on that device.  Make that first call before any
 * stream capture begins.
 * Concurrency: all calls on one device share the one scratch, so calls must
 * not overlap.  Issue them on one stream, or order them with events or
 * synchronisation.  Calls in flight at the same time race on the scratch and
 * give wrong results, whether they come from two streams, two threads or two
 * independent users of the library in one process.  Calls are asynchronous
 * on cuda_stream.
 *
 * precision: DE_PREC_BF16X3 or DE_PREC_TF32X3.  DE_PREC_FP64 returns
 *   DE_ERR_UNSUPPORTED (use de_eval, which needs no scratch for FP64).
 * objective: DE_OBJ_SPHERE .. DE_OBJ_ACKLEY.  Rosenbrock needs d <= 256.
 * d: 1..1920 (BF16X3) or 1..1280 (TF32X3).  scale: finite and nonzero
 *   (y = (x - o) scale).
 * shift_dev: device, d doubles, or NULL for o = 0.
 * rot_dev: device, d*d doubles row-major (z_j = sum_k M[j][k] y_k), or NULL
 *   for M = I.
 * x_dev: device, n rows of d doubles with row stride ld (>= d) doubles.
 * f_dev: device, n doubles.
 * All device buffers are caller-owned and must be on the current device.
 * cuda_stream: a cudaStream_t, or NULL for the legacy default stream.
 * Errors: DE_ERR_INVALID_ARG (arguments, or n beyond the scratch),
 * DE_ERR_UNSUPPORTED, DE_ERR_CUDA.  The message is in de_last_error(NULL). */
DE_API de_status de_eval_noalloc(int32_t precision, int32_t objective, int32_t d, double scale,
                                 const double* shift_dev, const double* rot_dev, const double* x_dev, int64_t ld,
                                 int32_t n, double* f_dev, void* cuda_stream);

/* ---- surrogate network ----------------------------------------------
 * The paper has no surrogate; it motivates costly objectives in its Abstract.
 * This network screens candidate trials in the surrogate-assisted workload.
 *
 * Architecture: MLP 20 -> 256 -> 256 -> 1 with ReLU, 71,425 parameters.
 *   h1 = relu(W1 x/100 + b1),  h2 = relu(W2 h1 + b2),  y = w3 . h2 + b3.
 * Parameter vector (FP32, DE_MLP_PARAMS entries, in this order):
 *   W1 (256 x 20, row-major), b1 (256), W2 (256 x 256), b2 (256), w3 (256), b3.
 *
 * Arithmetic: BF16 operands on the tensor cores (tcgen05) with FP32
 * accumulation; FP32 epilogues, FP32 master weights, Adam in FP32.
 * Training minimises the mean squared error over minibatches of 256 rows.
 * Adam uses beta1 = 0.9, beta2 = 0.999, eps = 1e-8.
 * Work goes on the stream given to de_mlp_create.  Calls that return host
 * data synchronise it. */
#define DE_MLP_PARAMS 71425
typedef struct de_mlp de_mlp;

/* Allocate the network on the current device.  Weights are He-uniform from
 * `seed`; biases and Adam moments start at zero. */
DE_API de_status de_mlp_create(uint64_t seed, void* cuda_stream, de_mlp** out);
DE_API de_status de_mlp_destroy(de_mlp* m);
/* Replace the parameters (host, DE_MLP_PARAMS floats) and reset Adam. */
DE_API de_status de_mlp_set_params(de_mlp* m, const float* params);
DE_API de_status de_mlp_get_params(de_mlp* m, float* params);
/* y_dev[i] = network(x_dev row i), for n rows of 20 doubles with stride ld (>= 20). */
DE_API de_status de_mlp_forward(de_mlp* m, const double* x_dev, int64_t ld, int32_t n, float* y_dev);
/* Gradient of the loss (1/256) sum (y - t)^2 over rows 0..255 of x_dev,
 * with targets t_dev (device, 256 floats), without changing the parameters.
 * grad (host, DE_MLP_PARAMS floats) and loss (host, one float) may be NULL. */
DE_API de_status de_mlp_grad(de_mlp* m, const double* x_dev, int64_t ld, const float* t_dev, float* grad,
                             float* loss);
/* `steps` Adam steps with learning rate lr.  Each minibatch holds 256 rows
 * drawn uniformly, with replacement, from the n rows of x_dev and t_dev.
 * The draws come from a Philox stream keyed by the seed and the step count.
 * *loss (may be NULL) receives the loss of the last minibatch. */
DE_API de_status de_mlp_train(de_mlp* m, const double* x_dev, int64_t ld, const float* t_dev, int32_t n,
                              int32_t steps, float lr, float* loss);

/* ---- surrogate-assisted generations (surrogate_k >= 2) ----------------
 * The paper has no surrogate.  This mode serves costly objectives, which its
 * Abstract motivates; every setting below is a choice of this library.
 *
 * Per generation, each target draws k candidate trials.  Candidate c uses
 * the STEP draws with cand = c; candidate 0 is the plain DE/rand/1/bin trial
 * of Eq. 2 / Eq. 3.  The surrogate network (de_mlp) predicts each
 * candidate's fitness, and only the candidate with the lowest prediction is
 * evaluated with the true objective.  Greedy selection then runs as in
 * plain DE.  Evaluations count true evaluations only.
 *
 * Each evaluated trial and its f enter an archive of 200,000 rows.  The
 * network trains on the most recent 20,000 rows: first after 5 plain
 * generations, then every 10 generations, with surrogate_steps Adam steps on
 * standardised log f.
 * The network's measured error decides whether it screens: after each generation the
 * Spearman correlation between its predictions and the true f of the
 * evaluated trials is measured, and the next generation screens k
 * candidates only when that correlation is at least 0.3.  Otherwise it
 * draws a single candidate, which is plain DE.
 *
 * Each generation synchronises the stream once, for that decision.
 * trainings, screened_generations, last_rho and k_now may each be NULL.
 * Returns DE_ERR_STATE for a handle without a surrogate. */
DE_API de_status de_get_surrogate_stats(de_handle* h, int64_t* trainings, int64_t* screened_generations,
                                        double* last_rho, int32_t* k_now);

/* Copy run `run`'s current population (np*d, host) and fitness (np, host)
 * out (the population and objective values of Sec. 2); either pointer may be
 * NULL.  Synchronises. */
DE_API de_status de_get_population(de_handle* h, int32_t run, double* x_host, double* f_host);

/* Replace run `run`'s population and fitness with host arrays (np*d, np)
 * (the population of Sec. 2).  x_host must be finite (DE_ERR_NONFINITE
 * otherwise); f_host may hold NaN, and may be NULL, in which case the
 * population is evaluated on the device.  Resets that run's stop flag and
 * recomputes its best record (Sec. 7.3.4); the generation counter is kept. */
DE_API de_status de_set_population(de_handle* h, int32_t run, const double* x_host, const double* f_host);

/* Set the generation counter of run `run` (the next de_step runs g + 1).
 * The counter selects the random numbers of a generation (Philox counter) and
 * the evaluation count NP (1 + g) of the stopping rule (Sec. 7.3.4). */
DE_API de_status de_set_generation(de_handle* h, int32_t run, int64_t generation);

/* jDE state of run `run` (cfg.jde set): the per-individual F_i and CR_i of
 * the current population (np doubles each, host; either may be NULL).
 * de_init and de_reset set every F_i to cfg.f and every CR_i to cfg.cr;
 * de_set_population keeps them.  Synchronises.
 * Errors: DE_ERR_STATE when the run does not use jDE; DE_ERR_INVALID_ARG for
 * de_set_adaptive values outside F in [0, 2], CR in [0, 1]. */
DE_API de_status de_get_adaptive(de_handle* h, int32_t run, double* f_host, double* cr_host);
DE_API de_status de_set_adaptive(de_handle* h, int32_t run, const double* f_host, const double* cr_host);

/* Self-test (no counterpart in the paper): converts n host doubles to FP32
 * with the library's integer round-to-nearest-even (the conversion used for
 * the split-precision operands) and with the GPU's conversion instruction,
 * and returns how many results differ (NaN equals NaN), or -1 on a CUDA
 * error or a NULL / negative argument.  Allocates and synchronises the
 * current device. */
DE_API int64_t de_selftest_f32_rounding(const double* x_host, int64_t n);

/* Self-test (no counterpart in the paper): the current device's FP64
 * fused multiply-add throughput in TFLOP/s (2 flops per DFMA), measured by a
 * kernel of independent DFMA chains on every SM (4 CTAs of 256 threads per
 * SM, 8 chains per thread, 1024 steps; CUDA events, best of 3).  This is the
 * measured peak the FP64 kernels' throughput is reported against.  Returns
 * -1 on a CUDA error.  Allocates and synchronises the current device. */
DE_API double de_selftest_fp64_rate(void);

/* Best record of run `run` (the best-so-far solution that the stopping rule
 * of Sec. 7.3.4 tests): best_f, its index (lowest index on ties), a copy of
 * its vector (host, d doubles, may be NULL), and generation/evaluation
 * counters. */
DE_API de_status de_get_best(de_handle* h, int32_t run, double* best_f, int32_t* best_index, double* best_x,
                      int64_t* generations, int64_t* evals, int32_t* stop_reason);

/* Copy the last generation's debug capture of run `run` (cfg.debug_capture
 * must have been set): the mutant indices r1, r2, r3 of Eq. 2, j_rand and the
 * crossover mask of Eq. 3, the repaired trials, their fitness and the
 * selection decisions (Sec. 2, Selection).  Synchronises. */
DE_API de_status de_get_debug(de_handle* h, int32_t run, const de_debug* out);

/* Number of runs in the handle, and run `run`'s np and d. */
DE_API de_status de_get_shape(de_handle* h, int32_t run, int32_t* np, int32_t* d, int32_t* nruns);

/* Which kernel path runs the generations of this handle:
 *   0  FP64: one fused kernel per generation
 *   1  split precision, three kernels per generation (trial, tensor-core
 *      fitness and selection, FP64 band), in CUDA graphs
 *   2  split precision, one persistent cluster kernel for many generations
 *   4  split precision, one cooperative persistent kernel for many
 *      generations in which every CTA owns at most 16 targets and runs their
 *      tensor-core products itself (a grid barrier between generations, no
 *      clusters); single runs of d <= 128 whose CTAs all fit at once
 *   5  split precision, one cooperative persistent kernel (one CTA per SM)
 *      for many generations of a batch of runs: work items are the runs'
 *      128-target tiles, each CTA owns a fixed slice of them, and in place of
 *      a grid barrier each run has an arrival counter (a run's next
 *      generation starts when every tile of its previous one is done; the
 *      stop rule of Sec. 7.3.4 applies per run); batches of at least two
 *      DE/rand/1/bin runs of d <= 128 whose operands fit one CTA's shared
 *      memory (TF32x3: d <= 112); de_init times it against path 1 and keeps
 *      the faster (DE_GB300_PERSIST_BATCH=1 / 0 forces path 5 / path 1)
 *   3  FP64, one cooperative persistent kernel for many generations of
 *      every run of the handle (grid barrier between generations; the same
 *      numbers as path 0; not with a surrogate, and only when every tile
 *      fits on the device at once; an island model's migrations and common
 *      stop run inside the loop, an extra grid barrier after each migration,
 *      except for the benchmark suite's objectives 5..20, whose islands run
 *      on path 0), or, for one run of at most 8
 *      tiles, the same loop as one thread-block cluster (cluster barrier);
 *      the FP64 autotuner chooses among path 0 and these when one times
 *      faster on the handle's problem; DE_GB300_FP64_PERSIST=0 / 1 / 2 forces
 *      path 0 / the cooperative launch / the cluster (where it applies)
 * cluster_size (may be NULL) receives the CTAs per cluster of path 2 or of
 * path 3 launched as one cluster, else 0;
 * each cluster owns up to 128 targets (a multiple of the cluster size, timed
 * at de_init; DE_GB300_PERSIST_ROWS fixes it).
 * Paths 2 and 4 apply to a single run, path 2 of d <= 105 (its FP64 band
 * gives each of the 7 member CTAs at most 15 outputs), path 4 of d <= 128;
 * de_init times both where both apply and keeps the faster (DE_GB300_PERSIST_MODE=cluster / cta keeps one form,
 * DE_GB300_PERSIST_CTA_ROWS fixes the targets per CTA of path 4); the
 * environment variable DE_GB300_PERSIST=0 disables both.
 * Test switch (failure detection, off by default): DE_GB300_TEST_GRID_TIMEOUT=k
 * at de_init makes CTA k - 1 of every persistent launch (paths 2, 3, 4 and 5)
 * leave out its first grid-barrier arrival (path 5: the arrival of its first
 * item's first generation) and the waits give up after a few thousand polls,
 * so that the bounded wait runs out and de_run returns DE_ERR_TIMEOUT. */
DE_API de_status de_get_plan(de_handle* h, int32_t* kernel_path, int32_t* cluster_size);

/* Counters of the split-precision selection of run `run` since de_init:
 * trials whose comparison (or best-record candidacy) was decided on FP64
 * re-evaluations, and trials evaluated in total.  Both are 0 in FP64
 * precision, where every comparison is FP64. */
DE_API de_status de_get_stats(de_handle* h, int32_t run, int64_t* fp64_reevals, int64_t* trials);

/* Write the state of every run (population, fitness, jDE parameters,
 * counters, best record: the state of the loop of Sec. 2 at a generation
 * boundary) to `path`, with a CRC32 over the payload and, per run, a 64-bit
 * hash of the problem (objective, F, CR, bounds, scale, seed, run_id,
 * precision, strategy, jDE, FP64 band policy, shift, rotation and
 * permutation).  de_load restores it into a handle created with the same
 * configurations; the stopping limits (target_error, max_evals,
 * max_generations) may differ.  de_load parses and checks the whole file on
 * the host before it copies anything to the device, so a refused file leaves
 * the handle unchanged.
 * Errors: DE_ERR_IO (open/write/read failure, bad magic, CRC mismatch,
 * truncation), DE_ERR_STATE (a run's shape or problem differs from the
 * handle's). */
DE_API de_status de_save(de_handle* h, const char* path);
DE_API de_status de_load(de_handle* h, const char* path);

/* Destroy the handle and free its device memory (h may be NULL). */
DE_API de_status de_destroy(de_handle* h);

/* Last error message of h (or of the last failed handle-less call when h is
 * NULL); an empty string after success.  Owned by the library. */
DE_API const char* de_last_error(de_handle* h);

/* Name of a status code. */
DE_API const char* de_status_string(de_status s);

#ifdef __cplusplus
}
#endif

#endif /* DE_GB300_H */
