/*
 * de_oracle.c -- plain, slow, FP64 CPU oracle of DE/rand/1/bin.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  The
 * product path (the CUDA library) never links it and shares no code with it.
 *
 * Everything here follows "GPU Based Differential Evolution: New Insights and
 * Comparative Study" (arXiv 2405.16551):
 *   - population model and the generation loop      Sec. 2 (opening paragraphs)
 *   - DE/rand/1 mutation                             Sec. 2, Eq. 2
 *   - binomial crossover with a forced j_rand        Sec. 2, Eq. 3
 *   - greedy selection (replacement)                 Sec. 2 (Selection item), Sec. 6.2.5
 *   - shift y = x - o, rotation z = M y, [-100,100]  Sec. 7.3.1
 *   - stopping rule: error 1e-8 or the FE budget     Sec. 7.3.4
 * Readings where the paper is silent (index draw method, bound repair, the
 * random-number layout, tie rules) are written next to the code that takes them.
 *
 * Arithmetic: IEEE binary64, round to nearest.  Build with -ffp-contract=off so
 * that the only fused multiply-adds are the explicit fma() calls below.
 * Loops are scalar and in the paper's order; no blocking, no reordering.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11).  The paper's GPU DEs draw from cuRAND (Sec. 4.4, */
/* Sec. 6.2.1); a counter-based generator lets this oracle and the GPU draw   */
/* the same numbers.  Round: two 32x32->64 products of counter words 0 and 2 */
/* with the published multipliers, the high halves xored with the other two  */
/* counter words and the key; the key is bumped by the published Weyl        */
/* constants between rounds.                                                 */
/* ------------------------------------------------------------------------- */
#define OR_PHILOX_M0 0xD2511F53u
#define OR_PHILOX_M1 0xCD9E8D57u
#define OR_PHILOX_W0 0x9E3779B9u
#define OR_PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += OR_PHILOX_W0;
        k1 += OR_PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream layout (a reading: the paper fixes no generator).
 *   key = (seed low 32 bits, seed high 32 bits)
 *   ctr = (d / 4, individual, generation, run_id << 12 | cand << 4 | purpose)
 *   draw d of a stream is word d % 4 of that block.                         */
enum { OR_PURPOSE_INIT = 1, OR_PURPOSE_STEP = 2, OR_PURPOSE_JDE = 6 };

uint32_t or_draw(uint64_t seed, uint32_t purpose, uint32_t run_id, uint32_t cand,
                 uint32_t generation, uint32_t individual, uint32_t d)
{
    uint32_t ctr[4], key[2], out[4];
    ctr[0] = d / 4u;
    ctr[1] = individual;
    ctr[2] = generation;
    ctr[3] = (run_id << 12) | ((cand & 0xFFu) << 4) | (purpose & 0xFu);
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
    or_philox4x32_10(ctr, key, out);
    return out[d % 4u];
}

/* u in [0, 2^32) -> integer in [0, n): floor(u * n / 2^32). */
uint32_t or_map(uint32_t u, uint32_t n)
{
    return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

/* Two words (a, b) -> a double in [0, 1) with 53 random bits. */
double or_u53(uint32_t a, uint32_t b)
{
    uint64_t bits = (((uint64_t)a << 32) | (uint64_t)b) >> 11;
    return (double)bits * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------- */
/* Objectives (Sec. 7.3.1): y = (x - o) * scale, z = M y (M row-major D x D, */
/* NULL means no rotation), then a basic function of z whose minimum 0 is at  */
/* z = 0, i.e. at x = o.                                                      */
/*                                                                            */
/* *sabs receives the scale S of the fitness tolerance tau = rel (|f| + S):  */
/* the sum of the magnitudes of the terms before cancellation, plus the      */
/* first-order effect of rounding the inputs of the terms,                   */
/* sum_j |df/dz_j| (G_j + |z_j|) with G_j = sum_k |M_jk y_k| (the size of    */
/* the dot product that forms z_j), and for Rosenbrock also |df/dt_j| |t_j|  */
/* for the rounding of t = z + 1.  A correct evaluation in another summation  */
/* order differs from this one by a small multiple of eps * S.                */
/* ------------------------------------------------------------------------- */
enum { OR_SPHERE = 0, OR_RASTRIGIN = 1, OR_ROSENBROCK = 2, OR_ACKLEY = 3, OR_ODE = 4 };

/* The ODE fitting objective (de_oracle_ode.c): o is the hidden parameter
 * vector, d must be 20, M and scale do not apply. */
double or_ode_objective_s(const double* x, const double* x_hat, int steps, double dt, double* sabs);

/* The benchmark suite's objectives 5..20 (de_oracle_suite.c). */
double or_suite_objective(int obj, int d, const double* o, const double* M, double scale, const int32_t* perm,
                          const double* x, double* sabs);

/* perm: the hybrid functions' permutation (d indices), NULL elsewhere. */
double or_objective_p(int obj, int d, const double* o, const double* M, double scale, const int32_t* perm,
                      const double* x, double* sabs)
{
    if (obj >= 5 && obj <= 20) return or_suite_objective(obj, d, o, M, scale, perm, x, sabs);
    if (obj == OR_ODE) {
        static const double zero[20] = {0};
        if (d != 20) {
            if (sabs) *sabs = NAN;
            return NAN;
        }
        return or_ode_objective_s(x, o ? o : zero, 2000, 1e-3, sabs);
    }
    double* y = (double*)malloc(sizeof(double) * (size_t)d);
    double* z = (double*)malloc(sizeof(double) * (size_t)d);
    double* G = (double*)malloc(sizeof(double) * (size_t)d);
    const double pi = 3.14159265358979323846, two_pi = 2.0 * pi;
    double f = 0.0, s = 0.0;
    for (int k = 0; k < d; ++k)
        y[k] = (x[k] - (o ? o[k] : 0.0)) * scale;
    for (int j = 0; j < d; ++j) {
        if (M) {
            double acc = 0.0, mag = 0.0;
            for (int k = 0; k < d; ++k) {
                acc += M[(size_t)j * d + k] * y[k];
                mag += fabs(M[(size_t)j * d + k] * y[k]);
            }
            z[j] = acc;
            G[j] = mag;
        } else {
            z[j] = y[j];
            G[j] = fabs(y[j]);
        }
    }
    if (obj == OR_SPHERE) {
        for (int j = 0; j < d; ++j) f += z[j] * z[j];
        s = f;
        for (int j = 0; j < d; ++j) s += 2.0 * fabs(z[j]) * (G[j] + fabs(z[j]));
    } else if (obj == OR_RASTRIGIN) {
        for (int j = 0; j < d; ++j) {
            double c = cos(two_pi * z[j]);
            f += z[j] * z[j] - 10.0 * c + 10.0;
            s += z[j] * z[j] + 10.0 * fabs(c) + 10.0;
            double g = 2.0 * fabs(z[j]) + 20.0 * pi * fabs(sin(two_pi * z[j]));
            s += g * (G[j] + fabs(z[j]));
        }
    } else if (obj == OR_ROSENBROCK) {
        /* evaluated at t = z + 1 so that the minimum sits at z = 0 (x = o) */
        for (int j = 0; j + 1 < d; ++j) {
            double t0 = z[j] + 1.0, t1 = z[j + 1] + 1.0;
            double a = t1 - t0 * t0, b = t0 - 1.0;
            f += 100.0 * a * a + b * b;
            s += 100.0 * a * a + b * b;
            /* d/dt0 and d/dt1 of this term, times the sizes of t0, t1 and z */
            double g0 = 400.0 * fabs(a) * fabs(t0) + 2.0 * fabs(b);
            double g1 = 200.0 * fabs(a);
            s += g0 * (G[j] + fabs(z[j]) + fabs(t0)) + g1 * (G[j + 1] + fabs(z[j + 1]) + fabs(t1));
            s += 200.0 * fabs(a) * t0 * t0;
        }
    } else if (obj == OR_ACKLEY) {
        double s1 = 0.0, s2 = 0.0, s2abs = 0.0;
        for (int j = 0; j < d; ++j) {
            double c = cos(two_pi * z[j]);
            s1 += z[j] * z[j];
            s2 += c;
            s2abs += fabs(c);
        }
        double r = sqrt(s1 / d);
        double e1 = exp(-0.2 * r);
        double e2 = exp(s2 / d);
        f = 20.0 + exp(1.0) - 20.0 * e1 - e2;
        s = 20.0 + exp(1.0) + 20.0 * e1 + exp(s2abs / d);
        for (int j = 0; j < d; ++j) {
            double g = (r > 0.0 ? 4.0 * e1 * fabs(z[j]) / (d * r) : 0.0)
                     + two_pi / d * fabs(sin(two_pi * z[j])) * e2;
            s += g * (G[j] + fabs(z[j]));
        }
        /* the square root amplifies the rounding of s1 near the optimum */
        s += (r > 0.0 ? 2.0 * e1 * r : 0.0);
    } else {
        f = NAN;
        s = NAN;
    }
    free(y);
    free(z);
    free(G);
    if (sabs) *sabs = s;
    return f;
}

double or_objective(int obj, int d, const double* o, const double* M, double scale,
                    const double* x, double* sabs)
{
    return or_objective_p(obj, d, o, M, scale, NULL, x, sabs);
}

/* n rows of x (row stride ld) -> f[n] (and sabs[n] if not NULL). */
void or_eval_p(int obj, int d, const double* o, const double* M, double scale, const int32_t* perm,
               const double* x, int64_t ld, int n, double* f, double* sabs, int threads)
{
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads > 0 ? threads : 1) schedule(static)
#else
    (void)threads;
#endif
    for (int i = 0; i < n; ++i) {
        double sa;
        f[i] = or_objective_p(obj, d, o, M, scale, perm, x + (size_t)i * (size_t)ld, &sa);
        if (sabs) sabs[i] = sa;
    }
}

void or_eval(int obj, int d, const double* o, const double* M, double scale,
             const double* x, int64_t ld, int n, double* f, double* sabs, int threads)
{
    or_eval_p(obj, d, o, M, scale, NULL, x, ld, n, f, sabs, threads);
}

/* ------------------------------------------------------------------------- */
/* Initialisation (Sec. 2; Sec. 6.2.1): every parameter uniform in [lo, hi).  */
/* Parameter j of individual i uses words 2j and 2j+1 of the INIT stream of   */
/* that individual at generation 0.                                           */
/* ------------------------------------------------------------------------- */
void or_init_population(int np, int d, double lo, double hi, uint64_t seed, uint32_t run_id,
                        double* X)
{
    for (int i = 0; i < np; ++i)
        for (int j = 0; j < d; ++j) {
            uint32_t a = or_draw(seed, OR_PURPOSE_INIT, run_id, 0, 0, (uint32_t)i, 2u * (uint32_t)j);
            uint32_t b = or_draw(seed, OR_PURPOSE_INIT, run_id, 0, 0, (uint32_t)i, 2u * (uint32_t)j + 1u);
            X[(size_t)i * d + j] = fma(hi - lo, or_u53(a, b), lo);
        }
}

/* ------------------------------------------------------------------------- */
/* Mutant indices (Eq. 2: r1, r2, r3 mutually distinct and different from i).*/
/* The paper's GPU DEs redraw until distinct (Sec. 6.2.3).  This oracle takes */
/* the same uniform ordered triple with exactly three draws: the k-th index   */
/* is drawn uniform over the NP - k values not yet taken, then moved past the */
/* taken values in ascending order.  Requires NP >= 4.                        */
/* ------------------------------------------------------------------------- */
static uint32_t or_skip_taken(uint32_t r, const uint32_t* taken, int ntaken)
{
    /* taken[] is visited in ascending order */
    uint32_t sorted[3];
    for (int a = 0; a < ntaken; ++a) sorted[a] = taken[a];
    for (int a = 0; a < ntaken; ++a)
        for (int b = a + 1; b < ntaken; ++b)
            if (sorted[b] < sorted[a]) { uint32_t t = sorted[a]; sorted[a] = sorted[b]; sorted[b] = t; }
    for (int a = 0; a < ntaken; ++a)
        if (r >= sorted[a]) r += 1u;
    return r;
}

void or_mutant_indices(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t i, uint32_t np,
                       uint32_t r[3])
{
    uint32_t taken[3];
    taken[0] = i;
    r[0] = or_skip_taken(or_map(w0, np - 1u), taken, 1);
    taken[1] = r[0];
    r[1] = or_skip_taken(or_map(w1, np - 2u), taken, 2);
    taken[2] = r[1];
    r[2] = or_skip_taken(or_map(w2, np - 3u), taken, 3);
}

/* CR -> integer threshold: rand_j <= CR with rand_j = w / 2^32 is w <= floor(CR 2^32). */
uint64_t or_cr_threshold(double cr)
{
    return (uint64_t)floor(cr * 4294967296.0);
}

/* ------------------------------------------------------------------------- */
/* One generation g >= 1 of DE/rand/1/bin, synchronous: every trial is built  */
/* from the generation-(g-1) population X, the next population goes to Xn.   */
/* Per target i, draws of the STEP stream: 0,1,2 -> r1,r2,r3; 3 -> j_rand;    */
/* 4 + j -> rand_j of Eq. 3.                                                  */
/* Optional outputs (any may be NULL): idx[np*3], jrand[np], mask[np*nw] with */
/* nw = ceil(d/32) (bit j%32 of word j/32), trial[np*d], ftrial[np],          */
/* sabs_trial[np], accept[np].                                                */
/* ------------------------------------------------------------------------- */
int or_best(int np, const double* f);

/* Variants of the trial construction (Sec. 2 names them: the base vector
 * "rand" or "best", "bin" or "exp" crossover; jDE adapts F and CR per
 * individual).  The formulas are the published ones, restated:
 *   strategy 0  DE/rand/1/bin   v = x_r1 + F (x_r2 - x_r3), binomial crossover
 *   strategy 1  DE/best/1/bin   v = x_best + F (x_r1 - x_r2), best = the best
 *                                individual of generation g-1 (lowest f, then
 *                                lowest index)
 *   strategy 2  DE/rand/1/exp   exponential crossover (Storn and Price): from
 *                                the start n = map(draw 3, D), L = 1 plus the
 *                                number of leading draws 4, 5, ... with
 *                                rand <= CR, at most D; coordinates n, n+1,
 *                                ..., n+L-1 (mod D) cross
 *   jDE (Brest et al., IEEE TEC 2006): per target, words w0..w3 of the JDE
 *   stream at (individual, generation); with probability tau = 0.1 each,
 *     F' = 0.1 + 0.9 u0  (one fma)       when w1 < floor(0.1 2^32),
 *     CR' = u2                            when w3 < floor(0.1 2^32),
 *   where u = w / 2^32; otherwise F' = F_i, CR' = CR_i.  The trial uses F'
 *   and CR'; they replace F_i and CR_i only when the trial is selected.
 * cand (may be NULL = all 0): per target, the candidate stream its trial is
 * drawn from.  Stream 0 is plain DE; streams 1, 2, ... give the other
 * candidate trials that a surrogate screens (the same construction with
 * independent draws). */
void or_step_ex(int np, int d, double F, double CR, double lo, double hi,
                int obj, const double* o, const double* M, const int32_t* perm, double scale,
                uint64_t seed, uint32_t run_id, uint32_t generation, const int32_t* cand,
                int strategy, int jde, const double* jF, const double* jCR, double* jFn, double* jCRn,
                const double* X, const double* fX, double* Xn, double* fXn,
                int32_t* idx, int32_t* jrand_out, uint32_t* mask, double* trial_out,
                double* ftrial_out, double* sabs_out, uint8_t* accept_out, int threads)
{
    const int nw = (d + 31) / 32;
    const uint64_t T = or_cr_threshold(CR);
    const uint32_t tau_thr = (uint32_t)floor(0.1 * 4294967296.0);
    /* DE/best/1: the lowest-index best; the paper does not cover a population
       without a finite fitness, where row 0 serves as the base */
    const int best = or_best(np, fX) < 0 ? 0 : or_best(np, fX);
    double* trial = (double*)malloc(sizeof(double) * (size_t)np * (size_t)d);
    double* ft = (double*)malloc(sizeof(double) * (size_t)np);
    double* sa = (double*)malloc(sizeof(double) * (size_t)np);
    double* Ft = (double*)malloc(sizeof(double) * (size_t)np);
    double* CRt = (double*)malloc(sizeof(double) * (size_t)np);

    /* mutation (Eq. 2), crossover (Eq. 3) and bound repair for every target */
    for (int i = 0; i < np; ++i) {
        const uint32_t ci = cand ? (uint32_t)cand[i] : 0u;
        uint32_t w[4];
        for (int k = 0; k < 4; ++k)
            w[k] = or_draw(seed, OR_PURPOSE_STEP, run_id, ci, generation, (uint32_t)i, (uint32_t)k);
        uint32_t r[3];
        or_mutant_indices(w[0], w[1], w[2], (uint32_t)i, (uint32_t)np, r);
        uint32_t jrand = or_map(w[3], (uint32_t)d);
        if (idx) { idx[3 * i] = (int32_t)r[0]; idx[3 * i + 1] = (int32_t)r[1]; idx[3 * i + 2] = (int32_t)r[2]; }
        if (jrand_out) jrand_out[i] = (int32_t)jrand;
        if (mask) for (int k = 0; k < nw; ++k) mask[(size_t)i * nw + k] = 0u;
        /* control parameters of this trial */
        double Fi = F, CRi = CR;
        uint64_t Ti = T;
        if (jde) {
            uint32_t a[4];
            for (int k = 0; k < 4; ++k)
                a[k] = or_draw(seed, OR_PURPOSE_JDE, run_id, ci, generation, (uint32_t)i, (uint32_t)k);
            Fi = a[1] < tau_thr ? fma(0.9, (double)a[0] * (1.0 / 4294967296.0), 0.1) : jF[i];
            CRi = a[3] < tau_thr ? (double)a[2] * (1.0 / 4294967296.0) : jCR[i];
            Ti = or_cr_threshold(CRi);
        }
        Ft[i] = Fi;
        CRt[i] = CRi;
        const double* xi = X + (size_t)i * d;
        const double* x1 = strategy == 1 ? X + (size_t)best * d : X + (size_t)r[0] * d;
        const double* x2 = strategy == 1 ? X + (size_t)r[0] * d : X + (size_t)r[1] * d;
        const double* x3 = strategy == 1 ? X + (size_t)r[1] * d : X + (size_t)r[2] * d;
        /* exponential crossover: the length of the crossed block */
        int L = 0;
        if (strategy == 2) {
            L = 1;
            while (L < d && (uint64_t)or_draw(seed, OR_PURPOSE_STEP, run_id, ci, generation, (uint32_t)i,
                                              4u + (uint32_t)(L - 1)) <= Ti)
                ++L;
        }
        for (int j = 0; j < d; ++j) {
            int crossed;
            if (strategy == 2) {
                crossed = ((j - (int)jrand + d) % d) < L;
            } else {
                uint32_t u = or_draw(seed, OR_PURPOSE_STEP, run_id, ci, generation, (uint32_t)i, 4u + (uint32_t)j);
                crossed = ((uint32_t)j == jrand) || ((uint64_t)u <= Ti);
            }
            double t;
            if (crossed) {
                /* Eq. 2: y_ij = x_base,j + F (x_a,j - x_b,j) */
                double v = fma(Fi, x2[j] - x3[j], x1[j]);
                /* bound repair (the paper is silent): a coordinate that leaves
                   [lo, hi] goes half way from the target's coordinate to the
                   violated bound */
                if (v < lo) v = (xi[j] + lo) * 0.5;
                else if (v > hi) v = (xi[j] + hi) * 0.5;
                t = v;
                if (mask) mask[(size_t)i * nw + j / 32] |= 1u << (j % 32);
            } else {
                t = xi[j];
            }
            trial[(size_t)i * d + j] = t;
        }
    }

    /* evaluate the trial population (Sec. 7.3.1) */
    or_eval_p(obj, d, o, M, scale, perm, trial, d, np, ft, sa, threads);

    /* greedy selection (Sec. 2, Selection): the trial replaces the target
       when it is no worse (ties go to the trial).  A NaN objective value has
       no quality and ranks below every number: a NaN trial never replaces,
       and any other trial replaces a NaN target. */
    for (int i = 0; i < np; ++i) {
        int acc = !isnan(ft[i]) && (isnan(fX[i]) || ft[i] <= fX[i]);
        if (accept_out) accept_out[i] = (uint8_t)acc;
        if (ftrial_out) ftrial_out[i] = ft[i];
        if (sabs_out) sabs_out[i] = sa[i];
        if (trial_out) memcpy(trial_out + (size_t)i * d, trial + (size_t)i * d, sizeof(double) * (size_t)d);
        if (Xn) memcpy(Xn + (size_t)i * d, acc ? trial + (size_t)i * d : X + (size_t)i * d, sizeof(double) * (size_t)d);
        if (fXn) fXn[i] = acc ? ft[i] : fX[i];
        if (jde) {
            if (jFn) jFn[i] = acc ? Ft[i] : jF[i];
            if (jCRn) jCRn[i] = acc ? CRt[i] : jCR[i];
        }
    }
    free(trial);
    free(ft);
    free(sa);
    free(Ft);
    free(CRt);
}

void or_step_cand(int np, int d, double F, double CR, double lo, double hi,
                  int obj, const double* o, const double* M, double scale,
                  uint64_t seed, uint32_t run_id, uint32_t generation, const int32_t* cand,
                  const double* X, const double* fX, double* Xn, double* fXn,
                  int32_t* idx, int32_t* jrand_out, uint32_t* mask, double* trial_out,
                  double* ftrial_out, double* sabs_out, uint8_t* accept_out, int threads)
{
    or_step_ex(np, d, F, CR, lo, hi, obj, o, M, NULL, scale, seed, run_id, generation, cand, 0, 0, NULL, NULL, NULL,
               NULL, X, fX, Xn, fXn, idx, jrand_out, mask, trial_out, ftrial_out, sabs_out, accept_out, threads);
}

void or_step(int np, int d, double F, double CR, double lo, double hi,
             int obj, const double* o, const double* M, double scale,
             uint64_t seed, uint32_t run_id, uint32_t generation,
             const double* X, const double* fX, double* Xn, double* fXn,
             int32_t* idx, int32_t* jrand_out, uint32_t* mask, double* trial_out,
             double* ftrial_out, double* sabs_out, uint8_t* accept_out, int threads)
{
    or_step_cand(np, d, F, CR, lo, hi, obj, o, M, scale, seed, run_id, generation, NULL, X, fX, Xn, fXn,
                 idx, jrand_out, mask, trial_out, ftrial_out, sabs_out, accept_out, threads);
}

/* Best individual: smallest f, lowest index on ties, NaN never best. */
int or_best(int np, const double* f)
{
    int b = -1;
    for (int i = 0; i < np; ++i) {
        if (f[i] != f[i]) continue;
        if (b < 0 || f[i] < f[b]) b = i;
    }
    return b;
}

/* ------------------------------------------------------------------------- */
/* A whole run (Sec. 2 loop; stopping rule Sec. 7.3.4): initialise, evaluate, */
/* then generations 1, 2, ... until the best error (f* = 0) is below target,  */
/* the evaluation count reaches max_evals, or max_generations have run.       */
/* Evaluations are counted from the initial population on (FE = NP (1 + g)). */
/* The stop test runs once per generation.                                    */
/* best_trace (may be NULL) receives the best f after init and after every    */
/* generation, max_generations + 1 entries.                                   */
/* Returns the number of generations run.                                     */
/* ------------------------------------------------------------------------- */
int64_t or_run_ex(int np, int d, double F, double CR, double lo, double hi,
                  int obj, const double* o, const double* M, const int32_t* perm, double scale,
                  uint64_t seed, uint32_t run_id, int strategy, int jde,
                  int64_t max_generations, int64_t max_evals, double target_error,
                  double* X, double* fX, double* jF, double* jCR, int64_t* evals_out, double* best_trace, int threads)
{
    double* Xn = (double*)malloc(sizeof(double) * (size_t)np * (size_t)d);
    double* fn = (double*)malloc(sizeof(double) * (size_t)np);
    double* jFn = (double*)malloc(sizeof(double) * (size_t)np);
    double* jCRn = (double*)malloc(sizeof(double) * (size_t)np);
    for (int i = 0; i < np && jde; ++i) {
        jF[i] = F;
        jCR[i] = CR;
    }
    or_init_population(np, d, lo, hi, seed, run_id, X);
    or_eval_p(obj, d, o, M, scale, perm, X, d, np, fX, NULL, threads);
    int64_t evals = np;
    int64_t g = 0;
    int b = or_best(np, fX);
    if (best_trace) best_trace[0] = b >= 0 ? fX[b] : NAN;
    while (1) {
        b = or_best(np, fX);
        if (b >= 0 && fX[b] < target_error) break;
        if (max_evals > 0 && evals >= max_evals) break;
        if (g >= max_generations) break;
        g += 1;
        or_step_ex(np, d, F, CR, lo, hi, obj, o, M, perm, scale, seed, run_id, (uint32_t)g, NULL, strategy, jde, jF, jCR,
                   jFn, jCRn, X, fX, Xn, fn, NULL, NULL, NULL, NULL, NULL, NULL, NULL, threads);
        memcpy(X, Xn, sizeof(double) * (size_t)np * (size_t)d);
        memcpy(fX, fn, sizeof(double) * (size_t)np);
        if (jde) {
            memcpy(jF, jFn, sizeof(double) * (size_t)np);
            memcpy(jCR, jCRn, sizeof(double) * (size_t)np);
        }
        evals += np;
        if (best_trace) { int bb = or_best(np, fX); best_trace[g] = bb >= 0 ? fX[bb] : NAN; }
    }
    free(Xn);
    free(fn);
    free(jFn);
    free(jCRn);
    if (evals_out) *evals_out = evals;
    return g;
}

int64_t or_run(int np, int d, double F, double CR, double lo, double hi,
               int obj, const double* o, const double* M, double scale,
               uint64_t seed, uint32_t run_id,
               int64_t max_generations, int64_t max_evals, double target_error,
               double* X, double* fX, int64_t* evals_out, double* best_trace, int threads)
{
    return or_run_ex(np, d, F, CR, lo, hi, obj, o, M, NULL, scale, seed, run_id, 0, 0, max_generations, max_evals,
                     target_error, X, fX, NULL, NULL, evals_out, best_trace, threads);
}
