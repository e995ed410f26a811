/*
 * de_oracle_islands.c -- plain FP64 CPU oracle of the island (multi-population)
 * model of DE: the coarse-grained parallel model of Sec. 3.2, on the GPU the
 * multi-population model of Sec. 5.4, named as future work for GPU DEs in the
 * Conclusion.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  The
 * product path (the CUDA library) never links it and shares no code with it.
 *
 * Readings (the paper describes the model, not its parameters):
 *   - m islands, island k is an ordinary DE run with run_id = run_id0 + k (its
 *     own random streams), all with the same problem and settings;
 *   - synchronous migration (Sec. 5.4: the generation kernels stop and a
 *     migration step runs) after every generation g with g % interval == 0,
 *     on a ring: the nmig best individuals of island k (ascending f, lower
 *     index first, NaN last) replace the nmig worst of island (k + 1) % m
 *     (descending f, NaN first, higher index first), the q-th best into the
 *     q-th worst; all migrants are taken from the populations before any
 *     replacement.  A migrant keeps its fitness (and, with jDE, its F and CR);
 *   - asynchronous migration (Sec. 3.2 names synchronous and asynchronous
 *     strategies; in the GPU form of Sec. 5.4 the asynchronous one migrates
 *     inside the generation kernel, so an island may receive migrants of
 *     another island that is ahead or behind it, which the paper notes makes
 *     runs irreproducible).  Read here with that staleness fixed to one
 *     interval: at every migration point each island posts its nmig best
 *     (the order above) to a mailbox, and takes, into its nmig worst, the
 *     migrants its ring predecessor posted at the previous migration point
 *     (none at the first).  No island then needs another island's state of
 *     the same generation, and the result does not depend on timing;
 *   - the model stops, all islands together, once the best f over all islands
 *     is below the target, or the per-island evaluations reach max_evals, or
 *     max_generations have run (tested before every generation, as a single
 *     run does).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void or_init_population(int np, int d, double lo, double hi, uint64_t seed, uint32_t run_id, double* X);
void or_eval_p(int obj, int d, const double* o, const double* M, double scale, const int32_t* perm,
               const double* x, int64_t ld, int n, double* f, double* sabs, int threads);
void or_step_ex(int np, int d, double F, double CR, double lo, double hi,
                int obj, const double* o, const double* M, const int32_t* perm, double scale,
                uint64_t seed, uint32_t run_id, uint32_t generation, const int32_t* cand,
                int strategy, int jde, const double* jF, const double* jCR, double* jFn, double* jCRn,
                const double* X, const double* fX, double* Xn, double* fXn,
                int32_t* idx, int32_t* jrand_out, uint32_t* mask, double* trial_out,
                double* ftrial_out, double* sabs_out, uint8_t* accept_out, int threads);
int or_best(int np, const double* f);

/* a is better than b: smaller f, NaN never better, lower index on ties */
static int better(const double* f, int a, int b)
{
    int na = f[a] != f[a], nb = f[b] != f[b];
    if (na != nb) return nb;
    if (!na && f[a] != f[b]) return f[a] < f[b];
    return a < b;
}

/* the n best (order[0] best) or the n worst (order[0] worst) indices */
void or_island_ranked(int np, const double* f, int n, int worst, int32_t* out)
{
    for (int q = 0; q < n; ++q) {
        int pick = -1;
        for (int i = 0; i < np; ++i) {
            int taken = 0;
            for (int t = 0; t < q; ++t)
                if (out[t] == i) taken = 1;
            if (taken) continue;
            if (pick < 0) pick = i;
            else if (worst ? better(f, pick, i) : better(f, i, pick)) pick = i;
        }
        out[q] = pick;
    }
}

/* X: m x np x d, fX: m x np, jF / jCR: m x np (jde only).  Returns the
   generations run; *evals_out the evaluations of one island. */
int64_t or_run_islands(int m, int interval, int nmig, int np, int d, double F, double CR, double lo, double hi,
                       int obj, const double* o, const double* M, const int32_t* perm, double scale,
                       uint64_t seed, uint32_t run_id0, int strategy, int jde,
                       int64_t max_generations, int64_t max_evals, double target_error,
                       double* X, double* fX, double* jF, double* jCR, int64_t* evals_out, int threads,
                       int async_mig)
{
    const size_t P = (size_t)np * d;
    double* Xn = (double*)malloc(sizeof(double) * P);
    double* fn = (double*)malloc(sizeof(double) * (size_t)np);
    double* jFn = (double*)malloc(sizeof(double) * (size_t)np);
    double* jCRn = (double*)malloc(sizeof(double) * (size_t)np);
    double* mx = (double*)malloc(sizeof(double) * (size_t)m * nmig * d);
    double* mf = (double*)malloc(sizeof(double) * (size_t)m * nmig);
    double* mF = (double*)malloc(sizeof(double) * (size_t)m * nmig);
    double* mC = (double*)malloc(sizeof(double) * (size_t)m * nmig);
    /* asynchronous migration: the migrants posted at the previous migration point */
    double* px = (double*)malloc(sizeof(double) * (size_t)m * nmig * d);
    double* pf = (double*)malloc(sizeof(double) * (size_t)m * nmig);
    double* pF = (double*)malloc(sizeof(double) * (size_t)m * nmig);
    double* pC = (double*)malloc(sizeof(double) * (size_t)m * nmig);
    int posted = 0;
    int32_t* best = (int32_t*)malloc(sizeof(int32_t) * (size_t)nmig);
    int32_t* worst = (int32_t*)malloc(sizeof(int32_t) * (size_t)nmig);
    for (int k = 0; k < m; ++k) {
        or_init_population(np, d, lo, hi, seed, run_id0 + (uint32_t)k, X + k * P);
        or_eval_p(obj, d, o, M, scale, perm, X + k * P, d, np, fX + (size_t)k * np, NULL, threads);
        for (int i = 0; i < np && jde; ++i) {
            jF[(size_t)k * np + i] = F;
            jCR[(size_t)k * np + i] = CR;
        }
    }
    int64_t evals = np, g = 0;
    while (1) {
        double fbest = INFINITY;
        for (int k = 0; k < m; ++k) {
            int b = or_best(np, fX + (size_t)k * np);
            if (b >= 0 && fX[(size_t)k * np + b] < fbest) fbest = fX[(size_t)k * np + b];
        }
        if (fbest < target_error) break;
        if (max_evals > 0 && evals >= max_evals) break;
        if (g >= max_generations) break;
        g += 1;
        for (int k = 0; k < m; ++k) {
            double* Xk = X + k * P;
            double* fk = fX + (size_t)k * np;
            double* Fk = jde ? jF + (size_t)k * np : NULL;
            double* Ck = jde ? jCR + (size_t)k * np : NULL;
            or_step_ex(np, d, F, CR, lo, hi, obj, o, M, perm, scale, seed, run_id0 + (uint32_t)k, (uint32_t)g, NULL,
                       strategy, jde, Fk, Ck, jFn, jCRn, Xk, fk, Xn, fn, NULL, NULL, NULL, NULL, NULL, NULL, NULL,
                       threads);
            memcpy(Xk, Xn, sizeof(double) * P);
            memcpy(fk, fn, sizeof(double) * (size_t)np);
            if (jde) {
                memcpy(Fk, jFn, sizeof(double) * (size_t)np);
                memcpy(Ck, jCRn, sizeof(double) * (size_t)np);
            }
        }
        evals += np;
        if (interval > 0 && m > 1 && g % interval == 0) {
            /* take every island's migrants first ... */
            for (int k = 0; k < m; ++k) {
                or_island_ranked(np, fX + (size_t)k * np, nmig, 0, best);
                for (int q = 0; q < nmig; ++q) {
                    size_t s = (size_t)k * nmig + q;
                    memcpy(mx + s * d, X + k * P + (size_t)best[q] * d, sizeof(double) * (size_t)d);
                    mf[s] = fX[(size_t)k * np + best[q]];
                    if (jde) {
                        mF[s] = jF[(size_t)k * np + best[q]];
                        mC[s] = jCR[(size_t)k * np + best[q]];
                    }
                }
            }
            /* ... then island (k + 1) % m takes island k's in place of its
               worst: this point's migrants (synchronous), or those posted at
               the previous point (asynchronous; none at the first point) */
            const double *ux = mx, *uf = mf, *uF = mF, *uC = mC;
            if (async_mig) {
                ux = px;
                uf = pf;
                uF = pF;
                uC = pC;
            }
            for (int k = 0; k < m && (!async_mig || posted); ++k) {
                int dst = (k + 1) % m;
                or_island_ranked(np, fX + (size_t)dst * np, nmig, 1, worst);
                for (int q = 0; q < nmig; ++q) {
                    size_t s = (size_t)k * nmig + q;
                    memcpy(X + dst * P + (size_t)worst[q] * d, ux + s * d, sizeof(double) * (size_t)d);
                    fX[(size_t)dst * np + worst[q]] = uf[s];
                    if (jde) {
                        jF[(size_t)dst * np + worst[q]] = uF[s];
                        jCR[(size_t)dst * np + worst[q]] = uC[s];
                    }
                }
            }
            if (async_mig) {
                /* this point's migrants become the posted ones */
                memcpy(px, mx, sizeof(double) * (size_t)m * nmig * d);
                memcpy(pf, mf, sizeof(double) * (size_t)m * nmig);
                memcpy(pF, mF, sizeof(double) * (size_t)m * nmig);
                memcpy(pC, mC, sizeof(double) * (size_t)m * nmig);
                posted = 1;
            }
        }
    }
    free(Xn);
    free(fn);
    free(jFn);
    free(jCRn);
    free(mx);
    free(mf);
    free(mF);
    free(mC);
    free(px);
    free(pf);
    free(pF);
    free(pC);
    free(best);
    free(worst);
    if (evals_out) *evals_out = evals;
    return g;
}
