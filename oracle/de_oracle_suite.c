/*
 * de_oracle_suite.c -- plain FP64 CPU oracle of the benchmark the paper
 * proposes for GPU DEs (Sec. 7.3, Table 2): its basic functions, the hybrid
 * functions (Sec. 7.3.2) and the composition functions (Sec. 7.3.3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  The
 * product path (the CUDA library) never links it and shares no code with it.
 *
 * The paper names the basic functions and takes their definitions from the
 * CEC'14 and CEC'17 suites; each is written here from its published
 * mathematical definition.  The shift, rotation and permutation data are
 * synthetic (the suites' data files are not used).  Readings where the
 * paper is silent are stated next to the code.
 *
 * Every basic function g has its minimum g = 0 at z = 0 (after the offsets
 * written next to it).  basic_eval also returns the scale S of the fitness
 * tolerance tau = rel (|f| + S): the sum of the term magnitudes plus
 * sum_k |dg/dz_k| e_k, where e_k bounds the size of the quantities whose
 * rounding formed z_k (so that a correct evaluation in another order, or
 * with another correctly rounded libm, differs by a small multiple of
 * eps * S).
 *
 * Arithmetic: IEEE binary64, round to nearest, built with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    G_SPHERE = 0, G_RASTRIGIN = 1, G_ROSENBROCK = 2, G_ACKLEY = 3,
    G_ZAKHAROV = 5, G_SCHWEFEL = 6, G_BENT_CIGAR = 7, G_HGBAT = 8, G_SCHAFFER_F6 = 9, G_KATSUURA = 10,
    G_HAPPYCAT = 11, G_GRIEWANK_ROSENBROCK = 12, G_ELLIPTIC = 13, G_GRIEWANK = 14,
    G_HYBRID1 = 15, G_HYBRID2 = 16, G_HYBRID3 = 17, G_COMPOSITION1 = 18, G_COMPOSITION2 = 19, G_COMPOSITION3 = 20
};

static const double OR_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------- */
/* Basic functions of z[0..n), i = k + 1 the 1-based position.               */
/* ------------------------------------------------------------------------- */

/* modified Schwefel term of t = z + 420.9687462275036 (CEC'14/'17 form): t sin
   sqrt|t| inside [-500, 500]; outside, the value folded back into the box
   with fmod and a quadratic penalty (t -+ 500)^2 / (10^4 n) */
static double schwefel_g(double t, int n)
{
    if (t > 500.0) {
        double m = fmod(t, 500.0);
        return (500.0 - m) * sin(sqrt(500.0 - m)) - (t - 500.0) * (t - 500.0) / (10000.0 * n);
    }
    if (t < -500.0) {
        double m = fmod(-t, 500.0);
        return (m - 500.0) * sin(sqrt(500.0 - m)) - (t + 500.0) * (t + 500.0) / (10000.0 * n);
    }
    return t * sin(sqrt(fabs(t)));
}

/* Schaffer's F6 of the pair (u, v) */
static double schaffer_pair(double u, double v, double* S, double eu, double ev)
{
    double s = u * u + v * v;
    double r = sqrt(s);
    double sn = sin(r);
    double den = 1.0 + 0.001 * s;
    double g = 0.5 + (sn * sn - 0.5) / (den * den);
    double dgs = (r > 0.0 ? fabs(sn * cos(r)) / r : 1.0) / (den * den)
               + 0.002 * fabs(sn * sn - 0.5) / (den * den * den);
    *S += 0.5 + fabs(sn * sn - 0.5) / (den * den) + dgs * (2.0 * fabs(u) * eu + 2.0 * fabs(v) * ev + 2.0 * s);
    return g;
}

/* Griewank's 1-D term of Rosenbrock's 2-D term of the pair (u, v) */
static double griewank_rosenbrock_pair(double zu, double zv, double eu, double ev, double* S)
{
    double u = zu + 1.0, v = zv + 1.0;
    double a = u * u - v, b = u - 1.0;
    double r = 100.0 * a * a + b * b;
    double g = r * r / 4000.0 - cos(r) + 1.0;
    double dgr = r / 2000.0 + fabs(sin(r));
    double dru = fabs(400.0 * a * u + 2.0 * b), drv = 200.0 * fabs(a);
    *S += r * r / 4000.0 + fabs(cos(r)) + 1.0
        + dgr * (dru * (eu + fabs(zu) + fabs(u)) + drv * (ev + fabs(zv) + fabs(v)) + 200.0 * fabs(a) * u * u + r);
    return g;
}

/* g(z) of basic function fn on n coordinates; e[k] >= |z[k]| bounds the
   rounding of z[k] (NULL: |z[k]|); *S receives the tolerance scale. */
double or_basic(int fn, int n, const double* z, const double* e, double* sabs)
{
    double f = 0.0, S = 0.0;
#define E(k) (e ? e[(k)] : fabs(z[(k)]))
    if (n < 1) {
        if (sabs) *sabs = NAN;
        return NAN;
    }
    switch (fn) {
    case G_SPHERE:
        for (int k = 0; k < n; ++k) f += z[k] * z[k];
        S = f;
        for (int k = 0; k < n; ++k) S += 2.0 * fabs(z[k]) * E(k);
        break;
    case G_RASTRIGIN:
        for (int k = 0; k < n; ++k) {
            double c = cos(2.0 * OR_PI * z[k]);
            f += z[k] * z[k] - 10.0 * c + 10.0;
            S += z[k] * z[k] + 10.0 * fabs(c) + 10.0
               + (2.0 * fabs(z[k]) + 20.0 * OR_PI * fabs(sin(2.0 * OR_PI * z[k]))) * E(k);
        }
        break;
    case G_ROSENBROCK:
        /* at t = z + 1: sum_{i<n} 100 (t_{i+1} - t_i^2)^2 + (t_i - 1)^2 */
        for (int k = 0; k + 1 < n; ++k) {
            double t0 = z[k] + 1.0, t1 = z[k + 1] + 1.0;
            double a = t1 - t0 * t0, b = t0 - 1.0;
            f += 100.0 * a * a + b * b;
            S += 100.0 * a * a + b * b + (400.0 * fabs(a) * fabs(t0) + 2.0 * fabs(b)) * (E(k) + fabs(t0))
               + 200.0 * fabs(a) * (E(k + 1) + fabs(t1)) + 200.0 * fabs(a) * t0 * t0;
        }
        break;
    case G_ACKLEY: {
        double s1 = 0.0, s2 = 0.0, s2abs = 0.0;
        for (int k = 0; k < n; ++k) {
            double c = cos(2.0 * OR_PI * z[k]);
            s1 += z[k] * z[k];
            s2 += c;
            s2abs += fabs(c);
        }
        double r = sqrt(s1 / n);
        double e1 = exp(-0.2 * r), e2 = exp(s2 / n);
        f = 20.0 + exp(1.0) - 20.0 * e1 - e2;
        S = 20.0 + exp(1.0) + 20.0 * e1 + exp(s2abs / n) + (r > 0.0 ? 2.0 * e1 * r : 0.0);
        for (int k = 0; k < n; ++k)
            S += ((r > 0.0 ? 4.0 * e1 * fabs(z[k]) / (n * r) : 0.0)
                  + 2.0 * OR_PI / n * fabs(sin(2.0 * OR_PI * z[k])) * e2) * E(k);
        break;
    }
    case G_ZAKHAROV: {
        /* sum z_i^2 + (sum 0.5 i z_i)^2 + (sum 0.5 i z_i)^4 */
        double a = 0.0, b = 0.0, bb = 0.0, be = 0.0;
        for (int k = 0; k < n; ++k) {
            a += z[k] * z[k];
            b += 0.5 * (k + 1) * z[k];
            bb += 0.5 * (k + 1) * fabs(z[k]);
            be += 0.5 * (k + 1) * E(k);
            S += 2.0 * fabs(z[k]) * E(k);
        }
        f = a + b * b + b * b * b * b;
        S += f + (2.0 * fabs(b) + 4.0 * fabs(b) * b * b) * (bb + be);
        break;
    }
    case G_SCHWEFEL: {
        /* 418.9828872724338 n - sum g(z_i + 420.9687462275036): the optimum of
           t sin sqrt|t| on [-500, 500] is at t = 420.9687462275036 with value
           418.9828872724338 (to double precision) */
        const double c0 = 420.9687462275036, fmax = 418.9828872724338;
        double s = 0.0;
        for (int k = 0; k < n; ++k) {
            double t = z[k] + c0;
            double g = schwefel_g(t, n);
            s += g;
            double at = fabs(t);
            S += fabs(g) + (1.0 + 0.5 * sqrt(at < 500.0 ? at : 500.0) + 2.0 * (at > 500.0 ? at - 500.0 : 0.0) / (10000.0 * n))
                         * (E(k) + at);
        }
        f = fmax * n - s;
        S += fmax * n;
        break;
    }
    case G_BENT_CIGAR:
        /* z_1^2 + 10^6 sum_{i>=2} z_i^2 */
        f = z[0] * z[0];
        S = 2.0 * fabs(z[0]) * E(0);
        for (int k = 1; k < n; ++k) {
            f += 1e6 * z[k] * z[k];
            S += 2e6 * fabs(z[k]) * E(k);
        }
        S += f;
        break;
    case G_HGBAT:
    case G_HAPPYCAT: {
        /* at x = z - 1 (minimum at z = 0), with a = sum x^2, b = sum x:
           HGBat    |a^2 - b^2|^(1/2) + (0.5 a + b) / n + 0.5
           HappyCat |a - n|^(1/4)     + (0.5 a + b) / n + 0.5 */
        double a = 0.0, b = 0.0, bb = 0.0;
        for (int k = 0; k < n; ++k) {
            double x = z[k] - 1.0;
            a += x * x;
            b += x;
            bb += fabs(x);
        }
        double h, dA, dB, cancel;
        if (fn == G_HGBAT) {
            double q = fabs(a * a - b * b);
            h = sqrt(q);
            dA = (h > 0.0 ? fabs(a) / h : HUGE_VAL) + 0.5 / n;
            dB = (h > 0.0 ? fabs(b) / h : HUGE_VAL) + 1.0 / n;
            cancel = h > 0.0 ? (a * a + b * b) / (2.0 * h) : HUGE_VAL;
        } else {
            double u = fabs(a - n);
            h = pow(u, 0.25);
            dA = (u > 0.0 ? 0.25 * h / u : HUGE_VAL) + 0.5 / n;
            dB = 1.0 / n;
            cancel = u > 0.0 ? 0.25 * h / u * (a + n) : HUGE_VAL;
        }
        f = h + (0.5 * a + b) / n + 0.5;
        S = h + (0.5 * a + fabs(b)) / n + 0.5 + cancel + dA * a + dB * bb;
        for (int k = 0; k < n; ++k) {
            double x = z[k] - 1.0;
            S += (dA * 2.0 * fabs(x) + dB) * (E(k) + fabs(x));
        }
        break;
    }
    case G_SCHAFFER_F6:
        /* expanded: sum over the cyclic pairs (z_i, z_{i+1}), (z_n, z_1) */
        for (int k = 0; k < n; ++k) {
            int k1 = (k + 1) % n;
            f += schaffer_pair(z[k], z[k1], &S, E(k), E(k1));
        }
        break;
    case G_KATSUURA: {
        /* (10 / n^2) prod_i (1 + i sum_{j=1}^{32} |2^j z_i - round(2^j z_i)| / 2^j)^(10 / n^1.2) - 10 / n^2 */
        const double ex = 10.0 / pow((double)n, 1.2), c = 10.0 / ((double)n * n);
        double P = 1.0, sens = 0.0;
        for (int k = 0; k < n; ++k) {
            double s = 0.0, p2 = 1.0;
            for (int j = 1; j <= 32; ++j) {
                p2 *= 2.0;
                double v = p2 * z[k];
                s += fabs(v - round(v)) / p2;
            }
            double base = 1.0 + (k + 1) * s;
            P *= pow(base, ex);
            /* each of the 32 sawtooth terms has slope +-1 in z */
            sens += ex * (k + 1) / base * (32.0 * (E(k) + fabs(z[k])) + s);
        }
        f = c * P - c;
        S = c * (P + 1.0) + c * P * sens;
        break;
    }
    case G_GRIEWANK_ROSENBROCK:
        /* expanded: sum of Griewank's 1-D term of Rosenbrock's 2-D term over the
           cyclic pairs, at t = z + 1 */
        for (int k = 0; k < n; ++k) {
            int k1 = (k + 1) % n;
            f += griewank_rosenbrock_pair(z[k], z[k1], E(k), E(k1), &S);
        }
        break;
    case G_ELLIPTIC:
        /* sum (10^6)^((i-1)/(n-1)) z_i^2 */
        for (int k = 0; k < n; ++k) {
            double ck = n > 1 ? pow(1e6, (double)k / (double)(n - 1)) : 1.0;
            f += ck * z[k] * z[k];
            S += 2.0 * ck * fabs(z[k]) * E(k);
        }
        S += f;
        break;
    case G_GRIEWANK: {
        /* sum z_i^2 / 4000 - prod cos(z_i / sqrt(i)) + 1 */
        double s = 0.0, P = 1.0;
        for (int k = 0; k < n; ++k) {
            s += z[k] * z[k] / 4000.0;
            P *= cos(z[k] / sqrt((double)(k + 1)));
            S += (fabs(z[k]) / 2000.0 + 1.0 / sqrt((double)(k + 1))) * (E(k) + fabs(z[k]));
        }
        f = s - P + 1.0;
        S += s + fabs(P) + 1.0;
        break;
    }
    default:
        f = NAN;
        S = NAN;
    }
#undef E
    if (sabs) *sabs = S;
    return f;
}

/* ------------------------------------------------------------------------- */
/* Suite tables (Table 2).                                                    */
/* ------------------------------------------------------------------------- */

/* Search-domain scale of each basic function inside a hybrid or composition
   function: [-100, 100] is mapped onto the function's customary domain
   (Sec. 7.3.1 says each function scales the range, without the factors; the
   factors of the CEC'14/'17 definitions are taken). */
double or_domain_scale(int fn)
{
    switch (fn) {
    case G_RASTRIGIN: return 5.12 / 100.0;
    case G_ROSENBROCK: return 2.048 / 100.0;
    case G_SCHWEFEL: return 1000.0 / 100.0;
    case G_GRIEWANK: return 600.0 / 100.0;
    case G_HGBAT:
    case G_HAPPYCAT:
    case G_KATSUURA:
    case G_GRIEWANK_ROSENBROCK: return 5.0 / 100.0;
    default: return 1.0;
    }
}

typedef struct {
    int n;           /* number of basic functions */
    int fn[5];
    int pct[5];      /* hybrid: share of the coordinates, percent */
    double sigma[5]; /* composition */
    double lambda[5];
    double bias[5];
} suite_spec;

static int suite_get(int obj, suite_spec* s)
{
    memset(s, 0, sizeof *s);
    switch (obj) {
    case G_HYBRID1: /* Bent Cigar, HGBat, Rastrigin; p = [0.3, 0.3, 0.4] */
        *s = (suite_spec){3, {G_BENT_CIGAR, G_HGBAT, G_RASTRIGIN}, {30, 30, 40}, {0}, {0}, {0}};
        return 1;
    case G_HYBRID2: /* Expanded Schaffer F6, HGBat, Rosenbrock, modified Schwefel; p = [0.2, 0.2, 0.3, 0.3] */
        *s = (suite_spec){4, {G_SCHAFFER_F6, G_HGBAT, G_ROSENBROCK, G_SCHWEFEL}, {20, 20, 30, 30}, {0}, {0}, {0}};
        return 1;
    case G_HYBRID3: /* Katsuura, HappyCat, Griewank-Rosenbrock, modified Schwefel, Ackley; p = [0.3, 0.2, 0.2, 0.1, 0.2] */
        *s = (suite_spec){5, {G_KATSUURA, G_HAPPYCAT, G_GRIEWANK_ROSENBROCK, G_SCHWEFEL, G_ACKLEY},
                          {30, 20, 20, 10, 20}, {0}, {0}, {0}};
        return 1;
    case G_COMPOSITION1: /* Rastrigin, Griewank, modified Schwefel */
        *s = (suite_spec){3, {G_RASTRIGIN, G_GRIEWANK, G_SCHWEFEL}, {0}, {10, 20, 30}, {1, 10, 1}, {0, 100, 200}};
        return 2;
    case G_COMPOSITION2: /* Ackley, high-conditioned elliptic, Griewank, Rastrigin */
        *s = (suite_spec){4, {G_ACKLEY, G_ELLIPTIC, G_GRIEWANK, G_RASTRIGIN}, {0}, {10, 20, 30, 40},
                          {10, 1e-6, 10, 1}, {0, 100, 200, 300}};
        return 2;
    case G_COMPOSITION3: /* Expanded Schaffer F6, modified Schwefel, Griewank, Rosenbrock, Rastrigin */
        *s = (suite_spec){5, {G_SCHAFFER_F6, G_SCHWEFEL, G_GRIEWANK, G_ROSENBROCK, G_RASTRIGIN}, {0},
                          {10, 20, 20, 30, 40}, {0.005, 1, 10, 1, 10}, {0, 100, 200, 300, 400}};
        return 2;
    default:
        return 0;
    }
}

/* Hybrid split of d coordinates: the first m - 1 parts take ceil(p_i d)
   coordinates each (integer arithmetic on the percentages), the last the
   rest.  Returns 0 when some part would be empty. */
int or_hybrid_segments(int obj, int d, int32_t* start /* m + 1 */)
{
    suite_spec s;
    if (suite_get(obj, &s) != 1) return 0;
    int used = 0;
    start[0] = 0;
    for (int c = 0; c + 1 < s.n; ++c) {
        int nc = (s.pct[c] * d + 99) / 100;
        used += nc;
        start[c + 1] = used;
    }
    start[s.n] = d;
    for (int c = 0; c < s.n; ++c)
        if (start[c + 1] - start[c] < 1) return 0;
    return s.n;
}

/* Number of (shift, rotation) pairs the objective takes: the composition
   functions one per basic function, everything else one. */
int or_suite_components(int obj)
{
    suite_spec s;
    return suite_get(obj, &s) == 2 ? s.n : 1;
}

/* z = M y (M row-major d x d, NULL = identity) and G_j = sum_k |M_jk y_k| */
static void rotate(int d, const double* M, const double* y, double* z, double* G)
{
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
}

/* One objective of the suite at x (obj 5..20; 0..3 are handled here too
   when they appear inside hybrid and composition functions).
   basic (5..14):  g(M ((x - o) scale))
   hybrid:         z = M ((x - o) scale), permuted, split into parts; part c
                   is scaled by its function's domain scale and evaluated by
                   that function as an n_c-dimensional function (Sec. 7.3.2:
                   one shift, one rotation, one permutation)
   composition:    sum_i omega_i (lambda_i g_i(M_i ((x - o_i) s_i)) + bias_i),
                   s_i the domain scale of g_i; omega_i = w_i / sum_k w_k with
                   w_i = exp(-D_i / (2 d sigma_i^2)) / sqrt(D_i),
                   D_i = sum_j (x_j - o_ij)^2 (Sec. 7.3.3).  The weights are
                   normalised in logarithms (ln w_i = -ln(D_i)/2 - D_i/(2 d
                   sigma_i^2), then exp(ln w_i - max_k ln w_k) / sum), the
                   same numbers without underflow; at x = o_i (D_i = 0,
                   w_i infinite) omega is 1 for the first such i.
   o: d values (composition: n x d), M: d x d (composition: n x d x d), both
   may be NULL; perm: d indices (hybrid), NULL = identity. */
double or_suite_objective(int obj, int d, const double* o, const double* M, double scale, const int32_t* perm,
                          const double* x, double* sabs)
{
    suite_spec s;
    int kind = suite_get(obj, &s);
    double* y = (double*)malloc(sizeof(double) * (size_t)d);
    double* z = (double*)malloc(sizeof(double) * (size_t)d);
    double* G = (double*)malloc(sizeof(double) * (size_t)d);
    double* w = (double*)malloc(sizeof(double) * (size_t)d);
    double* e = (double*)malloc(sizeof(double) * (size_t)d);
    double f = 0.0, S = 0.0;
    if (kind == 0) {
        for (int k = 0; k < d; ++k) y[k] = (x[k] - (o ? o[k] : 0.0)) * scale;
        rotate(d, M, y, z, G);
        for (int k = 0; k < d; ++k) e[k] = G[k] + fabs(z[k]);
        f = or_basic(obj, d, z, e, &S);
    } else if (kind == 1) {
        int32_t start[6];
        if (or_hybrid_segments(obj, d, start) != s.n) {
            f = NAN;
            S = NAN;
        } else {
            for (int k = 0; k < d; ++k) y[k] = (x[k] - (o ? o[k] : 0.0)) * scale;
            rotate(d, M, y, z, G);
            for (int c = 0; c < s.n; ++c) {
                double sc = or_domain_scale(s.fn[c]), Sc;
                int nc = start[c + 1] - start[c];
                for (int l = 0; l < nc; ++l) {
                    int src = perm ? perm[start[c] + l] : start[c] + l;
                    w[l] = sc * z[src];
                    e[l] = sc * (G[src] + fabs(z[src])) + fabs(w[l]);
                }
                f += or_basic(s.fn[c], nc, w, e, &Sc);
                S += Sc;
            }
        }
    } else {
        double g[5], Sg[5], D[5], lw[5], om[5];
        int hit = -1;
        for (int c = 0; c < s.n; ++c) {
            const double* oc = o ? o + (size_t)c * d : NULL;
            const double* Mc = M ? M + (size_t)c * d * d : NULL;
            double sc = or_domain_scale(s.fn[c]);
            D[c] = 0.0;
            for (int k = 0; k < d; ++k) {
                double diff = x[k] - (oc ? oc[k] : 0.0);
                D[c] += diff * diff;
                y[k] = diff * sc;
            }
            rotate(d, Mc, y, z, G);
            for (int k = 0; k < d; ++k) e[k] = G[k] + fabs(z[k]);
            g[c] = or_basic(s.fn[c], d, z, e, &Sg[c]);
            if (D[c] == 0.0 && hit < 0) hit = c;
        }
        if (hit >= 0) {
            for (int c = 0; c < s.n; ++c) om[c] = c == hit ? 1.0 : 0.0;
        } else {
            double m = -HUGE_VAL, sum = 0.0;
            for (int c = 0; c < s.n; ++c) {
                lw[c] = -0.5 * log(D[c]) - D[c] / (2.0 * d * s.sigma[c] * s.sigma[c]);
                if (lw[c] > m) m = lw[c];
            }
            for (int c = 0; c < s.n; ++c) {
                om[c] = exp(lw[c] - m);
                sum += om[c];
            }
            for (int c = 0; c < s.n; ++c) om[c] /= sum;
        }
        for (int c = 0; c < s.n; ++c) f += om[c] * (s.lambda[c] * g[c] + s.bias[c]);
        for (int c = 0; c < s.n; ++c) {
            double v = s.lambda[c] * g[c] + s.bias[c];
            double L = hit >= 0 ? 0.0 : D[c] / (2.0 * d * s.sigma[c] * s.sigma[c]) + 0.5 * fabs(log(D[c])) + 1.0;
            S += om[c] * (s.lambda[c] * (Sg[c] + fabs(g[c])) + s.bias[c]) + 2.0 * om[c] * fabs(v - f) * L;
        }
    }
    free(y);
    free(z);
    free(G);
    free(w);
    free(e);
    if (sabs) *sabs = S;
    return f;
}
