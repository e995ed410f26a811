/*
 * de_oracle_ode.c -- plain FP64 CPU oracle of the ODE parameter-fitting
 * objective (the expensive objective of the surrogate-assisted workload).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  The
 * product path never links it and shares no code with it.
 *
 * The paper motivates GPU DE with objectives whose evaluation dominates the
 * run time (Abstract) but defines no such problem.  This objective is a
 * reading, not the paper's:
 *   - ten unit masses in a chain, positions q_i and momenta p_i;
 *   - spring constants k_i to ground and dampers c_i on every mass;
 *   - neighbouring masses joined by springs of stiffness kappa = 1;
 *   - both chain ends tied to fixed walls (q_0 = q_11 = 0);
 *   - equations of motion: dq_i/dt = p_i,
 *         dp_i/dt = -k_i q_i - c_i p_i - kappa (2 q_i - q_{i-1} - q_{i+1});
 *   - parameters from x in [-100, 100]^20 by affine maps:
 *         k_i = 0.5 + 4.5 u_i and c_i = 0.01 + 0.49 u_{10+i},
 *         where u = (x + 100) / 200;
 *   - start q(0) = e_1, p(0) = 0;
 *   - classical fourth-order Runge-Kutta, step dt = 1e-3, 2000 steps;
 *   - observation: all ten positions after every step;
 *   - f(x) = mean over the 2000 x 10 observations of (q - q_hat)^2, where
 *     q_hat is the trajectory of the hidden parameter vector x_hat, so that
 *     f(x_hat) = 0.
 *
 * Order of operations (IEEE binary64, round to nearest; the only fused
 * multiply-adds are the explicit fma() calls: build with -ffp-contract=off):
 *   a(q, p) = fma(-c, p, fma(-(k + 2), q, q_left + q_right)),
 *     the same force as above with the two neighbour springs gathered;
 *   stage points fma(dt/2, kq, q) and fma(dt/2, kp, p), then with dt;
 *   update fma(dt/6, (k1 + k4) + ((k2 + k3) + (k2 + k3)), q), the same for p.
 * Any correct RK4 in another order differs from this one by rounding only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_ODE_N 10

/* Parameters (k, c) of the chain from a parameter vector x of length 20. */
void or_ode_params(const double* x, double* k, double* c)
{
    for (int i = 0; i < OR_ODE_N; ++i) {
        double uk = (x[i] + 100.0) / 200.0;
        double uc = (x[OR_ODE_N + i] + 100.0) / 200.0;
        k[i] = 0.5 + 4.5 * uk;
        c[i] = 0.01 + 0.49 * uc;
    }
}

/* Accelerations of the chain at (q, p): -k_i q_i - c_i p_i - (2 q_i - q_{i-1}
 * - q_{i+1}), gathered as (q_{i-1} + q_{i+1}) - (k_i + 2) q_i - c_i p_i. */
static void or_ode_accel(const double* k, const double* c, const double* q, const double* p, double* a)
{
    for (int i = 0; i < OR_ODE_N; ++i) {
        double ql = i > 0 ? q[i - 1] : 0.0;
        double qr = i + 1 < OR_ODE_N ? q[i + 1] : 0.0;
        double w = fma(-(k[i] + 2.0), q[i], ql + qr);
        a[i] = fma(-c[i], p[i], w);
    }
}

/* Trajectory of the chain with raw parameters k, c from q(0) = e_1, p(0) = 0:
 * out[s * 10 + i] = q_i after step s + 1, for s < steps. */
void or_ode_integrate(const double* k, const double* c, int steps, double dt, double* out)
{
    double q[OR_ODE_N], p[OR_ODE_N];
    double k1q[OR_ODE_N], k1p[OR_ODE_N], k2q[OR_ODE_N], k2p[OR_ODE_N];
    double k3q[OR_ODE_N], k3p[OR_ODE_N], k4q[OR_ODE_N], k4p[OR_ODE_N];
    double qs[OR_ODE_N], ps[OR_ODE_N];
    const double h = dt, hh = dt * 0.5, h6 = dt / 6.0;
    for (int i = 0; i < OR_ODE_N; ++i) {
        q[i] = i == 0 ? 1.0 : 0.0;
        p[i] = 0.0;
    }
    for (int s = 0; s < steps; ++s) {
        /* stage 1 at (q, p) */
        for (int i = 0; i < OR_ODE_N; ++i) k1q[i] = p[i];
        or_ode_accel(k, c, q, p, k1p);
        /* stage 2 at the half step along stage 1 */
        for (int i = 0; i < OR_ODE_N; ++i) {
            qs[i] = fma(hh, k1q[i], q[i]);
            ps[i] = fma(hh, k1p[i], p[i]);
            k2q[i] = ps[i];
        }
        or_ode_accel(k, c, qs, ps, k2p);
        /* stage 3 at the half step along stage 2 */
        for (int i = 0; i < OR_ODE_N; ++i) {
            qs[i] = fma(hh, k2q[i], q[i]);
            ps[i] = fma(hh, k2p[i], p[i]);
            k3q[i] = ps[i];
        }
        or_ode_accel(k, c, qs, ps, k3p);
        /* stage 4 at the full step along stage 3 */
        for (int i = 0; i < OR_ODE_N; ++i) {
            qs[i] = fma(h, k3q[i], q[i]);
            ps[i] = fma(h, k3p[i], p[i]);
            k4q[i] = ps[i];
        }
        or_ode_accel(k, c, qs, ps, k4p);
        /* weighted update (1, 2, 2, 1) / 6 */
        for (int i = 0; i < OR_ODE_N; ++i) {
            double mq = k2q[i] + k3q[i], mp = k2p[i] + k3p[i];
            q[i] = fma(h6, (k1q[i] + k4q[i]) + (mq + mq), q[i]);
            p[i] = fma(h6, (k1p[i] + k4p[i]) + (mp + mp), p[i]);
            out[(size_t)s * OR_ODE_N + i] = q[i];
        }
    }
}

/* Trajectory of the parameter vector x (2000 steps of 1e-3 in the objective;
 * other step counts and sizes serve the order tests). */
void or_ode_trajectory(const double* x, int steps, double dt, double* out)
{
    double k[OR_ODE_N], c[OR_ODE_N];
    or_ode_params(x, k, c);
    or_ode_integrate(k, c, steps, dt, out);
}

/* f(x) = mean squared difference between the trajectories of x and x_hat,
 * both integrated here with `steps` steps of size dt.  *sabs (if not NULL)
 * receives the tolerance scale: f plus the mean of 2 |q - q_hat| (|q| +
 * |q_hat|), the first-order effect of relative rounding in either trajectory. */
double or_ode_objective_s(const double* x, const double* x_hat, int steps, double dt, double* sabs)
{
    double* a = (double*)malloc(sizeof(double) * (size_t)steps * OR_ODE_N);
    double* b = (double*)malloc(sizeof(double) * (size_t)steps * OR_ODE_N);
    or_ode_trajectory(x, steps, dt, a);
    or_ode_trajectory(x_hat, steps, dt, b);
    double sum = 0.0, mag = 0.0;
    for (size_t e = 0; e < (size_t)steps * OR_ODE_N; ++e) {
        double r = a[e] - b[e];
        sum += r * r;
        mag += 2.0 * fabs(r) * (fabs(a[e]) + fabs(b[e]));
    }
    free(a);
    free(b);
    const double n = (double)steps * OR_ODE_N;
    if (sabs) *sabs = sum / n + mag / n;
    return sum / n;
}

double or_ode_objective(const double* x, const double* x_hat, int steps, double dt)
{
    return or_ode_objective_s(x, x_hat, steps, dt, NULL);
}
