/*
 * de_oracle_mlp.c -- plain FP64 CPU oracle of the surrogate network: a
 * multilayer perceptron nin -> nh -> nh -> 1 with ReLU hidden layers, its
 * mean-squared-error gradient by backpropagation, and the Adam update.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  The
 * product path never links it and shares no code with it.
 *
 * The paper has no surrogate: this part serves the surrogate-assisted
 * workload (screening several candidate trials per target on costly
 * objectives, which the paper's Abstract motivates).  Definitions:
 *   h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  y = w3 . h2 + b3,
 *   loss = (1/B) sum_b (y_b - t_b)^2,
 *   relu'(0) = 0 (the derivative is taken as 0 at the kink);
 *   Adam (Kingma and Ba, ICLR 2015): m = b1 m + (1 - b1) g,
 *     v = b2 v + (1 - b2) g^2, w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 * Matrices are row-major: W1[j][k] (nh x nin), W2[j][i] (nh x nh).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static double or_relu(double v) { return v > 0.0 ? v : 0.0; }

/* Hidden activations of one input row: h1[nh], h2[nh]; returns y. */
static double or_mlp_row(int nin, int nh, const double* x, const double* W1, const double* b1, const double* W2,
                         const double* b2, const double* w3, double b3, double* h1, double* h2)
{
    for (int j = 0; j < nh; ++j) {
        double s = b1[j];
        for (int k = 0; k < nin; ++k) s += W1[(size_t)j * nin + k] * x[k];
        h1[j] = or_relu(s);
    }
    for (int j = 0; j < nh; ++j) {
        double s = b2[j];
        for (int i = 0; i < nh; ++i) s += W2[(size_t)j * nh + i] * h1[i];
        h2[j] = or_relu(s);
    }
    double y = b3;
    for (int j = 0; j < nh; ++j) y += w3[j] * h2[j];
    return y;
}

/* y[b] for B rows of X (row stride nin). */
void or_mlp_forward(int B, int nin, int nh, const double* X, const double* W1, const double* b1, const double* W2,
                    const double* b2, const double* w3, const double* b3, double* y)
{
    double* h1 = (double*)malloc(sizeof(double) * (size_t)nh);
    double* h2 = (double*)malloc(sizeof(double) * (size_t)nh);
    for (int b = 0; b < B; ++b)
        y[b] = or_mlp_row(nin, nh, X + (size_t)b * nin, W1, b1, W2, b2, w3, *b3, h1, h2);
    free(h1);
    free(h2);
}

/* loss = (1/B) sum (y - t)^2 and its gradient with respect to every
 * parameter (same shapes as the parameters; overwritten). */
double or_mlp_loss_grad(int B, int nin, int nh, const double* X, const double* t, const double* W1, const double* b1,
                        const double* W2, const double* b2, const double* w3, const double* b3, double* gW1,
                        double* gb1, double* gW2, double* gb2, double* gw3, double* gb3)
{
    double* h1 = (double*)malloc(sizeof(double) * (size_t)nh);
    double* h2 = (double*)malloc(sizeof(double) * (size_t)nh);
    double* d2 = (double*)malloc(sizeof(double) * (size_t)nh);
    double* d1 = (double*)malloc(sizeof(double) * (size_t)nh);
    memset(gW1, 0, sizeof(double) * (size_t)nh * nin);
    memset(gb1, 0, sizeof(double) * (size_t)nh);
    memset(gW2, 0, sizeof(double) * (size_t)nh * nh);
    memset(gb2, 0, sizeof(double) * (size_t)nh);
    memset(gw3, 0, sizeof(double) * (size_t)nh);
    *gb3 = 0.0;
    double loss = 0.0;
    for (int b = 0; b < B; ++b) {
        const double* x = X + (size_t)b * nin;
        double y = or_mlp_row(nin, nh, x, W1, b1, W2, b2, w3, *b3, h1, h2);
        double r = y - t[b];
        loss += r * r;
        double dy = 2.0 * r / B;              /* d loss / d y_b */
        *gb3 += dy;
        for (int j = 0; j < nh; ++j) {
            gw3[j] += dy * h2[j];
            d2[j] = h2[j] > 0.0 ? dy * w3[j] : 0.0;   /* d loss / d (pre-activation of layer 2) */
        }
        for (int i = 0; i < nh; ++i) {
            double s = 0.0;
            for (int j = 0; j < nh; ++j) s += W2[(size_t)j * nh + i] * d2[j];
            d1[i] = h1[i] > 0.0 ? s : 0.0;              /* d loss / d (pre-activation of layer 1) */
        }
        for (int j = 0; j < nh; ++j) {
            gb2[j] += d2[j];
            for (int i = 0; i < nh; ++i) gW2[(size_t)j * nh + i] += d2[j] * h1[i];
        }
        for (int i = 0; i < nh; ++i) {
            gb1[i] += d1[i];
            for (int k = 0; k < nin; ++k) gW1[(size_t)i * nin + k] += d1[i] * x[k];
        }
    }
    free(h1);
    free(h2);
    free(d2);
    free(d1);
    return loss / B;
}

/* One Adam update of n parameters; `step` counts from 1. */
void or_adam(int n, double* w, const double* g, double* m, double* v, int step, double lr, double beta1,
             double beta2, double eps)
{
    const double c1 = 1.0 - pow(beta1, step), c2 = 1.0 - pow(beta2, step);
    for (int e = 0; e < n; ++e) {
        m[e] = beta1 * m[e] + (1.0 - beta1) * g[e];
        v[e] = beta2 * v[e] + (1.0 - beta2) * g[e] * g[e];
        w[e] -= lr * (m[e] / c1) / (sqrt(v[e] / c2) + eps);
    }
}
