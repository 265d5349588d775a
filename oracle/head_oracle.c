/*
 * head_oracle.c -- FP64 reference of SplatAD's per-ray lidar decoder (Sec. 3.3: the
 * rendered features concatenated with the ray direction are decoded to intensity and
 * ray-drop probability by a small MLP; App. B: lightweight, two hidden layers; loss terms
 * lambda_intens L2(intensity) and lambda_raydrop BCE(ray drop), Eq. loss_fn, App. B
 * weights 1.0 and 0.1).  TEST INFRASTRUCTURE ONLY (tests, smoke, benchmark baseline).
 *
 * Network: x[32] -> relu(W1^T x + b1)[64] -> relu(W2^T h1 + b2)[64] -> W3^T h2 + b3 [2]
 * with out[0] the intensity logit (intensity = sigmoid) and out[1] the drop logit.
 * Weights are given already rounded to BF16 (the library stores them in BF16); every
 * product and sum here is FP64.  Row-major W1[32][64], W2[64][64], W3[64][2].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HI 32
#define HH 64
#define HO 2

static double relu(double v) { return v > 0 ? v : 0; }
static double sigmoid(double v) { return 1.0 / (1.0 + exp(-v)); }

static void head_one(const double *x, const double *W1, const double *b1, const double *W2, const double *b2,
                     const double *W3, const double *b3, double *h1, double *h2, double *o) {
    for (int j = 0; j < HH; j++) {
        double s = b1[j];
        for (int i = 0; i < HI; i++) s += x[i] * W1[i * HH + j];
        h1[j] = relu(s);
    }
    for (int j = 0; j < HH; j++) {
        double s = b2[j];
        for (int i = 0; i < HH; i++) s += h1[i] * W2[i * HH + j];
        h2[j] = relu(s);
    }
    for (int k = 0; k < HO; k++) {
        double s = b3[k];
        for (int i = 0; i < HH; i++) s += h2[i] * W3[i * HO + k];
        o[k] = s;
    }
}

/* Public: raw outputs (intensity logit, drop logit) for R rays. */
int head_forward(int64_t R, const double *x, const double *W1, const double *b1, const double *W2, const double *b2,
                 const double *W3, const double *b3, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < R; r++) {
        double h1[HH], h2[HH];
        head_one(x + HI * r, W1, b1, W2, b2, W3, b3, h1, h2, out + HO * r);
    }
    return 0;
}

/* Public: loss = lam_i * mean_r (sigmoid(o0) - y_int)^2 + lam_d * mean_r BCE(o1, y_drop)
 * and its gradients (accumulated, +=) with respect to the weights, biases and, if gx is
 * not NULL, the inputs.  Returns the loss. */
double head_loss_backward(int64_t R, const double *x, const double *W1, const double *b1, const double *W2,
                          const double *b2, const double *W3, const double *b3, const double *y_int,
                          const double *y_drop, double lam_i, double lam_d, double *gW1, double *gb1, double *gW2,
                          double *gb2, double *gW3, double *gb3, double *gx) {
    double loss = 0;
    for (int64_t r = 0; r < R; r++) {
        double h1[HH], h2[HH], o[HO];
        const double *xr = x + HI * r;
        head_one(xr, W1, b1, W2, b2, W3, b3, h1, h2, o);
        const double s = sigmoid(o[0]);
        const double e = s - y_int[r];
        /* BCE with logits, written stably */
        const double z = o[1], y = y_drop[r];
        const double bce = (z > 0 ? z : 0) - z * y + log1p(exp(-fabs(z)));
        loss += lam_i * e * e / R + lam_d * bce / R;
        double dO[HO];
        dO[0] = lam_i * 2.0 * e * s * (1.0 - s) / R;
        dO[1] = lam_d * (sigmoid(z) - y) / R;
        double dh2[HH], dh1[HH];
        for (int k = 0; k < HO; k++) gb3[k] += dO[k];
        for (int i = 0; i < HH; i++) {
            double s2 = 0;
            for (int k = 0; k < HO; k++) {
                gW3[i * HO + k] += h2[i] * dO[k];
                s2 += W3[i * HO + k] * dO[k];
            }
            dh2[i] = h2[i] > 0 ? s2 : 0;
        }
        for (int j = 0; j < HH; j++) gb2[j] += dh2[j];
        for (int i = 0; i < HH; i++) {
            double s1 = 0;
            for (int j = 0; j < HH; j++) {
                gW2[i * HH + j] += h1[i] * dh2[j];
                s1 += W2[i * HH + j] * dh2[j];
            }
            dh1[i] = h1[i] > 0 ? s1 : 0;
        }
        for (int j = 0; j < HH; j++) gb1[j] += dh1[j];
        for (int i = 0; i < HI; i++) {
            double s0 = 0;
            for (int j = 0; j < HH; j++) {
                gW1[i * HH + j] += xr[i] * dh1[j];
                s0 += W1[i * HH + j] * dh1[j];
            }
            if (gx) gx[HI * r + i] += s0;
        }
    }
    return loss;
}

/* Public: one Adam step (Kingma & Ba, with bias correction; epsilon added to the square
 * root of the corrected second moment) on n parameters; step counts from 1. */
int head_adam(int64_t n, double *p, const double *g, double *m, double *v, double lr, double beta1, double beta2,
              double eps, int64_t step) {
    const double c1 = 1.0 - pow(beta1, (double)step), c2 = 1.0 - pow(beta2, (double)step);
    for (int64_t i = 0; i < n; i++) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        const double mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
    return 0;
}
