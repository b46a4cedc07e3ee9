/*
 * Oracle (test infrastructure only): the learned surrogates (temperature: one output;
 * chemistry source: ten outputs).
 *
 * The paper has no surrogate; this is the plain FP64 reference for the learned forms of
 * the per-node temperature solve and of the finite-rate source: a 7 -> 64 -> 64 -> n_out
 * perceptron with the tanh form of GELU after both hidden layers,
 * gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) (Hendrycks & Gimpel),
 * mean-squared-error loss averaged over samples and outputs, back-propagation written
 * out layer by layer, and the Adam update (Kingma & Ba) with bias correction.
 * Parameter vector layout: W1[64][7], b1[64], W2[64][64], b2[64], W3[n_out][64],
 * b3[n_out] (n_out = 1: w3[64], b3).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define NI 7
#define NH 64
#define NO_MAX 16
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + NH * NI)
#define OFF_W2 (OFF_B1 + NH)
#define OFF_B2 (OFF_W2 + NH * NH)
#define OFF_W3 (OFF_B2 + NH)
#define OFF_B3(no) (OFF_W3 + (no) * NH)

int or_mlp_nparams_n(int n_out) { return OFF_B3(n_out) + n_out; }
int or_mlp_nparams(void) { return or_mlp_nparams_n(1); }

double or_gelu(double x) {
  const double k = sqrt(2.0 / M_PI);
  return 0.5 * x * (1.0 + tanh(k * (x + 0.044715 * x * x * x)));
}

double or_gelu_d(double x) {
  const double k = sqrt(2.0 / M_PI);
  double z = k * (x + 0.044715 * x * x * x);
  double t = tanh(z);
  double dz = k * (1.0 + 3.0 * 0.044715 * x * x);
  return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * dz;
}

/* one sample: pre-activations a1, a2, activations h1, h2 and the n_out outputs y */
static void forward1(const double* p, int no, const double* x, double* a1, double* h1, double* a2,
                     double* h2, double* y) {
  for (int j = 0; j < NH; ++j) {
    double s = p[OFF_B1 + j];
    for (int i = 0; i < NI; ++i) s += p[OFF_W1 + j * NI + i] * x[i];
    a1[j] = s;
    h1[j] = or_gelu(s);
  }
  for (int j = 0; j < NH; ++j) {
    double s = p[OFF_B2 + j];
    for (int i = 0; i < NH; ++i) s += p[OFF_W2 + j * NH + i] * h1[i];
    a2[j] = s;
    h2[j] = or_gelu(s);
  }
  for (int o = 0; o < no; ++o) {
    double s = p[OFF_B3(no) + o];
    for (int i = 0; i < NH; ++i) s += p[OFF_W3 + o * NH + i] * h2[i];
    y[o] = s;
  }
}

int or_mlp_forward_n(const double* p, int no, int n, const double* X, double* Y) {
  if (no < 1 || no > NO_MAX) return 1;
  double a1[NH], h1[NH], a2[NH], h2[NH];
  for (int s = 0; s < n; ++s) forward1(p, no, X + (size_t)s * NI, a1, h1, a2, h2, Y + (size_t)s * no);
  return 0;
}

void or_mlp_forward(const double* p, int n, const double* X, double* y) { or_mlp_forward_n(p, 1, n, X, y); }

/* First-order statistical model of the error of the network's evaluation on the GPU with
 * BF16 operands (reading R18s of the learned chemistry source).  The GPU rounds the
 * standardised inputs, W1, W2 and the first hidden layer's activations to BF16, accumulates
 * in FP32, evaluates GELU with a tanh approximation of absolute error at most eps_t and the
 * output layer in FP32.  Each rounding is modelled as an independent zero-mean error,
 * uniform within its bound (variance (u |v|)^2 / 3 for a value v rounded with unit
 * roundoff u, eps_t^2 / 3 for the tanh error), and propagated to first order (GELU through
 * its derivative).
 *   u_round: unit roundoff of the BF16 roundings (2^-8 against the exact network; 0 against
 *            a network that rounds exactly where the GPU does);
 *   u_flip:  against such an emulation, a first hidden activation of the GPU (off from the
 *            emulation's by its FP32 sums and tanh) can round to the neighbouring BF16 value,
 *            a rare jump of 2 u_flip |a| that no variance describes: FLIP [n][n_out] (when
 *            not NULL) receives, per output, the largest first-order effect of one such jump
 *            over the 64 hidden units, sum_j |W3_oj| |gelu'(z2_j)| |W2_ji| 2 u_flip |a_i|;
 *   x_rel:   a relative error of the raw inputs (an input state in FP32), in units of |x| + 1.
 * Returns the exact FP64 outputs Y [n][n_out] and the standard deviations SD [n][n_out] of
 * the GPU's difference from the reference under the model. */
int or_mlp_forward_sd_n(const double* p, int no, int n, const double* X, double u, double u_flip,
                        double eps_t, double x_rel, double* Y, double* SD, double* FLIP) {
  if (no < 1 || no > NO_MAX) return 1;
  const double u32 = ldexp(1.0, -23);  /* FP32 accumulation, one rounding per addition */
  const double third = 1.0 / 3.0;
  double a1[NH], h1[NH], a2[NH], h2[NH];
  double vx[NI], va1[NH], va2[NH];
  for (int s = 0; s < n; ++s) {
    const double* x = X + (size_t)s * NI;
    double* y = Y + (size_t)s * no;
    double* sd = SD + (size_t)s * no;
    forward1(p, no, x, a1, h1, a2, h2, y);
    for (int i = 0; i < NI; ++i) {
      const double r = u * fabs(x[i]), q = x_rel * (fabs(x[i]) + 1.0);
      vx[i] = third * (r * r + q * q);
    }
    /* layer 1: rounded inputs and weights, FP32 sum of 7 products and the bias */
    for (int j = 0; j < NH; ++j) {
      double v = 0.0, mag = fabs(p[OFF_B1 + j]);
      for (int i = 0; i < NI; ++i) {
        const double w = p[OFF_W1 + j * NI + i];
        v += w * w * vx[i] + third * (u * w * x[i]) * (u * w * x[i]);
        mag += fabs(w * x[i]);
      }
      v += third * (NI + 1) * (u32 * mag) * (u32 * mag);
      const double g = or_gelu_d(a1[j]), t = 0.5 * a1[j] * eps_t;
      /* GELU (derivative, tanh approximation, a few FP32 operations), then BF16 rounding */
      const double vg = g * g * v + third * t * t + third * 4.0 * (u32 * h1[j]) * (u32 * h1[j]);
      va1[j] = vg + third * (u * h1[j]) * (u * h1[j]);
    }
    /* layer 2: rounded activations and weights, FP32 sum of 64 products and the bias */
    for (int j = 0; j < NH; ++j) {
      double v = 0.0, mag = fabs(p[OFF_B2 + j]);
      for (int i = 0; i < NH; ++i) {
        const double w = p[OFF_W2 + j * NH + i];
        v += w * w * va1[i] + third * (u * w * h1[i]) * (u * w * h1[i]);
        mag += fabs(w * h1[i]);
      }
      v += third * (NH + 1) * (u32 * mag) * (u32 * mag);
      const double g = or_gelu_d(a2[j]), t = 0.5 * a2[j] * eps_t;
      va2[j] = g * g * v + third * t * t + third * 4.0 * (u32 * h2[j]) * (u32 * h2[j]);
    }
    /* output layer in FP32 with FP32 weights */
    for (int o = 0; o < no; ++o) {
      double v = 0.0, mag = fabs(p[OFF_B3(no) + o]);
      for (int i = 0; i < NH; ++i) {
        const double w = p[OFF_W3 + o * NH + i];
        v += w * w * va2[i];
        mag += fabs(w * h2[i]);
      }
      v += third * (NH + 1) * (u32 * mag) * (u32 * mag);
      sd[o] = sqrt(v);
    }
    if (FLIP && u_flip > 0.0) {
      double gd2[NH];
      for (int j = 0; j < NH; ++j) gd2[j] = fabs(or_gelu_d(a2[j]));
      for (int o = 0; o < no; ++o) {
        double worst = 0.0;
        for (int i = 0; i < NH; ++i) {
          double e = 0.0;
          for (int j = 0; j < NH; ++j)
            e += fabs(p[OFF_W3 + o * NH + j]) * gd2[j] * fabs(p[OFF_W2 + j * NH + i]);
          e *= 2.0 * u_flip * fabs(h1[i]);
          if (e > worst) worst = e;
        }
        FLIP[(size_t)s * no + o] = worst;
      }
    } else if (FLIP) {
      for (int o = 0; o < no; ++o) FLIP[(size_t)s * no + o] = 0.0;
    }
  }
  return 0;
}

/* loss = (1/(n n_out)) sum_s sum_o (y_so - t_so)^2 and its gradient with respect to every
 * parameter; returns the loss (negative on invalid n_out) */
double or_mlp_loss_grad_n(const double* p, int no, int n, const double* X, const double* t, double* g) {
  if (no < 1 || no > NO_MAX) return -1.0;
  double a1[NH], h1[NH], a2[NH], h2[NH], d2[NH], d1[NH], y[NO_MAX], dy[NO_MAX];
  memset(g, 0, sizeof(double) * or_mlp_nparams_n(no));
  double loss = 0.0;
  const double scale = 1.0 / ((double)n * no);
  for (int s = 0; s < n; ++s) {
    const double* x = X + (size_t)s * NI;
    forward1(p, no, x, a1, h1, a2, h2, y);
    for (int o = 0; o < no; ++o) {
      double r = y[o] - t[(size_t)s * no + o];
      loss += r * r;
      dy[o] = 2.0 * r * scale;
      g[OFF_B3(no) + o] += dy[o];
      for (int i = 0; i < NH; ++i) g[OFF_W3 + o * NH + i] += dy[o] * h2[i];
    }
    for (int i = 0; i < NH; ++i) {
      double back = 0.0;
      for (int o = 0; o < no; ++o) back += dy[o] * p[OFF_W3 + o * NH + i];
      d2[i] = back * or_gelu_d(a2[i]);
    }
    for (int j = 0; j < NH; ++j) {
      g[OFF_B2 + j] += d2[j];
      for (int i = 0; i < NH; ++i) g[OFF_W2 + j * NH + i] += d2[j] * h1[i];
    }
    for (int i = 0; i < NH; ++i) {
      double s2 = 0.0;
      for (int j = 0; j < NH; ++j) s2 += p[OFF_W2 + j * NH + i] * d2[j];
      d1[i] = s2 * or_gelu_d(a1[i]);
    }
    for (int j = 0; j < NH; ++j) {
      g[OFF_B1 + j] += d1[j];
      for (int i = 0; i < NI; ++i) g[OFF_W1 + j * NI + i] += d1[j] * x[i];
    }
  }
  return loss * scale;
}

double or_mlp_loss_grad(const double* p, int n, const double* X, const double* t, double* g) {
  return or_mlp_loss_grad_n(p, 1, n, X, t, g);
}

/* Adam with bias correction; step counts from 1 */
void or_adam_step(double* p, double* m, double* v, const double* g, int np_, int step, double lr,
                  double b1, double b2, double eps) {
  const double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
  for (int i = 0; i < np_; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}
