/*
 * Oracle (test infrastructure only): the learned temperature surrogate.
 *
 * The paper has no surrogate; this is the plain FP64 reference for the learned form
 * of the per-node temperature solve: a 7 -> 64 -> 64 -> 1 perceptron with the tanh
 * form of GELU, gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))
 * (Hendrycks & Gimpel), mean-squared-error loss, back-propagation written out layer
 * by layer, and the Adam update (Kingma & Ba) with bias correction.
 * Parameter vector layout: W1[64][7], b1[64], W2[64][64], b2[64], w3[64], b3.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define NI 7
#define NH 64
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + NH * NI)
#define OFF_W2 (OFF_B1 + NH)
#define OFF_B2 (OFF_W2 + NH * NH)
#define OFF_W3 (OFF_B2 + NH)
#define OFF_B3 (OFF_W3 + NH)
#define NPARAM (OFF_B3 + 1)

int or_mlp_nparams(void) { return NPARAM; }

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

/* one sample: pre-activations a1, a2 and activations h1, h2; returns the output */
static double forward1(const double* p, const double* x, double* a1, double* h1, double* a2,
                       double* h2) {
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
  double y = p[OFF_B3];
  for (int i = 0; i < NH; ++i) y += p[OFF_W3 + i] * h2[i];
  return y;
}

void or_mlp_forward(const double* p, int n, const double* X, double* y) {
  double a1[NH], h1[NH], a2[NH], h2[NH];
  for (int s = 0; s < n; ++s) y[s] = forward1(p, X + (size_t)s * NI, a1, h1, a2, h2);
}

/* loss = (1/n) sum (y - t)^2 and its gradient with respect to every parameter */
double or_mlp_loss_grad(const double* p, int n, const double* X, const double* t, double* g) {
  double a1[NH], h1[NH], a2[NH], h2[NH], d2[NH], d1[NH];
  memset(g, 0, sizeof(double) * NPARAM);
  double loss = 0.0;
  for (int s = 0; s < n; ++s) {
    const double* x = X + (size_t)s * NI;
    double y = forward1(p, x, a1, h1, a2, h2);
    double r = y - t[s];
    loss += r * r;
    double dy = 2.0 * r / n;
    g[OFF_B3] += dy;
    for (int i = 0; i < NH; ++i) {
      g[OFF_W3 + i] += dy * h2[i];
      d2[i] = dy * p[OFF_W3 + i] * or_gelu_d(a2[i]);
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
  return loss / n;
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
