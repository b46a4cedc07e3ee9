// One-dimensional LGL collocation basis for the library (host side, set-up only).
//
// The paper collocates on Gauss-Lobatto-Legendre nodes (Eqs. lagrange_3d, lag)
// with D_jn = l_n'(X_j).  Construction used here:
//   nodes   : the N+1 zeros of q(x) = P_{N+1}(x) - P_{N-1}(x), proportional to
//             (1 - x^2) P_N'(x); Newton with q'(x) = (2N+1) P_N(x), started from
//             the Chebyshev extrema;
//   weights : w_i = 2 / (N (N+1) P_N(x_i)^2);
//   D       : the closed form for LGL collocation,
//             D_ij = P_N(x_i) / (P_N(x_j) (x_i - x_j))  (i != j),
//             D_00 = -N(N+1)/4, D_NN = N(N+1)/4, other diagonal entries 0;
//   modes   : orthonormal Legendre p_j = sqrt((2j+1)/2) P_j; the nodal-to-modal
//             map is the LGL quadrature projection, whose norm for the top mode
//             is (2N+1)/N instead of 1.
#include <math.h>
#include "dg_internal.h"

static double legendre(int n, double x) {
  if (n == 0) return 1.0;
  double pm = 1.0, p = x;
  for (int k = 1; k < n; ++k) {
    double pn = ((2 * k + 1) * x * p - k * pm) / (k + 1);
    pm = p;
    p = pn;
  }
  return p;
}

int dg_host_basis(int N, DgHostBasis* b) {
  if (N < 1 || N > DG_MAXN) return 1;
  b->N = N;
  const int n1 = N + 1;
  for (int i = 0; i < n1; ++i) {
    double x = -cos(M_PI * i / N);
    if (i > 0 && i < N) {
      for (int it = 0; it < 200; ++it) {
        double q = legendre(N + 1, x) - legendre(N - 1, x);
        double dq = (2 * N + 1) * legendre(N, x);
        double dx = q / dq;
        x -= dx;
        if (fabs(dx) < 1e-17) break;
      }
    }
    b->x[i] = x;
  }
  // enforce exact antisymmetry of the node set
  for (int i = 0; i < n1 / 2; ++i) {
    double a = 0.5 * (b->x[N - i] - b->x[i]);
    b->x[i] = -a;
    b->x[N - i] = a;
  }
  if (N % 2 == 0) b->x[N / 2] = 0.0;
  double PN[DG_MAXN + 1];
  for (int i = 0; i < n1; ++i) {
    PN[i] = legendre(N, b->x[i]);
    b->w[i] = 2.0 / (N * (N + 1.0) * PN[i] * PN[i]);
  }
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n1; ++j) {
      double v;
      if (i != j) v = PN[i] / (PN[j] * (b->x[i] - b->x[j]));
      else if (i == 0) v = -N * (N + 1.0) / 4.0;
      else if (i == N) v = N * (N + 1.0) / 4.0;
      else v = 0.0;
      b->D[i * n1 + j] = v;
    }
  for (int j = 0; j < n1; ++j) {
    double norm = (j < N) ? 1.0 : (2.0 * N + 1.0) / N;
    for (int i = 0; i < n1; ++i) {
      double pj = sqrt((2.0 * j + 1.0) / 2.0) * legendre(j, b->x[i]);
      b->Vinv[j * n1 + i] = b->w[i] * pj / norm;
    }
  }
  return 0;
}
