/*
 * Oracle (test infrastructure only): one-dimensional LGL basis.
 *
 * The paper collocates on Gauss-Lobatto-Legendre points with Lagrange
 * polynomials (Eqs. lagrange_3d, lag) and defines D_jn = dl_n(X_j)/dX
 * (text after Eq. fluxes_discrete_strong).  Readings:
 *   nodes  = -1, +1 and the roots of P_N' in between (Newton on P_N'),
 *   weights w_i = 2 / (N (N+1) P_N(x_i)^2),
 *   D_ij   = l_j'(x_i) from barycentric weights,
 *   modal basis for the shock indicator = orthonormal Legendre polynomials.
 */
#include <math.h>
#include <string.h>
#include <stdlib.h>
#include "oracle.h"

/* P_n(x) and P_n'(x) by the three-term recurrence. */
void or_legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    double d2 = d0 + (2.0 * k + 1.0) * p1;   /* P'_{k+1} = P'_{k-1} + (2k+1) P_k */
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1; *dP = d1;
}

int or_lgl(int N, double* x, double* w) {
  if (N < 1 || N > OR_MAX_N) return 1;
  x[0] = -1.0; x[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double xi = -cos(M_PI * i / N);  /* Chebyshev-Gauss-Lobatto start */
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      or_legendre(N, xi, &P, &dP);
      /* Legendre ODE: (1-x^2) P'' = 2x P' - N(N+1) P */
      double d2P = (2.0 * xi * dP - N * (N + 1.0) * P) / (1.0 - xi * xi);
      double dx = dP / d2P;
      xi -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    x[i] = xi;
  }
  /* exact symmetry about 0 */
  for (int i = 0; i <= N / 2; ++i) {
    double s = 0.5 * (x[N - i] - x[i]);
    x[i] = -s; x[N - i] = s;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  for (int i = 0; i <= N; ++i) {
    double P, dP;
    or_legendre(N, x[i], &P, &dP);
    w[i] = 2.0 / (N * (N + 1.0) * P * P);
  }
  return 0;
}

void or_dmat(int N, const double* x, double* D) {
  double lam[OR_MAX_N + 1];
  for (int j = 0; j <= N; ++j) {
    double p = 1.0;
    for (int k = 0; k <= N; ++k)
      if (k != j) p *= (x[j] - x[k]);
    lam[j] = 1.0 / p;
  }
  for (int i = 0; i <= N; ++i) {
    double s = 0.0;
    for (int j = 0; j <= N; ++j) {
      if (j == i) continue;
      D[i * (N + 1) + j] = (lam[j] / lam[i]) / (x[i] - x[j]);
      s += D[i * (N + 1) + j];
    }
    D[i * (N + 1) + i] = -s;
  }
}

/* V_ij = sqrt((2j+1)/2) P_j(x_i): nodal values of the orthonormal modes. */
void or_vandermonde_legendre(int N, const double* x, double* V) {
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N; ++j) {
      double P, dP;
      or_legendre(j, x[i], &P, &dP);
      V[i * (N + 1) + j] = sqrt((2.0 * j + 1.0) / 2.0) * P;
    }
}

/* Gauss-Jordan inverse with partial pivoting (small dense matrices). */
int or_invert(int n, const double* A, double* Ainv) {
  double* M = (double*)malloc(sizeof(double) * n * 2 * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j)
      M[i * 2 * n + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[r * 2 * n + c]) > fabs(M[piv * 2 * n + c])) piv = r;
    if (M[piv * 2 * n + c] == 0.0) { free(M); return 1; }
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) {
        double t = M[c * 2 * n + j]; M[c * 2 * n + j] = M[piv * 2 * n + j]; M[piv * 2 * n + j] = t;
      }
    double d = M[c * 2 * n + c];
    for (int j = 0; j < 2 * n; ++j) M[c * 2 * n + j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = M[r * 2 * n + c];
      for (int j = 0; j < 2 * n; ++j) M[r * 2 * n + j] -= f * M[c * 2 * n + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = M[i * 2 * n + n + j];
  free(M);
  return 0;
}

/* number of OpenMP threads of the oracle's element loops (timing only; <= 0 leaves it) */
#ifdef _OPENMP
#include <omp.h>
#endif
int or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
