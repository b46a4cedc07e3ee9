/*
 * Oracle (test infrastructure only): metric terms of the curvilinear map.
 *
 * The paper maps each element to [-1,1]^d (Eq. mapp), defines the Jacobian
 * J_ij = dx_i/dX_j (Eq. jacobian) and writes the transformed flux
 * |J| dX_i/dx_j F_j (Eq. mapped_equation).  It does not say how the
 * contravariant vectors Ja^i = |J| grad(X_i) are discretised.  Reading:
 *   - geometry is the degree-N nodal interpolant of the map (node_xyz given at
 *     the LGL nodes),
 *   - 3D: Kopriva's conservative curl form
 *       Ja^i_n = - [ curl_xi ( x_l grad_xi x_m ) ]_i ,  (n, m, l) cyclic,
 *     with every derivative taken by the LGL derivative matrix,
 *   - 2D: Ja^1 = ( y_eta, -x_eta ),  Ja^2 = ( -y_xi, x_xi ),
 *   - J = det(dx/dxi) from the same derivatives.
 *   - the undifferentiated factor x_l is taken relative to the element's first
 *     node: a constant shift c changes the curl form by c curl_xi grad_xi x_m,
 *     which vanishes (the tensor-product derivative matrices of different
 *     directions commute), and without it the products x_l grad x_m of size
 *     |x| h cancel to Ja of size h^2, which amplifies rounding by |x| / h.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static int ipow(int b, int e) { int r = 1; while (e--) r *= b; return r; }

/* derivative of nodal field f along reference direction d, at node n */
static double dref(int dim, int N, const double* D, const double* f, int d, int n) {
  int s = ipow(N + 1, d);
  int pos = (n / s) % (N + 1);
  int base = n - pos * s;
  double acc = 0.0;
  for (int l = 0; l <= N; ++l) acc += D[pos * (N + 1) + l] * f[base + l * s];
  (void)dim;
  return acc;
}

int or_geometry(int dim, int N, int64_t K, const double* xyz, double* Ja, double* J) {
  if (dim < 2 || dim > 3 || N < 1 || N > OR_MAX_N) return 1;
  double x[OR_MAX_N + 1], w[OR_MAX_N + 1], D[(OR_MAX_N + 1) * (OR_MAX_N + 1)];
  or_lgl(N, x, w);
  or_dmat(N, x, D);
  int np = ipow(N + 1, dim);
  double* V = (double*)malloc(sizeof(double) * 3 * np);
  for (int64_t k = 0; k < K; ++k) {
    const double* X = xyz + (size_t)k * dim * np;
    double* JA = Ja + (size_t)k * dim * dim * np;
    double* JJ = J + (size_t)k * np;
    /* a[n][j] = d x_n / d xi_j at every node */
    for (int node = 0; node < np; ++node) {
      double a[3][3];
      for (int n = 0; n < dim; ++n)
        for (int j = 0; j < dim; ++j) a[n][j] = dref(dim, N, D, X + n * np, j, node);
      if (dim == 2) {
        JJ[node] = a[0][0] * a[1][1] - a[0][1] * a[1][0];
        /* Ja[i][n]: i = reference direction, n = physical component */
        JA[(0 * 2 + 0) * np + node] = a[1][1];
        JA[(0 * 2 + 1) * np + node] = -a[0][1];
        JA[(1 * 2 + 0) * np + node] = -a[1][0];
        JA[(1 * 2 + 1) * np + node] = a[0][0];
      } else {
        JJ[node] = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
                   a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                   a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
      }
    }
    if (dim == 3) {
      for (int n = 0; n < 3; ++n) {
        int m = (n + 1) % 3, l = (n + 2) % 3;
        /* V_j = (x_l - x_l(first node)) * d x_m / d xi_j  (nodal interpolant of
           the product) */
        const double c = X[l * np];
        for (int node = 0; node < np; ++node)
          for (int j = 0; j < 3; ++j)
            V[j * np + node] = (X[l * np + node] - c) * dref(3, N, D, X + m * np, j, node);
        for (int node = 0; node < np; ++node) {
          double c0 = dref(3, N, D, V + 2 * np, 1, node) - dref(3, N, D, V + 1 * np, 2, node);
          double c1 = dref(3, N, D, V + 0 * np, 2, node) - dref(3, N, D, V + 2 * np, 0, node);
          double c2 = dref(3, N, D, V + 1 * np, 0, node) - dref(3, N, D, V + 0 * np, 1, node);
          JA[(0 * 3 + n) * np + node] = -c0;
          JA[(1 * 3 + n) * np + node] = -c1;
          JA[(2 * 3 + n) * np + node] = -c2;
        }
      }
    }
    for (int node = 0; node < np; ++node)
      if (!(JJ[node] > 0.0)) { free(V); return 2; }
  }
  free(V);
  return 0;
}
