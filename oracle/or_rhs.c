/*
 * Oracle (test infrastructure only): semi-discrete right-hand side,
 * time step, low-storage RK and domain integrals.
 *
 * Advective part (Eqs. strong_form, fluxes_discrete_strong, fluxdiffcons):
 *   du_i/dt = -(1/J_i) sum_dir [ sum_{l != i} 2 D_il F#(u_i, u_l; (Ja_i+Ja_l)/2)
 *                                + delta_iN F*_N / w_N - delta_i0 F*_0 / w_0 ]
 * which is the paper's form with 2 D and the (F* - F) surface terms once the
 * LGL identities 2 D_00 = -1/w_0, 2 D_NN = 1/w_N are used (reading of the
 * index/sign conventions, which differ between Eqs. fluxes_discrete_strong and
 * fluxdiff).  Interface fluxes follow Eqs. riemann_problem1-3 with the element's
 * own face metric Ja^dir as the (unnormalised) normal; a conforming partner
 * face sees the same normal up to rounding.
 * Shock capturing (Eqs. DGvec, fluxes_discrete_with_fv, finitevolumeder,
 * finitevolumeflux), reading of Hennemann et al.: per line, the (N+2)-vectors
 * of subcell fluxes carry the element's face fluxes F*_0, F*_N at both ends for
 * the high-order and the finite-volume part alike; du_i/dt = -(1/(J_i w_i))
 * sum_dir Delta[(1-alpha) Fbar + alpha F^FV]_i.  Curved subcell normals:
 * n_{j+1/2} = Ja_0 + sum_{m<=j} w_m (D Ja)_m.
 * Viscous part (Eqs. visc_fluxes, stress, auxil, auxstrongf), reading:
 * BR1 on primitive gradients W = (v, theta = p/rho), interface values
 * W* = (W- + W+)/2, strong form Q = D W + M^{-1} B (W* - W) per reference
 * direction (the sign that makes sum_i w_i Q_i = W*_r - W*_l), physical
 * gradient (1/J) sum_i Ja^i Q^i; viscous flux f^v_x = (0, sigma_.x,
 * sigma_.x . v + kappa dT/dx) with sigma per Eq. stress (lambda = 0) and
 * kappa dT/dx = mu gamma / ((gamma-1) Pr) dtheta/dx (mu and kappa scaled per node by
 * Sutherland's law, Eq. sutherland, when it is on); interface viscous flux
 * = average of both sides' f^v, dotted with the face normal; it enters as
 * + (1/J)[D Fv + M^{-1} B (Fv* - Fv)].
 * Viscous boundaries (weakly, through W* and Fv*; reading of the boundary paragraph of the
 * numerical-results section): supersonic inflow W* = (W + W_ext)/2, Fv* = mean of f^v of
 * the interior gradient with the interior and with the external state; outflow W* = W,
 * Fv* = f^v; no-slip walls W* = (0, theta) (adiabatic) or (0, theta_wall) (isothermal),
 * Fv* = f^v of the interior gradient at wall velocity 0, with the heat flux set to 0 on an
 * adiabatic wall.  The advective part of a no-slip wall is the slip-wall flux (mirrored
 * normal velocity through the Riemann solver); Navier-Stokes slip walls are not modelled.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static int ipow(int b, int e) { int r = 1; while (e--) r *= b; return r; }

typedef struct {
  int dim, N, np, nf, nv, nsp;
  double x[OR_MAX_N + 1], w[OR_MAX_N + 1], D[(OR_MAX_N + 1) * (OR_MAX_N + 1)];
} basis;

static void make_basis(const or_problem* P, basis* b) {
  b->dim = P->dim; b->N = P->N;
  b->np = ipow(P->N + 1, P->dim);
  b->nf = 2 * P->dim;
  b->nsp = P->n_species > 0 ? P->n_species : 1;
  b->nv = b->nsp + P->dim + 1;
  or_lgl(P->N, b->x, b->w);
  or_dmat(P->N, b->x, b->D);
}

static void node_u(const basis* b, const double* u, int64_t k, int node, double* uu) {
  for (int v = 0; v < b->nv; ++v) uu[v] = u[((size_t)k * b->nv + v) * b->np + node];
}

static void node_metric(const or_problem* P, const basis* b, int64_t k, int d, int node,
                        double* n) {
  for (int c = 0; c < 3; ++c) n[c] = 0.0;
  for (int c = 0; c < b->dim; ++c)
    n[c] = P->Ja[(((size_t)k * b->dim + d) * b->dim + c) * b->np + node];
}

static int line_pos(const basis* b, int d, int node) {
  int s = ipow(b->N + 1, d);
  return (node / s) % (b->N + 1);
}

/* partner node across face f (conforming, aligned faces: + pairs with -) */
static int nbr_node(const basis* b, int f, int node) {
  int d = f / 2, s = ipow(b->N + 1, d), pos = (node / s) % (b->N + 1);
  int target = (f % 2 == 1) ? 0 : b->N;
  return node + (target - pos) * s;
}

/* mu(T) / mu by Sutherland's law (Eq. sutherland) at a node; 1 when it is off */
static double mu_ratio(const or_problem* P, const or_prim* q) {
  double s = P->sutherland_s;
  if (!(s > 0.0)) return 1.0;
  double th = q->p / (q->rho * P->sutherland_rt);
  return (1.0 + s) * pow(th, 1.5) / (th + s);
}

static int check_mesh(const or_problem* P) {
  int nf = 2 * P->dim;
  if (P->sutherland_s < 0.0 || (P->sutherland_s > 0.0 && !(P->sutherland_rt > 0.0))) return 1;
  if (P->sutherland_s > 0.0 && P->n_species > 0) return 1;
  if (P->indicator_var != 0 && P->indicator_var != 1) return 1;
  for (int64_t k = 0; k < P->K; ++k)
    for (int f = 0; f < nf; ++f) {
      int64_t nb = P->nbr_elem[k * nf + f];
      if (nb >= 0) {
        if (nb >= P->K) return 1;
        if (P->nbr_face[k * nf + f] != (f ^ 1)) return 1;
      } else {
        int64_t bc = -(nb + 1);
        if (bc >= P->n_bc) return 1;
        int kind = P->bc_kind[bc];
        if (kind < OR_BC_INFLOW || kind > OR_BC_ISOTHERMAL) return 1;
        if (P->equations == OR_NAVIER_STOKES && (kind == OR_BC_SLIP_WALL || P->n_species > 0)) return 1;
      }
    }
  return 0;
}

/* External (ghost) state for a boundary face.  Returns 1 for "flux is the
 * physical flux of *ug" (inflow/outflow), 0 for "use the Riemann solver". */
static int boundary_state(const or_problem* P, const basis* b, int bc, const double* uo,
                          const or_prim* qo, const double* n, double* ug, or_prim* qg,
                          int* err) {
  int kind = P->bc_kind[bc];
  if (kind == OR_BC_INFLOW) {
    or_prim_to_cons(P, P->bc_prim + (size_t)bc * b->nv, ug);
    if (or_cons_to_prim(P, ug, qg)) *err = 1;
    return 1;
  }
  if (kind == OR_BC_OUTFLOW) {
    memcpy(ug, uo, sizeof(double) * b->nv);
    *qg = *qo;
    return 1;
  }
  /* slip and no-slip walls: mirror the normal velocity */
  double nn = 0.0, vn = 0.0;
  for (int d = 0; d < b->dim; ++d) nn += n[d] * n[d];
  nn = sqrt(nn);
  for (int d = 0; d < b->dim; ++d) vn += qo->v[d] * n[d] / nn;
  memcpy(ug, uo, sizeof(double) * b->nv);
  for (int d = 0; d < b->dim; ++d) ug[b->nsp + d] = qo->rho * (qo->v[d] - 2.0 * vn * n[d] / nn);
  *qg = *qo;
  for (int d = 0; d < b->dim; ++d) qg->v[d] = qo->v[d] - 2.0 * vn * n[d] / nn;
  return 0;
}

/* numerical flux in +dir orientation at node of element k on face f */
static void face_flux(const or_problem* P, const basis* b, const double* u, int64_t k, int f,
                      int node, const double* uo, const or_prim* qo, double* F, int* err) {
  double n[3];
  node_metric(P, b, k, f / 2, node, n);
  int64_t nb = P->nbr_elem[k * b->nf + f];
  double ux[OR_MAX_NV];
  or_prim qx;
  if (nb >= 0) {
    node_u(b, u, nb, nbr_node(b, f, node), ux);
    if (or_cons_to_prim(P, ux, &qx)) *err = 1;
  } else {
    if (boundary_state(P, b, (int)(-(nb + 1)), uo, qo, n, ux, &qx, err)) {
      or_phys_flux(P, &qx, ux, n, F);
      return;
    }
  }
  if (f % 2 == 1) or_surface_flux(P, uo, qo, ux, &qx, n, F);
  else or_surface_flux(P, ux, &qx, uo, qo, n, F);
}

/* ---------- shock indicator (Hennemann-Gassner, reading of Eq. fluxes_discrete_with_fv) */
static int element_alpha_raw(const or_problem* P, const basis* b, const double* u, int64_t k,
                             double* alpha) {
  int N = b->N, n1 = N + 1, np = b->np;
  double V[(OR_MAX_N + 1) * (OR_MAX_N + 1)], Vi[(OR_MAX_N + 1) * (OR_MAX_N + 1)];
  or_vandermonde_legendre(N, b->x, V);
  or_invert(n1, V, Vi);
  double* f = (double*)malloc(sizeof(double) * np);
  double* m = (double*)malloc(sizeof(double) * np);
  double* t = (double*)malloc(sizeof(double) * np);
  int err = 0;
  for (int node = 0; node < np; ++node) {
    double uu[OR_MAX_NV];
    or_prim q;
    node_u(b, u, k, node, uu);
    if (or_cons_to_prim(P, uu, &q)) err = 1;
    f[node] = P->indicator_var ? q.p : q.rho * q.p;
  }
  /* modal coefficients: apply V^{-1} along every direction */
  memcpy(m, f, sizeof(double) * np);
  for (int d = 0; d < b->dim; ++d) {
    int s = ipow(n1, d);
    for (int node = 0; node < np; ++node) {
      int pos = (node / s) % n1, base = node - pos * s;
      double acc = 0.0;
      for (int l = 0; l < n1; ++l) acc += Vi[pos * n1 + l] * m[base + l * s];
      t[node] = acc;
    }
    memcpy(m, t, sizeof(double) * np);
  }
  /* energy of all modes, of the modes up to degree N-1, and of the highest (degree N) and
   * second-highest (degree N-1) modes, summed directly (no cancellation) */
  double Etot = 0.0, E1 = 0.0, Eh1 = 0.0, Eh2 = 0.0;
  for (int node = 0; node < np; ++node) {
    int mx = 0;
    for (int d = 0; d < b->dim; ++d) {
      int pos = line_pos(b, d, node);
      if (pos > mx) mx = pos;
    }
    double e = m[node] * m[node];
    Etot += e;
    if (mx <= N - 1) E1 += e;
    if (mx == N) Eh1 += e;
    if (mx == N - 1) Eh2 += e;
  }
  double frac1 = Etot > 0.0 ? Eh1 / Etot : 0.0;
  double frac2 = E1 > 0.0 ? Eh2 / E1 : 0.0;
  double E = frac1 > frac2 ? frac1 : frac2;
  double thr = 0.5 * pow(10.0, -1.8 * pow(N + 1.0, 0.25));
  double s = log((1.0 - 1e-4) / 1e-4);
  double a = 1.0 / (1.0 + exp(-(s / thr) * (E - thr)));
  if (a < 1e-3) a = 0.0;
  if (a > P->alpha_max) a = P->alpha_max;
  *alpha = a;
  free(f); free(m); free(t);
  return err;
}

int or_indicator(const or_problem* P, const double* u, double* alpha) {
  basis b;
  make_basis(P, &b);
  double* raw = (double*)malloc(sizeof(double) * P->K);
  int err = 0;
#pragma omp parallel for reduction(| : err)
  for (int64_t k = 0; k < P->K; ++k) err |= element_alpha_raw(P, &b, u, k, raw + k);
  for (int64_t k = 0; k < P->K; ++k) {
    double a = raw[k];
    for (int f = 0; f < b.nf; ++f) {
      int64_t nb = P->nbr_elem[k * b.nf + f];
      if (nb >= 0 && 0.5 * raw[nb] > a) a = 0.5 * raw[nb];
    }
    alpha[k] = a;
  }
  free(raw);
  return err;
}

/* ---------- BR1 gradients of W = (v_1..v_dim, theta) ---------- */
static void node_W(const or_problem* P, const basis* b, const double* u, int64_t k, int node,
                   double* W, int* err) {
  double uu[OR_MAX_NV];
  or_prim q;
  node_u(b, u, k, node, uu);
  if (or_cons_to_prim(P, uu, &q)) *err = 1;
  for (int d = 0; d < b->dim; ++d) W[d] = q.v[d];
  W[b->dim] = q.p / q.rho;
}

/* primitive external state of boundary id bc (from its primitive description) */
static void bc_prim_state(const or_problem* P, const basis* b, int bc, or_prim* q, int* err) {
  double ug[OR_MAX_NV];
  or_prim_to_cons(P, P->bc_prim + (size_t)bc * b->nv, ug);
  if (or_cons_to_prim(P, ug, q)) *err = 1;
}

/* BR1 boundary value W* at a boundary face node with interior value Wn */
static void boundary_W(const or_problem* P, const basis* b, int bc, const double* Wn, double* Ws,
                       int* err) {
  int dim = b->dim, kind = P->bc_kind[bc];
  or_prim qe;
  for (int c = 0; c <= dim; ++c) Ws[c] = Wn[c];
  if (kind == OR_BC_INFLOW) {
    bc_prim_state(P, b, bc, &qe, err);
    for (int d = 0; d < dim; ++d) Ws[d] = 0.5 * (Wn[d] + qe.v[d]);
    Ws[dim] = 0.5 * (Wn[dim] + qe.p / qe.rho);
  } else if (kind == OR_BC_NOSLIP_ADIABATIC || kind == OR_BC_ISOTHERMAL) {
    for (int d = 0; d < dim; ++d) Ws[d] = 0.0;
    if (kind == OR_BC_ISOTHERMAL) {
      bc_prim_state(P, b, bc, &qe, err);
      Ws[dim] = qe.p / qe.rho;
    }
  }
}

static int br1_gradients(const or_problem* P, const basis* b, const double* u, double* G) {
  int dim = b->dim, nW = dim + 1, np = b->np, N = b->N;
  int err = 0;
#pragma omp parallel for reduction(| : err)
  for (int64_t k = 0; k < P->K; ++k) {
    for (int node = 0; node < np; ++node) {
      double Q[3][OR_MAX_NV];
      double Wn[4];
      node_W(P, b, u, k, node, Wn, &err);
      for (int d = 0; d < dim; ++d) {
        int s = ipow(N + 1, d), pos = line_pos(b, d, node), base = node - pos * s;
        for (int c = 0; c < nW; ++c) Q[d][c] = 0.0;
        for (int l = 0; l <= N; ++l) {
          double Wm[4];
          node_W(P, b, u, k, base + l * s, Wm, &err);
          for (int c = 0; c < nW; ++c) Q[d][c] += b->D[pos * (N + 1) + l] * Wm[c];
        }
        for (int side = 0; side < 2; ++side) {
          int f = 2 * d + side;
          if (pos != (side ? N : 0)) continue;
          int64_t nb = P->nbr_elem[k * b->nf + f];
          double Ws[4];
          if (nb >= 0) {
            double Wx[4];
            node_W(P, b, u, nb, nbr_node(b, f, node), Wx, &err);
            for (int c = 0; c < nW; ++c) Ws[c] = 0.5 * (Wn[c] + Wx[c]);
          } else {
            boundary_W(P, b, (int)(-(nb + 1)), Wn, Ws, &err);
          }
          for (int c = 0; c < nW; ++c) {
            if (side) Q[d][c] += (Ws[c] - Wn[c]) / b->w[N];
            else Q[d][c] -= (Ws[c] - Wn[c]) / b->w[0];
          }
        }
      }
      double Jn = P->J[(size_t)k * np + node];
      for (int x = 0; x < dim; ++x)
        for (int c = 0; c < nW; ++c) {
          double acc = 0.0;
          for (int d = 0; d < dim; ++d) {
            double n[3];
            node_metric(P, b, k, d, node, n);
            acc += n[x] * Q[d][c];
          }
          G[(((size_t)k * dim + x) * nW + c) * np + node] = acc / Jn;
        }
    }
  }
  return err;
}

/* physical viscous flux f^v_x (x = physical direction) at a node */
static void visc_flux(const or_problem* P, const basis* b, const double* G, int64_t k, int node,
                      const or_prim* q, double (*fv)[OR_MAX_NV]) {
  const double* v = q->v;
  int dim = b->dim, nW = dim + 1, np = b->np;
  double gv[3][3], gth[3];
  for (int x = 0; x < dim; ++x) {
    for (int a = 0; a < dim; ++a) gv[a][x] = G[(((size_t)k * dim + x) * nW + a) * np + node];
    gth[x] = G[(((size_t)k * dim + x) * nW + dim) * np + node];
  }
  double div = 0.0;
  for (int a = 0; a < dim; ++a) div += gv[a][a];
  double mu = P->mu * mu_ratio(P, q), g = P->gamma;
  double kap = mu * g / ((g - 1.0) * P->Pr);
  for (int x = 0; x < dim; ++x) {
    fv[x][0] = 0.0;
    double work = 0.0;
    for (int a = 0; a < dim; ++a) {
      double sig = mu * (gv[a][x] + gv[x][a]) - (a == x ? 2.0 / 3.0 * mu * div : 0.0);
      fv[x][1 + a] = sig;
      work += v[a] * sig;
    }
    fv[x][1 + dim] = work + kap * gth[x];
  }
}

/* ---------- the right-hand side ---------- */
int or_rhs(const or_problem* P, const double* u, double* rhs, double* alpha_out,
           double* gradW_out) {
  basis b;
  if (P->dim < 2 || P->dim > 3 || P->N < 1 || P->N > OR_MAX_N) return 1;
  if (check_mesh(P)) return 1;
  make_basis(P, &b);
  /* the Ranocha, Kennedy-Gruber, Pirozzoli and Morinishi forms are single-gas fluxes */
  if (P->n_species > 0 && P->volume_flux != OR_VF_DUCROS && P->volume_flux != OR_VF_CENTRAL) return 1;
  if (P->n_species > 0 && P->equations == OR_NAVIER_STOKES) return 1;
  int dim = b.dim, N = b.N, np = b.np, nv = b.nv;
  double* alpha = NULL;
  int err = 0;
  if (P->alpha_max > 0.0 || P->alpha_override >= 0.0) {
    alpha = (double*)malloc(sizeof(double) * P->K);
    if (P->alpha_override >= 0.0)
      for (int64_t k = 0; k < P->K; ++k) alpha[k] = P->alpha_override;
    else
      err |= or_indicator(P, u, alpha);
    if (alpha_out) memcpy(alpha_out, alpha, sizeof(double) * P->K);
  }
#pragma omp parallel for reduction(| : err)
  for (int64_t k = 0; k < P->K; ++k) {
    double* acc = (double*)calloc((size_t)nv * np, sizeof(double));
    double* ue = (double*)malloc(sizeof(double) * nv * np);
    or_prim* qe = (or_prim*)malloc(sizeof(or_prim) * np);
    for (int node = 0; node < np; ++node) {
      node_u(&b, u, k, node, ue + node * nv);
      if (or_cons_to_prim(P, ue + node * nv, qe + node)) err |= 1;
    }
    if (!alpha) {
      /* volume: sum_{l != i} 2 D_il F#(u_i, u_l) per direction */
      for (int node = 0; node < np; ++node)
        for (int d = 0; d < dim; ++d) {
          int s = ipow(N + 1, d), pos = line_pos(&b, d, node), base = node - pos * s;
          double ni[3];
          node_metric(P, &b, k, d, node, ni);
          for (int l = 0; l <= N; ++l) {
            if (l == pos) continue;
            int m = base + l * s;
            double nm[3], na[3], F[OR_MAX_NV];
            node_metric(P, &b, k, d, m, nm);
            for (int c = 0; c < 3; ++c) na[c] = 0.5 * (ni[c] + nm[c]);
            or_volume_flux(P, ue + node * nv, qe + node, ue + m * nv, qe + m, na, F);
            for (int v = 0; v < nv; ++v) acc[v * np + node] += 2.0 * b.D[pos * (N + 1) + l] * F[v];
          }
        }
      /* surface: + F*_N / w_N at the + face, - F*_0 / w_0 at the - face */
      for (int node = 0; node < np; ++node)
        for (int d = 0; d < dim; ++d) {
          int pos = line_pos(&b, d, node);
          for (int side = 0; side < 2; ++side) {
            if (pos != (side ? N : 0)) continue;
            double F[OR_MAX_NV];
            face_flux(P, &b, u, k, 2 * d + side, node, ue + node * nv, qe + node, F, &err);
            for (int v = 0; v < nv; ++v)
              acc[v * np + node] += side ? F[v] / b.w[N] : -F[v] / b.w[0];
          }
        }
    } else {
      /* blended DG / subcell FV, one line at a time */
      double a = alpha[k];
      for (int d = 0; d < dim; ++d) {
        int s = ipow(N + 1, d);
        for (int node0 = 0; node0 < np; ++node0) {
          if (line_pos(&b, d, node0) != 0) continue;
          int ln[OR_MAX_N + 1];
          for (int j = 0; j <= N; ++j) ln[j] = node0 + j * s;
          double FDG[OR_MAX_N + 2][OR_MAX_NV], FFV[OR_MAX_N + 2][OR_MAX_NV];
          double Fs0[OR_MAX_NV], FsN[OR_MAX_NV];
          face_flux(P, &b, u, k, 2 * d, ln[0], ue + ln[0] * nv, qe + ln[0], Fs0, &err);
          face_flux(P, &b, u, k, 2 * d + 1, ln[N], ue + ln[N] * nv, qe + ln[N], FsN, &err);
          for (int v = 0; v < nv; ++v) {
            FDG[0][v] = FFV[0][v] = Fs0[v];
            FDG[N + 1][v] = FFV[N + 1][v] = FsN[v];
          }
          /* high-order subcell fluxes Fbar_j, Eq. DGvec */
          for (int j = 1; j <= N; ++j) {
            for (int v = 0; v < nv; ++v) FDG[j][v] = 0.0;
            for (int p = j; p <= N; ++p)
              for (int q = 0; q <= j - 1; ++q) {
                double nq[3], npp[3], na[3], F[OR_MAX_NV];
                node_metric(P, &b, k, d, ln[q], nq);
                node_metric(P, &b, k, d, ln[p], npp);
                for (int c = 0; c < 3; ++c) na[c] = 0.5 * (nq[c] + npp[c]);
                or_volume_flux(P, ue + ln[q] * nv, qe + ln[q], ue + ln[p] * nv, qe + ln[p], na, F);
                for (int v = 0; v < nv; ++v)
                  FDG[j][v] += 2.0 * b.w[q] * b.D[q * (N + 1) + p] * F[v];
              }
          }
          /* finite-volume subcell fluxes, Eq. finitevolumeflux, curved normals */
          double nh[3];
          node_metric(P, &b, k, d, ln[0], nh);
          for (int j = 1; j <= N; ++j) {
            int m = j - 1; /* advance the normal across subcell m */
            for (int l = 0; l <= N; ++l) {
              double nl[3];
              node_metric(P, &b, k, d, ln[l], nl);
              for (int c = 0; c < 3; ++c) nh[c] += b.w[m] * b.D[m * (N + 1) + l] * nl[c];
            }
            or_surface_flux(P, ue + ln[j - 1] * nv, qe + ln[j - 1], ue + ln[j] * nv, qe + ln[j],
                            nh, FFV[j]);
          }
          for (int i = 0; i <= N; ++i)
            for (int v = 0; v < nv; ++v) {
              double dg = FDG[i + 1][v] - FDG[i][v];
              double fv = FFV[i + 1][v] - FFV[i][v];
              acc[v * np + ln[i]] += ((1.0 - a) * dg + a * fv) / b.w[i];
            }
        }
      }
    }
    for (int node = 0; node < np; ++node) {
      double Jn = P->J[(size_t)k * np + node];
      for (int v = 0; v < nv; ++v)
        rhs[((size_t)k * nv + v) * np + node] = -acc[v * np + node] / Jn;
    }
    /* finite-rate species sources (Eq. source_term) */
    if (P->n_reactions > 0 && P->n_species == 5) {
      for (int node = 0; node < np; ++node) {
        double S[5];
        or_chem_source(P->species, P->n_reactions, P->reactions, qe[node].rhos, qe[node].T,
                       P->chem_dt, S);
        for (int s = 0; s < 5; ++s) rhs[((size_t)k * nv + s) * np + node] += S[s];
      }
    }
    free(acc); free(ue); free(qe);
  }
  if (P->equations == OR_NAVIER_STOKES) {
    int nW = dim + 1;
    double* G = (double*)malloc(sizeof(double) * (size_t)P->K * dim * nW * np);
    err |= br1_gradients(P, &b, u, G);
    if (gradW_out) memcpy(gradW_out, G, sizeof(double) * (size_t)P->K * dim * nW * np);
#pragma omp parallel for reduction(| : err)
    for (int64_t k = 0; k < P->K; ++k) {
      double* Fv = (double*)malloc(sizeof(double) * dim * nv * np); /* [d][v][node] */
      double* acc = (double*)calloc((size_t)nv * np, sizeof(double));
      for (int node = 0; node < np; ++node) {
        double uu[OR_MAX_NV], fv[3][OR_MAX_NV];
        or_prim q;
        node_u(&b, u, k, node, uu);
        if (or_cons_to_prim(P, uu, &q)) err |= 1;
        visc_flux(P, &b, G, k, node, &q, fv);
        for (int d = 0; d < dim; ++d) {
          double n[3];
          node_metric(P, &b, k, d, node, n);
          for (int v = 0; v < nv; ++v) {
            double s = 0.0;
            for (int x = 0; x < dim; ++x) s += n[x] * fv[x][v];
            Fv[((size_t)d * nv + v) * np + node] = s;
          }
        }
      }
      for (int node = 0; node < np; ++node)
        for (int d = 0; d < dim; ++d) {
          int s = ipow(N + 1, d), pos = line_pos(&b, d, node), base = node - pos * s;
          for (int l = 0; l <= N; ++l)
            for (int v = 0; v < nv; ++v)
              acc[v * np + node] += b.D[pos * (N + 1) + l] * Fv[((size_t)d * nv + v) * np + base + l * s];
          for (int side = 0; side < 2; ++side) {
            int f = 2 * d + side;
            if (pos != (side ? N : 0)) continue;
            int64_t nb = P->nbr_elem[k * b.nf + f];
            int mn = nbr_node(&b, f, node);
            double uu[OR_MAX_NV], fo[3][OR_MAX_NV], fx[3][OR_MAX_NV], n[3];
            or_prim q;
            node_u(&b, u, k, node, uu);
            or_cons_to_prim(P, uu, &q);
            visc_flux(P, &b, G, k, node, &q, fo);
            int kind = nb >= 0 ? 0 : P->bc_kind[-(nb + 1)];
            if (nb >= 0) {
              node_u(&b, u, nb, mn, uu);
              or_cons_to_prim(P, uu, &q);
              visc_flux(P, &b, G, nb, mn, &q, fx);
            } else if (kind == OR_BC_INFLOW) {
              or_prim qe;
              bc_prim_state(P, &b, (int)(-(nb + 1)), &qe, &err);
              visc_flux(P, &b, G, k, node, &qe, fx);    /* interior gradient, external state */
            } else if (kind == OR_BC_OUTFLOW) {
              memcpy(fx, fo, sizeof(fx));
            } else {                                     /* no-slip walls: wall velocity 0 */
              or_prim qw = q;
              for (int c = 0; c < dim; ++c) qw.v[c] = 0.0;
              visc_flux(P, &b, G, k, node, &qw, fx);
              if (kind == OR_BC_NOSLIP_ADIABATIC)
                for (int x = 0; x < dim; ++x) fx[x][1 + dim] = 0.0;
              memcpy(fo, fx, sizeof(fx));               /* Fv* = the wall flux itself */
            }
            node_metric(P, &b, k, d, node, n);
            for (int v = 0; v < nv; ++v) {
              double Fs = 0.0;
              for (int x = 0; x < dim; ++x) Fs += 0.5 * (fo[x][v] + fx[x][v]) * n[x];
              double jump = Fs - Fv[((size_t)d * nv + v) * np + node];
              acc[v * np + node] += side ? jump / b.w[N] : -jump / b.w[0];
            }
          }
        }
      for (int node = 0; node < np; ++node) {
        double Jn = P->J[(size_t)k * np + node];
        for (int v = 0; v < nv; ++v) rhs[((size_t)k * nv + v) * np + node] += acc[v * np + node] / Jn;
      }
      free(Fv); free(acc);
    }
    free(G);
  }
  free(alpha);
  return err;
}

int or_prim_to_cons_field(const or_problem* P, const double* w, double* u) {
  basis b;
  make_basis(P, &b);
  int err = 0;
  for (int64_t k = 0; k < P->K; ++k)
    for (int node = 0; node < b.np; ++node) {
      double ww[OR_MAX_NV], uu[OR_MAX_NV];
      for (int v = 0; v < b.nv; ++v) ww[v] = w[((size_t)k * b.nv + v) * b.np + node];
      err |= or_prim_to_cons(P, ww, uu);
      for (int v = 0; v < b.nv; ++v) u[((size_t)k * b.nv + v) * b.np + node] = uu[v];
    }
  return err;
}

/* ---------- time step: dt = cfl * 2 / ((N+1) max lambda), lambda = sum_i (|v.Ja^i| + c|Ja^i|)/J;
 * Navier-Stokes adds dt_v = cfl * 4 / ((N+1)^2 max gamma mu(T)/(Pr rho) sum_i |Ja^i|^2 / J^2) */
double or_max_dt(const or_problem* P, const double* u, double cfl) {
  basis b;
  make_basis(P, &b);
  double lam = 0.0, lamv = 0.0;
  for (int64_t k = 0; k < P->K; ++k)
    for (int node = 0; node < b.np; ++node) {
      double uu[OR_MAX_NV];
      or_prim q;
      node_u(&b, u, k, node, uu);
      or_cons_to_prim(P, uu, &q);
      double Jn = P->J[(size_t)k * b.np + node], l = 0.0, lv = 0.0;
      for (int d = 0; d < b.dim; ++d) {
        double n[3], vn = 0.0, nn = 0.0;
        node_metric(P, &b, k, d, node, n);
        for (int c = 0; c < b.dim; ++c) { vn += q.v[c] * n[c]; nn += n[c] * n[c]; }
        l += fabs(vn) + q.c * sqrt(nn);
        lv += nn;
      }
      l /= Jn;
      lv = P->gamma * P->mu * mu_ratio(P, &q) / (P->Pr * q.rho) * lv / (Jn * Jn);
      if (l > lam) lam = l;
      if (lv > lamv) lamv = lv;
    }
  double dt = cfl * 2.0 / ((P->N + 1) * lam);
  if (P->equations == OR_NAVIER_STOKES && lamv > 0.0) {
    double dtv = cfl * 4.0 / ((P->N + 1.0) * (P->N + 1.0) * lamv);
    if (dtv < dt) dt = dtv;
  }
  return dt;
}

/* Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage coefficients */
void or_ck45(double* A, double* B, double* c) {
  A[0] = 0.0;
  A[1] = -567301805773.0 / 1357537059087.0;
  A[2] = -2404267990393.0 / 2016746695238.0;
  A[3] = -3550918686646.0 / 2091501179385.0;
  A[4] = -1275806237668.0 / 842570457699.0;
  B[0] = 1432997174477.0 / 9575080441755.0;
  B[1] = 5161836677717.0 / 13612068292357.0;
  B[2] = 1720146321549.0 / 2090206949498.0;
  B[3] = 3134564353537.0 / 4481467310338.0;
  B[4] = 2277821191437.0 / 14882151754819.0;
  c[0] = 0.0;
  c[1] = 1432997174477.0 / 9575080441755.0;
  c[2] = 2526269341429.0 / 6820363962896.0;
  c[3] = 2006345519317.0 / 3224310063776.0;
  c[4] = 2802321613138.0 / 2924317926251.0;
}

int or_step_rk(const or_problem* P, double* u, int nsteps, double cfl, double dt_fixed,
               double* t) {
  basis b;
  make_basis(P, &b);
  size_t n = (size_t)P->K * b.nv * b.np;
  double* du = (double*)calloc(n, sizeof(double));
  double* r = (double*)malloc(sizeof(double) * n);
  double A[5], B[5], c[5];
  or_ck45(A, B, c);
  int err = 0;
  for (int st = 0; st < nsteps && !err; ++st) {
    double dt = dt_fixed > 0.0 ? dt_fixed : or_max_dt(P, u, cfl);
    for (int s = 0; s < 5 && !err; ++s) {
      or_problem Q = *P;
      Q.chem_dt = dt; /* point-implicit scaling of the chemistry source uses the step */
      err |= or_rhs(&Q, u, r, NULL, NULL);
      for (size_t i = 0; i < n; ++i) {
        du[i] = (s == 0 ? 0.0 : A[s] * du[i]) + dt * r[i];
        u[i] += B[s] * du[i];
      }
      if (P->positivity_eps > 0.0) err |= or_positivity(P, u, P->positivity_eps, NULL);
    }
    *t += dt;
  }
  free(du); free(r);
  return err;
}

/* Zhang-Shu positivity limiter (the positivity-preserving limiter the paper applies to
 * its shock problems), one calorically perfect gas.  Per element, with the quadrature
 * weights W_i = w_i J_i and the element mean ubar = sum W_i u_i / sum W_i:
 *   1. density: if min rho_i < eps, rho_i <- rhobar + th1 (rho_i - rhobar) with
 *      th1 = (rhobar - eps) / (rhobar - min rho_i);
 *   2. pressure: for every node with p(u_i) < eps, t_i in (0, 1) solves
 *      p(ubar + t (u_i - ubar)) = eps, i.e. the quadratic
 *      (E(t) - eps/(gamma-1)) rho(t) - |m(t)|^2 / 2 = 0; th2 = min t_i and every variable
 *      u_i <- ubar + th2 (u_i - ubar).
 * Both steps keep the element mean.  Returns 1 when an element mean itself is not
 * admissible (rhobar <= eps or p(ubar) <= eps).  n_limited (may be NULL) counts the
 * elements changed. */
/* Zhang-Shu limiter for a mixture (reading of the positivity-preservation remark for the
 * reacting cases): per element, with J-weighted means, (1) the partial densities move
 * toward their means by one common factor th1 until every rho_s >= min(eps, mean rho_s);
 * (2) every variable moves toward its mean by th2 until T >= OR_T_FLOOR at every node,
 * i.e. g(u) = (E - sum_s rho_s e_s(T_floor)) rho - |m|^2 / 2 >= 0 (e(T) increases with T),
 * th2 the smallest root in [0, 1] of the quadratic g(ubar + t (u - ubar)) = 0. */
static int positivity_mixture(const or_problem* P, const basis* b, double* u, double eps, int* n_limited) {
  const int dim = b->dim, np = b->np, nv = b->nv, ns = P->n_species;
  double ef[OR_MAX_SPECIES];
  for (int s = 0; s < ns; ++s) ef[s] = or_species_energy(P->species + 8 * s, OR_T_FLOOR);
  int err = 0, nlim = 0;
  double* W = (double*)malloc(sizeof(double) * np);
  for (int64_t k = 0; k < P->K; ++k) {
    double* ue = u + (size_t)k * nv * np;
    double Wsum = 0.0, ubar[OR_MAX_NV] = {0};
    for (int node = 0; node < np; ++node) {
      double wq = 1.0;
      for (int d = 0; d < dim; ++d) wq *= b->w[line_pos(b, d, node)];
      W[node] = wq * P->J[(size_t)k * np + node];
      Wsum += W[node];
      for (int v = 0; v < nv; ++v) ubar[v] += W[node] * ue[v * np + node];
    }
    for (int v = 0; v < nv; ++v) ubar[v] /= Wsum;
    /* g at the mean and the mean's admissibility */
    double rbar = 0.0, Ebar = ubar[ns + dim], mb2 = 0.0;
    int bad = 0;
    for (int s = 0; s < ns; ++s) {
      rbar += ubar[s];
      Ebar -= ubar[s] * ef[s];
      bad |= !(ubar[s] >= 0.0);
    }
    for (int d = 0; d < dim; ++d) mb2 += ubar[ns + d] * ubar[ns + d];
    if (bad || !(rbar > 0.0) || !(Ebar * rbar - 0.5 * mb2 > 0.0)) {
      err = 1;
      continue;
    }
    int changed = 0;
    /* 1. partial densities, one common factor */
    double th1 = 1.0;
    for (int s = 0; s < ns; ++s) {
      const double es = fmin(eps, ubar[s]);
      double mn = ue[s * np];
      for (int node = 1; node < np; ++node) mn = fmin(mn, ue[s * np + node]);
      if (mn < es) th1 = fmin(th1, (ubar[s] - es) / (ubar[s] - mn));
    }
    if (th1 < 1.0) {
      for (int s = 0; s < ns; ++s)
        for (int node = 0; node < np; ++node) ue[s * np + node] = ubar[s] + th1 * (ue[s * np + node] - ubar[s]);
      changed = 1;
    }
    /* 2. temperature floor */
    double th2 = 1.0;
    for (int node = 0; node < np; ++node) {
      double r = 0.0, Ep = ue[(ns + dim) * np + node], m2 = 0.0, dr = 0.0, dE = 0.0, mdm = 0.0, dm2 = 0.0;
      for (int s = 0; s < ns; ++s) {
        r += ue[s * np + node];
        Ep -= ue[s * np + node] * ef[s];
        dr += ue[s * np + node] - ubar[s];
        dE -= (ue[s * np + node] - ubar[s]) * ef[s];
      }
      dE += ue[(ns + dim) * np + node] - ubar[ns + dim];
      for (int d = 0; d < dim; ++d) {
        const double m = ue[(ns + d) * np + node], dm = m - ubar[ns + d];
        m2 += m * m;
        mdm += ubar[ns + d] * dm;
        dm2 += dm * dm;
      }
      if (Ep * r - 0.5 * m2 >= 0.0 && r > 0.0) continue;
      const double a = dE * dr - 0.5 * dm2;
      const double bq = dE * rbar + Ebar * dr - mdm;
      const double c = Ebar * rbar - 0.5 * mb2; /* > 0 */
      double t;
      if (fabs(a) < 1e-14 * (fabs(bq) + fabs(c))) {
        t = -c / bq;
      } else {
        const double disc = fmax(0.0, bq * bq - 4.0 * a * c);
        const double q = -0.5 * (bq + copysign(sqrt(disc), bq));
        const double t1 = q / a, t2 = c / q;
        t = (t1 >= 0.0 && t1 <= 1.0) ? t1 : t2;
      }
      th2 = fmin(th2, fmin(1.0, fmax(0.0, t)));
    }
    if (th2 < 1.0) {
      for (int v = 0; v < nv; ++v)
        for (int node = 0; node < np; ++node) ue[v * np + node] = ubar[v] + th2 * (ue[v * np + node] - ubar[v]);
      changed = 1;
    }
    nlim += changed;
  }
  free(W);
  if (n_limited) *n_limited = nlim;
  return err;
}

int or_positivity(const or_problem* P, double* u, double eps, int* n_limited) {
  basis b;
  make_basis(P, &b);
  const int dim = b.dim, np = b.np, nv = b.nv;
  if (P->n_species > 0) return positivity_mixture(P, &b, u, eps, n_limited);
  const double g1 = P->gamma - 1.0;
  int err = 0, nlim = 0;
  double* W = (double*)malloc(sizeof(double) * np);
  for (int64_t k = 0; k < P->K; ++k) {
    double* ue = u + (size_t)k * nv * np;
    double Wsum = 0.0, ubar[OR_MAX_NV] = {0};
    for (int node = 0; node < np; ++node) {
      double wq = 1.0;
      for (int d = 0; d < dim; ++d) wq *= b.w[line_pos(&b, d, node)];
      W[node] = wq * P->J[(size_t)k * np + node];
      Wsum += W[node];
      for (int v = 0; v < nv; ++v) ubar[v] += W[node] * ue[v * np + node];
    }
    for (int v = 0; v < nv; ++v) ubar[v] /= Wsum;
    double mb2 = 0.0;
    for (int d = 0; d < dim; ++d) mb2 += ubar[1 + d] * ubar[1 + d];
    const double pbar = g1 * (ubar[1 + dim] - 0.5 * mb2 / ubar[0]);
    if (!(ubar[0] > eps) || !(pbar > eps)) {
      err = 1;
      continue;
    }
    int changed = 0;
    /* 1. density */
    double rmin = ue[0];
    for (int node = 1; node < np; ++node) rmin = fmin(rmin, ue[node]);
    if (rmin < eps) {
      const double th1 = (ubar[0] - eps) / (ubar[0] - rmin);
      for (int node = 0; node < np; ++node) ue[node] = ubar[0] + th1 * (ue[node] - ubar[0]);
      changed = 1;
    }
    /* 2. pressure */
    const double ep = eps / g1;
    double th2 = 1.0;
    for (int node = 0; node < np; ++node) {
      double m2 = 0.0;
      for (int d = 0; d < dim; ++d) m2 += ue[(1 + d) * np + node] * ue[(1 + d) * np + node];
      const double p = g1 * (ue[(1 + dim) * np + node] - 0.5 * m2 / ue[node]);
      if (p >= eps) continue;
      const double dr = ue[node] - ubar[0], dE = ue[(1 + dim) * np + node] - ubar[1 + dim];
      double mdm = 0.0, dm2 = 0.0;
      for (int d = 0; d < dim; ++d) {
        const double dm = ue[(1 + d) * np + node] - ubar[1 + d];
        mdm += ubar[1 + d] * dm;
        dm2 += dm * dm;
      }
      const double a = dE * dr - 0.5 * dm2;
      const double bq = dE * ubar[0] + (ubar[1 + dim] - ep) * dr - mdm;
      const double c = (ubar[1 + dim] - ep) * ubar[0] - 0.5 * mb2;  /* > 0 */
      double t;
      if (fabs(a) < 1e-14 * (fabs(bq) + fabs(c))) {
        t = -c / bq;
      } else {
        const double disc = fmax(0.0, bq * bq - 4.0 * a * c);
        const double q = -0.5 * (bq + copysign(sqrt(disc), bq));
        const double t1 = q / a, t2 = c / q;
        t = (t1 >= 0.0 && t1 <= 1.0) ? t1 : t2;
      }
      t = fmin(1.0, fmax(0.0, t));
      th2 = fmin(th2, t);
    }
    if (th2 < 1.0) {
      for (int v = 0; v < nv; ++v)
        for (int node = 0; node < np; ++node) ue[v * np + node] = ubar[v] + th2 * (ue[v * np + node] - ubar[v]);
      changed = 1;
    }
    nlim += changed;
  }
  free(W);
  if (n_limited) *n_limited = nlim;
  return err;
}

/* domain integrals with the LGL quadrature:
 * out = [KE/|Omega|, enstrophy/|Omega|, int S, int rho, int rho E, |Omega|,
 *        int (mu(T)/mu) (div v)^2 / |Omega|, int (mu(T)/mu) |omega|^2 / |Omega|] (the
 *        integrals of Eqs. TGV_DD and TGV_SD; mu(T)/mu = 1 without Sutherland's law);
 *        vorticity from element-local derivatives. */
int or_diagnostics(const or_problem* P, const double* u, double* out) {
  basis b;
  make_basis(P, &b);
  int dim = b.dim, N = b.N, np = b.np;
  double vol = 0.0, ke = 0.0, ens = 0.0, ent = 0.0, mass = 0.0, en = 0.0, dil = 0.0, sol = 0.0;
  int err = 0;
  for (int64_t k = 0; k < P->K; ++k) {
    for (int node = 0; node < np; ++node) {
      double wq = 1.0;
      for (int d = 0; d < dim; ++d) wq *= b.w[line_pos(&b, d, node)];
      double Jn = P->J[(size_t)k * np + node];
      double uu[OR_MAX_NV];
      or_prim q;
      node_u(&b, u, k, node, uu);
      if (or_cons_to_prim(P, uu, &q)) err = 1;
      double v2 = 0.0;
      for (int d = 0; d < dim; ++d) v2 += q.v[d] * q.v[d];
      /* grad v: dv_a/dx_x = (1/J) sum_d Ja^d_x (D_d v_a) */
      double gv[3][3] = {{0}};
      for (int a = 0; a < dim; ++a)
        for (int d = 0; d < dim; ++d) {
          int s = ipow(N + 1, d), pos = line_pos(&b, d, node), base = node - pos * s;
          double dv = 0.0;
          for (int l = 0; l <= N; ++l) {
            double um[OR_MAX_NV];
            or_prim qm;
            node_u(&b, u, k, base + l * s, um);
            or_cons_to_prim(P, um, &qm);
            dv += b.D[pos * (N + 1) + l] * qm.v[a];
          }
          double n[3];
          node_metric(P, &b, k, d, node, n);
          for (int x = 0; x < dim; ++x) gv[a][x] += n[x] * dv / Jn;
        }
      double w2;
      if (dim == 3) {
        double wx = gv[2][1] - gv[1][2], wy = gv[0][2] - gv[2][0], wz = gv[1][0] - gv[0][1];
        w2 = wx * wx + wy * wy + wz * wz;
      } else {
        double wz = gv[1][0] - gv[0][1];
        w2 = wz * wz;
      }
      double div = 0.0;
      for (int a = 0; a < dim; ++a) div += gv[a][a];
      double dV = wq * Jn;
      vol += dV;
      ke += dV * 0.5 * q.rho * v2;
      ens += dV * 0.5 * q.rho * w2;
      ent += P->n_species == 0 ? dV * or_entropy(P, &q) : 0.0;
      mass += dV * q.rho;
      en += dV * q.rhoE;
      double mr = P->n_species == 0 ? mu_ratio(P, &q) : 1.0;
      dil += dV * mr * div * div;
      sol += dV * mr * w2;
    }
  }
  out[0] = ke / vol; out[1] = ens / vol; out[2] = ent; out[3] = mass; out[4] = en;
  out[5] = vol; out[6] = dil / vol; out[7] = sol / vol;
  return err;
}

/* temperature of every node (mixtures: Newton from 1000 K; one gas: p / rho) */
int or_temperature_field(const or_problem* P, const double* u, double* T) {
  basis b;
  make_basis(P, &b);
  int err = 0;
  for (int64_t k = 0; k < P->K; ++k)
    for (int node = 0; node < b.np; ++node) {
      double uu[OR_MAX_NV];
      or_prim q;
      node_u(&b, u, k, node, uu);
      err |= or_cons_to_prim(P, uu, &q);
      T[(size_t)k * b.np + node] = q.T;
    }
  return err;
}
