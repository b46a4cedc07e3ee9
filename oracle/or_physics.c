/*
 * Oracle (test infrastructure only): pointwise physics.
 *
 * Conserved variables U = (rho_1..rho_Ns, rho v, rho E) (Eq. Uconserv);
 * advective flux (Eq. adevctive_flux); E = e + |v|^2/2 (Eq. total_energy);
 * e = sum rho_s e_s / rho (Eq. internal_energies); Dalton p = sum rho_s R_s T
 * (Eq. eos).  With n_species == 0 the gas is a single calorically perfect
 * gas, p = (gamma-1)(rho E - rho|v|^2/2).
 *
 * Readings where the paper names a flux without defining it:
 *   EC volume flux: Ranocha's entropy-conserving, kinetic-energy-preserving
 *     flux (ideal gas), logarithmic means evaluated by the artanh series for
 *     nearly equal arguments (|x-y|^2/(x+y)^2 < 1e-4) and the closed form
 *     otherwise;
 *   mixture volume flux: Ducros split form {{rho phi}}{{v.n}} + {{p}} n;
 *   LLF: 0.5 (f_L + f_R).n - 0.5 lambda (u_R - u_L),
 *     lambda = max(|v_L.n| + c_L |n|, |v_R.n| + c_R |n|);
 *   HLLC: Toro's three-wave solver with Davis speed estimates, evaluated
 *     along n/|n| and scaled by |n|.
 * Mixture thermodynamics (stand-in for the RRHO database of the appendix,
 * Eq. Internal_energy): each species has cp/R = a1 + a2 T + .. + a5 T^4 and
 *   e_s(T) = R_s (a1 T + a2 T^2/2 + a3 T^3/3 + a4 T^4/4 + a5 T^5/5 + a6 - T).
 * T is recovered from e by Newton iteration (stop |dT| <= 1e-12 T, at most 50
 * steps, T kept in [200, 1e4] K).
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

#define OR_RU 8.314462618

double or_R_univ(void) { return OR_RU; }

int or_nv(int dim, int n_species) { return (n_species > 0 ? n_species : 1) + dim + 1; }

double or_species_energy(const double* sp, double T) {
  double R = OR_RU / sp[0];
  const double* a = sp + 1;
  double h = a[0] * T + a[1] * T * T / 2.0 + a[2] * T * T * T / 3.0 +
             a[3] * T * T * T * T / 4.0 + a[4] * T * T * T * T * T / 5.0 + a[5];
  return R * (h - T);
}

double or_species_cv(const double* sp, double T) {
  double R = OR_RU / sp[0];
  const double* a = sp + 1;
  double cp = a[0] + a[1] * T + a[2] * T * T + a[3] * T * T * T + a[4] * T * T * T * T;
  return R * (cp - 1.0);
}

double or_mixture_energy(int ns, const double* species, const double* Y, double T) {
  double e = 0.0;
  for (int s = 0; s < ns; ++s) e += Y[s] * or_species_energy(species + 8 * s, T);
  return e;
}

double or_mixture_cv(int ns, const double* species, const double* Y, double T) {
  double c = 0.0;
  for (int s = 0; s < ns; ++s) c += Y[s] * or_species_cv(species + 8 * s, T);
  return c;
}

int or_temperature(int ns, const double* species, const double* Y, double e, double T0,
                   double* T, int* iters) {
  double t = T0;
  for (int it = 1; it <= 50; ++it) {
    double r = or_mixture_energy(ns, species, Y, t) - e;
    double dT = r / or_mixture_cv(ns, species, Y, t);
    double tn = t - dT;
    if (tn < 200.0) tn = 200.0;
    if (tn > 1.0e4) tn = 1.0e4;
    double step = fabs(tn - t);
    t = tn;
    if (step <= 1e-12 * t) { *T = t; if (iters) *iters = it; return 0; }
  }
  *T = t;
  if (iters) *iters = 50;
  return 1;
}

int or_cons_to_prim(const or_problem* P, const double* u, or_prim* q) {
  int dim = P->dim, ns = P->n_species, nsp = ns > 0 ? ns : 1;
  double rho = 0.0;
  for (int s = 0; s < nsp; ++s) { q->rhos[s] = u[s]; rho += u[s]; }
  q->rho = rho;
  q->v[0] = q->v[1] = q->v[2] = 0.0;
  double v2 = 0.0;
  for (int d = 0; d < dim; ++d) { q->v[d] = u[nsp + d] / rho; v2 += q->v[d] * q->v[d]; }
  q->rhoE = u[nsp + dim];
  if (!(rho > 0.0)) return 1;
  if (ns == 0) {
    q->p = (P->gamma - 1.0) * (q->rhoE - 0.5 * rho * v2);
    q->T = q->p / rho;
    if (!(q->p > 0.0)) return 1;
    q->c = sqrt(P->gamma * q->p / rho);
  } else {
    double Y[OR_MAX_SPECIES], e = q->rhoE / rho - 0.5 * v2, T, Rmix = 0.0;
    for (int s = 0; s < ns; ++s) Y[s] = q->rhos[s] / rho;
    if (or_temperature(ns, P->species, Y, e, 1000.0, &T, NULL)) return 2;
    for (int s = 0; s < ns; ++s) Rmix += Y[s] * OR_RU / P->species[8 * s];
    q->T = T;
    q->p = rho * Rmix * T;
    double cv = or_mixture_cv(ns, P->species, Y, T);
    double gam = (cv + Rmix) / cv;
    q->c = sqrt(gam * q->p / rho);
  }
  return 0;
}

int or_prim_to_cons(const or_problem* P, const double* w, double* u) {
  int dim = P->dim, ns = P->n_species, nsp = ns > 0 ? ns : 1;
  double rho = 0.0, v2 = 0.0;
  for (int s = 0; s < nsp; ++s) { u[s] = w[s]; rho += w[s]; }
  for (int d = 0; d < dim; ++d) { u[nsp + d] = rho * w[nsp + d]; v2 += w[nsp + d] * w[nsp + d]; }
  if (ns == 0) {
    u[nsp + dim] = w[nsp + dim] / (P->gamma - 1.0) + 0.5 * rho * v2;
  } else {
    double Y[OR_MAX_SPECIES];
    for (int s = 0; s < ns; ++s) Y[s] = w[s] / rho;
    u[nsp + dim] = rho * (or_mixture_energy(ns, P->species, Y, w[nsp + dim]) + 0.5 * v2);
  }
  return rho > 0.0 ? 0 : 1;
}

/* contravariant advective flux f(u) . n */
void or_phys_flux(const or_problem* P, const or_prim* q, const double* u, const double* n,
                  double* f) {
  int dim = P->dim, nsp = P->n_species > 0 ? P->n_species : 1;
  double vn = 0.0;
  for (int d = 0; d < dim; ++d) vn += q->v[d] * n[d];
  for (int s = 0; s < nsp; ++s) f[s] = u[s] * vn;
  for (int d = 0; d < dim; ++d) f[nsp + d] = u[nsp + d] * vn + q->p * n[d];
  f[nsp + dim] = (q->rhoE + q->p) * vn;
}

/* logarithmic mean (y - x) / ln(y / x) */
double or_ln_mean(double x, double y) {
  double f2 = (x - y) * (x - y) / ((x + y) * (x + y));
  if (f2 < 1e-4)
    return (x + y) / (2.0 + f2 * (2.0 / 3.0 + f2 * (2.0 / 5.0 + f2 * (2.0 / 7.0))));
  return (y - x) / log(y / x);
}

void or_volume_flux(const or_problem* P, const double* uL, const or_prim* qL,
                    const double* uR, const or_prim* qR, const double* n, double* f) {
  int dim = P->dim, ns = P->n_species, nsp = ns > 0 ? ns : 1;
  int nv = nsp + dim + 1;
  if (P->volume_flux == OR_VF_CENTRAL) {
    double fL[OR_MAX_NV], fR[OR_MAX_NV];
    or_phys_flux(P, qL, uL, n, fL);
    or_phys_flux(P, qR, uR, n, fR);
    for (int v = 0; v < nv; ++v) f[v] = 0.5 * (fL[v] + fR[v]);
    return;
  }
  double vnL = 0.0, vnR = 0.0;
  for (int d = 0; d < dim; ++d) { vnL += qL->v[d] * n[d]; vnR += qR->v[d] * n[d]; }
  if (P->volume_flux == OR_VF_DUCROS) {
    double vn = 0.5 * (vnL + vnR);
    for (int s = 0; s < nsp; ++s) f[s] = 0.5 * (uL[s] + uR[s]) * vn;
    for (int d = 0; d < dim; ++d)
      f[nsp + d] = 0.5 * (uL[nsp + d] + uR[nsp + d]) * vn + 0.5 * (qL->p + qR->p) * n[d];
    f[nsp + dim] = 0.5 * (qL->rhoE + qL->p + qR->rhoE + qR->p) * vn;
    return;
  }
  if (P->volume_flux == OR_VF_KG || P->volume_flux == OR_VF_PIROZZOLI) {
    /* Kennedy-Gruber and Pirozzoli split forms (single gas), as two-point fluxes: products
     * of arithmetic means, {{rho}} {{v.n}} for mass; momentum f_rho {{v}} + {{p}} n; energy
     * f_rho {{E/rho}} + {{p}} {{v.n}} (Kennedy-Gruber) or f_rho {{(E + p)/rho}} (Pirozzoli) */
    double frho = 0.5 * (qL->rho + qR->rho) * 0.5 * (vnL + vnR);
    f[0] = frho;
    for (int d = 0; d < dim; ++d)
      f[1 + d] = frho * 0.5 * (qL->v[d] + qR->v[d]) + 0.5 * (qL->p + qR->p) * n[d];
    if (P->volume_flux == OR_VF_KG)
      f[1 + dim] = frho * 0.5 * (qL->rhoE / qL->rho + qR->rhoE / qR->rho) +
                   0.5 * (qL->p + qR->p) * 0.5 * (vnL + vnR);
    else
      f[1 + dim] = frho * 0.5 * ((qL->rhoE + qL->p) / qL->rho + (qR->rhoE + qR->p) / qR->rho);
    return;
  }
  if (P->volume_flux == OR_VF_MORINISHI) {
    /* Morinishi's form (single gas): mass {{rho v}}.n in divergence form, momentum
     * f_rho {{v}} + {{p}} n (skew-symmetric), enthalpy g/(g-1) {{p v}}.n in divergence
     * form and kinetic energy f_rho v_L.v_R / 2 */
    double frho = 0.0, pv = 0.0, vv = 0.0;
    for (int d = 0; d < dim; ++d) {
      frho += 0.5 * (uL[1 + d] + uR[1 + d]) * n[d];
      vv += qL->v[d] * qR->v[d];
    }
    pv = 0.5 * (qL->p * vnL + qR->p * vnR);
    f[0] = frho;
    for (int d = 0; d < dim; ++d)
      f[1 + d] = frho * 0.5 * (qL->v[d] + qR->v[d]) + 0.5 * (qL->p + qR->p) * n[d];
    f[1 + dim] = P->gamma / (P->gamma - 1.0) * pv + frho * 0.5 * vv;
    return;
  }
  /* Ranocha EC flux (single ideal gas) */
  double g = P->gamma;
  double rho_m = or_ln_mean(qL->rho, qR->rho);
  double beta_m = or_ln_mean(qL->rho / qL->p, qR->rho / qR->p); /* mean of rho/p */
  double vv = 0.0;
  for (int d = 0; d < dim; ++d) vv += qL->v[d] * qR->v[d];
  double frho = rho_m * 0.5 * (vnL + vnR);
  f[0] = frho;
  for (int d = 0; d < dim; ++d)
    f[1 + d] = frho * 0.5 * (qL->v[d] + qR->v[d]) + 0.5 * (qL->p + qR->p) * n[d];
  f[1 + dim] = frho * (0.5 * vv + 1.0 / ((g - 1.0) * beta_m)) + 0.5 * (qL->p * vnR + qR->p * vnL);
  (void)nv;
}

void or_surface_flux(const or_problem* P, const double* uL, const or_prim* qL,
                     const double* uR, const or_prim* qR, const double* n, double* f) {
  int dim = P->dim, nsp = P->n_species > 0 ? P->n_species : 1;
  int nv = nsp + dim + 1;
  if (P->surface_flux == OR_SF_EC) { or_volume_flux(P, uL, qL, uR, qR, n, f); return; }
  double nn = 0.0;
  for (int d = 0; d < dim; ++d) nn += n[d] * n[d];
  nn = sqrt(nn);
  double vnL = 0.0, vnR = 0.0;
  for (int d = 0; d < dim; ++d) { vnL += qL->v[d] * n[d]; vnR += qR->v[d] * n[d]; }
  double fL[OR_MAX_NV], fR[OR_MAX_NV];
  or_phys_flux(P, qL, uL, n, fL);
  or_phys_flux(P, qR, uR, n, fR);
  if (P->surface_flux == OR_SF_LLF) {
    double lL = fabs(vnL) + qL->c * nn, lR = fabs(vnR) + qR->c * nn;
    double lam = lL > lR ? lL : lR;
    for (int v = 0; v < nv; ++v) f[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * lam * (uR[v] - uL[v]);
    return;
  }
  /* HLLC along the unit normal, scaled by |n| */
  double uL_n = vnL / nn, uR_n = vnR / nn, nh[3] = {0, 0, 0};
  for (int d = 0; d < dim; ++d) nh[d] = n[d] / nn;
  double SL = fmin(uL_n - qL->c, uR_n - qR->c);
  double SR = fmax(uL_n + qL->c, uR_n + qR->c);
  if (SL >= 0.0) { for (int v = 0; v < nv; ++v) f[v] = fL[v]; return; }
  if (SR <= 0.0) { for (int v = 0; v < nv; ++v) f[v] = fR[v]; return; }
  if (P->surface_flux == OR_SF_HLL) {
    /* HLL (Harten, Lax, van Leer) with the same Davis speeds: one intermediate state */
    for (int v = 0; v < nv; ++v)
      f[v] = (SR * fL[v] - SL * fR[v] + nn * SL * SR * (uR[v] - uL[v])) / (SR - SL);
    return;
  }
  double Ss = (qR->p - qL->p + qL->rho * uL_n * (SL - uL_n) - qR->rho * uR_n * (SR - uR_n)) /
              (qL->rho * (SL - uL_n) - qR->rho * (SR - uR_n));
  const double* uK = Ss >= 0.0 ? uL : uR;
  const or_prim* qK = Ss >= 0.0 ? qL : qR;
  const double* fK = Ss >= 0.0 ? fL : fR;
  double SK = Ss >= 0.0 ? SL : SR, unK = Ss >= 0.0 ? uL_n : uR_n;
  double fac = (SK - unK) / (SK - Ss);
  double us[OR_MAX_NV];
  for (int s = 0; s < nsp; ++s) us[s] = uK[s] * fac;
  for (int d = 0; d < dim; ++d) us[nsp + d] = qK->rho * fac * (qK->v[d] + (Ss - unK) * nh[d]);
  us[nsp + dim] = qK->rho * fac *
                  (qK->rhoE / qK->rho + (Ss - unK) * (Ss + qK->p / (qK->rho * (SK - unK))));
  /* fK already carries |n|; the jump term is scaled by |n| */
  for (int v = 0; v < nv; ++v) f[v] = fK[v] + nn * SK * (us[v] - uK[v]);
}

void or_entropy_vars(const or_problem* P, const or_prim* q, double* wv) {
  int dim = P->dim;
  double g = P->gamma, v2 = 0.0;
  for (int d = 0; d < dim; ++d) v2 += q->v[d] * q->v[d];
  double s = log(q->p) - g * log(q->rho);
  wv[0] = (g - s) / (g - 1.0) - 0.5 * q->rho * v2 / q->p;
  for (int d = 0; d < dim; ++d) wv[1 + d] = q->rho * q->v[d] / q->p;
  wv[1 + dim] = -q->rho / q->p;
}

double or_entropy(const or_problem* P, const or_prim* q) {
  double s = log(q->p) - P->gamma * log(q->rho);
  return -q->rho * s / (P->gamma - 1.0);
}

/* single-state entry points used by the pin tests */
int or_flux_pair(const or_problem* P, const double* uL, const double* uR, const double* n,
                 int which, double* f) {
  or_prim qL, qR;
  if (or_cons_to_prim(P, uL, &qL) || or_cons_to_prim(P, uR, &qR)) return 1;
  if (which == 0) or_volume_flux(P, uL, &qL, uR, &qR, n, f);
  else if (which == 1) or_surface_flux(P, uL, &qL, uR, &qR, n, f);
  else or_phys_flux(P, &qL, uL, n, f);
  return 0;
}

int or_entropy_vars_u(const or_problem* P, const double* u, double* wv) {
  or_prim q;
  if (or_cons_to_prim(P, u, &q)) return 1;
  or_entropy_vars(P, &q, wv);
  return 0;
}

/* vectorised helpers for the pin tests: e(T), cv(T), T(e) over n states */
int or_mixture_eval(int ns, const double* species, int n, const double* Y, const double* T,
                    double* e, double* cv) {
  for (int i = 0; i < n; ++i) {
    e[i] = or_mixture_energy(ns, species, Y + (size_t)i * ns, T[i]);
    cv[i] = or_mixture_cv(ns, species, Y + (size_t)i * ns, T[i]);
  }
  return 0;
}

int or_mixture_temperature(int ns, const double* species, int n, const double* Y,
                           const double* e, const double* T0, double* T, int* iters) {
  int bad = 0;
  for (int i = 0; i < n; ++i)
    bad |= or_temperature(ns, species, Y + (size_t)i * ns, e[i], T0 ? T0[i] : 1000.0, T + i,
                          iters ? iters + i : NULL);
  return bad;
}
