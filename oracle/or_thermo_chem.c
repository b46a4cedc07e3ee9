/*
 * Oracle (test infrastructure only): finite-rate chemistry source (appendix, Chemical
 * Kinetics: Eqs. chemreact, nrp, forward_rate, backward, kedef, calc_prod) for the
 * seeded stand-in mechanism.  Readings where the paper is garbled or silent:
 *   - concentrations in mol/cm^3 (the units of Park-type rate constants):
 *     c_s = 1e-6 rho_s / W_s (rho_s in kg/m^3, W_s in kg/mol);
 *   - k_f = A T^beta exp(-theta/T) (theta = E/R_u); k_b = k_f / K_c (Eq. backward prints
 *     k_f = K_eq k_b with the roles swapped);
 *   - ln K_c = -sum_s dnu_s g_s/(R_u T) + (sum_s dnu_s) ln(1e-6 p0/(R_u T)) with the
 *     standard-state Gibbs energy of each species from its thermally perfect polynomial,
 *     g/(R T) = h/(R T) - s/R (h/(RT) = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5
 *     + a6/T, s/R = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7), p0 = 101325 Pa
 *     (Eq. kedef prints 1 Pa);
 *   - rate of progress R_r = [k_f prod c^nu' - k_b prod c^nu''] (times sum_s eff_s c_s
 *     for third-body reactions, Eq. nrp);
 *   - omega_s = 1e6 W_s sum_r (nu''_sr - nu'_sr) R_r in kg/(m^3 s) (Eq. calc_prod, sum
 *     over reactions);
 *   - point-implicit source: S_s = omega_s / (1 + dt max(0, -d omega_s / d rho_s)) with
 *     the analytic diagonal Jacobian at fixed T.
 * Reaction rows: [nu'(5), nu''(5), third_body, eff(5), A, beta, theta].
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

#define NSP_CHEM 5
#define OR_P0 101325.0

static double g_over_RT(const double* sp, double T) {
  const double* a = sp + 1;
  double h = a[0] + a[1] * T / 2.0 + a[2] * T * T / 3.0 + a[3] * T * T * T / 4.0 +
             a[4] * T * T * T * T / 5.0 + a[5] / T;
  double s = a[0] * log(T) + a[1] * T + a[2] * T * T / 2.0 + a[3] * T * T * T / 3.0 +
             a[4] * T * T * T * T / 4.0 + a[6];
  return h - s;
}

/* omega (kg/m^3/s) and the diagonal d omega_s / d rho_s at fixed T */
int or_chem_omega(const double* species, int nr, const double* reac, const double* rhos, double T,
                  double* omega, double* jdiag) {
  double c[NSP_CHEM], g[NSP_CHEM];
  for (int s = 0; s < NSP_CHEM; ++s) {
    c[s] = 1e-6 * rhos[s] / species[8 * s];
    g[s] = g_over_RT(species + 8 * s, T);
    omega[s] = 0.0;
    if (jdiag) jdiag[s] = 0.0;
  }
  for (int r = 0; r < nr; ++r) {
    const double* row = reac + 19 * r;
    const double* nf = row;
    const double* nb = row + 5;
    const int tb = row[10] != 0.0;
    const double* eff = row + 11;
    const double A = row[16], beta = row[17], theta = row[18];
    double kf = A * pow(T, beta) * exp(-theta / T);
    double dg = 0.0, dn = 0.0;
    for (int s = 0; s < NSP_CHEM; ++s) {
      dg += (nb[s] - nf[s]) * g[s];
      dn += nb[s] - nf[s];
    }
    double lnKc = -dg + dn * log(1e-6 * OR_P0 / (or_R_univ() * T));
    double kb = kf / exp(lnKc);
    double pf = kf, pb = kb;
    for (int s = 0; s < NSP_CHEM; ++s) {
      pf *= pow(c[s], nf[s]);
      pb *= pow(c[s], nb[s]);
    }
    double M = 1.0;
    if (tb) {
      M = 0.0;
      for (int s = 0; s < NSP_CHEM; ++s) M += eff[s] * c[s];
    }
    double Rr = (pf - pb) * M;
    for (int s = 0; s < NSP_CHEM; ++s) omega[s] += 1e6 * species[8 * s] * (nb[s] - nf[s]) * Rr;
    if (jdiag) {
      /* d R_r / d c_s, then d omega_s / d rho_s = dnu_s dR_r/dc_s (the 1e6 W_s and 1e-6/W_s cancel) */
      for (int s = 0; s < NSP_CHEM; ++s) {
        double dpf = nf[s] > 0 ? kf * nf[s] * pow(c[s], nf[s] - 1) : 0.0;
        double dpb = nb[s] > 0 ? kb * nb[s] * pow(c[s], nb[s] - 1) : 0.0;
        for (int q = 0; q < NSP_CHEM; ++q) {
          if (q == s) continue;
          dpf *= pow(c[q], nf[q]);
          dpb *= pow(c[q], nb[q]);
        }
        double dR = (dpf - dpb) * M + (tb ? (pf - pb) * eff[s] : 0.0);
        jdiag[s] += (nb[s] - nf[s]) * dR;
      }
    }
  }
  return 0;
}

int or_chem_source(const double* species, int nr, const double* reac, const double* rhos, double T,
                   double dt, double* S) {
  double om[NSP_CHEM], jd[NSP_CHEM];
  or_chem_omega(species, nr, reac, rhos, T, om, jd);
  for (int s = 0; s < NSP_CHEM; ++s) {
    double d = dt > 0.0 && -jd[s] > 0.0 ? -jd[s] : 0.0;
    S[s] = om[s] / (1.0 + dt * d);
  }
  return 0;
}

/* vectorised entry for the pin tests: n states of (rho_s[5], T) */
int or_chem_eval(const double* species, int nr, const double* reac, int n, const double* rhos,
                 const double* T, double dt, double* omega, double* jdiag, double* S) {
  for (int i = 0; i < n; ++i) {
    or_chem_omega(species, nr, reac, rhos + 5 * i, T[i], omega + 5 * i, jdiag + 5 * i);
    or_chem_source(species, nr, reac, rhos + 5 * i, T[i], dt, S + 5 * i);
  }
  return 0;
}
