/*
 * Plain FP64 CPU oracle of the entropy-stable DGSEM right-hand side
 * (H3PC, arXiv 2511.17551).  TEST INFRASTRUCTURE ONLY: the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark call it; the GPU
 * library never links, includes or calls anything in this directory.
 *
 * Every routine is the simplest loop nest that follows the paper's
 * statement of the method (section "Methodology", Eqs. mapped_equation,
 * strong_form, fluxes_discrete_strong, differencing, fluxdiffcons, DGvec,
 * fluxes_discrete_with_fv, finitevolumeflux, auxil, auxstrongf) and, where
 * the paper is silent or garbled, the readings written next to each routine.
 *
 * Layouts (all row-major, node index fastest):
 *   node  = i + (N+1) j + (N+1)^2 k              (x fastest)
 *   u     [K][nv][np]   conserved (rho_1..rho_ns, rho v_1..rho v_dim, rho E)
 *   w     [K][nv][np]   primitive (rho_1..rho_ns, v_1..v_dim, p  or  T)
 *   xyz   [K][dim][np]  node coordinates
 *   Ja    [K][dim][dim][np]  Ja[k][i][n][node] = J d(xi_i)/d(x_n)
 *   J     [K][np]
 *   faces ordered -xi,+xi,-eta,+eta,-zeta,+zeta;  nbr_elem[k][f] >= 0 is the
 *   neighbour element, < 0 encodes boundary id  -(bc+1).
 */
#ifndef DG_ORACLE_H
#define DG_ORACLE_H
#include <stdint.h>

#define OR_MAX_N 15
#define OR_MAX_SPECIES 8
#define OR_MAX_NV (OR_MAX_SPECIES + 4)

enum { OR_EULER = 0, OR_NAVIER_STOKES = 1 };
enum { OR_VF_RANOCHA = 0, OR_VF_DUCROS = 1, OR_VF_CENTRAL = 2, OR_VF_KG = 3, OR_VF_PIROZZOLI = 4,
       OR_VF_MORINISHI = 5 };
enum { OR_SF_LLF = 0, OR_SF_HLLC = 1, OR_SF_EC = 2, OR_SF_HLL = 3 };
/* no-slip walls: the advective part is the slip-wall flux, the no-slip condition enters
 * through the viscous terms; isothermal walls take T_wall from the bc state's p / rho */
enum { OR_BC_INFLOW = 1, OR_BC_OUTFLOW = 2, OR_BC_SLIP_WALL = 3, OR_BC_NOSLIP_ADIABATIC = 4,
       OR_BC_ISOTHERMAL = 5 };

typedef struct {
  int dim, N;
  int64_t K;
  int n_species;       /* 0: single calorically perfect gas */
  int equations;       /* OR_EULER | OR_NAVIER_STOKES */
  int volume_flux;     /* OR_VF_* */
  int surface_flux;    /* OR_SF_* */
  double gamma;        /* ideal gas only */
  double mu, Pr;       /* NS: constant dynamic viscosity, Prandtl number */
  double alpha_max;    /* > 0 switches on DG / subcell-FV blending */
  const int64_t* nbr_elem;  /* [K][2dim] */
  const int8_t* nbr_face;   /* [K][2dim] */
  int n_bc;
  const int* bc_kind;       /* [n_bc] */
  const double* bc_prim;    /* [n_bc][nv] primitive external states */
  const double* species;    /* [ns][8] = W (kg/mol), a1..a7 */
  const double* Ja;         /* [K][dim][dim][np] */
  const double* J;          /* [K][np] */
  double alpha_override;    /* >= 0: use this blending factor on every element */
  int n_reactions;          /* finite-rate chemistry (5 species), 0 = frozen */
  const double* reactions;  /* [n_reactions][19] */
  double chem_dt;           /* point-implicit time scale of the source; 0 = explicit */
  double positivity_eps;    /* > 0: Zhang-Shu positivity limiter after every RK stage: one gas,
                               density and pressure >= eps; mixtures, partial densities >= eps
                               (or their element mean, if smaller) and T >= OR_T_FLOOR */
  /* NS, one gas: s > 0 switches on Sutherland's law (Eq. sutherland),
   * mu(T) = mu (1 + s) th^1.5 / (th + s), th = (p / rho) / rt; mu is the viscosity at th = 1 */
  double sutherland_s, sutherland_rt;
  int indicator_var;        /* shock-indicator quantity: 0 = rho p, 1 = p */
} or_problem;

typedef struct {
  double rho;                     /* total density */
  double rhos[OR_MAX_SPECIES];    /* species densities (mixtures) */
  double v[3];
  double p;
  double T;                       /* mixtures: temperature; ideal gas: p/rho */
  double c;                       /* frozen sound speed */
  double rhoE;
} or_prim;

/* ---- basis (or_basis.c) ---- */
void or_legendre(int n, double x, double* P, double* dP);
int or_lgl(int N, double* x, double* w);
void or_dmat(int N, const double* x, double* D);
void or_vandermonde_legendre(int N, const double* x, double* V);
int or_invert(int n, const double* A, double* Ainv);

/* ---- geometry (or_geometry.c) ---- */
int or_geometry(int dim, int N, int64_t K, const double* xyz, double* Ja, double* J);

/* ---- physics (or_physics.c) ---- */
int or_nv(int dim, int n_species);
double or_R_univ(void);
double or_species_energy(const double* sp, double T);  /* e_s(T) per unit mass */
double or_species_cv(const double* sp, double T);
double or_mixture_energy(int ns, const double* species, const double* Y, double T);
double or_mixture_cv(int ns, const double* species, const double* Y, double T);
int or_temperature(int ns, const double* species, const double* Y, double e, double T0,
                   double* T, int* iters);
int or_cons_to_prim(const or_problem* P, const double* u, or_prim* q);
int or_prim_to_cons(const or_problem* P, const double* w, double* u);
void or_phys_flux(const or_problem* P, const or_prim* q, const double* u, const double* n,
                  double* f);
void or_volume_flux(const or_problem* P, const double* uL, const or_prim* qL,
                    const double* uR, const or_prim* qR, const double* n, double* f);
void or_surface_flux(const or_problem* P, const double* uL, const or_prim* qL,
                     const double* uR, const or_prim* qR, const double* n, double* f);
double or_ln_mean(double x, double y);
void or_entropy_vars(const or_problem* P, const or_prim* q, double* wv);
double or_entropy(const or_problem* P, const or_prim* q);
int or_flux_pair(const or_problem* P, const double* uL, const double* uR, const double* n,
                 int which, double* f);
int or_entropy_vars_u(const or_problem* P, const double* u, double* wv);
int or_mixture_eval(int ns, const double* species, int n, const double* Y, const double* T,
                    double* e, double* cv);
int or_mixture_temperature(int ns, const double* species, int n, const double* Y,
                           const double* e, const double* T0, double* T, int* iters);

/* ---- right-hand side, time stepping, diagnostics (or_rhs.c) ---- */
int or_prim_to_cons_field(const or_problem* P, const double* w, double* u);
int or_rhs(const or_problem* P, const double* u, double* rhs, double* alpha_out,
           double* gradW_out);
int or_indicator(const or_problem* P, const double* u, double* alpha);
double or_max_dt(const or_problem* P, const double* u, double cfl);
int or_step_rk(const or_problem* P, double* u, int nsteps, double cfl, double dt_fixed,
               double* t);
int or_diagnostics(const or_problem* P, const double* u, double* out);
#define OR_T_FLOOR 200.0  /* temperature floor of the mixture limiter (the Newton clamp) */
int or_positivity(const or_problem* P, double* u, double eps, int* n_limited);
void or_ck45(double* A, double* B, double* c);
int or_temperature_field(const or_problem* P, const double* u, double* T);

/* ---- finite-rate chemistry (or_thermo_chem.c) ---- */
int or_chem_omega(const double* species, int nr, const double* reac, const double* rhos, double T,
                  double* omega, double* jdiag);
int or_chem_source(const double* species, int nr, const double* reac, const double* rhos, double T,
                   double dt, double* S);
int or_chem_eval(const double* species, int nr, const double* reac, int n, const double* rhos,
                 const double* T, double dt, double* omega, double* jdiag, double* S);

/* ---- learned surrogates: temperature (1 output), chemistry source (10) (or_mlp.c) ---- */
int or_mlp_nparams(void);
int or_mlp_nparams_n(int n_out);
int or_mlp_forward_n(const double* p, int n_out, int n, const double* X, double* Y);
int or_mlp_forward_sd_n(const double* p, int n_out, int n, const double* X, double u, double u_flip,
                        double eps_t, double x_rel, double* Y, double* SD, double* FLIP);
double or_mlp_loss_grad_n(const double* p, int n_out, int n, const double* X, const double* t,
                          double* g);
double or_gelu(double x);
double or_gelu_d(double x);
void or_mlp_forward(const double* p, int n, const double* X, double* y);
double or_mlp_loss_grad(const double* p, int n, const double* X, const double* t, double* g);
void or_adam_step(double* p, double* m, double* v, const double* g, int np_, int step, double lr,
                  double b1, double b2, double eps);

int or_set_threads(int n);
#endif
