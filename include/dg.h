/*
 * dg.h -- C ABI of libdg, a GB300 (sm_103a) implementation of the right-hand
 * side and low-storage Runge-Kutta stepping of the entropy-stable DGSEM of
 * Peyvan, Shukla & Karniadakis, "H3PC" (arXiv 2511.17551).
 *
 * The calls follow the paper's problem statement  dU/dt + div F = S  with
 * boundary data U = Phi and initial data U(x,0) = Psi (Methodology, Eq. system)
 * and its semi-discrete form (Eqs. strong_form, fluxes_discrete_strong).
 *
 * Conventions shared by every entry point
 *  - Layouts are row-major with the node index fastest; node = i + (N+1) j
 *    + (N+1)^2 k.  A state is [K][nv][np]: nv = n_sp + dim + 1 conserved
 *    variables (rho_1..rho_nsp, rho v_1..rho v_dim, rho E; Eq. Uconserv),
 *    n_sp = max(1, n_species), np = (N+1)^dim.  Primitive states use the same
 *    shape with (rho_s, v, p) for one gas and (rho_s, v, T) for mixtures.
 *  - Faces are ordered -xi,+xi,-eta,+eta,-zeta,+zeta.  nbr_elem[k][f] >= 0
 *    names the neighbour element; a negative value -(b+1) names boundary b.
 *    Face f of k must meet face f^1 of its neighbour with orientation 0
 *    (conforming, aligned hexahedra/quadrilaterals).
 *  - Host pointers passed to dg_init_mesh are read during the call and not
 *    retained.  Device pointers passed to dg_rhs are borrowed for the call.
 *    libdg owns every internal buffer (state, RK register, metric terms,
 *    gradients, temperature cache, surrogate weights) and frees them in
 *    dg_destroy.
 *  - Arguments are validated before any work is queued; an invalid call
 *    returns DG_EINVAL and changes nothing.  Work is queued on the context
 *    stream.  Errors detected on the device (non-physical state, Newton
 *    failure) are latched in a device status word and returned by the next
 *    dg_sync / dg_step_rk / dg_get_state; kernels never trap.
 *  - No call falls back to a CPU implementation: without a usable CUDA device
 *    dg_init_mesh returns DG_ECUDA.
 */
#ifndef DG_H
#define DG_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_ctx dg_ctx;

typedef enum {
  DG_OK = 0,
  DG_EINVAL = 1,    /* bad argument or unsupported combination */
  DG_ENOMEM = 2,    /* device allocation failed */
  DG_ECUDA = 3,     /* CUDA runtime error, or no device */
  DG_ENONPHYS = 4,  /* rho <= 0, p <= 0 or NaN met on the device */
  DG_ENEWTON = 5,   /* temperature Newton iteration did not converge */
  DG_ETIMEOUT = 6,  /* a bounded wait on the device ran out */
  DG_ESTATE = 7     /* call out of order (e.g. no state set) */
} dg_status;

enum { DG_EULER = 0, DG_NAVIER_STOKES = 1 };
/* two-point volume flux F# of Eq. fluxdiffcons */
/* DG_VF_CENTRAL = {{f(u).n}}, the standard DG form; DG_VF_DUCROS = {{u}}{{v.n}} + {{p}} */
enum { DG_VF_RANOCHA = 0, DG_VF_DUCROS = 1, DG_VF_CENTRAL = 2,
       /* split forms the paper lists beside Ducros (one gas): Kennedy-Gruber
          ({{rho}}{{v.n}}, f_rho {{v}} + {{p}} n, f_rho {{E/rho}} + {{p}}{{v.n}}), Pirozzoli
          (energy f_rho {{(E + p)/rho}}) and Morinishi (f_rho = {{rho v}}.n, f_rho {{v}} + {{p}} n,
          g/(g-1) {{p v}}.n + f_rho v_L.v_R / 2) */
       DG_VF_KG = 3, DG_VF_PIROZZOLI = 4, DG_VF_MORINISHI = 5 };
/* interface flux F^Rie of Eqs. riemann_problem1-3; DG_SF_EC uses F# itself */
enum { DG_SF_LLF = 0, DG_SF_HLLC = 1, DG_SF_EC = 2,
       /* HLL with the Davis wave speeds (the third solver the paper names) */
       DG_SF_HLL = 3 };
enum { DG_FP64 = 0, DG_MIXED = 1 };
/* temperature floor of the mixture positivity limiter: the clamp of the temperature solve (K) */
#define DG_T_FLOOR 200.0
enum { DG_THERMO_NEWTON = 0, DG_THERMO_MLP = 1 };
/* boundary kinds (weak, through the numerical fluxes).  Inflow: advective flux f(u_ext).n;
 * outflow: f(u).n; walls: the mirror state (normal velocity reversed) through the Riemann
 * solver.  Navier-Stokes adds the BR1 boundary value W* of W = (v, p/rho) and the viscous
 * boundary flux Fv*: inflow W* = (W + W_ext)/2, Fv* = mean of f^v of the interior gradient
 * with the interior and with the external state; outflow W* = W, Fv* = f^v; no-slip walls
 * W* = (0, p/rho) (adiabatic) or (0, T_wall) (isothermal, T_wall = p/rho of the id's
 * bc_prim state), Fv* = f^v of the interior gradient at zero velocity, heat flux 0 on an
 * adiabatic wall.  DG_BC_SLIP_WALL is Euler-only. */
enum { DG_BC_INFLOW = 1, DG_BC_OUTFLOW = 2, DG_BC_SLIP_WALL = 3, DG_BC_NOSLIP_ADIABATIC = 4,
       DG_BC_ISOTHERMAL = 5 };

typedef struct {
  int dim;                  /* 2 or 3 */
  int N;                    /* polynomial degree on LGL nodes, 1..7 */
  int64_t K;                /* number of elements, >= 1, < 2^31 */
  const double* node_xyz;   /* host [K][dim][np]: geometry sampled at the LGL nodes
                               returned by dg_lgl_nodes (degree-N map, Eq. mapp) */
  const int64_t* nbr_elem;  /* host [K][2 dim] */
  const int8_t* nbr_face;   /* host [K][2 dim], must equal f^1 */
  const int8_t* nbr_orient; /* host [K][2 dim] or NULL; must be 0 */
} dg_mesh_desc;

typedef struct {
  int equations;            /* DG_EULER | DG_NAVIER_STOKES (one gas; no slip walls) */
  int n_species;            /* 0: one calorically perfect gas; 1..8: mixture */
  double gamma;             /* ratio of specific heats (one gas) */
  double mu, Pr;            /* Navier-Stokes: dynamic viscosity, Prandtl number */
  const double* species;    /* host [n_species][8] = W (kg/mol), a1..a7, or NULL */
  int volume_flux;          /* DG_VF_* */
  int surface_flux;         /* DG_SF_* */
  double alpha_max;         /* > 0 turns on DG / subcell-FV blending, alpha in [0, alpha_max] */
  int precision;            /* DG_FP64 | DG_MIXED (FP32 fluxes and sums, FP64 reductions) */
  int thermo;               /* DG_THERMO_NEWTON | DG_THERMO_MLP (mixtures) */
  int n_bc;                 /* number of boundary ids */
  const int* bc_kind;       /* host [n_bc]: DG_BC_* */
  const double* bc_prim;    /* host [n_bc][nv]: external primitive states */
  void* stream;             /* cudaStream_t to queue work on, or NULL for a private stream */
  const double* reactions;  /* host [n_reactions][19] finite-rate mechanism (mixtures):
                               nu'(5), nu''(5), third-body flag, efficiencies(5), A, beta,
                               theta = E/R_u (appendix, Eqs. chemreact..calc_prod), or NULL;
                               stoichiometric coefficients in {0, 1, 2, 3}, else DG_EINVAL */
  int n_reactions;          /* 0: frozen mixture; 1..64 */
  double p_ref;             /* one gas: pressure offset p_ref; the momentum components of
                               every numerical flux use p - p_ref (a constant pressure adds
                               nothing to the discrete right-hand side, so the result is the
                               same in exact arithmetic) and the pressure of the mixed form is
                               recovered from the compensated energy relative to
                               p_ref / (gamma - 1): low-Mach fluctuations keep their FP32
                               digits.  0 for none; must be 0 for mixtures. */
  double positivity_eps;    /* > 0 applies the Zhang-Shu positivity limiter (the limiter the
                               paper uses for its shock problems) to the state after every RK
                               stage of dg_step_rk, per element by scaling toward the element
                               mean (which it keeps).  One gas: density, then pressure >=
                               positivity_eps at every node.  Mixtures: partial densities >=
                               min(positivity_eps, their element mean), by one common factor,
                               then T >= DG_T_FLOOR (internal energy >= e(DG_T_FLOOR)).  The
                               next step's CFL time step uses the wave speeds of the last stage
                               before limiting.  0 for none. */
  double sutherland_s;      /* one gas, Navier-Stokes: > 0 switches on Sutherland's law
                               (Eq. sutherland), mu(T) = mu (1 + s) th^1.5 / (th + s) with
                               th = (p / rho) / sutherland_rt, in the viscous fluxes (kappa
                               scales with mu), the viscous time-step bound and the weights of
                               the dissipation integrals of dg_diagnostics; s = S / T_ref
                               (0.4042 in the paper's supersonic TGV); mu is the viscosity at
                               T_ref.  0 for a constant viscosity. */
  double sutherland_rt;     /* p / rho at T_ref (R T_ref); > 0 when sutherland_s > 0 */
  int indicator_variable;   /* shock-indicator quantity: 0 = rho p (Hennemann-Gassner's
                               default), 1 = p (the paper's supersonic TGV) */
} dg_physics_desc;

/* LGL nodes and weights used by libdg for degree N (host arrays of N+1).
 * Reading of Eqs. lagrange_3d and lag: -1, +1 and the roots of P_N'. */
dg_status dg_lgl_nodes(int N, double* nodes, double* weights);

/* Build a context: copies geometry and topology to the device and computes
 * the metric terms Ja^i = J grad(xi_i) (curl form) and J (Eqs. mapped_equation,
 * jacobian) on the GPU.  *out receives the context or NULL on failure. */
dg_status dg_init_mesh(const dg_mesh_desc* mesh, const dg_physics_desc* phys, dg_ctx** out);

/* Set the state from FP64 conserved variables [K][nv][np] (host or device
 * pointer, copied; converted to the compensated FP32 pair in DG_MIXED).  t is the
 * solution time.  In DG_MIXED a page-locked host buffer (cudaHostAlloc /
 * cudaHostRegister) is read by the conversion kernel directly, without a staging copy.
 * Synchronises.  Mixtures: the per-node temperature cache restarts cold (Newton from
 * 1000 K). */
dg_status dg_set_state(dg_ctx* ctx, const double* u, int on_device, double t);

/* Set the state from FP64 primitive variables (Eq. total_energy / eos applied
 * on the device).  Mixtures: the given temperatures seed the temperature cache. */
dg_status dg_set_state_primitive(dg_ctx* ctx, const double* w, int on_device, double t);

/* Copy the current state to u (FP64 [K][nv][np], host or device) and its time
 * to *t (may be NULL).  In DG_MIXED a page-locked host buffer is written by the
 * conversion kernel directly.  Synchronises the context stream. */
dg_status dg_get_state(dg_ctx* ctx, double* u, int on_device, double* t);

/* rhs = du/dt evaluated at u (Eq. strong_form with the split volume term of
 * Eq. fluxdiffcons and, for Navier-Stokes, the BR1 terms of Eqs. auxil and
 * auxstrongf).  u and rhs are device pointers of the context's precision
 * (double*, or float* in DG_MIXED), [K][nv][np]; u and rhs must not overlap.
 * Queued on the context stream; returns before the work finishes. */
dg_status dg_rhs(dg_ctx* ctx, const void* u, void* rhs, double t);

/* Advance the internal state by nsteps steps of the Carpenter-Kennedy
 * five-stage fourth-order 2N-storage Runge-Kutta scheme.  dt_fixed > 0 uses
 * that step; otherwise dt = cfl * 2 / ((N+1) max lambda) per step with
 * lambda = sum_i (|v.Ja^i| + c |Ja^i|) / J (plus a viscous bound for
 * Navier-Stokes), reduced on the device.  *t_inout is advanced by the elapsed
 * time.  Synchronises at the end and returns any latched device error. */
dg_status dg_step_rk(dg_ctx* ctx, int nsteps, double cfl, double dt_fixed, double* t_inout);

/* FP64 domain integrals of the current state (Eqs. TGV_KE, TGV_SD, TGV_DD):
 * out[8] = { KE/|Omega|, enstrophy/|Omega|, int S, int rho, int rho E, |Omega|,
 *            int (mu(T)/mu) (div v)^2 / |Omega|, int (mu(T)/mu) |omega|^2 / |Omega| },
 * KE = int rho|v|^2/2, enstrophy = int rho|omega|^2/2, S = -rho s/(gamma-1) (one gas, else 0);
 * mu(T)/mu is Sutherland's ratio (1 for a constant viscosity), so that
 * eps_s = L^2/(Re U^2) out[7] and eps_d = L^2/(3 Re U^2) out[6].  Synchronises. */
dg_status dg_diagnostics(dg_ctx* ctx, double out[8]);

/* Temperature of the current state of a mixture context (Eqs. total_energy,
 * internal_energies, eos; T recovered from e per node), FP64 [K][np] host.
 * Runs the temperature solve of the context's thermo mode on the current state.
 * DG_EINVAL for a single-gas context. Synchronises. */
dg_status dg_get_temperature(dg_ctx* ctx, double* T);

/* ---- learned surrogates (no counterpart in the paper).  Both are a perceptron
 * 7 -> 64 -> 64 -> n_out with the tanh form of GELU after the hidden layers, evaluated
 * with BF16 tensor-core MMAs (FP32 accumulation) and always checked against the plain
 * FP64 computation they replace, which remains the fallback.  Parameter vector (FP32,
 * P = dg_mlp_nparams(n_out)): W1[64][7], b1[64], W2[64][64], b2[64], W3[n_out][64],
 * b3[n_out].
 *
 * DG_SURROGATE_TEMPERATURE (n_out = 1): the per-node temperature solve of Eqs.
 *   total_energy / internal_energies / eos.  Inputs standardised (Y_1..Y_5, ln rho, e),
 *   output standardised T; stats (FP64, 16): mean[7], std[7], mean_T, std_T.  Every
 *   prediction gets one FP64 Newton step and is accepted when the next correction would
 *   be <= 1e-6 T, otherwise the plain Newton iteration runs (per node).
 * DG_SURROGATE_SOURCE (n_out = 10): the finite-rate source of Eqs. nrp / forward_rate /
 *   backward / calc_prod with its point-implicit terms.  Inputs standardised
 *   (Y_1..Y_5, ln rho, T); outputs the standardised z_s = asinh(omega_s / omega_ref) and
 *   z_{5+s} = asinh(jpi_s / jpi_ref), jpi_s = max(0, -d omega_s / d rho_s), so that
 *   S_s = omega_s / (1 + dt jpi_s) for any RK step dt.  Stats (FP64, DG_SRC_NSTATS)
 *   indexed by the DG_SRC_* offsets below.  Acceptance per tile of 32 consecutive nodes:
 *   every node's raw features inside the training box, every node's raw rates
 *   mass-balanced (|sum omega| <= tol_mass sum |omega| + floor), every node's learned
 *   update positive (rho_s + dt S_s >= 0, dt the running step), and, at one node per tile drawn
 *   anew each evaluation, |S_learned - S_plain| <= tol_check sum_s |S_plain| + floor for
 *   every species; rejected tiles are recomputed with the plain FP64 source.  Accepted
 *   rates are projected onto exact mass balance, omega_s -= |omega_s| sum omega / sum|omega|. */
enum { DG_SURROGATE_TEMPERATURE = 0, DG_SURROGATE_SOURCE = 1 };
enum {
  DG_SRC_X_MEAN = 0,      /* [7] feature means (Y_1..Y_5, ln rho, T) */
  DG_SRC_X_STD = 7,       /* [7] feature standard deviations */
  DG_SRC_Y_MEAN = 14,     /* [10] target means (asinh images) */
  DG_SRC_Y_STD = 24,      /* [10] target standard deviations */
  DG_SRC_OMEGA_REF = 34,  /* omega_ref, kg/(m^3 s) */
  DG_SRC_JPI_REF = 35,    /* jpi_ref, 1/s */
  DG_SRC_BOX_LO = 36,     /* [7] trust box: smallest raw feature values of the training set */
  DG_SRC_BOX_HI = 43,     /* [7] largest */
  DG_SRC_TOL_CHECK = 50,  /* sampled-node check, relative tolerance */
  DG_SRC_TOL_MASS = 51,   /* raw mass-balance tolerance */
  DG_SRC_FLOOR = 52,      /* absolute floor of both rate checks, kg/(m^3 s) */
  DG_SRC_NSTATS = 53
};

/* Load (params, stats: host arrays) into a mixture context and switch the temperature
 * solve (which = DG_SURROGATE_TEMPERATURE) or the chemistry source (which =
 * DG_SURROGATE_SOURCE, reacting contexts only) to the learned form described above.
 * params == NULL switches back to the plain computation.  DG_EINVAL for a single-gas
 * context, a frozen mixture with DG_SURROGATE_SOURCE, or non-positive deviations. */
dg_status dg_set_surrogate(dg_ctx* ctx, int which, const float* params, const double* stats);

/* Plain correction of the learned source (reacting contexts).  period 0 (the default)
 * switches it off.  period k >= 1: a refresh evaluation takes the plain FP64 source at
 * every node and stores per node the plain rates minus the network's decoded rates
 * (omega_s - omega^_s and jpi_s - jpi'_s, jpi' the decoded jpi before its clamp at 0;
 * FP32, 40 bytes per node, allocated here); the learned evaluations that follow add these
 * differences to the decoded rates (omega^_s + c_s, max(0, jpi'_s + c_{5+s})) before the
 * acceptance tests above.  At a refresh every node is also checked: its uncorrected learned
 * source against the plain one with the sampled check's test; a tile with a failing node
 * takes the plain source at every evaluation until the next refresh (flag 4 in
 * dg_get_source).  Refreshes happen at the first source evaluation of each
 * dg_step_rk call, at the first RK stage of every k-th step after it, and at the first
 * dg_rhs after the state, the network or the period was set.  Reading R18s step 9: the
 * corrected network is exact at the refresh state; the checks still decide acceptance.
 * DG_EINVAL for a context without chemistry or a negative period. */
dg_status dg_set_source_refresh(dg_ctx* ctx, int period);

/* Nodes accepted and nodes recomputed plainly by the surrogate `which` since the last
 * call (host int64[2]); resets the counters.  Refresh evaluations of the source are
 * counted in neither. */
dg_status dg_surrogate_stats(dg_ctx* ctx, int which, int64_t* accepted_fallback);

/* The species source of the last evaluation (the appendix's finite-rate source with its
 * point-implicit factor, Eqs. nrp .. calc_prod; learned where the surrogate's tile was
 * accepted): S [K][5][np] FP64 host (converted from the form precision).  flags (host,
 * (K np + 31) / 32 bytes, or NULL) receives the per-tile decision of that evaluation:
 * 0 learned, 1 rejected by the trust box, the mass balance or the positivity test, 2
 * rejected by the sampled check, 3 a refresh evaluation (plain everywhere), 4 not trusted
 * since the last refresh (255 everywhere when the learned source is off); *call (or NULL) the evaluation
 * counter that drew the tiles' sampled nodes (-1 before the first learned evaluation).
 * DG_EINVAL for a context without chemistry, DG_ESTATE before any evaluation.  Waits for
 * the context stream (bounded). */
dg_status dg_get_source(dg_ctx* ctx, double* S, unsigned char* flags, int64_t* call);

/* Training data from the plain solver: runs the temperature solve on the current state,
 * then writes n samples drawn with splitmix64(seed + j) over all nodes:
 * X [n][7] raw features (Y_1..Y_5, ln rho, e) and T [n] (device float arrays). */
dg_status dg_thermo_sample(dg_ctx* ctx, int64_t n, uint64_t seed, float* X, float* T);

/* Training data for the source surrogate (reacting contexts): runs the temperature solve
 * on the current state, then for n nodes drawn with splitmix64(seed + j): X [n][7] raw
 * features (Y_1..Y_5, ln rho, T) (device float) and targets [n][10] = (omega_1..5,
 * jpi_1..5) of the plain FP64 source (device double). */
dg_status dg_chem_sample(dg_ctx* ctx, int64_t n, uint64_t seed, float* X, double* targets);

/* ---- training and checking kernels (device pointers, queued on `stream`) */
/* Parameter count for n_out outputs (1..16), -1 otherwise. */
int dg_mlp_nparams(int n_out);
/* Workspace bytes that dg_mlp_grad / dg_mlp_train_step need for a batch (0 if invalid). */
size_t dg_mlp_workspace_bytes(int batch, int n_out);
/* Gradient of loss = mean over samples and outputs of (y - t)^2 (FP32 back-propagation,
 * fixed-order reduction): params [P], X [batch][7] standardised inputs, t [batch][n_out]
 * standardised targets, grad [P] out, loss (device double*, may be NULL). */
dg_status dg_mlp_grad(const float* params, int n_out, const float* X, const float* t, int batch,
                      float* grad, double* loss, float* workspace, size_t ws_bytes, void* stream);
/* One Adam step (beta = 0.9, 0.999, eps = 1e-8, bias-corrected, step >= 1) on the same
 * loss; params, m, v updated in place. */
dg_status dg_mlp_train_step(float* params, int n_out, float* m, float* v, const float* X,
                            const float* t, int batch, int step, float lr, double* loss,
                            float* workspace, size_t ws_bytes, void* stream);
/* y[n][n_out] = network(X[n][7]) for standardised X; tensor_cores = 1 uses the warp-level
 * BF16 MMA path of the inference kernels, 2 the tcgen05 path (128-row tiles, tensor-memory
 * accumulators; DG_ETIMEOUT if a bounded wait inside ran out), both for n_out 1 or 10 and
 * synchronising; 0 the FP32 path. */
dg_status dg_mlp_forward(const float* params, int n_out, const float* X, float* y, int64_t n,
                         int tensor_cores, void* stream);

/* Data preparation of the learned surrogates (no counterpart in the paper; the steps
 * that turn the plain solver's samples into training arrays), on the device, with
 * fixed-order reductions (deterministic).  Sample arrays are row-major [n][d] device arrays
 * of FP32 (is_f64 = 0) or FP64 values; `ref` (host, [d] positive, or NULL) maps each value
 * v of column c to asinh(v / ref[c]) first.  Each call synchronises `stream`.
 *
 * dg_column_stats: out (host, [4][d]) = per column mean, standard deviation (divisor
 *   n - 1), min and max of the (mapped) values; n >= 2, d <= 64. */
dg_status dg_column_stats(const void* X, int is_f64, int64_t n, int d, const double* ref, double* out,
                          void* stream);
/* dg_standardize: out[i][c] = (mapped X[i][c] - mean[c]) / std[c] as FP32 (device [n][d]);
 *   mean, std host [d], std > 0. */
dg_status dg_standardize(const void* X, int is_f64, int64_t n, int d, const double* ref, const double* mean,
                         const double* std_dev, float* out, void* stream);
/* dg_abs_quantile: the q-quantile (0 <= q <= 1) of |Y[i][c]| over all rows and the columns
 *   c0 .. c0 + nc - 1 of an FP64 device array Y [n][d]: the order statistics around
 *   position q (m - 1), m = n nc, found exactly by bisection on their bit patterns, and
 *   linear interpolation between them; *out on the host. */
dg_status dg_abs_quantile(const double* Y, int64_t n, int d, int c0, int nc, double q, double* out, void* stream);
/* dg_gather_rows: out[r][:] = X[idx[r]][:] for r < m (device arrays; idx int64 in range). */
dg_status dg_gather_rows(const float* X, int d, const int64_t* idx, int64_t m, float* out, void* stream);
/* dg_mlp_loss: *loss (host) = mean over the n samples and n_out outputs of
 *   (network(X) - t)^2 with the FP32 forward (params, X [n][7], t [n][n_out] device). */
dg_status dg_mlp_loss(const float* params, int n_out, const float* X, const float* t, int64_t n, double* loss,
                      void* stream);

/* Blending factors alpha [K] used by the last right-hand side (FP64, host). */
dg_status dg_get_alpha(dg_ctx* ctx, double* alpha);

/* Metric terms of the context (Methodology, curvilinear mapping: Eqs. mapp, jacobian;
 * contravariant terms in the conservative curl form), FP64: Ja [K][dim][dim][np] with
 * Ja[k][i][n][node] = Ja^i_n, invJ [K][np] = 1/J.  Host buffers (on_device = 0) or
 * device buffers (1) of the caller; the copies are queued on the context stream and
 * waited for (bounded).  These are the arrays dg_rhs_ns_noalloc takes. */
dg_status dg_get_metrics(dg_ctx* ctx, double* Ja, double* invJ, int on_device);

/* BR1 gradients of (v, p/rho) (Eq. auxstrongf), [K][dim][dim+1][np] FP64 host: of the input
 * of the last dg_rhs call, or, once dg_step_rk has run since, of the current state.
 * DG_ESTATE before any Navier-Stokes right-hand side. Synchronises. */
dg_status dg_get_gradients(dg_ctx* ctx, double* grad);

/* Per-kernel device timing (tracing).  While enabled, every kernel launch of the
 * context is bracketed by CUDA events recorded on the context stream.
 * dg_profile_read waits for the stream and returns, per kernel kind, the summed
 * device milliseconds and the number of launches since the last read
 * (kinds: DG_PROF_RHS, DG_PROF_GRAD, DG_PROF_INDICATOR, DG_PROF_LAMBDA,
 * DG_PROF_THERMO, DG_PROF_MLP, DG_PROF_CHEM, DG_PROF_OTHER, DG_PROF_LIMITER); then it
 * resets them.  ms and launches are host arrays of n entries (n <= DG_PROF_KINDS). */
enum { DG_PROF_RHS = 0, DG_PROF_GRAD = 1, DG_PROF_INDICATOR = 2, DG_PROF_LAMBDA = 3,
       DG_PROF_THERMO = 4, DG_PROF_MLP = 5, DG_PROF_CHEM = 6, DG_PROF_OTHER = 7,
       DG_PROF_LIMITER = 8, DG_PROF_KINDS = 9 };
dg_status dg_profile(dg_ctx* ctx, int enable);
dg_status dg_profile_read(dg_ctx* ctx, double* ms, int64_t* launches, int n);

/* Apply the positivity limiter (eps = positivity_eps of the context, which must be > 0)
 * once to the current state, e.g. to a raw initial condition.  Synchronises; returns
 * DG_ENONPHYS when an element mean is not admissible. */
dg_status dg_limit_state(dg_ctx* ctx);

/* Elements changed by the positivity limiter since the last call (host int64); resets
 * the count.  0 when the limiter is off. */
dg_status dg_limiter_stats(dg_ctx* ctx, int64_t* elements);

/* Measured arithmetic peak of the current device (no counterpart in the paper; the
 * roofline denominator of arithmetic-bound kernels): chains of fused multiply-adds in
 * FP64 (precision = DG_FP64) or FP32 (DG_MIXED), iters FMAs per chain, CUDA-event
 * timed; *tflops = 2 flops per FMA / time.  Synchronises the device. */
dg_status dg_peak_flops(int precision, int iters, double* tflops);

/* Wait (bounded) for the context stream, then return and clear the latched
 * device status. */
dg_status dg_sync(dg_ctx* ctx);

/* Element index of the first latched device error, or -1. */
int64_t dg_error_element(dg_ctx* ctx);

const char* dg_status_string(dg_status s);

void dg_destroy(dg_ctx* ctx);

/* Allocation-free FP64 Navier-Stokes right-hand side.  The paper has no
 * counterpart: it exists for callers that may not allocate device memory (a
 * host framework that owns all device memory and passes a library only inputs
 * and outputs, or a loop where cudaMalloc's implicit synchronisation and
 * run-time failure are not acceptable), and so cannot create a context.
 * Computes the same operator as dg_rhs for a 3D, single-gas, fully periodic
 * Navier-Stokes problem.  Inputs and output are caller-owned device arrays:
 *   nbr  int32 [K][6] neighbour element per face (faces -x,+x,-y,+y,-z,+z),
 *   Ja   [K][3][3][np] metric terms Ja^i_n, invJ [K][np] = 1/J,
 *   u    [K][5][np] conserved state, rhs [K][5][np] output (must not overlap u).
 * Scratch (the BR1 gradients, K (N+1)^3 12 doubles, and a status word) lives in
 * one static device array of DG_NOALLOC_SCRATCH_BYTES that every GPU loading
 * the library holds until exit; larger problems return DG_EINVAL.  No device
 * memory is allocated or freed.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and uploads the basis tables, so make
 * that first call before any stream capture.  All calls share the one array:
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it; serialise them.  The problem must be fully periodic: every nbr
 * entry must lie in [0, K).  The call copies nbr into the scratch first and
 * replaces an entry outside that range by the element's own index (so that no
 * kernel reads outside u), latching DG_EINVAL with that element; the output is
 * then not valid.  The status word is cleared at every call; device-side errors
 * (DG_EINVAL for a bad nbr entry, DG_ENONPHYS for rho <= 0, p <= 0 or NaN) are
 * latched there and read by dg_noalloc_status.  Queued on `stream`
 * (cudaStream_t, NULL = legacy default); returns before the work finishes.
 * Concurrent first calls from several host threads are safe (the set-up is
 * serialised). */
#define DG_NOALLOC_SCRATCH_BYTES (16u << 20)
dg_status dg_rhs_ns_noalloc(int N, int64_t K, const int32_t* nbr, const double* Ja,
                            const double* invJ, double gamma, double mu, double Pr,
                            int volume_flux, int surface_flux, const double* u, double* rhs,
                            void* stream);

/* Status word latched by the last dg_rhs_ns_noalloc call on the current device
 * (no counterpart in the paper).  Copies the 8-byte word into *status_out (a
 * host variable; (code << 56) | element, 0 when clean) after the work queued on
 * `stream` before it, waiting for the stream (bounded: DG_ETIMEOUT after 600 s),
 * and returns DG_OK, DG_EINVAL (a neighbour index outside [0, K)) or
 * DG_ENONPHYS.  Allocates no device memory.  Does not clear the word. */
dg_status dg_noalloc_status(void* stream, uint64_t* status_out);

#ifdef __cplusplus
}
#endif
#endif
