// Internal interface between the C-ABI layer (dg_capi.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define DG_MAXN 7
#define DG_MAX_SPECIES 8
#define DG_MAX_NV (DG_MAX_SPECIES + 4)

// device status word: (code << 56) | element
#define DG_ST_NONPHYS 4ull
#define DG_ST_NEWTON 5ull
#define DG_ST_TIMEOUT 6ull  // a bounded wait inside a kernel ran out

// Everything a right-hand-side / RK-stage launch needs, passed by value.
struct DgArgs {
  int64_t K;
  int dim, N, nsp, nv, np;
  int n_bc;
  int has_bnd;            // the mesh has boundary faces
  int vf, sf;             // DG_VF_*, DG_SF_*
  int mode;               // 0: write rhs, 1: RK stage
  int stage;              // RK stage 0..4
  int want_lambda;        // mode 1: accumulate wave speeds of the new state
  int lam_cur;            // slot holding the current step's wave-speed maxima
  int ns;                 // Navier-Stokes terms on
  double gamma, mu, kappa_fac;   // kappa_fac = mu gamma / ((gamma-1) Pr)
  double pref;                   // pressure offset of the momentum fluxes (one gas)
  double visc_coef;              // gamma mu / Pr (viscous time-step bound)
  double suth_s, suth_rt;        // Sutherland's law: s = S / T_ref (0: constant mu), p/rho at T_ref
  int ind_var;                   // shock indicator on 0: rho p, 1: p
  double pos_ef[8];              // mixture limiter: e_s(T_floor) per unit mass of each species
  double cfl, dt_fixed, rkA, rkB;
  const void* u;          // [K][nv][np] input state
  void* out;              // mode 0: rhs; mode 1: new state
  void* du;               // mode 1: 2N-storage register
  void* ulo;              // mode 1, FP32 form: low part of the compensated input state (or null)
  void* ulo_out;          // mode 1, FP32 form: low part of the new state (a second buffer: other
                          // CTAs still read their neighbours' input low parts)
  const void* Ja;         // [K][dim][dim][np]
  const void* invJ;       // [K][np]
  void* gradW;            // [K][dim][dim+1][np] (Navier-Stokes): grad_mode 0 the contravariant
                          // viscous fluxes [d][c] = sum_x Ja^d_x f^v_{x,c}; 1 the gradients [x][c]
  int grad_mode;
  const void* alpha_raw;  // [K] unsmoothed blending factors, or null
  double* alpha_used;     // [K] smoothed factors actually applied (FP64), or null
  const int* nbr;         // [K][2 dim]
  const int* bc_kind;     // [n_bc]
  const void* bc_u;       // [n_bc][nv] conserved boundary states
  const void* pc;         // mixtures: [K][2][np] pressure and sound speed
  const void* bc_pc;      // mixtures: [n_bc][2]
  const void* src;        // mixtures with chemistry: [K][nsp][np] species source, or null
  double* scal;           // device scalars: [0] t, [1] dt of the running step
  unsigned long long* lam;  // [2 slots][2] wave-speed maxima as ordered double bits
  unsigned long long* status;
};

struct DgHostBasis {
  int N;
  double x[DG_MAXN + 1], w[DG_MAXN + 1];
  double D[(DG_MAXN + 1) * (DG_MAXN + 1)];
  double Vinv[(DG_MAXN + 1) * (DG_MAXN + 1)];  // nodal -> orthonormal Legendre modes
};

// host basis (dg_basis.cpp)
int dg_host_basis(int N, DgHostBasis* b);

// kernel translation units
// generic-flux halves of the right-hand-side kernels (called by dg_f64_rhs / dg_f32_rhs
// for non-production flux pairs; their basis tables are uploaded with the production ones)
cudaError_t dg_f64g_upload_basis();
cudaError_t dg_f32g_upload_basis();
cudaError_t dg_f32s_upload_basis();
cudaError_t dg_f32s_rhs(const DgArgs& a, cudaStream_t s);
cudaError_t dg_f64g_rhs(const DgArgs& a, cudaStream_t s);
cudaError_t dg_f32g_rhs(const DgArgs& a, cudaStream_t s);
// Zhang-Shu positivity limiter on a state of the context's precision (one gas)
cudaError_t dg_f64_positivity(const DgArgs& a, void* u, void* ulo, double eps, unsigned long long* nlim,
                              cudaStream_t s);
cudaError_t dg_f32_positivity(const DgArgs& a, void* u, void* ulo, double eps, unsigned long long* nlim,
                              cudaStream_t s);
cudaError_t dg_f64_upload_basis();
cudaError_t dg_f32_upload_basis();
cudaError_t dg_f64_rhs(const DgArgs& a, cudaStream_t s);
cudaError_t dg_f32_rhs(const DgArgs& a, cudaStream_t s);
cudaError_t dg_f64_gradients(const DgArgs& a, cudaStream_t s);
cudaError_t dg_f32_gradients(const DgArgs& a, cudaStream_t s);
cudaError_t dg_f64_lambda(const DgArgs& a, int slot, cudaStream_t s);
cudaError_t dg_f32_lambda(const DgArgs& a, int slot, cudaStream_t s);
cudaError_t dg_f64_step_dt(const DgArgs& a, int slot, int advance_time, cudaStream_t s);
cudaError_t dg_f32_step_dt(const DgArgs& a, int slot, int advance_time, cudaStream_t s);
cudaError_t dg_f64_indicator(const DgArgs& a, double alpha_max, void* alpha_raw, cudaStream_t s);
cudaError_t dg_f32_indicator(const DgArgs& a, double alpha_max, void* alpha_raw, cudaStream_t s);
