// Mixture thermodynamics on the device (temperature from internal energy,
// pressure, frozen sound speed) for the multi-species Euler form.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct DgThermo {
  int64_t K;
  int np, dim, ns, mode, f32;
  double* species;     // device [ns][8] e(T) polynomial coefficient rows per species
  float* coef32;       // device [ns][8] FP32 copy
  double* T;           // device [K][np] temperature cache (FP64)
  void* pc;            // device [K][2][np] pressure, sound speed (form precision)
  void* bc_pc;         // device [n_bc][2]
  unsigned long long* status;
  double* species_raw; // device [ns][16] chemistry coefficient rows (dg_chem.cu)
  double* reac;        // device [nr][20] reaction rows (ln A in slot 16)
  int nr;              // number of reactions, 0 = frozen
  void* src;           // device [K][ns][np] chemistry source (form precision)
  void* mlp;           // temperature surrogate weights (device) or null
  unsigned long long* mlp_stats;  // [accepted, fallback] node counts of the surrogate
  void* chem_mlp;                 // chemistry-source surrogate (device) or null
  unsigned long long* chem_stats; // [accepted, fallback] node counts of the source surrogate
  unsigned char* chem_flags;      // per 32-node tile: 0 accepted, otherwise recomputed plainly
  unsigned long long chem_calls;  // learned-source evaluations so far (moves each tile's sampled node)
  int src_valid;                  // src holds an evaluation
  float* chem_corr;               // [10][K np] plain-minus-network corrections of the learned source
  int refresh_period;             // 0: no correction; k: refresh at stage 0 of every k-th RK step
  int corr_valid;                 // chem_corr holds the corrections of a refresh
  unsigned char* chem_trust;      // per 32-node tile: 1 when the network passed the last refresh's full check
};

cudaError_t dg_thermo_upload_basis();
cudaError_t dg_thermo_init(DgThermo* th, int64_t K, int np, int dim, const double* species_host,
                           int mode, int f32, unsigned long long* status);
void dg_thermo_free(DgThermo* th);
cudaError_t dg_thermo_reset(DgThermo* th, cudaStream_t s);
cudaError_t dg_thermo_update(DgThermo* th, const void* u, int f32, cudaStream_t s);
cudaError_t dg_thermo_boundary(DgThermo* th, const double* bw, int n_bc, void* bc_u, cudaStream_t s);
cudaError_t dg_thermo_prim2cons(DgThermo* th, const double* w, void* u, cudaStream_t s);
// chemistry (dg_chem.cu)
cudaError_t dg_chem_init(DgThermo* th, const double* species_host, const double* reac_host, int nr);
// refresh != 0 (learned source with corrections only): plain source everywhere, and the
// corrections of this state stored for the evaluations that follow
cudaError_t dg_chem_source(DgThermo* th, const void* u, int f32, const double* dt_dev, int refresh,
                           cudaStream_t s);
// learned source (dg_chem.cu): set / clear (params null) and plain-source training samples
cudaError_t dg_chem_mlp_set(DgThermo* th, const float* params_host, const double* stats_host);
cudaError_t dg_chem_sample_dev(DgThermo* th, const void* u, int f32, int64_t n, uint64_t seed, float* X,
                           double* targets, cudaStream_t s);
// surrogate (dg_mlp.cu)
cudaError_t dg_mlp_set(DgThermo* th, const float* params_host, const double* stats_host);
cudaError_t dg_mlp_thermo_update(DgThermo* th, const void* u, int f32, cudaStream_t s);
cudaError_t dg_mlp_sample(DgThermo* th, const void* u, int f32, int64_t n, uint64_t seed, float* X,
                          float* T, cudaStream_t s);
