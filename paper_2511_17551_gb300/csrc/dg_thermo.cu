// Mixture thermodynamics on the device: temperature from internal energy by Newton
// iteration, Dalton pressure and frozen sound speed, per node.
//
// Thermally perfect species (stand-in for the RRHO database of the appendix,
// Eq. Internal_energy): cp_s/R_s = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4 and
//   e_s(T) = R_s (a1 T + a2 T^2/2 + a3 T^3/3 + a4 T^4/4 + a5 T^5/5 + a6 - T),
// e = sum Y_s e_s (Eq. internal_energies), p = sum rho_s R_s T (Eq. eos).
// At set-up every species becomes one row of a coefficient table
//   [R_s a6, R_s (a1-1), R_s a2/2, R_s a3/3, R_s a4/4, R_s a5/5, R_s, 0],
// so a node folds its mixture into e(T) = b0 + b1 T + ... + b5 T^5 with 30 multiply-adds
// (no divisions) and evaluates e and cv = de/dT by Horner's rule.  Newton
// T <- T - (e(T) - e)/cv(T) is warm-started from the node's previous temperature and
// stops at |dT| <= 1e-12 T (at most 50 steps, T kept in [200, 1e4] K); failure latches
// DG_ENEWTON.  Mixed form: FP32 Newton on e(T) - b0 = e - b0 (the constant b0 is
// removed so FP32 resolves the residual) to |dT| <= 1e-6 T, then FP64 Newton steps on
// the FP64 residual (normally one).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "dg_internal.h"
#include "dg_thermo.h"

#define DG_RU 8.314462618
#define NSPEC 5

namespace {

__device__ __forceinline__ void latch(unsigned long long* st, unsigned long long code, int64_t e) {
  atomicCAS(st, 0ull, (code << 56) | (unsigned long long)(e & 0x00ffffffffffffffll));
}

template <typename R>
struct Poly {
  R b[6];  // e(T) = sum b_k T^k
  R Rmix;
  __device__ __forceinline__ R e(R T) const {
    return b[0] + T * (b[1] + T * (b[2] + T * (b[3] + T * (b[4] + T * b[5]))));
  }
  __device__ __forceinline__ R e_noconst(R T) const {
    return T * (b[1] + T * (b[2] + T * (b[3] + T * (b[4] + T * b[5]))));
  }
  __device__ __forceinline__ R cv(R T) const {
    return b[1] + T * (R(2) * b[2] + T * (R(3) * b[3] + T * (R(4) * b[4] + T * (R(5) * b[5]))));
  }
};

template <typename R>
__device__ __forceinline__ void build_poly(const R* cf, const R* Y, Poly<R>& P) {
#pragma unroll
  for (int k = 0; k < 6; ++k) P.b[k] = R(0);
  P.Rmix = R(0);
#pragma unroll
  for (int s = 0; s < NSPEC; ++s) {
#pragma unroll
    for (int k = 0; k < 6; ++k) P.b[k] += Y[s] * cf[8 * s + k];
    P.Rmix += Y[s] * cf[8 * s + 6];
  }
}

__device__ __forceinline__ double clampT(double T) { return T < 200.0 ? 200.0 : (T > 1e4 ? 1e4 : T); }
__device__ __forceinline__ float clampTf(float T) { return T < 200.f ? 200.f : (T > 1e4f ? 1e4f : T); }

// FP64 Newton from T; returns true on convergence
__device__ __forceinline__ bool newton64(const Poly<double>& P, double e, double& T) {
  for (int it = 0; it < 50; ++it) {
    const double Tn = clampT(T - (P.e(T) - e) / P.cv(T));
    const double step = fabs(Tn - T);
    T = Tn;
    if (step <= 1e-12 * T) return true;
  }
  return false;
}

template <typename T>
__global__ void thermo_update_kernel(const T* u, int64_t K, int np, int dim, const double* cf,
                                     const float* cf32, double* Tc, T* pc,
                                     unsigned long long* status, int mixed) {
  const int nv = NSPEC + dim + 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K * np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / np;
    const int node = (int)(i % np);
    const T* uu = u + k * nv * np + node;
    double Y[NSPEC], rho = 0.0, ke = 0.0;
#pragma unroll
    for (int s = 0; s < NSPEC; ++s) {
      Y[s] = (double)uu[s * np];
      rho += Y[s];
    }
    for (int d = 0; d < dim; ++d) {
      const double m = (double)uu[(NSPEC + d) * np];
      ke += m * m;
    }
    const double ir = 1.0 / rho;
    const double e = (double)uu[(NSPEC + dim) * np] * ir - 0.5 * ke * ir * ir;
    double Tk = Tc[k * np + node];
    if (!(Tk >= 200.0 && Tk <= 1e4)) Tk = 1000.0;
    Poly<double> P;
    if (mixed) {
      // FP32 mixture polynomial for the Newton iteration; in FP64 only the large constant
      // b0 (formation energies), from density-weighted sums
      Poly<float> Pf;
      float Yf[NSPEC];
      double b0 = 0.0;
      const float irf = (float)ir;
#pragma unroll
      for (int s = 0; s < NSPEC; ++s) {
        Yf[s] = (float)Y[s] * irf;
        b0 += Y[s] * cf[8 * s];
      }
      b0 *= ir;
      build_poly<float>(cf32, Yf, Pf);
      const float er = (float)(e - b0);
      float Tf = (float)Tk;
      bool conv = false;
      for (int it = 0; it < 12; ++it) {
        const float Tn = clampTf(Tf - (Pf.e_noconst(Tf) - er) / Pf.cv(Tf));
        const float step = fabsf(Tn - Tf);
        Tf = Tn;
        if (step <= 1e-6f * Tf) {
          conv = true;
          break;
        }
      }
      // the FP64 final residual: one Newton correction on e64(T) - e, evaluated in FP64
      // with the FP64 constant b0 and the FP32-rounded temperature coefficients (their
      // rounding moves e by ~1e-7 relative, i.e. T by ~1e-4 K); cv in FP32 only scales the
      // correction.  The full FP64 iteration runs only where the FP32 stage did not converge.
      double T64 = (double)Tf;
      const double r = (b0 + T64 * ((double)Pf.b[1] + T64 * ((double)Pf.b[2] + T64 * ((double)Pf.b[3] +
                        T64 * ((double)Pf.b[4] + T64 * (double)Pf.b[5]))))) - e;
      T64 = clampT(T64 - r * (double)(1.0f / Pf.cv(Tf)));
      bool ok = rho > 0.0;
      if (ok && !conv) {
#pragma unroll
        for (int s = 0; s < NSPEC; ++s) Y[s] *= ir;
        build_poly<double>(cf, Y, P);
        ok = newton64(P, e, T64);
      }
      if (!ok) latch(status, DG_ST_NEWTON, k);
      Tc[k * np + node] = T64;
      const float Tq = (float)T64, rhof = (float)rho;
      const float pf = rhof * Pf.Rmix * Tq, cvf = Pf.cv(Tq);
      pc[(k * 2 + 0) * np + node] = (T)pf;
      pc[(k * 2 + 1) * np + node] = (T)sqrtf((cvf + Pf.Rmix) / cvf * pf / rhof);
      continue;
    }
#pragma unroll
    for (int s = 0; s < NSPEC; ++s) Y[s] *= ir;
    build_poly<double>(cf, Y, P);
    const bool ok = rho > 0.0 && newton64(P, e, Tk);
    if (!ok) latch(status, DG_ST_NEWTON, k);
    Tc[k * np + node] = Tk;
    const double p = rho * P.Rmix * Tk;
    const double cv = P.cv(Tk);
    pc[(k * 2 + 0) * np + node] = (T)p;
    pc[(k * 2 + 1) * np + node] = (T)sqrt((cv + P.Rmix) / cv * p * ir);
  }
}

// (rho_s, v, T) -> conserved and (p, c); also seeds the temperature cache
template <typename T>
__global__ void thermo_prim2cons_kernel(const double* w, T* u, int64_t K, int np, int dim,
                                        const double* cf, double* Tc, T* pc) {
  const int nv = NSPEC + dim + 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K * np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / np;
    const int node = (int)(i % np);
    const double* ww = w + k * nv * np + node;
    T* uu = u + k * nv * np + node;
    double rho = 0.0, Y[NSPEC];
#pragma unroll
    for (int s = 0; s < NSPEC; ++s) {
      Y[s] = ww[s * np];
      rho += Y[s];
      uu[s * np] = (T)ww[s * np];
    }
#pragma unroll
    for (int s = 0; s < NSPEC; ++s) Y[s] /= rho;
    double ke = 0.0;
    for (int d = 0; d < dim; ++d) {
      const double v = ww[(NSPEC + d) * np];
      uu[(NSPEC + d) * np] = (T)(rho * v);
      ke += v * v;
    }
    const double Tk = ww[(NSPEC + dim) * np];
    Poly<double> P;
    build_poly<double>(cf, Y, P);
    uu[(NSPEC + dim) * np] = (T)(rho * (P.e(Tk) + 0.5 * ke));
    if (Tc) Tc[k * np + node] = Tk;
    if (pc) {
      const double p = rho * P.Rmix * Tk, cv = P.cv(Tk);
      pc[(k * 2 + 0) * np + node] = (T)p;
      pc[(k * 2 + 1) * np + node] = (T)sqrt((cv + P.Rmix) / cv * p / rho);
    }
  }
}

__global__ void fill_kernel(double* a, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

unsigned grid_of(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t dg_thermo_upload_basis() { return cudaSuccess; }

cudaError_t dg_thermo_init(DgThermo* th, int64_t K, int np, int dim, const double* species_host,
                           int mode, int f32, unsigned long long* status) {
  memset(th, 0, sizeof(*th));
  th->K = K;
  th->np = np;
  th->dim = dim;
  th->ns = NSPEC;
  th->mode = mode;
  th->f32 = f32;
  th->status = status;
  // per-species coefficient rows (see the header comment)
  double cf[8 * NSPEC];
  float cf32[8 * NSPEC];
  for (int s = 0; s < NSPEC; ++s) {
    const double* sp = species_host + 8 * s;
    const double Rs = DG_RU / sp[0];
    const double* a = sp + 1;
    const double row[8] = {Rs * a[5], Rs * (a[0] - 1.0), Rs * a[1] / 2.0, Rs * a[2] / 3.0,
                           Rs * a[3] / 4.0, Rs * a[4] / 5.0, Rs, 0.0};
    for (int k = 0; k < 8; ++k) {
      cf[8 * s + k] = row[k];
      cf32[8 * s + k] = (float)row[k];
    }
  }
  const size_t rs = f32 ? sizeof(float) : sizeof(double);
  cudaError_t e = cudaMalloc((void**)&th->species, sizeof(cf));
  if (e == cudaSuccess) e = cudaMemcpy(th->species, cf, sizeof(cf), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&th->coef32, sizeof(cf32));
  if (e == cudaSuccess) e = cudaMemcpy(th->coef32, cf32, sizeof(cf32), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&th->T, sizeof(double) * K * np);
  if (e == cudaSuccess) e = cudaMalloc(&th->pc, rs * 2 * K * np);
  if (e == cudaSuccess) e = cudaMalloc(&th->bc_pc, rs * 2 * 64);
  if (e == cudaSuccess) {
    fill_kernel<<<grid_of(K * np), 256>>>(th->T, K * np, 1000.0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e;
}

void dg_thermo_free(DgThermo* th) {
  if (th->mlp) cudaFree(th->mlp);
  if (th->mlp_stats) cudaFree(th->mlp_stats);
  if (th->chem_mlp) cudaFree(th->chem_mlp);
  if (th->chem_stats) cudaFree(th->chem_stats);
  if (th->chem_flags) cudaFree(th->chem_flags);
  if (th->chem_corr) cudaFree(th->chem_corr);
  if (th->chem_trust) cudaFree(th->chem_trust);
  if (th->species) cudaFree(th->species);
  if (th->coef32) cudaFree(th->coef32);
  if (th->species_raw) cudaFree(th->species_raw);
  if (th->reac) cudaFree(th->reac);
  if (th->src) cudaFree(th->src);
  if (th->T) cudaFree(th->T);
  if (th->pc) cudaFree(th->pc);
  if (th->bc_pc) cudaFree(th->bc_pc);
  memset(th, 0, sizeof(*th));
}

// cold start: every node's Newton iteration restarts from 1000 K
cudaError_t dg_thermo_reset(DgThermo* th, cudaStream_t s) {
  fill_kernel<<<grid_of(th->K * th->np), 256, 0, s>>>(th->T, th->K * th->np, 1000.0);
  return cudaGetLastError();
}

cudaError_t dg_thermo_update(DgThermo* th, const void* u, int f32, cudaStream_t s) {
  if (th->mode == 1 && th->mlp) return dg_mlp_thermo_update(th, u, f32, s);
  if (f32)
    thermo_update_kernel<float><<<grid_of(th->K * th->np), 256, 0, s>>>(
        (const float*)u, th->K, th->np, th->dim, th->species, th->coef32, th->T, (float*)th->pc,
        th->status, 1);
  else
    thermo_update_kernel<double><<<grid_of(th->K * th->np), 256, 0, s>>>(
        (const double*)u, th->K, th->np, th->dim, th->species, th->coef32, th->T,
        (double*)th->pc, th->status, 0);
  return cudaGetLastError();
}

cudaError_t dg_thermo_boundary(DgThermo* th, const double* bw, int n_bc, void* bc_u, cudaStream_t s) {
  if (n_bc > 64) return cudaErrorInvalidValue;
  if (th->f32)
    thermo_prim2cons_kernel<float><<<1, 64, 0, s>>>(bw, (float*)bc_u, n_bc, 1, th->dim, th->species,
                                                     NULL, (float*)th->bc_pc);
  else
    thermo_prim2cons_kernel<double><<<1, 64, 0, s>>>(bw, (double*)bc_u, n_bc, 1, th->dim, th->species,
                                                      NULL, (double*)th->bc_pc);
  return cudaGetLastError();
}

cudaError_t dg_thermo_prim2cons(DgThermo* th, const double* w, void* u, cudaStream_t s) {
  if (th->f32)
    thermo_prim2cons_kernel<float><<<grid_of(th->K * th->np), 256, 0, s>>>(
        w, (float*)u, th->K, th->np, th->dim, th->species, th->T, (float*)th->pc);
  else
    thermo_prim2cons_kernel<double><<<grid_of(th->K * th->np), 256, 0, s>>>(
        w, (double*)u, th->K, th->np, th->dim, th->species, th->T, (double*)th->pc);
  return cudaGetLastError();
}
