// Finite-rate chemistry source on the device (appendix, Chemical Kinetics: Eqs. nrp,
// forward_rate, backward, kedef, calc_prod), FP64, one thread per node.
//
// Concentrations c_s = 1e-6 rho_s / W_s (mol/cm^3, the units of Park-type constants);
// k_f = exp(ln A + beta ln T - theta/T); k_b = k_f / K_c with
// ln K_c = -sum dnu_s g_s/(R_u T) + (sum dnu_s) ln(1e-6 p0 / (R_u T)), p0 = 101325 Pa,
// g/(RT) = h/(RT) - s/R from each species' polynomial; rate of progress
// R_r = (k_f prod c^nu' - k_b prod c^nu'') (times sum eff_s c_s for third-body steps);
// omega_s = 1e6 W_s sum_r dnu_sr R_r (kg/m^3/s); point-implicit source
// S_s = omega_s / (1 + dt max(0, -d omega_s/d rho_s)) with the analytic diagonal
// Jacobian at fixed T, dt = the running RK step (0 outside RK stepping).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "dg_internal.h"
#include "dg_thermo.h"

#define NSPEC 5
#define DG_RU 8.314462618
#define DG_P0 101325.0

namespace {

// c^nu for the small non-negative integer stoichiometric coefficients (0..3 here)
__device__ __forceinline__ double ipow012(double c, double nu) {
  double r = 1.0;
  for (int q = 0; q < (int)nu; ++q) r *= c;
  return r;
}

template <typename T>
__global__ void chem_kernel(const T* u, const double* Tc, int64_t K, int np, int dim,
                            const double* sp_raw, const double* reac, int nr, const double* dtp,
                            T* src) {
  const int nv = NSPEC + dim + 1;
  const double dt = dtp ? *dtp : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K * np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / np;
    const int node = (int)(i % np);
    const T* uu = u + k * nv * np + node;
    const double Tk = Tc[k * np + node];
    const double lnT = log(Tk), iT = 1.0 / Tk;
    double c[NSPEC], g[NSPEC], om[NSPEC], jd[NSPEC];
#pragma unroll
    for (int s = 0; s < NSPEC; ++s) {
      const double* a = sp_raw + 8 * s + 1;
      c[s] = 1e-6 * (double)uu[s * np] / sp_raw[8 * s];
      const double h = a[0] + Tk * (a[1] / 2.0 + Tk * (a[2] / 3.0 + Tk * (a[3] / 4.0 + Tk * a[4] / 5.0))) + a[5] * iT;
      const double sr = a[0] * lnT + Tk * (a[1] + Tk * (a[2] / 2.0 + Tk * (a[3] / 3.0 + Tk * a[4] / 4.0))) + a[6];
      g[s] = h - sr;
      om[s] = 0.0;
      jd[s] = 0.0;
    }
    const double lnP = log(1e-6 * DG_P0 / (DG_RU * Tk));
    for (int r = 0; r < nr; ++r) {
      const double* row = reac + 20 * r;  // [nu'(5), nu''(5), tb, eff(5), lnA, beta, theta, 0]
      double dg = 0.0, dn = 0.0;
#pragma unroll
      for (int s = 0; s < NSPEC; ++s) {
        const double d = row[5 + s] - row[s];
        dg += d * g[s];
        dn += d;
      }
      const double lnkf = row[16] + row[17] * lnT - row[18] * iT;
      const double kf = exp(lnkf);
      const double kb = exp(lnkf + dg - dn * lnP);
      double pf = kf, pb = kb;
#pragma unroll
      for (int s = 0; s < NSPEC; ++s) {
        pf *= ipow012(c[s], row[s]);
        pb *= ipow012(c[s], row[5 + s]);
      }
      double M = 1.0;
      const bool tb = row[10] != 0.0;
      if (tb) {
        M = 0.0;
#pragma unroll
        for (int s = 0; s < NSPEC; ++s) M += row[11 + s] * c[s];
      }
      const double Rr = (pf - pb) * M;
#pragma unroll
      for (int s = 0; s < NSPEC; ++s) {
        const double d = row[5 + s] - row[s];
        om[s] += 1e6 * sp_raw[8 * s] * d * Rr;
        // d R_r / d c_s (explicit products when c_s = 0)
        double dpf = 0.0, dpb = 0.0;
        if (c[s] > 0.0) {
          dpf = row[s] > 0.0 ? pf * row[s] / c[s] : 0.0;
          dpb = row[5 + s] > 0.0 ? pb * row[5 + s] / c[s] : 0.0;
        } else {
          if (row[s] == 1.0) {
            dpf = kf;
            for (int q = 0; q < NSPEC; ++q) if (q != s) dpf *= ipow012(c[q], row[q]);
          }
          if (row[5 + s] == 1.0) {
            dpb = kb;
            for (int q = 0; q < NSPEC; ++q) if (q != s) dpb *= ipow012(c[q], row[5 + q]);
          }
        }
        jd[s] += d * ((dpf - dpb) * M + (tb ? (pf - pb) * row[11 + s] : 0.0));
      }
    }
    T* so = src + k * NSPEC * np + node;
#pragma unroll
    for (int s = 0; s < NSPEC; ++s) {
      const double dj = -jd[s] > 0.0 ? -jd[s] : 0.0;
      so[s * np] = (T)(om[s] / (1.0 + dt * dj));
    }
  }
}

unsigned grid_of(int64_t n) {
  int64_t g = (n + 127) / 128;
  if (g > 152 * 64) g = 152 * 64;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t dg_chem_init(DgThermo* th, const double* species_host, const double* reac_host, int nr) {
  if (nr < 1 || nr > 64) return cudaErrorInvalidValue;
  double* rows = (double*)malloc(sizeof(double) * 20 * nr);
  if (!rows) return cudaErrorMemoryAllocation;
  for (int r = 0; r < nr; ++r) {
    for (int q = 0; q < 16; ++q) rows[20 * r + q] = reac_host[19 * r + q];
    rows[20 * r + 16] = log(reac_host[19 * r + 16]);
    rows[20 * r + 17] = reac_host[19 * r + 17];
    rows[20 * r + 18] = reac_host[19 * r + 18];
    rows[20 * r + 19] = 0.0;
  }
  const size_t rs = th->f32 ? sizeof(float) : sizeof(double);
  cudaError_t e = cudaMalloc((void**)&th->reac, sizeof(double) * 20 * nr);
  if (e == cudaSuccess) e = cudaMemcpy(th->reac, rows, sizeof(double) * 20 * nr, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&th->species_raw, sizeof(double) * 8 * NSPEC);
  if (e == cudaSuccess)
    e = cudaMemcpy(th->species_raw, species_host, sizeof(double) * 8 * NSPEC, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&th->src, rs * NSPEC * th->K * th->np);
  free(rows);
  th->nr = nr;
  return e;
}

cudaError_t dg_chem_source(DgThermo* th, const void* u, int f32, const double* dt_dev, cudaStream_t s) {
  if (f32)
    chem_kernel<float><<<grid_of(th->K * th->np), 128, 0, s>>>(
        (const float*)u, th->T, th->K, th->np, th->dim, th->species_raw, th->reac, th->nr, dt_dev,
        (float*)th->src);
  else
    chem_kernel<double><<<grid_of(th->K * th->np), 128, 0, s>>>(
        (const double*)u, th->T, th->K, th->np, th->dim, th->species_raw, th->reac, th->nr, dt_dev,
        (double*)th->src);
  return cudaGetLastError();
}
