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
#include <stdlib.h>
#include <string.h>

#include "../../include/dg.h"
#include "dg_internal.h"
#include "dg_mlp.cuh"
#include "dg_mlp_tc5.cuh"
#include "dg_thermo.h"

#define NSPEC 5
#define DG_RU 8.314462618
#define DG_P0 101325.0

namespace {

// Device tables (built by dg_chem_init from the species and reaction arrays):
// species rows [16]: 1e-6/W, 1e6 W, g/(RT) = h/(RT) - s/R as the coefficients of 1, T, T^2,
//   T^3, T^4 (from a1..a5 and a7), the 1/T coefficient a6 and the ln T coefficient a1,
//   1e-6 p0 / R_u and its reciprocal, slots 11-13 unused, ln(1e-6 p0 / R_u), 0;
// reaction rows [32]: nu'(5), nu''(5), third_body, eff(5), ln A, beta, theta,
//   dn = sum dnu, dnu(5), then (slot 25, as raw bits) the integer form of the row, and
//   dnu_s eff_s (5, slots 26-30); the integer form holds 2 bits
//   per species of nu' in {0..3} (bits 0-9) and nu'' (bits 10-19), the third-body flag (bit 20) and
//   one bit per species with dnu != 0 (bits 21-25), and, where k_b may be formed as a product
//   (sum |dnu_s| <= 15 and |dn| <= 3), sum |dnu_s| (bits 26-29) with bit 30 set.  The
//   integer form drives the uniform
//   branches of the reaction loop, so that no FP64 compare or conversion is spent on them.
#define SP_W 16
#define RX_W 32
#define RX_META 25

// c^nu for the stoichiometric coefficients nu in {1, 2, 3} (c2 = c c)
__device__ __forceinline__ double pow123(int nu, double c, double c2) {
  return nu == 1 ? c : (nu == 2 ? c2 : c2 * c);
}

// x^n for n in {-3..3} \ {0} from x and 1/x
__device__ __forceinline__ double ipow_pm3(int n, double x, double xi) {
  const double b = n > 0 ? x : xi;
  const int m = n > 0 ? n : -n;
  return m == 1 ? b : (m == 2 ? b * b : b * b * b);
}

// Plain FP64 source at one node: omega_s (kg/m^3/s) and the point-implicit terms
// jpi_s = max(0, -d omega_s / d rho_s) of the analytic diagonal Jacobian at fixed T.
// uu points at the node's first species density, stride np between variables.
// The Jacobian of reaction r with respect to c_s is M (nu'_s pf - nu''_s pb) / c_s plus, for
// third-body reactions, eff_s (pf - pb); the first part is summed over the reactions and
// divided by c_s once after the loop (c_s > 0), the explicit products are kept for c_s = 0.
template <typename T>
__device__ __forceinline__ void chem_node(const T* uu, int np, double Tk, const double* sp,
                                          const double* reac, int nr, double* om, double* jpi) {
  const double lnT = log(Tk), iT = 1.0 / Tk;
  // ln(1e-6 p0 / (R_u T)) = ln(1e-6 p0 / R_u) - ln T (the constant sits in species row 0)
  const double lnP = sp[14] - lnT;
  double c[NSPEC], c2[NSPEC], g[NSPEC], jd[NSPEC], j1[NSPEC];
  bool pos[NSPEC];
  double gmax = 0.0;
#pragma unroll
  for (int s = 0; s < NSPEC; ++s) {
    const double* q = sp + SP_W * s;
    c[s] = q[0] * (double)uu[s * np];
    c2[s] = c[s] * c[s];
    pos[s] = c[s] > 0.0;
    // g/(RT) = h/(RT) - s/R as one polynomial in T plus the 1/T and ln T terms
    g[s] = q[2] + Tk * (q[3] + Tk * (q[4] + Tk * (q[5] + Tk * q[6]))) + q[7] * iT - q[8] * lnT;
    gmax = fmax(gmax, fabs(g[s]));
    om[s] = 0.0;
    jd[s] = 0.0;
    j1[s] = 0.0;
  }
  // k_b = k_f X with X = exp(sum dnu_s g_s) P^-dn, P = 1e-6 p0 / (R_u T): from E_s = exp(g_s)
  // taken once per node, X is a product of powers of E_s, 1/E_s and P.  A reaction takes it
  // when every partial product stays inside the double range: sum |dnu_s| max|g_s| < 650
  // (the integer gcap bounds sum |dnu_s|; |P^-dn| adds at most e^42 for |dn| <= 3 and
  // 200 K <= T <= 10^4 K) and k_f is a normal number; otherwise one exp of the whole exponent.
  double E[NSPEC], Ei[NSPEC];
  const double P = sp[9] * iT, Pi = Tk * sp[10];
  const int gcap = gmax < 650.0 ? (gmax > 0.0 ? (int)fmin(650.0 / gmax, 64.0) : 64) : 0;
  if (gcap) {
#pragma unroll
    for (int s = 0; s < NSPEC; ++s) {
      E[s] = exp(g[s]);
      Ei[s] = 1.0 / E[s];
    }
  }
#pragma unroll 1
  for (int r = 0; r < nr; ++r) {
    const double* row = reac + RX_W * r;
    const int meta = (int)__double_as_longlong(row[RX_META]);
    const double lnkf = row[16] + row[17] * lnT - row[18] * iT;
    const double kf = exp(lnkf);
    double kb;
    // bits 26-29: sum |dnu_s|; bit 30: |dn| <= 3 (set at init)
    if ((meta >> 30) & 1 && ((meta >> 26) & 15) <= gcap && lnkf > -700.0) {
      double X = 1.0;
      int dn = 0;
#pragma unroll
      for (int s = 0; s < NSPEC; ++s) {
        const int ds = ((meta >> (10 + 2 * s)) & 3) - ((meta >> (2 * s)) & 3);
        dn += ds;
        if (ds) X *= ipow_pm3(ds, E[s], Ei[s]);
      }
      if (dn) X *= ipow_pm3(-dn, P, Pi);
      kb = kf * X;
    } else {
      double dg = 0.0;
#pragma unroll
      for (int s = 0; s < NSPEC; ++s)
        if (meta & (1 << (21 + s))) dg += row[20 + s] * g[s];
      kb = exp(lnkf + dg - row[19] * lnP);
    }
    double pf = kf, pb = kb;
#pragma unroll
    for (int s = 0; s < NSPEC; ++s) {
      const int a = (meta >> (2 * s)) & 3, b = (meta >> (10 + 2 * s)) & 3;
      if (a) pf *= pow123(a, c[s], c2[s]);
      if (b) pb *= pow123(b, c[s], c2[s]);
    }
    double M = 1.0;
    const bool tb = meta & (1 << 20);
    if (tb) {
      M = 0.0;
#pragma unroll
      for (int s = 0; s < NSPEC; ++s) M += row[11 + s] * c[s];
    }
    const double dp = pf - pb, Rr = dp * M;
#pragma unroll
    for (int s = 0; s < NSPEC; ++s) {
      if (!(meta & (1 << (21 + s)))) continue;  // the same for every node: no divergence
      const double d = row[20 + s];
      om[s] += d * Rr;
      if (tb) jd[s] += row[26 + s] * dp;  // dnu_s eff_s (pf - pb)
      const int a = (meta >> (2 * s)) & 3, b = (meta >> (10 + 2 * s)) & 3;
      if (!(a | b)) continue;
      if (pos[s]) {
        // nu'_s pf - nu''_s pb (the stoichiometric coefficients are exact small integers)
        const double t = row[s] * pf - row[5 + s] * pb;
        j1[s] += (tb ? d * M : d) * t;
      } else {
        // c_s = 0: the explicit products for nu = 1 (higher powers have zero derivative)
        double dpf = 0.0, dpb = 0.0;
        if (a == 1) {
          dpf = kf;
#pragma unroll
          for (int q = 0; q < NSPEC; ++q)
            if (q != s) {
              const int aq = (meta >> (2 * q)) & 3;
              if (aq) dpf *= pow123(aq, c[q], c2[q]);
            }
        }
        if (b == 1) {
          dpb = kb;
#pragma unroll
          for (int q = 0; q < NSPEC; ++q)
            if (q != s) {
              const int bq = (meta >> (10 + 2 * q)) & 3;
              if (bq) dpb *= pow123(bq, c[q], c2[q]);
            }
        }
        jd[s] += d * (dpf - dpb) * M;
      }
    }
  }
  // omega in kg/(m^3 s); d omega_s / d rho_s = 1e6 W_s (1e-6 / W_s) d(...)/dc_s = jd_s
#pragma unroll
  for (int s = 0; s < NSPEC; ++s) {
    if (pos[s]) jd[s] += j1[s] / c[s];
    om[s] *= sp[SP_W * s + 1];
    jpi[s] = -jd[s] > 0.0 ? -jd[s] : 0.0;
  }
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
    double om[NSPEC], jpi[NSPEC];
    chem_node<T>(u + k * nv * np + node, np, Tc[i], sp_raw, reac, nr, om, jpi);
    T* so = src + k * NSPEC * np + node;
#pragma unroll
    for (int s = 0; s < NSPEC; ++s) so[s * np] = (T)(om[s] / (1.0 + dt * jpi[s]));
  }
}

// ------------------------------------------------------------------ learned source
// Surrogate of (omega, jpi): 7 -> 64 -> 64 -> 10 perceptron on standardised features
// (Y_1..Y_5, ln rho, T); outputs are the standardised asinh images
// z_s = asinh(omega_s / omega_ref), z_{5+s} = asinh(jpi_s / jpi_ref).
// Acceptance, per tile of 32 nodes (one warp): every node inside the training box, every
// node's raw rates mass-balanced (|sum omega| <= tol_mass sum|omega| + floor), every
// node's learned update positive (rho_s + dt S_s >= 0), and one sampled node per tile
// (moved each call) within tol_check of the plain FP64 source; otherwise the tile's source
// is recomputed plainly.  Accepted rates are projected onto exact mass balance:
// omega_s -= |omega_s| sum(omega) / sum|omega|.
// With a refresh period (plain correction): a refresh evaluation takes the plain source at
// every node and stores, per node, the plain rates minus the network's decoded ones; the
// evaluations until the next refresh add those differences to the decoded rates before the
// tests, so the corrected network is exact at the refresh state.
struct __align__(16) DgChemMlp {
  DgMlpW<10> w;
  float mean[7], inv_std[7], muY[10], sdY[10], lo[7], hi[7];
  float w_ref, j_ref, tol_mass, floor32;
  double tol_check, floor;
};

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// raw features of one node: Y_1..Y_5, ln rho, T
template <typename T>
__device__ __forceinline__ void chem_features(const T* uu, int np, double Tk, float* x) {
  double r[NSPEC], rho = 0.0;
#pragma unroll
  for (int s = 0; s < NSPEC; ++s) {
    r[s] = (double)uu[s * np];
    rho += r[s];
  }
  const double ir = 1.0 / rho;
#pragma unroll
  for (int s = 0; s < NSPEC; ++s) x[s] = (float)(r[s] * ir);
  x[5] = (float)log(rho);
  x[6] = (float)Tk;
}

// The learned source on the fifth-generation tensor cores: CTAs of 128 threads take
// 128-node tiles through the tcgen05 tile engine (dg_mlp_tc5.cuh); each thread forms its
// node's features (and the trust-box test) before the two tensor-core layers and decodes
// its node's ten outputs after them (species sources, mass-balance test).  Flags per
// 32-node (warp) tile: 0 accepted, 1 rejected; a tile whose tensor-core waits ran out is
// rejected too, so the plain fallback recomputes it.
// corr ([10][K np], FP32) with cmode 1: the decoded rates are corrected by the stored
// plain-minus-network differences before the tests (omega_s + c_s, max(0, jpi'_s + c_5+s));
// cmode 2 (refresh): only the decoded rates (jpi' before its clamp) are written to corr,
// for chem_refresh_kernel to turn into corrections.
template <typename T>
__global__ void __launch_bounds__(dgtc5::THREADS, 1)
chem_mlp_tc5_kernel(const T* u, const double* Tc, int64_t K, int np, int dim, const DgChemMlp* mlp,
                    const double* dtp, T* src, unsigned char* flags, float* corr, const unsigned char* trust,
                    int cmode) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  dgtc5::Smem<10>& s = *reinterpret_cast<dgtc5::Smem<10>*>(smem_raw);
  __shared__ DgChemMlp m;
  dgmlp::copy_to_smem(m, mlp);
  __syncthreads();
  dgtc5::load_weights<10>(s, m.w);
  const int nv = NSPEC + dim + 1;
  const int64_t total = K * np;
  const float dt = dtp ? (float)*dtp : 0.f;
  auto prod = [&](int64_t i, float* x) {
    float raw[7];
    bool ok = true;
    if (i < total) {
      chem_features<T>(u + (i / np) * nv * np + (i % np), np, Tc[i], raw);
#pragma unroll
      for (int q = 0; q < 7; ++q) ok = ok && raw[q] >= m.lo[q] && raw[q] <= m.hi[q];
    } else {
#pragma unroll
      for (int q = 0; q < 7; ++q) raw[q] = m.mean[q];
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) x[q] = (raw[q] - m.mean[q]) * m.inv_std[q];
    x[7] = 0.f;
    return ok;
  };
  auto cons = [&](int64_t i, const float* y, bool ok, bool valid) {
    if (cmode == 2) {  // uniform over the grid: no lane reaches the vote below
      if (i < total && valid) {
#pragma unroll
        for (int q = 0; q < NSPEC; ++q) {
          corr[q * total + i] = m.w_ref * sinhf(m.muY[q] + m.sdY[q] * y[q]);
          corr[(5 + q) * total + i] = m.j_ref * sinhf(m.muY[5 + q] + m.sdY[5 + q] * y[5 + q]);
        }
      }
      return;
    }
    ok = ok && valid;
    if (i < total && valid) {
      float om[NSPEC], jp[NSPEC], msum = 0.f, asum = 0.f;
#pragma unroll
      for (int q = 0; q < NSPEC; ++q) {
        om[q] = m.w_ref * sinhf(m.muY[q] + m.sdY[q] * y[q]);
        float jr = m.j_ref * sinhf(m.muY[5 + q] + m.sdY[5 + q] * y[5 + q]);
        if (cmode == 1) {
          om[q] += corr[q * total + i];
          jr += corr[(5 + q) * total + i];
        }
        jp[q] = fmaxf(0.f, jr);
        msum += om[q];
        asum += fabsf(om[q]);
      }
      ok = ok && isfinite(asum) && fabsf(msum) <= m.tol_mass * asum + m.floor32;
      const float f = asum > 0.f ? msum / asum : 0.f;
      T* so = src + (i / np) * NSPEC * np + (i % np);
      // positivity of the learned update: rho_s + dt S_s >= 0 (the plain point-implicit
      // source never consumes a species faster than the step allows; a learned one can)
      const T* uu = u + (i / np) * nv * np + (i % np);
#pragma unroll
      for (int q = 0; q < NSPEC; ++q) {
        const float Sq = (om[q] - fabsf(om[q]) * f) / (1.f + dt * jp[q]);
        ok = ok && ((float)uu[q * np] + dt * Sq >= 0.f);
        so[q * np] = (T)Sq;
      }
    }
    const bool tile_ok = __all_sync(0xffffffffu, ok);
    const int64_t base = i - (threadIdx.x & 31);  // first node of this warp's 32-node tile
    if ((threadIdx.x & 31) == 0 && base < total) {
      // with corrections, a tile whose network missed the plain source at the last refresh
      // is not trusted until the next one
      const bool trusted = cmode != 1 || trust[base >> 5];
      flags[base >> 5] = !trusted ? 4 : (tile_ok ? 0 : 1);
    }
  };
  dgtc5::run_tiles<10>(s, total, prod, cons);
}

// one thread per tile still accepted: compare the learned source at the tile's sampled
// node with the plain FP64 source there
template <typename T>
__global__ void chem_check_kernel(const T* u, const double* Tc, int64_t K, int np, int dim,
                                  const double* sp_raw, const double* reac, int nr, const DgChemMlp* mlp,
                                  const double* dtp, const T* src, unsigned char* flags, uint64_t call) {
  const int nv = NSPEC + dim + 1;
  const int64_t total = K * np, ntiles = (total + 31) / 32;
  const double dt = dtp ? *dtp : 0.0;
  const double tol = mlp->tol_check, floor_ = mlp->floor;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (flags[t]) continue;
    const int64_t in_tile = total - t * 32 < 32 ? total - t * 32 : 32;
    const int64_t i = t * 32 + (int64_t)(splitmix64(call * 0x100000001B3ull + (uint64_t)t) % (uint64_t)in_tile);
    const int64_t k = i / np;
    const int node = (int)(i % np);
    double om[NSPEC], jpi[NSPEC], Sp[NSPEC], scale = 0.0;
    chem_node<T>(u + k * nv * np + node, np, Tc[i], sp_raw, reac, nr, om, jpi);
#pragma unroll
    for (int s = 0; s < NSPEC; ++s) {
      Sp[s] = om[s] / (1.0 + dt * jpi[s]);
      scale += fabs(Sp[s]);
    }
    bool ok = true;
#pragma unroll
    for (int s = 0; s < NSPEC; ++s) {
      const double Sm = (double)src[(k * NSPEC + s) * np + node];
      ok = ok && fabs(Sm - Sp[s]) <= tol * scale + floor_;
    }
    if (!ok) flags[t] = 2;
  }
}

// one warp per tile: recompute rejected tiles with the plain source; count nodes
template <typename T>
__global__ void __launch_bounds__(128)
chem_fallback_kernel(const T* u, const double* Tc, int64_t K, int np, int dim, const double* sp_raw,
                     const double* reac, int nr, const double* dtp, T* src, const unsigned char* flags,
                     unsigned long long* stats) {
  const int nv = NSPEC + dim + 1;
  const int lane = threadIdx.x & 31;
  const int64_t total = K * np, ntiles = (total + 31) / 32;
  const double dt = dtp ? *dtp : 0.0;
  unsigned long long n_ok = 0, n_fb = 0;
  for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < ntiles;
       t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t i = t * 32 + lane;
    if (i >= total) continue;
    if (!flags[t]) {
      ++n_ok;
      continue;
    }
    ++n_fb;
    const int64_t k = i / np;
    const int node = (int)(i % np);
    double om[NSPEC], jpi[NSPEC];
    chem_node<T>(u + k * nv * np + node, np, Tc[i], sp_raw, reac, nr, om, jpi);
    T* so = src + k * NSPEC * np + node;
#pragma unroll
    for (int s = 0; s < NSPEC; ++s) so[s * np] = (T)(om[s] / (1.0 + dt * jpi[s]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    n_ok += __shfl_xor_sync(0xffffffffu, n_ok, o);
    n_fb += __shfl_xor_sync(0xffffffffu, n_fb, o);
  }
  if (lane == 0 && (n_ok | n_fb)) {
    atomicAdd(&stats[0], n_ok);
    atomicAdd(&stats[1], n_fb);
  }
}

// refresh of the corrections: every node takes the plain FP64 source, and corr (holding
// the network's decoded rates of this state, written by chem_mlp_tc5_kernel in cmode 2)
// becomes the plain-minus-network differences; every tile is flagged 3 (plain).  The full
// check: each node's uncorrected learned source (projection, point-implicit factor) against
// the plain one with the sampled check's test; a tile is trusted until the next refresh when
// all of its nodes pass.  Threads are grouped in warps over whole 32-node tiles.
template <typename T>
__global__ void __launch_bounds__(128)
chem_refresh_kernel(const T* u, const double* Tc, int64_t K, int np, int dim, const double* sp_raw,
                    const double* reac, int nr, const DgChemMlp* mlp, const double* dtp, T* src, float* corr,
                    unsigned char* flags, unsigned char* trust) {
  const int nv = NSPEC + dim + 1;
  const int64_t total = K * np;
  const double dt = dtp ? *dtp : 0.0;
  const double tol = mlp->tol_check, floor_ = mlp->floor;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;  // a multiple of 32
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i - lane < total; i += stride) {
    bool ok = true;
    if (i < total) {
      const int64_t k = i / np;
      const int node = (int)(i % np);
      double om[NSPEC], jpi[NSPEC], Sp[NSPEC], oh[NSPEC], jh[NSPEC], scale = 0.0, msum = 0.0, asum = 0.0;
      chem_node<T>(u + k * nv * np + node, np, Tc[i], sp_raw, reac, nr, om, jpi);
      T* so = src + k * NSPEC * np + node;
#pragma unroll
      for (int s = 0; s < NSPEC; ++s) {
        Sp[s] = om[s] / (1.0 + dt * jpi[s]);
        so[s * np] = (T)Sp[s];
        scale += fabs(Sp[s]);
        oh[s] = (double)corr[s * total + i];
        jh[s] = (double)corr[(5 + s) * total + i];
        msum += oh[s];
        asum += fabs(oh[s]);
      }
      const double f = asum > 0.0 ? msum / asum : 0.0;
      ok = isfinite(asum);
#pragma unroll
      for (int s = 0; s < NSPEC; ++s) {
        const double Sl = (oh[s] - fabs(oh[s]) * f) / (1.0 + dt * fmax(0.0, jh[s]));
        ok = ok && fabs(Sl - Sp[s]) <= tol * scale + floor_;
        corr[s * total + i] = (float)(om[s] - oh[s]);
        corr[(5 + s) * total + i] = (float)(jpi[s] - jh[s]);
      }
    }
    const bool tile_ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) {
      flags[i >> 5] = 3;
      trust[i >> 5] = tile_ok ? 1 : 0;
    }
  }
}

// training data: raw features and the plain (omega, jpi) at counter-sampled nodes
template <typename T>
__global__ void chem_sample_kernel(const T* u, const double* Tc, int64_t K, int np, int dim,
                                   const double* sp_raw, const double* reac, int nr, int64_t n, uint64_t seed,
                                   float* X, double* Y) {
  const int nv = NSPEC + dim + 1;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (int64_t)(splitmix64(seed + (uint64_t)j) % (uint64_t)(K * np));
    const int64_t k = i / np;
    const int node = (int)(i % np);
    const T* uu = u + k * nv * np + node;
    chem_features<T>(uu, np, Tc[i], X + j * 7);
    chem_node<T>(uu, np, Tc[i], sp_raw, reac, nr, Y + j * 10, Y + j * 10 + 5);
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
  double* rows = (double*)calloc((size_t)RX_W * nr + SP_W * NSPEC, sizeof(double));
  if (!rows) return cudaErrorMemoryAllocation;
  for (int r = 0; r < nr; ++r) {
    const double* in = reac_host + 19 * r;  // [nu'(5), nu''(5), tb, eff(5), A, beta, theta]
    double* o = rows + RX_W * r;
    for (int q = 0; q < 16; ++q) o[q] = in[q];
    o[16] = log(in[16]);
    o[17] = in[17];
    o[18] = in[18];
    double dn = 0.0;
    long long meta = 0;
    for (int s = 0; s < NSPEC; ++s) {
      o[20 + s] = in[5 + s] - in[s];
      dn += o[20 + s];
      const double a = in[s], b = in[5 + s];
      if (!(a == 0.0 || a == 1.0 || a == 2.0 || a == 3.0) || !(b == 0.0 || b == 1.0 || b == 2.0 || b == 3.0)) {
        free(rows);  // the integer form holds nu in {0, 1, 2, 3}
        return cudaErrorInvalidValue;
      }
      meta |= (long long)a << (2 * s);
      meta |= (long long)b << (10 + 2 * s);
      if (o[20 + s] != 0.0) meta |= 1ll << (21 + s);
    }
    if (in[10] != 0.0) meta |= 1ll << 20;
    int sabs = 0, dnt = 0;
    for (int s = 0; s < NSPEC; ++s) {
      const int ds = (int)in[5 + s] - (int)in[s];
      sabs += ds < 0 ? -ds : ds;
      dnt += ds;
    }
    if (sabs <= 15 && dnt >= -3 && dnt <= 3) meta |= ((long long)sabs << 26) | (1ll << 30);
    o[19] = dn;
    memcpy(&o[RX_META], &meta, sizeof(meta));
    for (int s = 0; s < NSPEC; ++s) o[26 + s] = o[20 + s] * in[11 + s];  // dnu_s eff_s
  }
  double* sp = rows + (size_t)RX_W * nr;
  for (int s = 0; s < NSPEC; ++s) {
    const double* in = species_host + 8 * s;  // [W, a1..a7]
    double* o = sp + SP_W * s;
    // g/(RT) = h/(RT) - s/R = (a1 - a7) + T (a2/2 - a2) + T^2 (a3/3 - a3/2) + T^3 (a4/4 - a4/3)
    //         + T^4 (a5/5 - a5/4) + a6 / T - a1 ln T
    o[0] = 1e-6 / in[0];
    o[1] = 1e6 * in[0];
    o[2] = in[1] - in[7];
    o[3] = in[2] / 2.0 - in[2];
    o[4] = in[3] / 3.0 - in[3] / 2.0;
    o[5] = in[4] / 4.0 - in[4] / 3.0;
    o[6] = in[5] / 5.0 - in[5] / 4.0;
    o[7] = in[6];
    o[8] = in[1];
    o[9] = 1e-6 * DG_P0 / DG_RU;  // P = o[9] / T
    o[10] = DG_RU / (1e-6 * DG_P0);  // 1/P = o[10] T
    o[14] = log(1e-6 * DG_P0 / DG_RU);
  }
  const size_t rs = th->f32 ? sizeof(float) : sizeof(double);
  cudaError_t e = cudaMalloc((void**)&th->reac, sizeof(double) * RX_W * nr);
  if (e == cudaSuccess) e = cudaMemcpy(th->reac, rows, sizeof(double) * RX_W * nr, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&th->species_raw, sizeof(double) * SP_W * NSPEC);
  if (e == cudaSuccess) e = cudaMemcpy(th->species_raw, sp, sizeof(double) * SP_W * NSPEC, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&th->src, rs * NSPEC * th->K * th->np);
  free(rows);
  th->nr = nr;
  return e;
}

template <typename T>
static cudaError_t chem_learned(DgThermo* th, const T* u, const double* dt_dev, int refresh, cudaStream_t s) {
  const int64_t total = th->K * th->np, ntiles = (total + 31) / 32;
  const DgChemMlp* m = (const DgChemMlp*)th->chem_mlp;
  // tensor-core tiles of 128 nodes; the dynamic shared memory is padded to 60 KB so that at
  // most 3 CTAs (3 x 128 tensor-memory columns) share an SM
  const size_t smem = sizeof(dgtc5::Smem<10>) > 60 * 1024 ? sizeof(dgtc5::Smem<10>) : 60 * 1024;
  auto k1 = chem_mlp_tc5_kernel<T>;
  cudaError_t e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t t128 = (total + dgtc5::ROWS - 1) / dgtc5::ROWS;
  const unsigned g1 = (unsigned)(t128 < 152 * 3 ? t128 : 152 * 3);
  if (refresh) {
    if (!th->chem_corr || !th->chem_trust) return cudaErrorInvalidValue;
    k1<<<g1, dgtc5::THREADS, smem, s>>>(u, th->T, th->K, th->np, th->dim, m, dt_dev, (T*)th->src,
                                        th->chem_flags, th->chem_corr, th->chem_trust, 2);
    chem_refresh_kernel<T><<<grid_of(ntiles * 32), 128, 0, s>>>(u, th->T, th->K, th->np, th->dim,
                                                                th->species_raw, th->reac, th->nr, m, dt_dev,
                                                                (T*)th->src, th->chem_corr, th->chem_flags,
                                                                th->chem_trust);
    e = cudaGetLastError();
    if (e == cudaSuccess) th->corr_valid = 1;
    return e;
  }
  const int cmode = th->chem_corr && th->chem_trust && th->corr_valid ? 1 : 0;
  k1<<<g1, dgtc5::THREADS, smem, s>>>(u, th->T, th->K, th->np, th->dim, m, dt_dev, (T*)th->src, th->chem_flags,
                                      th->chem_corr, th->chem_trust, cmode);
  chem_check_kernel<T><<<grid_of(ntiles), 128, 0, s>>>(u, th->T, th->K, th->np, th->dim, th->species_raw,
                                                       th->reac, th->nr, m, dt_dev, (const T*)th->src,
                                                       th->chem_flags, th->chem_calls++);
  int64_t g3 = (ntiles + 3) / 4;
  if (g3 > 152 * 64) g3 = 152 * 64;
  chem_fallback_kernel<T><<<(unsigned)g3, 128, 0, s>>>(u, th->T, th->K, th->np, th->dim, th->species_raw,
                                                        th->reac, th->nr, dt_dev, (T*)th->src, th->chem_flags,
                                                        th->chem_stats);
  return cudaGetLastError();
}

cudaError_t dg_chem_source(DgThermo* th, const void* u, int f32, const double* dt_dev, int refresh,
                           cudaStream_t s) {
  if (th->chem_mlp)
    return f32 ? chem_learned<float>(th, (const float*)u, dt_dev, refresh, s)
               : chem_learned<double>(th, (const double*)u, dt_dev, refresh, s);
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

cudaError_t dg_chem_mlp_set(DgThermo* th, const float* params_host, const double* st) {
  th->corr_valid = 0;
  if (!params_host) {
    if (th->chem_mlp) cudaFree(th->chem_mlp);
    th->chem_mlp = NULL;
    return cudaSuccess;
  }
  DgChemMlp* h = (DgChemMlp*)calloc(1, sizeof(DgChemMlp));
  if (!h) return cudaErrorMemoryAllocation;
  dg_mlp_pack<10>(params_host, &h->w);
  for (int q = 0; q < 7; ++q) {
    h->mean[q] = (float)st[DG_SRC_X_MEAN + q];
    h->inv_std[q] = (float)(1.0 / st[DG_SRC_X_STD + q]);
    h->lo[q] = (float)st[DG_SRC_BOX_LO + q];
    h->hi[q] = (float)st[DG_SRC_BOX_HI + q];
  }
  for (int q = 0; q < 10; ++q) {
    h->muY[q] = (float)st[DG_SRC_Y_MEAN + q];
    h->sdY[q] = (float)st[DG_SRC_Y_STD + q];
  }
  h->w_ref = (float)st[DG_SRC_OMEGA_REF];
  h->j_ref = (float)st[DG_SRC_JPI_REF];
  h->tol_mass = (float)st[DG_SRC_TOL_MASS];
  h->tol_check = st[DG_SRC_TOL_CHECK];
  h->floor = st[DG_SRC_FLOOR];
  h->floor32 = (float)st[DG_SRC_FLOOR];
  const int64_t ntiles = (th->K * th->np + 31) / 32;
  cudaError_t e = cudaSuccess;
  if (!th->chem_mlp) e = cudaMalloc(&th->chem_mlp, sizeof(DgChemMlp));
  if (e == cudaSuccess && !th->chem_stats) e = cudaMalloc((void**)&th->chem_stats, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess && !th->chem_flags) e = cudaMalloc((void**)&th->chem_flags, (size_t)ntiles);
  if (e == cudaSuccess) e = cudaMemset(th->chem_stats, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemcpy(th->chem_mlp, h, sizeof(DgChemMlp), cudaMemcpyHostToDevice);
  free(h);
  return e;
}

cudaError_t dg_chem_sample_dev(DgThermo* th, const void* u, int f32, int64_t n, uint64_t seed, float* X,
                           double* targets, cudaStream_t s) {
  if (f32)
    chem_sample_kernel<float><<<grid_of(n), 128, 0, s>>>((const float*)u, th->T, th->K, th->np, th->dim,
                                                         th->species_raw, th->reac, th->nr, n, seed, X, targets);
  else
    chem_sample_kernel<double><<<grid_of(n), 128, 0, s>>>((const double*)u, th->T, th->K, th->np, th->dim,
                                                          th->species_raw, th->reac, th->nr, n, seed, X, targets);
  return cudaGetLastError();
}
