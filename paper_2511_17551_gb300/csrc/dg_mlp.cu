// Learned surrogates: training kernels (FP32, any number of outputs up to 16) and the
// temperature surrogate's BF16 tensor-core inference fused with the per-node FP64
// Newton polish and the Newton fallback.
//
// Temperature surrogate: x in R^7 -> 64 -> 64 -> 1, x = standardised (Y_1..Y_5, ln rho,
// e), output = standardised T.  Inference (dg_thermo_update in surrogate mode): 128-node
// tiles on the tcgen05 tensor cores (dg_mlp_tc5.cuh), then per node: one Newton step from
// the prediction, accept when the next correction would be <= 1e-6 T, otherwise run the
// plain Newton iteration (fallback, counted).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "../../include/dg.h"
#include "dg_internal.h"
#include "dg_mlp.cuh"
#include "dg_mlp_tc5.cuh"
#include "dg_thermo.h"

#define NI DG_MLP_NI
#define NH DG_MLP_NH
#define NO_MAX DG_MLP_NO_MAX
#define DG_RU 8.314462618
#define NSPEC 5

// temperature surrogate: weights and input / output standardisation
struct __align__(16) DgMlpDev {
  DgMlpW<1> w;
  float mean[NI], inv_std[NI];
  float muT, sigT;
};

namespace {
using namespace dgmlp;

struct PolyD {
  double b[6], Rmix;
  __device__ __forceinline__ double e(double T) const {
    return b[0] + T * (b[1] + T * (b[2] + T * (b[3] + T * (b[4] + T * b[5]))));
  }
  __device__ __forceinline__ double cv(double T) const {
    return b[1] + T * (2.0 * b[2] + T * (3.0 * b[3] + T * (4.0 * b[4] + T * (5.0 * b[5]))));
  }
};

// mixture polynomial from the per-species coefficient rows of the context
// ([R a6, R (a1-1), R a2/2, R a3/3, R a4/4, R a5/5, R, 0] per species)
__device__ __forceinline__ void poly_d(const double* cf, const double* Y, PolyD& P) {
#pragma unroll
  for (int k = 0; k < 6; ++k) P.b[k] = 0.0;
  P.Rmix = 0.0;
#pragma unroll
  for (int s = 0; s < NSPEC; ++s) {
#pragma unroll
    for (int k = 0; k < 6; ++k) P.b[k] += Y[s] * cf[8 * s + k];
    P.Rmix += Y[s] * cf[8 * s + 6];
  }
}

__device__ __forceinline__ double clampT(double T) { return T < 200.0 ? 200.0 : (T > 1e4 ? 1e4 : T); }

#define MLP_WARPS 4

// Temperature surrogate on the fifth-generation tensor cores: CTAs of 128 threads take
// 128-node tiles through the tcgen05 tile engine (dg_mlp_tc5.cuh).  Each thread forms its
// node's features before the two tensor-core layers and, after them, polishes the
// predicted temperature by one Newton step with the residual check, or runs the plain
// Newton iteration (fallback, counted; also when the engine's waits ran out).
template <typename T>
__global__ void __launch_bounds__(dgtc5::THREADS, 1)
thermo_mlp_kernel(const T* u, int64_t K, int np, int dim, const double* sp, const float* sp32, double* Tc,
                  T* pc, unsigned long long* status, const DgMlpDev* mlp, unsigned long long* stats) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  dgtc5::Smem<1>& sm = *reinterpret_cast<dgtc5::Smem<1>*>(smem_raw);
  __shared__ DgMlpDev m;
  copy_to_smem(m, mlp);
  __syncthreads();
  dgtc5::load_weights<1>(sm, m.w);
  const int nv = NSPEC + dim + 1;
  const int64_t total = K * np;
  unsigned long long n_ok = 0, n_fb = 0;
  double Y[NSPEC], rho = 1.0, e = 0.0;  // this thread's node, carried from features to polish
  auto prod = [&](int64_t i, float* x) {
    if (i < total) {
      const T* uu = u + (i / np) * nv * np + (i % np);
      rho = 0.0;
#pragma unroll
      for (int q = 0; q < NSPEC; ++q) {
        Y[q] = (double)uu[q * np];
        rho += Y[q];
      }
      double ke = 0.0;
      for (int d = 0; d < dim; ++d) {
        const double mm = (double)uu[(NSPEC + d) * np];
        ke += mm * mm;
      }
      const double ir = 1.0 / rho;
      e = (double)uu[(NSPEC + dim) * np] * ir - 0.5 * ke * ir * ir;
#pragma unroll
      for (int q = 0; q < NSPEC; ++q) Y[q] *= ir;
    } else {
      rho = 1.0;
      e = 0.0;
#pragma unroll
      for (int q = 0; q < NSPEC; ++q) Y[q] = 0.2;
    }
    float f[NI];
#pragma unroll
    for (int q = 0; q < NSPEC; ++q) f[q] = (float)Y[q];
    f[5] = logf((float)rho);
    f[6] = (float)e;
#pragma unroll
    for (int q = 0; q < NI; ++q) x[q] = (f[q] - m.mean[q]) * m.inv_std[q];
    x[7] = 0.f;
    return true;
  };
  // the plain FP64 Newton iteration from T1 (fallback); false when it did not converge
  auto newton = [&](const PolyD& P, double& T1) {
    for (int it = 0; it < 50; ++it) {
      const double Tn = clampT(T1 - (P.e(T1) - e) / P.cv(T1));
      const double step = fabs(Tn - T1);
      T1 = Tn;
      if (step <= 1e-12 * T1) return true;
    }
    return false;
  };
  auto cons = [&](int64_t i, const float* y, bool, bool valid) {
    if (i >= total) return;
    const int64_t k = i / np;
    const int node = (int)(i % np);
    if (sizeof(T) == 4) {
      // mixed form: the same equation as its plain solve -- FP64 formation-energy constant
      // b0, FP32-rounded temperature coefficients, FP64 residual -- so accepted nodes and
      // the plain path agree to the acceptance tolerance
      float c32[6], R32 = 0.f;
      double b0 = 0.0;
#pragma unroll
      for (int q = 0; q < 6; ++q) c32[q] = 0.f;
#pragma unroll
      for (int q = 0; q < NSPEC; ++q) {
        b0 += Y[q] * sp[8 * q];
        const float yf = (float)Y[q];
#pragma unroll
        for (int r = 1; r < 6; ++r) c32[r] += yf * sp32[8 * q + r];
        R32 += yf * sp32[8 * q + 6];
      }
      auto e64 = [&](double t) {
        return b0 + t * ((double)c32[1] + t * ((double)c32[2] + t * ((double)c32[3] +
                         t * ((double)c32[4] + t * (double)c32[5]))));
      };
      auto cv32 = [&](float t) {
        return c32[1] + t * (2.f * c32[2] + t * (3.f * c32[3] + t * (4.f * c32[4] + t * 5.f * c32[5])));
      };
      double T1 = 1000.0;
      bool acc = false;
      if (valid) {
        const double T0 = clampT((double)(m.muT + m.sigT * y[0]));
        const float cv0 = cv32((float)T0);
        T1 = clampT(T0 - (e64(T0) - e) * (double)(1.0f / cv0));
        acc = fabs(e64(T1) - e) <= 1e-6 * (double)cv0 * T1;
      }
      if (acc) {
        ++n_ok;
      } else {
        ++n_fb;
        PolyD P;
        poly_d(sp, Y, P);
        if (!newton(P, T1)) atomicCAS(status, 0ull, (DG_ST_NEWTON << 56) | (unsigned long long)k);
      }
      Tc[k * np + node] = T1;
      const float Tq = (float)T1, rhof = (float)rho;
      const float pf = rhof * R32 * Tq, cvf = cv32(Tq);
      pc[(k * 2 + 0) * np + node] = (T)pf;
      pc[(k * 2 + 1) * np + node] = (T)sqrtf((cvf + R32) / cvf * pf / rhof);
    } else {
      PolyD P;
      poly_d(sp, Y, P);
      double T1 = 1000.0;
      bool acc = false;
      if (valid) {
        const double T0 = clampT((double)(m.muT + m.sigT * y[0]));
        // FP64 residuals; cv only scales the correction, FP32 is enough for it
        const float cv0 = (float)P.b[1] + (float)T0 * (2.f * (float)P.b[2] + (float)T0 *
                          (3.f * (float)P.b[3] + (float)T0 * (4.f * (float)P.b[4] + (float)T0 * 5.f * (float)P.b[5])));
        T1 = clampT(T0 - (P.e(T0) - e) / (double)cv0);
        acc = fabs(P.e(T1) - e) <= 1e-6 * (double)cv0 * T1;
      }
      if (acc) {
        ++n_ok;
      } else {
        ++n_fb;
        if (!newton(P, T1)) atomicCAS(status, 0ull, (DG_ST_NEWTON << 56) | (unsigned long long)k);
      }
      Tc[k * np + node] = T1;
      const double p = rho * P.Rmix * T1, cv = P.cv(T1);
      pc[(k * 2 + 0) * np + node] = (T)p;
      pc[(k * 2 + 1) * np + node] = (T)sqrt((cv + P.Rmix) / cv * p / rho);
    }
  };
  dgtc5::run_tiles<1>(sm, total, prod, cons);
  if (stats) {
    for (int o = 16; o > 0; o >>= 1) {
      n_ok += __shfl_xor_sync(0xffffffffu, n_ok, o);
      n_fb += __shfl_xor_sync(0xffffffffu, n_fb, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats[0], n_ok);
      atomicAdd(&stats[1], n_fb);
    }
  }
}

// plain tensor-core forward for standardised inputs X[n][7] -> y[n][NO] (checks)
template <int NO>
__global__ void __launch_bounds__(32 * MLP_WARPS)
mlp_forward_tc_kernel(const DgMlpW<NO>* mlp, const float* X, float* y, int64_t n) {
  __shared__ DgMlpW<NO> m;
  __shared__ float feat[MLP_WARPS][16][17];
  __shared__ float yv[MLP_WARPS][NO][16];
  copy_to_smem(m, mlp);
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t base = ((int64_t)blockIdx.x * MLP_WARPS + w) * 16; base < n;
       base += (int64_t)gridDim.x * MLP_WARPS * 16) {
    if (lane < 16) {
      const int64_t i = base + lane;
#pragma unroll
      for (int q = 0; q < 17; ++q) feat[w][lane][q] = (i < n && q < NI) ? X[i * NI + q] : 0.f;
    }
    __syncwarp();
    mlp16<NO>(m, feat[w], yv[w]);
    __syncwarp();
    if (lane < 16 && base + lane < n)
      for (int o = 0; o < NO; ++o) y[(base + lane) * NO + o] = yv[w][o][lane];
    __syncwarp();
  }
}

// FP32 SIMT forward of one sample per thread (reference path of the device code)
__global__ void mlp_forward_f32_kernel(const float* P, int no, const float* X, float* y, int64_t n) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    float h1[NH], h2[NH];
    for (int j = 0; j < NH; ++j) {
      float a = P[NH * NI + j];
      for (int k = 0; k < NI; ++k) a += P[j * NI + k] * X[s * NI + k];
      h1[j] = gelu_f(a);
    }
    for (int j = 0; j < NH; ++j) {
      float a = P[NH * NI + NH + NH * NH + j];
      for (int i = 0; i < NH; ++i) a += P[NH * NI + NH + j * NH + i] * h1[i];
      h2[j] = gelu_f(a);
    }
    for (int o = 0; o < no; ++o) {
      float out = P[dg_mlp_off_b3(no) + o];
      for (int j = 0; j < NH; ++j) out += P[dg_mlp_off_w3() + o * NH + j] * h2[j];
      y[s * no + o] = out;
    }
  }
}

// ------------------------------------------------------------------ training (FP32)
#define TS 32  // samples per tile
#define OFF_W1 0
#define OFF_B1 (NH * NI)
#define OFF_W2 (OFF_B1 + NH)
#define OFF_B2 (OFF_W2 + NH * NH)
struct TrainSmem {
  float W1[NH * NI], b1[NH], W2[NH * NH], W2T[NH * NH], b2[NH], W3[NO_MAX * NH], b3[NO_MAX];
  float X[TS][NI], a1[TS][NH], h1[TS][NH], a2[TS][NH], h2[TS][NH];
  float dy[TS][NO_MAX], r2[TS][NO_MAX];
  float g[dg_mlp_np(NO_MAX)];  // gW2 stored transposed [i][j]
  float loss;
};

// per-CTA partial gradients of loss = (1/(B no)) sum_s sum_o (y_so - t_so)^2 over the
// CTA's tiles
__global__ void __launch_bounds__(NH) mlp_grad_kernel(const float* P, int no, const float* X, const float* t,
                                                      int B, float* partial) {
  extern __shared__ __align__(16) unsigned char raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(raw);
  const int j = threadIdx.x;
  const int OW3 = dg_mlp_off_w3(), OB3 = dg_mlp_off_b3(no), NPAR = dg_mlp_np(no);
  for (int q = j; q < NH * NI; q += NH) S.W1[q] = P[OFF_W1 + q];
  for (int q = j; q < NH * NH; q += NH) {
    S.W2[q] = P[OFF_W2 + q];
    S.W2T[(q % NH) * NH + q / NH] = P[OFF_W2 + q];
  }
  S.b1[j] = P[OFF_B1 + j];
  S.b2[j] = P[OFF_B2 + j];
  for (int o = 0; o < no; ++o) S.W3[o * NH + j] = P[OW3 + o * NH + j];
  if (j < no) S.b3[j] = P[OB3 + j];
  if (j == 0) S.loss = 0.f;
  for (int q = j; q < NPAR; q += NH) S.g[q] = 0.f;
  __syncthreads();
  const float inv = 1.0f / ((float)B * (float)no);
  for (int s0 = blockIdx.x * TS; s0 < B; s0 += gridDim.x * TS) {
    const int ns = min(TS, B - s0);
    for (int q = j; q < TS * NI; q += NH) S.X[q / NI][q % NI] = q / NI < ns ? X[(int64_t)s0 * NI + q] : 0.f;
    __syncthreads();
    for (int s = 0; s < ns; ++s) {
      float a = S.b1[j];
#pragma unroll
      for (int k = 0; k < NI; ++k) a += S.W1[j * NI + k] * S.X[s][k];
      S.a1[s][j] = a;
      S.h1[s][j] = gelu_f(a);
    }
    __syncthreads();
    for (int s = 0; s < ns; ++s) {
      float a = S.b2[j];
      for (int i = 0; i < NH; ++i) a += S.W2T[i * NH + j] * S.h1[s][i];
      S.a2[s][j] = a;
      S.h2[s][j] = gelu_f(a);
    }
    __syncthreads();
    for (int q = j; q < ns * no; q += NH) {
      const int s = q / no, o = q % no;
      float y = S.b3[o];
      for (int i = 0; i < NH; ++i) y += S.W3[o * NH + i] * S.h2[s][i];
      const float r = y - t[(int64_t)(s0 + s) * no + o];
      S.dy[s][o] = 2.0f * r * inv;
      S.r2[s][o] = r * r * inv;
    }
    __syncthreads();
    if (j == 0)  // fixed order: deterministic
      for (int s = 0; s < ns; ++s)
        for (int o = 0; o < no; ++o) S.loss += S.r2[s][o];
    float gb2 = 0.f;
    for (int o = 0; o < no; ++o) {
      float gw3 = 0.f;
      for (int s = 0; s < ns; ++s) gw3 += S.dy[s][o] * S.h2[s][j];
      S.g[OW3 + o * NH + j] += gw3;
    }
    for (int s = 0; s < ns; ++s) {
      float back = 0.f;
      for (int o = 0; o < no; ++o) back += S.dy[s][o] * S.W3[o * NH + j];
      const float d2 = back * gelu_d_f(S.a2[s][j]);
      S.a2[s][j] = d2;  // a2 now holds delta2
      gb2 += d2;
    }
    S.g[OFF_B2 + j] += gb2;
    if (j < no) {
      float gb3 = 0.f;
      for (int s = 0; s < ns; ++s) gb3 += S.dy[s][j];
      S.g[OB3 + j] += gb3;
    }
    __syncthreads();
    // thread j: row j of dW2 (stored transposed) and delta1 of hidden unit j
    for (int i = 0; i < NH; ++i) {
      float acc = 0.f;
      for (int s = 0; s < ns; ++s) acc += S.a2[s][j] * S.h1[s][i];
      S.g[OFF_W2 + i * NH + j] += acc;
    }
    float gb1 = 0.f, gw1[NI] = {0, 0, 0, 0, 0, 0, 0};
    for (int s = 0; s < ns; ++s) {
      float acc = 0.f;
      for (int q = 0; q < NH; ++q) acc += S.W2[q * NH + j] * S.a2[s][q];
      const float d1 = acc * gelu_d_f(S.a1[s][j]);
      gb1 += d1;
#pragma unroll
      for (int k = 0; k < NI; ++k) gw1[k] += d1 * S.X[s][k];
    }
    S.g[OFF_B1 + j] += gb1;
#pragma unroll
    for (int k = 0; k < NI; ++k) S.g[OFF_W1 + j * NI + k] += gw1[k];
    __syncthreads();
  }
  float* out = partial + (int64_t)blockIdx.x * (NPAR + 1);
  for (int q = j; q < NPAR; q += NH) {
    if (q >= OFF_W2 && q < OFF_W2 + NH * NH) {  // back to row-major [j][i]
      const int i = (q - OFF_W2) / NH, jj = (q - OFF_W2) % NH;
      out[OFF_W2 + jj * NH + i] = S.g[q];
    } else {
      out[q] = S.g[q];
    }
  }
  if (j == 0) out[NPAR] = S.loss;
}

// fixed-order sum of the partial gradients, then (optionally) one Adam step
__global__ void mlp_reduce_adam_kernel(const float* partial, int nb, int npar, float* grad, float* P, float* mo,
                                       float* vo, int step, float lr, float b1, float b2, float eps,
                                       double* loss) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > npar) return;
  float s = 0.f;
  for (int b = 0; b < nb; ++b) s += partial[(int64_t)b * (npar + 1) + q];
  if (q == npar) {
    if (loss) *loss = (double)s;
    return;
  }
  if (grad) grad[q] = s;
  if (P) {
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    const float m = b1 * mo[q] + (1.0f - b1) * s;
    const float v = b2 * vo[q] + (1.0f - b2) * s * s;
    mo[q] = m;
    vo[q] = v;
    P[q] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}

// counter-based sampling of node states (splitmix64 of seed + index)
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

template <typename T>
__global__ void sample_kernel(const T* u, const double* Tc, int64_t K, int np, int dim, int64_t n,
                              uint64_t seed, float* X, float* Tout) {
  const int nv = NSPEC + dim + 1;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (int64_t)(splitmix64(seed + (uint64_t)j) % (uint64_t)(K * np));
    const int64_t k = i / np;
    const int node = (int)(i % np);
    const T* uu = u + k * nv * np + node;
    double rho = 0.0, ke = 0.0;
    for (int s = 0; s < NSPEC; ++s) rho += (double)uu[s * np];
    for (int d = 0; d < dim; ++d) {
      const double mm = (double)uu[(NSPEC + d) * np];
      ke += mm * mm;
    }
    for (int s = 0; s < NSPEC; ++s) X[j * NI + s] = (float)((double)uu[s * np] / rho);
    X[j * NI + 5] = (float)log(rho);
    X[j * NI + 6] = (float)((double)uu[(NSPEC + dim) * np] / rho - 0.5 * ke / (rho * rho));
    Tout[j] = (float)Tc[i];
  }
}

unsigned grid_of(int64_t n, int bs) {
  int64_t g = (n + bs - 1) / bs;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

void pack_host(const float* params, const double* stats, DgMlpDev* h) {
  memset(h, 0, sizeof(*h));
  dg_mlp_pack<1>(params, &h->w);
  for (int q = 0; q < NI; ++q) {
    h->mean[q] = (float)stats[q];
    h->inv_std[q] = (float)(1.0 / stats[NI + q]);
  }
  h->muT = (float)stats[2 * NI];
  h->sigT = (float)stats[2 * NI + 1];
}

}  // namespace

// ---------------------------------------------------------------- thermo hooks
cudaError_t dg_mlp_set(DgThermo* th, const float* params_host, const double* stats_host) {
  if (!params_host) {
    if (th->mlp) cudaFree(th->mlp);
    th->mlp = NULL;
    return cudaSuccess;
  }
  DgMlpDev h;
  pack_host(params_host, stats_host, &h);
  cudaError_t e = cudaSuccess;
  if (!th->mlp) e = cudaMalloc(&th->mlp, sizeof(DgMlpDev));
  if (e == cudaSuccess && !th->mlp_stats) e = cudaMalloc((void**)&th->mlp_stats, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(th->mlp_stats, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemcpy(th->mlp, &h, sizeof(h), cudaMemcpyHostToDevice);
  return e;
}

cudaError_t dg_mlp_thermo_update(DgThermo* th, const void* u, int f32, cudaStream_t s) {
  const int64_t n = th->K * th->np;
  // tensor-core tiles of 128 nodes; the dynamic shared memory is padded to 60 KB so that at
  // most 3 CTAs (3 x 128 tensor-memory columns) share an SM
  const size_t smem = sizeof(dgtc5::Smem<1>) > 60 * 1024 ? sizeof(dgtc5::Smem<1>) : 60 * 1024;
  const int64_t t128 = (n + dgtc5::ROWS - 1) / dgtc5::ROWS;
  const unsigned grid = (unsigned)(t128 < 152 * 3 ? t128 : 152 * 3);
  cudaError_t e;
  if (f32) {
    auto k = thermo_mlp_kernel<float>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, dgtc5::THREADS, smem, s>>>((const float*)u, th->K, th->np, th->dim, th->species, th->coef32, th->T,
                                         (float*)th->pc, th->status, (const DgMlpDev*)th->mlp, th->mlp_stats);
  } else {
    auto k = thermo_mlp_kernel<double>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, dgtc5::THREADS, smem, s>>>((const double*)u, th->K, th->np, th->dim, th->species, th->coef32,
                                         th->T, (double*)th->pc, th->status, (const DgMlpDev*)th->mlp,
                                         th->mlp_stats);
  }
  return cudaGetLastError();
}

cudaError_t dg_mlp_sample(DgThermo* th, const void* u, int f32, int64_t n, uint64_t seed, float* X,
                          float* T, cudaStream_t s) {
  if (f32)
    sample_kernel<float><<<grid_of(n, 256), 256, 0, s>>>((const float*)u, th->T, th->K, th->np, th->dim,
                                                         n, seed, X, T);
  else
    sample_kernel<double><<<grid_of(n, 256), 256, 0, s>>>((const double*)u, th->T, th->K, th->np, th->dim,
                                                          n, seed, X, T);
  return cudaGetLastError();
}

// tcgen05 forward: persistent CTAs of 128 threads over 128-row tiles; the dynamic
// shared memory is padded to 60 KB so that at most 3 CTAs (3 x 128 tensor-memory columns)
// share an SM
__device__ unsigned g_tc5_err;
template <int NO>
static dg_status forward_tc5(const float* P, const float* X, float* y, int64_t n, cudaStream_t st) {
  const size_t smem = sizeof(dgtc5::Smem<NO>) > 60 * 1024 ? sizeof(dgtc5::Smem<NO>) : 60 * 1024;
  auto k = dgtc5::mlp_forward_tc5_kernel<NO>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return DG_ECUDA;
  unsigned* err = NULL;
  if (cudaGetSymbolAddress((void**)&err, g_tc5_err) != cudaSuccess) return DG_ECUDA;
  if (cudaMemsetAsync(err, 0, sizeof(unsigned), st) != cudaSuccess) return DG_ECUDA;
  const int64_t tiles = (n + dgtc5::ROWS - 1) / dgtc5::ROWS;
  const unsigned grid = (unsigned)(tiles < 152 * 3 ? tiles : 152 * 3);
  k<<<grid, dgtc5::THREADS, smem, st>>>(P, X, y, n, err);
  if (cudaGetLastError() != cudaSuccess) return DG_ECUDA;
  unsigned h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DG_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return DG_ECUDA;
  return h ? DG_ETIMEOUT : DG_OK;
}

template <int NO>
static dg_status forward_tc(const float* hp, const float* X, float* y, int64_t n, cudaStream_t st) {
  DgMlpW<NO> h;
  memset(&h, 0, sizeof(h));
  dg_mlp_pack<NO>(hp, &h);
  DgMlpW<NO>* d = NULL;
  if (cudaMalloc((void**)&d, sizeof(h)) != cudaSuccess) return DG_ENOMEM;
  cudaError_t e = cudaMemcpy(d, &h, sizeof(h), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    mlp_forward_tc_kernel<NO><<<grid_of((n + 15) / 16, MLP_WARPS), 32 * MLP_WARPS, 0, st>>>(d, X, y, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  return e == cudaSuccess ? DG_OK : DG_ECUDA;
}

// FP32 forward launch for the data-preparation module (dg_data.cu)
cudaError_t dg_mlp_forward_f32_launch(const float* P, int no, const float* X, float* y, int64_t n, cudaStream_t s) {
  mlp_forward_f32_kernel<<<grid_of(n, 128), 128, 0, s>>>(P, no, X, y, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- C ABI (training)
extern "C" {

int dg_mlp_nparams(int n_out) { return n_out >= 1 && n_out <= NO_MAX ? dg_mlp_np(n_out) : -1; }

size_t dg_mlp_workspace_bytes(int batch, int n_out) {
  if (batch < 1 || n_out < 1 || n_out > NO_MAX) return 0;
  int nb = (batch + TS - 1) / TS;
  if (nb > 152) nb = 152;
  return sizeof(float) * (size_t)nb * (dg_mlp_np(n_out) + 1);
}

static dg_status grad_common(const float* P, int no, const float* X, const float* t, int B, float* ws,
                             size_t ws_bytes, cudaStream_t st, int* nb_out) {
  if (!P || !X || !t || !ws || B < 1 || no < 1 || no > NO_MAX) return DG_EINVAL;
  if (ws_bytes < dg_mlp_workspace_bytes(B, no)) return DG_EINVAL;
  int nb = (B + TS - 1) / TS;
  if (nb > 152) nb = 152;
  const size_t smem = sizeof(TrainSmem);
  if (cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return DG_ECUDA;
  mlp_grad_kernel<<<nb, NH, smem, st>>>(P, no, X, t, B, ws);
  if (cudaGetLastError() != cudaSuccess) return DG_ECUDA;
  *nb_out = nb;
  return DG_OK;
}

dg_status dg_mlp_grad(const float* params, int n_out, const float* X, const float* t, int batch, float* grad,
                      double* loss, float* workspace, size_t ws_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int nb = 0;
  dg_status r = grad_common(params, n_out, X, t, batch, workspace, ws_bytes, st, &nb);
  if (r != DG_OK) return r;
  if (!grad) return DG_EINVAL;
  const int npar = dg_mlp_np(n_out);
  mlp_reduce_adam_kernel<<<(npar + 1 + 255) / 256, 256, 0, st>>>(workspace, nb, npar, grad, NULL, NULL, NULL, 0,
                                                                 0.f, 0.f, 0.f, 0.f, loss);
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_ECUDA;
}

dg_status dg_mlp_train_step(float* params, int n_out, float* m, float* v, const float* X, const float* t,
                            int batch, int step, float lr, double* loss, float* workspace, size_t ws_bytes,
                            void* stream) {
  if (!m || !v || step < 1 || !(lr > 0.f)) return DG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int nb = 0;
  dg_status r = grad_common(params, n_out, X, t, batch, workspace, ws_bytes, st, &nb);
  if (r != DG_OK) return r;
  const int npar = dg_mlp_np(n_out);
  mlp_reduce_adam_kernel<<<(npar + 1 + 255) / 256, 256, 0, st>>>(workspace, nb, npar, NULL, params, m, v, step,
                                                                 lr, 0.9f, 0.999f, 1e-8f, loss);
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_ECUDA;
}

dg_status dg_mlp_forward(const float* params, int n_out, const float* X, float* y, int64_t n, int tensor_cores,
                         void* stream) {
  if (!params || !X || !y || n < 1 || n_out < 1 || n_out > NO_MAX) return DG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!tensor_cores) {
    mlp_forward_f32_kernel<<<grid_of(n, 128), 128, 0, st>>>(params, n_out, X, y, n);
    return cudaGetLastError() == cudaSuccess ? DG_OK : DG_ECUDA;
  }
  if (n_out != 1 && n_out != 10) return DG_EINVAL;  // the surrogates' output counts
  if (tensor_cores == 2) return n_out == 1 ? forward_tc5<1>(params, X, y, n, st) : forward_tc5<10>(params, X, y, n, st);
  if (tensor_cores != 1) return DG_EINVAL;
  const int npar = dg_mlp_np(n_out);
  float* hp = (float*)malloc(sizeof(float) * npar);
  if (!hp) return DG_ENOMEM;
  if (cudaMemcpy(hp, params, sizeof(float) * npar, cudaMemcpyDeviceToHost) != cudaSuccess) {
    free(hp);
    return DG_ECUDA;
  }
  dg_status r = n_out == 1 ? forward_tc<1>(hp, X, y, n, st) : forward_tc<10>(hp, X, y, n, st);
  free(hp);
  return r;
}

}  // extern "C"
