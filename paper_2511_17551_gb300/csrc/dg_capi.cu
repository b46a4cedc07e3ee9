// C ABI of libdg (see include/dg.h): context management, set-up kernels (metric
// terms, primitive -> conserved), state transfer, RK driver and FP64 domain
// integrals.  The right-hand-side kernels live in dg_rhs_f64.cu / dg_rhs_f32.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <utility>

#include "../../include/dg.h"
#include "dg_internal.h"
#include "dg_thermo.h"

struct dg_ctx {
  int dev;
  int dim, N, np, nv, nsp, nf;
  int64_t K;
  int equations, n_species, vf, sf, precision, thermo, n_bc;
  int has_bnd;  // the mesh has boundary faces
  double gamma, mu, Pr, alpha_max, p_ref, pos_eps;
  double suth_s, suth_rt;
  int ind_var;
  double pos_ef[8];  // mixture limiter: e_s(T_floor) per unit mass
  unsigned long long* pos_count;  // elements changed by the positivity limiter
  cudaStream_t stream;
  bool own_stream;
  size_t rs;  // bytes per real of the form
  int* nbr;
  double *Ja64, *J64, *invJ64;
  float *Ja32, *invJ32;
  void* u[2];
  float* ulo;      // mixed form: low part of the compensated current state
  float* ulo_alt;  // the other buffer: an RK stage writes the new state's low part there
  int cur;
  void* du;
  void* gradW;
  void* alpha_raw;
  double* alpha_used;
  int* bc_kind;
  void* bc_u;
  double* scal;
  unsigned long long* lam;
  int lam_slot;
  int64_t rk_step;  // step index within the running dg_step_rk call
  // mixtures: the temperature cache and (p, c) hold the solve of the state thermo_u while
  // thermo_ok (cleared by every write to a state buffer)
  const void* thermo_u;
  bool thermo_ok;
  unsigned long long* status;
  double* partial;
  int diag_blocks;
  double* stage64;  // FP64 staging buffer for host <-> device state transfers
  bool have_state, have_grad, have_alpha;
  bool grad_is_gradient;  // gradW holds the gradients of the last dg_rhs input (not fluxes)
  DgThermo th;  // mixtures
  // tracing: CUDA events around each launch while profiling is on
  int prof;
  cudaEvent_t* ev;
  int* ev_kind;
  int ev_cap, ev_used;
  double prof_ms[DG_PROF_KINDS];
  int64_t prof_n[DG_PROF_KINDS];
};

namespace {

__constant__ double c_D64[(DG_MAXN + 1) * (DG_MAXN + 1)];
__constant__ double c_w64[DG_MAXN + 1];
int g_basis_uploaded_for = -1;  // device id

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return DG_ECUDA;     \
  } while (0)

cudaError_t upload_all_bases(int dev) {
  if (g_basis_uploaded_for == dev) return cudaSuccess;
  cudaError_t e = dg_f64_upload_basis();
  if (e == cudaSuccess) e = dg_f32_upload_basis();
  if (e == cudaSuccess) e = dg_thermo_upload_basis();
  if (e == cudaSuccess) g_basis_uploaded_for = dev;
  return e;
}

cudaError_t upload_local_basis(int N) {
  DgHostBasis b;
  if (dg_host_basis(N, &b)) return cudaErrorInvalidValue;
  double D[(DG_MAXN + 1) * (DG_MAXN + 1)] = {0}, w[DG_MAXN + 1] = {0};
  for (int i = 0; i < (N + 1) * (N + 1); ++i) D[i] = b.D[i];
  for (int i = 0; i <= N; ++i) w[i] = b.w[i];
  cudaError_t e = cudaMemcpyToSymbol(c_D64, D, sizeof(D));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w64, w, sizeof(w));
  return e;
}

__device__ __forceinline__ int ipow_d(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// derivative along reference direction d of nodal field f (stride 1 over nodes)
__device__ double dref(const double* f, int N, int d, int node) {
  const int n1 = N + 1, s = ipow_d(n1, d), pos = (node / s) % n1, base = node - pos * s;
  double acc = 0.0;
  for (int l = 0; l < n1; ++l) acc += c_D64[pos * n1 + l] * f[base + l * s];
  return acc;
}

// Metric terms, one CTA per element.  3D: conservative curl form
// Ja^i_n = -[curl_xi (x_l grad_xi x_m)]_i, (n,m,l) cyclic; 2D: Ja^1 = (y_eta, -x_eta),
// Ja^2 = (-y_xi, x_xi).  J = det(dx/dxi).
__global__ void metrics_kernel(int dim, int N, int64_t K, const double* xyz, double* Ja,
                               double* J, double* invJ, unsigned long long* status) {
  extern __shared__ double sm[];
  const int np = ipow_d(N + 1, dim);
  double* X = sm;               // [dim][np]
  double* V = X + dim * np;     // [3][np]
  const int64_t k = blockIdx.x;
  for (int i = threadIdx.x; i < dim * np; i += blockDim.x) X[i] = xyz[k * dim * np + i];
  __syncthreads();
  double* JA = Ja + k * dim * dim * np;
  for (int node = threadIdx.x; node < np; node += blockDim.x) {
    double a[3][3];
    for (int n = 0; n < dim; ++n)
      for (int j = 0; j < dim; ++j) a[n][j] = dref(X + n * np, N, j, node);
    double det;
    if (dim == 2) {
      det = a[0][0] * a[1][1] - a[0][1] * a[1][0];
      JA[0 * np + node] = a[1][1];
      JA[1 * np + node] = -a[0][1];
      JA[2 * np + node] = -a[1][0];
      JA[3 * np + node] = a[0][0];
    } else {
      det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
            a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
            a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    }
    J[k * np + node] = det;
    invJ[k * np + node] = 1.0 / det;
    if (!(det > 0.0)) atomicCAS(status, 0ull, (4ull << 56) | (unsigned long long)k);
  }
  if (dim == 3) {
    // curl form Ja^i_n = -[curl_xi(x_l grad_xi x_m)]_i with x_l taken relative to the
    // element's first node: the shift adds c curl grad x_m = 0 (the derivative matrices of
    // different directions commute) and keeps the products of size h^2 instead of |x| h,
    // so that rounding is not amplified by |x| / h in the cancellation
    for (int n = 0; n < 3; ++n) {
      const int m = (n + 1) % 3, l = (n + 2) % 3;
      __syncthreads();
      const double c = X[l * np];
      for (int node = threadIdx.x; node < np; node += blockDim.x)
        for (int j = 0; j < 3; ++j) V[j * np + node] = (X[l * np + node] - c) * dref(X + m * np, N, j, node);
      __syncthreads();
      for (int node = threadIdx.x; node < np; node += blockDim.x) {
        double c0 = dref(V + 2 * np, N, 1, node) - dref(V + 1 * np, N, 2, node);
        double c1 = dref(V + 0 * np, N, 2, node) - dref(V + 2 * np, N, 0, node);
        double c2 = dref(V + 1 * np, N, 0, node) - dref(V + 0 * np, N, 1, node);
        JA[(0 * 3 + n) * np + node] = -c0;
        JA[(1 * 3 + n) * np + node] = -c1;
        JA[(2 * 3 + n) * np + node] = -c2;
      }
    }
  }
}

template <typename T>
__global__ void cvt_kernel(const double* a, T* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (T)a[i];
}
template <typename T>
__global__ void cvt_back_kernel(const T* a, double* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// compensated FP32 state of the mixed form: u = hi + lo, hi = fl32(u), lo = fl32(u - hi)
__global__ void split_kernel(const double* a, float* hi, float* lo, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float h = (float)a[i];
    hi[i] = h;
    lo[i] = (float)(a[i] - (double)h);
  }
}
__global__ void merge_kernel(const float* hi, const float* lo, double* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)hi[i] + (double)lo[i];
}
// The same two conversions for 16-byte aligned buffers, built for the host link (a
// page-locked host buffer read or written in place): pairs of values as 16-byte accesses,
// four independent ones in flight per thread, so that the link's latency is covered by
// bytes in flight rather than by resident threads.  n2 = n / 2 pairs; an odd last value
// goes through the scalar kernels.
__global__ void split_kernel_x4(const double2* a, float2* hi, float2* lo, int64_t n2) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + 3 * st < n2; i += 4 * st) {
    double2 v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = a[i + j * st];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float hx = (float)v[j].x, hy = (float)v[j].y;
      hi[i + j * st] = make_float2(hx, hy);
      lo[i + j * st] = make_float2((float)(v[j].x - (double)hx), (float)(v[j].y - (double)hy));
    }
  }
  for (; i < n2; i += st) {
    const double2 v = a[i];
    const float hx = (float)v.x, hy = (float)v.y;
    hi[i] = make_float2(hx, hy);
    lo[i] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
  }
}
__global__ void merge_kernel_x4(const float2* hi, const float2* lo, double2* b, int64_t n2) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + 3 * st < n2; i += 4 * st) {
    float2 h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      h[j] = hi[i + j * st];
      l[j] = lo[i + j * st];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      b[i + j * st] = make_double2((double)h[j].x + (double)l[j].x, (double)h[j].y + (double)l[j].y);
  }
  for (; i < n2; i += st) {
    const float2 hh = hi[i], ll = lo[i];
    b[i] = make_double2((double)hh.x + (double)ll.x, (double)hh.y + (double)ll.y);
  }
}
// split / merge of n values: the 16-byte kernels where every pointer allows, the odd last
// value (and unaligned buffers) by the scalar ones
unsigned grid_for(int64_t n, int bs);
bool host_aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }
void launch_split(const double* src, float* hi, float* lo, int64_t n, cudaStream_t st) {
  if (host_aligned16(src) && host_aligned16(hi) && host_aligned16(lo)) {
    const int64_t n2 = n / 2;
    if (n2 > 0)
      split_kernel_x4<<<grid_for((n2 + 3) / 4, 256), 256, 0, st>>>((const double2*)src, (float2*)hi,
                                                                    (float2*)lo, n2);
    if (n & 1) split_kernel<<<1, 32, 0, st>>>(src + 2 * n2, hi + 2 * n2, lo + 2 * n2, 1);
  } else {
    split_kernel<<<grid_for(n, 256), 256, 0, st>>>(src, hi, lo, n);
  }
}
void launch_merge(const float* hi, const float* lo, double* dst, int64_t n, cudaStream_t st) {
  if (host_aligned16(dst) && host_aligned16(hi) && host_aligned16(lo)) {
    const int64_t n2 = n / 2;
    if (n2 > 0)
      merge_kernel_x4<<<grid_for((n2 + 3) / 4, 256), 256, 0, st>>>((const float2*)hi, (const float2*)lo,
                                                                    (double2*)dst, n2);
    if (n & 1) merge_kernel<<<1, 32, 0, st>>>(hi + 2 * n2, lo + 2 * n2, dst + 2 * n2, 1);
  } else {
    merge_kernel<<<grid_for(n, 256), 256, 0, st>>>(hi, lo, dst, n);
  }
}

// one-gas primitive (rho, v, p) -> conserved, written in the form precision
// (lo: the FP32 form's compensation part, or null)
template <typename T>
__global__ void prim2cons_kernel(const double* w, T* u, float* lo, int64_t K, int dim, int np, double gamma) {
  const int nv = dim + 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K * np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / np;
    const int node = (int)(i % np);
    const double* ww = w + k * nv * np + node;
    T* uu = u + k * nv * np + node;
    double rho = ww[0], ke = 0.0, c[8];
    c[0] = rho;
    for (int d = 0; d < dim; ++d) {
      c[1 + d] = rho * ww[(1 + d) * np];
      ke += ww[(1 + d) * np] * ww[(1 + d) * np];
    }
    c[1 + dim] = ww[(1 + dim) * np] / (gamma - 1.0) + 0.5 * rho * ke;
    for (int v = 0; v < nv; ++v) {
      uu[v * np] = (T)c[v];
      if (lo) lo[k * nv * np + v * np + node] = (float)(c[v] - (double)(T)c[v]);
    }
  }
}

// FP64 domain integrals, per block partial sums (deterministic: fixed order later)
template <typename T>
__global__ void diag_kernel(const T* u, const double* Ja, const double* J, int64_t K, int dim,
                            int N, int nsp, double gamma, int single_gas, double suth_s,
                            double suth_rt, double* partial) {
  const int np = ipow_d(N + 1, dim), nv = nsp + dim + 1;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K * np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / np;
    const int node = (int)(i % np);
    const T* uu = u + k * nv * np;
    double wq = 1.0;
    for (int d = 0; d < dim; ++d) wq *= c_w64[(node / ipow_d(N + 1, d)) % (N + 1)];
    const double Jn = J[k * np + node];
    double rho = 0.0;
    for (int s = 0; s < nsp; ++s) rho += (double)uu[s * np + node];
    double v[3] = {0, 0, 0}, v2 = 0.0;
    for (int d = 0; d < dim; ++d) {
      v[d] = (double)uu[(nsp + d) * np + node] / rho;
      v2 += v[d] * v[d];
    }
    const double rhoE = (double)uu[(nsp + dim) * np + node];
    double gv[3][3] = {{0}};
    const int n1 = N + 1;
    for (int a = 0; a < dim; ++a)
      for (int d = 0; d < dim; ++d) {
        const int s = ipow_d(n1, d), pos = (node / s) % n1, base = node - pos * s;
        double dv = 0.0;
        for (int l = 0; l < n1; ++l) {
          const int m = base + l * s;
          double rm = 0.0;
          for (int q = 0; q < nsp; ++q) rm += (double)uu[q * np + m];
          dv += c_D64[pos * n1 + l] * ((double)uu[(nsp + a) * np + m] / rm);
        }
        for (int x = 0; x < dim; ++x) gv[a][x] += Ja[((k * dim + d) * dim + x) * np + node] * dv / Jn;
      }
    double w2;
    if (dim == 3) {
      double wx = gv[2][1] - gv[1][2], wy = gv[0][2] - gv[2][0], wz = gv[1][0] - gv[0][1];
      w2 = wx * wx + wy * wy + wz * wz;
    } else {
      double wz = gv[1][0] - gv[0][1];
      w2 = wz * wz;
    }
    double div = 0.0;
    for (int a = 0; a < dim; ++a) div += gv[a][a];
    const double dV = wq * Jn;
    acc[0] += dV;
    acc[1] += dV * 0.5 * rho * v2;
    acc[2] += dV * 0.5 * rho * w2;
    if (single_gas) {
      double p = (gamma - 1.0) * (rhoE - 0.5 * rho * v2);
      acc[3] += dV * (-rho * (log(p) - gamma * log(rho)) / (gamma - 1.0));
    }
    acc[4] += dV * rho;
    acc[5] += dV * rhoE;
    // Sutherland weight mu(T)/mu of the dissipation integrals (Eqs. TGV_SD, TGV_DD)
    double mr = 1.0;
    if (single_gas && suth_s > 0.0) {
      const double th = (gamma - 1.0) * (rhoE - 0.5 * rho * v2) / (rho * suth_rt);
      mr = (1.0 + suth_s) * th * sqrt(th) / (th + suth_s);
    }
    acc[6] += dV * mr * div * div;
    acc[7] += dV * mr * w2;
  }
  __shared__ double red[8][256];
  for (int q = 0; q < 8; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 8; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 8; ++q) partial[blockIdx.x * 8 + q] = red[q][0];
}

__global__ void diag_final_kernel(const double* partial, int nb, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = 0; b < nb; ++b)
    for (int q = 0; q < 8; ++q) s[q] += partial[b * 8 + q];
  out[0] = s[1] / s[0];
  out[1] = s[2] / s[0];
  out[2] = s[3];
  out[3] = s[4];
  out[4] = s[5];
  out[5] = s[0];
  out[6] = s[6] / s[0];
  out[7] = s[7] / s[0];
}

void rk_ck45(double* A, double* B) {
  // Carpenter & Kennedy (1994), five-stage fourth-order 2N-storage
  A[0] = 0.0;
  A[1] = -567301805773.0 / 1357537059087.0;
  A[2] = -2404267990393.0 / 2016746695238.0;
  A[3] = -3550918686646.0 / 2091501179385.0;
  A[4] = -1275806237668.0 / 842570457699.0;
  B[0] = 1432997174477.0 / 9575080441755.0;
  B[1] = 5161836677717.0 / 13612068292357.0;
  B[2] = 1720146321549.0 / 2090206949498.0;
  B[3] = 3134564353537.0 / 4481467310338.0;
  B[4] = 2277821191437.0 / 14882151754819.0;
}

unsigned grid_for(int64_t n, int bs) {
  int64_t g = (n + bs - 1) / bs;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

DgArgs base_args(dg_ctx* c) {
  DgArgs a;
  memset(&a, 0, sizeof(a));
  a.K = c->K;
  a.dim = c->dim;
  a.N = c->N;
  a.nsp = c->nsp;
  a.nv = c->nv;
  a.np = c->np;
  a.n_bc = c->n_bc;
  a.has_bnd = c->has_bnd;
  a.vf = c->vf;
  a.sf = c->sf;
  a.ns = c->equations == DG_NAVIER_STOKES;
  a.gamma = c->gamma;
  a.pref = c->p_ref;
  a.mu = c->mu;
  a.kappa_fac = a.ns ? c->mu * c->gamma / ((c->gamma - 1.0) * c->Pr) : 0.0;
  a.visc_coef = a.ns ? c->gamma * c->mu / c->Pr : 0.0;
  a.suth_s = a.ns ? c->suth_s : 0.0;
  a.suth_rt = c->suth_rt;
  a.ind_var = c->ind_var;
  for (int q = 0; q < 8; ++q) a.pos_ef[q] = c->pos_ef[q];
  const bool f32 = c->precision == DG_MIXED;
  a.Ja = f32 ? (const void*)c->Ja32 : (const void*)c->Ja64;
  a.invJ = f32 ? (const void*)c->invJ32 : (const void*)c->invJ64;
  a.gradW = c->gradW;
  a.nbr = c->nbr;
  a.bc_kind = c->bc_kind;
  a.bc_u = c->bc_u;
  a.scal = c->scal;
  a.lam = c->lam;
  a.status = c->status;
  if (c->n_species > 0) {
    a.pc = c->th.pc;
    a.bc_pc = c->th.bc_pc;
  }
  return a;
}

void prof_flush(dg_ctx* c) {
  if (c->ev_used == 0) return;
  cudaEventSynchronize(c->ev[c->ev_used - 1]);
  for (int i = 0; i < c->ev_used / 2; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) == cudaSuccess) {
      c->prof_ms[c->ev_kind[i]] += ms;
      c->prof_n[c->ev_kind[i]] += 1;
    }
  }
  c->ev_used = 0;
}

template <typename F>
cudaError_t timed(dg_ctx* c, int kind, F f) {
  if (!c->prof) return f();
  if (c->ev_used + 2 > c->ev_cap) prof_flush(c);
  cudaEventRecord(c->ev[c->ev_used], c->stream);
  cudaError_t r = f();
  cudaEventRecord(c->ev[c->ev_used + 1], c->stream);
  c->ev_kind[c->ev_used / 2] = kind;
  c->ev_used += 2;
  return r;
}

cudaError_t run_rhs(dg_ctx* c, DgArgs& a) {
  return timed(c, DG_PROF_RHS, [&] {
    return c->precision == DG_MIXED ? dg_f32_rhs(a, c->stream) : dg_f64_rhs(a, c->stream);
  });
}
cudaError_t run_grad(dg_ctx* c, DgArgs& a) {
  return timed(c, DG_PROF_GRAD, [&] {
    return c->precision == DG_MIXED ? dg_f32_gradients(a, c->stream) : dg_f64_gradients(a, c->stream);
  });
}
cudaError_t run_ind(dg_ctx* c, DgArgs& a) {
  return timed(c, DG_PROF_INDICATOR, [&] {
    return c->precision == DG_MIXED ? dg_f32_indicator(a, c->alpha_max, c->alpha_raw, c->stream)
                                    : dg_f64_indicator(a, c->alpha_max, c->alpha_raw, c->stream);
  });
}
cudaError_t run_lambda(dg_ctx* c, DgArgs& a, int slot) {
  return timed(c, DG_PROF_LAMBDA, [&] {
    return c->precision == DG_MIXED ? dg_f32_lambda(a, slot, c->stream) : dg_f64_lambda(a, slot, c->stream);
  });
}
cudaError_t run_step_dt(dg_ctx* c, DgArgs& a, int slot, int advance) {
  return timed(c, DG_PROF_OTHER, [&] {
    return c->precision == DG_MIXED ? dg_f32_step_dt(a, slot, advance, c->stream)
                                    : dg_f64_step_dt(a, slot, advance, c->stream);
  });
}
cudaError_t run_thermo(dg_ctx* c, const void* u) {
  const cudaError_t e = timed(c, DG_PROF_THERMO, [&] {
    return dg_thermo_update(&c->th, u, c->precision == DG_MIXED, c->stream);
  });
  c->thermo_u = u;
  c->thermo_ok = e == cudaSuccess;
  return e;
}

cudaError_t run_positivity(dg_ctx* c, const DgArgs& b) {
  return timed(c, DG_PROF_LIMITER, [&] {
    return c->precision == DG_MIXED ? dg_f32_positivity(b, b.out, b.ulo_out ? b.ulo_out : c->ulo, c->pos_eps,
                                                        c->pos_count, c->stream)
                                    : dg_f64_positivity(b, b.out, nullptr, c->pos_eps, c->pos_count, c->stream);
  });
}

// everything that precedes the main kernel of one right-hand side at state u
cudaError_t pre_rhs(dg_ctx* c, DgArgs& a) {
  cudaError_t e = cudaSuccess;
  if (c->n_species > 0) {
    // an RK stage whose state was just solved (the first stage after the previous step's
    // wave-speed solve) reuses that solve
    if (!(a.mode == 1 && c->thermo_ok && c->thermo_u == a.u)) e = run_thermo(c, a.u);
    if (e != cudaSuccess) return e;
    if (c->th.nr > 0) {
      // species sources; point-implicit with the running step in RK stages
      // plain correction of the learned source: refresh at the first evaluation after the
      // corrections were invalidated (new state, new network, new dg_step_rk call) and at
      // the first stage of every k-th step
      const int kref = c->th.refresh_period;
      const int refresh = c->th.chem_mlp && kref > 0 &&
                          (!c->th.corr_valid || (a.mode == 1 && a.stage == 0 && c->rk_step % kref == 0));
      e = timed(c, DG_PROF_CHEM, [&] {
        return dg_chem_source(&c->th, a.u, c->precision == DG_MIXED, a.mode == 1 ? c->scal + 1 : NULL,
                              refresh, c->stream);
      });
      if (e != cudaSuccess) return e;
      c->th.src_valid = 1;
      a.src = c->th.src;
    }
  }
  if (c->equations == DG_NAVIER_STOKES) {
    e = run_grad(c, a);
    if (e != cudaSuccess) return e;
    c->have_grad = true;
  }
  if (c->alpha_max > 0.0) {
    e = run_ind(c, a);
    if (e != cudaSuccess) return e;
    a.alpha_raw = c->alpha_raw;
    a.alpha_used = c->alpha_used;
    c->have_alpha = true;
  }
  return e;
}

dg_status wait_stream(dg_ctx* c) {
  // bounded wait: poll for up to 600 s of wall time; the first 2 ms without sleeping (a
  // sleep overshoots by the timer slack, tens of microseconds, on every short wait), then
  // with 20 us sleeps
  struct timespec t0, t1;
  clock_gettime(CLOCK_MONOTONIC, &t0);
  for (;;) {
    cudaError_t q = cudaStreamQuery(c->stream);
    if (q == cudaSuccess) return DG_OK;
    if (q != cudaErrorNotReady) return DG_ECUDA;
    clock_gettime(CLOCK_MONOTONIC, &t1);
    const double el = (double)(t1.tv_sec - t0.tv_sec) + 1e-9 * (double)(t1.tv_nsec - t0.tv_nsec);
    if (el > 600.0) return DG_ETIMEOUT;
    if (el > 2e-3) {
      struct timespec ts = {0, 20000};
      nanosleep(&ts, NULL);
    }
  }
}

dg_status take_status(dg_ctx* c, int64_t* elem) {
  unsigned long long st = 0;
  if (cudaMemcpy(&st, c->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return DG_ECUDA;
  if (elem) *elem = st ? (int64_t)(st & 0x00ffffffffffffffull) : -1;
  if (!st) return DG_OK;
  unsigned long long code = st >> 56;
  return code == DG_ST_NEWTON ? DG_ENEWTON : (code == DG_ST_TIMEOUT ? DG_ETIMEOUT : DG_ENONPHYS);
}

void free_ctx(dg_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->dev);
  void* ptrs[] = {c->nbr, c->Ja64, c->J64, c->invJ64, c->Ja32, c->invJ32, c->u[0], c->u[1],
                  c->du, c->ulo, c->ulo_alt, c->pos_count, c->gradW, c->alpha_raw, c->alpha_used, c->bc_kind, c->bc_u, c->scal,
                  c->lam, c->status, c->partial, c->stage64};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  dg_thermo_free(&c->th);
  if (c->ev) {
    for (int i = 0; i < c->ev_cap; ++i) cudaEventDestroy(c->ev[i]);
    free(c->ev);
    free(c->ev_kind);
  }
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  free(c);
}

bool supported_degree(int dim, int N, int ns) {
  if (ns > 0) return dim == 3 && (N == 3 || N == 4);
  return N == 2 || N == 3 || N == 4 || N == 7;
}

}  // namespace

extern "C" {

dg_status dg_lgl_nodes(int N, double* nodes, double* weights) {
  if (N < 1 || N > DG_MAXN || !nodes) return DG_EINVAL;
  DgHostBasis b;
  if (dg_host_basis(N, &b)) return DG_EINVAL;
  for (int i = 0; i <= N; ++i) {
    nodes[i] = b.x[i];
    if (weights) weights[i] = b.w[i];
  }
  return DG_OK;
}

const char* dg_status_string(dg_status s) {
  switch (s) {
    case DG_OK: return "ok";
    case DG_EINVAL: return "invalid argument";
    case DG_ENOMEM: return "device allocation failed";
    case DG_ECUDA: return "CUDA error";
    case DG_ENONPHYS: return "non-physical state";
    case DG_ENEWTON: return "temperature Newton iteration failed";
    case DG_ETIMEOUT: return "device wait timed out";
    case DG_ESTATE: return "call out of order";
  }
  return "unknown";
}

dg_status dg_init_mesh(const dg_mesh_desc* m, const dg_physics_desc* p, dg_ctx** out) {
  if (!out) return DG_EINVAL;
  *out = NULL;
  if (!m || !p || !m->node_xyz || !m->nbr_elem || !m->nbr_face) return DG_EINVAL;
  if (m->dim < 2 || m->dim > 3 || m->K < 1 || m->K >= (1ll << 31)) return DG_EINVAL;
  if (p->n_species < 0 || p->n_species > DG_MAX_SPECIES) return DG_EINVAL;
  if (!supported_degree(m->dim, m->N, p->n_species)) return DG_EINVAL;
  if (p->n_species > 0 && (p->n_species != 5 || !p->species || p->n_bc > 64)) return DG_EINVAL;
  if (p->n_reactions < 0 || p->n_reactions > 64 || (p->n_reactions > 0 && (!p->reactions || p->n_species != 5)))
    return DG_EINVAL;
  if (p->equations != DG_EULER && p->equations != DG_NAVIER_STOKES) return DG_EINVAL;
  if (p->equations == DG_NAVIER_STOKES && (p->n_species > 0 || m->dim != 3 || !(p->mu > 0) ||
                                           !(p->Pr > 0)))
    return DG_EINVAL;
  if (p->volume_flux < 0 || p->volume_flux > DG_VF_MORINISHI || p->surface_flux < 0 || p->surface_flux > DG_SF_HLL)
    return DG_EINVAL;
  if (p->n_species > 0 && (p->volume_flux == DG_VF_RANOCHA || p->volume_flux == DG_VF_KG ||
                           p->volume_flux == DG_VF_PIROZZOLI || p->volume_flux == DG_VF_MORINISHI))
    return DG_EINVAL;
  if (p->n_species == 0 && !(p->gamma > 1.0)) return DG_EINVAL;
  if (!(p->p_ref >= 0.0) || (p->n_species > 0 && p->p_ref != 0.0)) return DG_EINVAL;
  if (!(p->positivity_eps >= 0.0)) return DG_EINVAL;
  if (!(p->sutherland_s >= 0.0) || (p->sutherland_s > 0.0 && (!(p->sutherland_rt > 0.0) || p->n_species > 0)))
    return DG_EINVAL;
  if (p->indicator_variable != 0 && p->indicator_variable != 1) return DG_EINVAL;
  if (p->precision != DG_FP64 && p->precision != DG_MIXED) return DG_EINVAL;
  if (p->thermo != DG_THERMO_NEWTON && p->thermo != DG_THERMO_MLP) return DG_EINVAL;
  if (p->alpha_max < 0.0 || p->alpha_max > 1.0) return DG_EINVAL;
  if (p->n_bc < 0 || (p->n_bc > 0 && (!p->bc_kind || !p->bc_prim))) return DG_EINVAL;
  const int dim = m->dim, nf = 2 * dim, N = m->N;
  const int64_t K = m->K;
  for (int b = 0; b < p->n_bc; ++b)
    if (p->bc_kind[b] < DG_BC_INFLOW || p->bc_kind[b] > DG_BC_ISOTHERMAL ||
        (p->equations == DG_NAVIER_STOKES && p->bc_kind[b] == DG_BC_SLIP_WALL))
      return DG_EINVAL;
  int* nbr_h = (int*)malloc(sizeof(int) * K * nf);
  if (!nbr_h) return DG_ENOMEM;
  bool any_bnd = false;
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < nf; ++f) {
      const int64_t nb = m->nbr_elem[k * nf + f];
      bool ok = true;
      if (nb >= 0) {
        ok = nb < K && m->nbr_face[k * nf + f] == (f ^ 1) &&
             (!m->nbr_orient || m->nbr_orient[k * nf + f] == 0);
      } else {
        ok = -(nb + 1) < p->n_bc;
      }
      if (!ok) {
        free(nbr_h);
        return DG_EINVAL;
      }
      nbr_h[k * nf + f] = (int)nb;
      any_bnd |= nb < 0;
    }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    free(nbr_h);
    return DG_ECUDA;
  }
  dg_ctx* c = (dg_ctx*)calloc(1, sizeof(dg_ctx));
  cudaGetDevice(&c->dev);
  c->dim = dim;
  c->N = N;
  c->K = K;
  c->nf = nf;
  c->np = 1;
  for (int d = 0; d < dim; ++d) c->np *= (N + 1);
  c->n_species = p->n_species;
  c->nsp = p->n_species > 0 ? p->n_species : 1;
  c->nv = c->nsp + dim + 1;
  c->equations = p->equations;
  c->vf = p->volume_flux;
  c->sf = p->surface_flux;
  c->precision = p->precision;
  c->thermo = p->thermo;
  c->n_bc = p->n_bc;
  c->has_bnd = any_bnd ? 1 : 0;
  c->gamma = p->gamma;
  c->p_ref = p->p_ref;
  c->pos_eps = p->positivity_eps;
  c->suth_s = p->sutherland_s;
  c->suth_rt = p->sutherland_s > 0.0 ? p->sutherland_rt : 1.0;
  c->ind_var = p->indicator_variable;
  // the mixture limiter's energy floor: e_s(T_floor) = R_s (a1 T + a2 T^2/2 + ... + a6 - T)
  for (int q = 0; q < p->n_species; ++q) {
    const double* sp = p->species + 8 * q;
    const double T = DG_T_FLOOR, Rs = 8.314462618 / sp[0];
    c->pos_ef[q] = Rs * (sp[1] * T + sp[2] * T * T / 2.0 + sp[3] * T * T * T / 3.0 + sp[4] * T * T * T * T / 4.0 +
                         sp[5] * T * T * T * T * T / 5.0 + sp[6] - T);
  }
  c->mu = p->mu;
  c->Pr = p->Pr;
  c->alpha_max = p->alpha_max;
  c->rs = c->precision == DG_MIXED ? sizeof(float) : sizeof(double);
  dg_status st = DG_OK;
#define TRY(x)                    \
  do {                            \
    if ((x) != cudaSuccess) {     \
      st = DG_ECUDA;              \
      goto fail;                  \
    }                             \
  } while (0)
#define TRYM(ptr, bytes)                                     \
  do {                                                       \
    if (cudaMalloc((void**)&(ptr), (bytes)) != cudaSuccess) { \
      st = DG_ENOMEM;                                        \
      goto fail;                                             \
    }                                                        \
  } while (0)
  {
    if (p->stream) {
      c->stream = (cudaStream_t)p->stream;
    } else {
      TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    TRY(upload_all_bases(c->dev));
    TRY(upload_local_basis(N));
    const int64_t nst = K * c->nv * c->np;
    TRYM(c->nbr, sizeof(int) * K * nf);
    TRYM(c->Ja64, sizeof(double) * K * dim * dim * c->np);
    TRYM(c->J64, sizeof(double) * K * c->np);
    TRYM(c->invJ64, sizeof(double) * K * c->np);
    if (c->precision == DG_MIXED) {
      TRYM(c->Ja32, sizeof(float) * K * dim * dim * c->np);
      TRYM(c->invJ32, sizeof(float) * K * c->np);
    }
    TRYM(c->u[0], c->rs * nst);
    TRYM(c->u[1], c->rs * nst);
    TRYM(c->du, c->rs * nst);
    if (c->precision == DG_MIXED) {
      TRYM(c->ulo, sizeof(float) * nst);
      TRYM(c->ulo_alt, sizeof(float) * nst);
    }
    if (c->pos_eps > 0.0) {
      TRYM(c->pos_count, sizeof(unsigned long long));
      TRY(cudaMemset(c->pos_count, 0, sizeof(unsigned long long)));
    }
    if (c->equations == DG_NAVIER_STOKES) TRYM(c->gradW, c->rs * K * dim * (dim + 1) * c->np);
    if (c->alpha_max > 0.0) {
      TRYM(c->alpha_raw, c->rs * K);
      TRYM(c->alpha_used, sizeof(double) * K);
    }
    TRYM(c->bc_kind, sizeof(int) * (p->n_bc > 0 ? p->n_bc : 1));
    TRYM(c->bc_u, c->rs * c->nv * (p->n_bc > 0 ? p->n_bc : 1));
    TRYM(c->scal, sizeof(double) * 4);
    TRYM(c->lam, sizeof(unsigned long long) * 4);
    TRYM(c->status, sizeof(unsigned long long));
    c->diag_blocks = 152 * 4;
    TRYM(c->partial, sizeof(double) * 8 * c->diag_blocks);
    TRYM(c->stage64, sizeof(double) * nst);
    TRY(cudaMemset(c->status, 0, sizeof(unsigned long long)));
    TRY(cudaMemset(c->scal, 0, sizeof(double) * 4));
    TRY(cudaMemset(c->lam, 0, sizeof(unsigned long long) * 4));
    TRY(cudaMemcpy(c->nbr, nbr_h, sizeof(int) * K * nf, cudaMemcpyHostToDevice));
    if (p->n_bc > 0) TRY(cudaMemcpy(c->bc_kind, p->bc_kind, sizeof(int) * p->n_bc, cudaMemcpyHostToDevice));
    // geometry -> metric terms
    double* xyz = NULL;
    TRYM(xyz, sizeof(double) * K * dim * c->np);
    if (cudaMemcpy(xyz, m->node_xyz, sizeof(double) * K * dim * c->np, cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      cudaFree(xyz);
      st = DG_ECUDA;
      goto fail;
    }
    const size_t msm = sizeof(double) * (dim + 3) * c->np;
    if (msm > 48 * 1024)
      cudaFuncSetAttribute(metrics_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msm);
    metrics_kernel<<<(unsigned)K, 128, msm, c->stream>>>(dim, N, K, xyz, c->Ja64, c->J64,
                                                          c->invJ64, c->status);
    cudaError_t ke = cudaGetLastError();
    if (ke == cudaSuccess) ke = cudaStreamSynchronize(c->stream);
    cudaFree(xyz);
    TRY(ke);
    int64_t bad = -1;
    if (take_status(c, &bad) != DG_OK) {
      st = DG_EINVAL;  // inverted element
      goto fail;
    }
    if (c->precision == DG_MIXED) {
      cvt_kernel<float><<<grid_for(K * dim * dim * c->np, 256), 256, 0, c->stream>>>(
          c->Ja64, c->Ja32, K * dim * dim * c->np);
      cvt_kernel<float><<<grid_for(K * c->np, 256), 256, 0, c->stream>>>(c->invJ64, c->invJ32,
                                                                          K * c->np);
      TRY(cudaGetLastError());
    }
    if (c->n_species > 0) {
      if (dg_thermo_init(&c->th, K, c->np, dim, p->species, p->thermo, c->precision == DG_MIXED,
                         c->status) != cudaSuccess) {
        st = DG_ENOMEM;
        goto fail;
      }
      if (p->n_reactions > 0) {
        const cudaError_t ce = dg_chem_init(&c->th, p->species, p->reactions, p->n_reactions);
        if (ce != cudaSuccess) {
          st = ce == cudaErrorInvalidValue ? DG_EINVAL : DG_ENOMEM;
          goto fail;
        }
      }
    }
    // boundary states (primitive -> conserved on the device)
    if (p->n_bc > 0) {
      double* bw = NULL;
      TRYM(bw, sizeof(double) * p->n_bc * c->nv);
      cudaMemcpy(bw, p->bc_prim, sizeof(double) * p->n_bc * c->nv, cudaMemcpyHostToDevice);
      cudaError_t e2;
      if (c->n_species == 0) {
        if (c->precision == DG_MIXED)
          prim2cons_kernel<float><<<1, 32, 0, c->stream>>>(bw, (float*)c->bc_u, NULL, p->n_bc, dim, 1, c->gamma);
        else
          prim2cons_kernel<double><<<1, 32, 0, c->stream>>>(bw, (double*)c->bc_u, NULL, p->n_bc, dim, 1, c->gamma);
        e2 = cudaGetLastError();
      } else {
        e2 = dg_thermo_boundary(&c->th, bw, p->n_bc, c->bc_u, c->stream);
      }
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(c->stream);
      cudaFree(bw);
      TRY(e2);
    }
    TRY(cudaStreamSynchronize(c->stream));
  }
  free(nbr_h);
  *out = c;
  return DG_OK;
fail:
  free(nbr_h);
  free_ctx(c);
  return st;
#undef TRY
#undef TRYM
}

void dg_destroy(dg_ctx* c) { free_ctx(c); }

// device address of page-locked host memory (cudaHostAlloc / cudaHostRegister), or null:
// kernels then read or write the host buffer directly over the CPU-GPU link, which folds
// the copy into the split / merge pass of the mixed form
const void* pinned_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

dg_status dg_set_state(dg_ctx* c, const double* u, int on_device, double t) {
  if (!c || !u) return DG_EINVAL;
  const int64_t n = c->K * c->nv * c->np;
  cudaSetDevice(c->dev);
  const double* src = u;
  const void* hp = (!on_device && c->precision == DG_MIXED) ? pinned_device_ptr(u) : nullptr;
  if (hp) {
    src = (const double*)hp;
  } else if (!on_device) {
    CK(cudaMemcpyAsync(c->stage64, u, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    src = c->stage64;
  }
  if (c->precision == DG_MIXED) {
    launch_split(src, (float*)c->u[c->cur], c->ulo, n, c->stream);
  } else {
    CK(cudaMemcpyAsync(c->u[c->cur], src, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
  }
  CK(cudaGetLastError());
  if (c->n_species > 0) CK(dg_thermo_reset(&c->th, c->stream));
  c->th.corr_valid = 0;
  c->thermo_ok = false;
  CK(cudaMemcpyAsync(c->scal, &t, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  c->have_state = true;
  return wait_stream(c);
}

dg_status dg_set_state_primitive(dg_ctx* c, const double* w, int on_device, double t) {
  if (!c || !w) return DG_EINVAL;
  const int64_t n = c->K * c->nv * c->np;
  cudaSetDevice(c->dev);
  const double* src = w;
  if (!on_device) {
    CK(cudaMemcpyAsync(c->stage64, w, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    src = c->stage64;
  }
  if (c->n_species == 0) {
    if (c->precision == DG_MIXED)
      prim2cons_kernel<float><<<grid_for(c->K * c->np, 256), 256, 0, c->stream>>>(
          src, (float*)c->u[c->cur], c->ulo, c->K, c->dim, c->np, c->gamma);
    else
      prim2cons_kernel<double><<<grid_for(c->K * c->np, 256), 256, 0, c->stream>>>(
          src, (double*)c->u[c->cur], NULL, c->K, c->dim, c->np, c->gamma);
    CK(cudaGetLastError());
  } else {
    // also seeds the temperature cache with the given temperatures; the compensation part
    // of a mixture state starts at zero (the FP32-rounded initial state)
    CK(dg_thermo_prim2cons(&c->th, src, c->u[c->cur], c->stream));
    if (c->ulo) CK(cudaMemsetAsync(c->ulo, 0, sizeof(float) * n, c->stream));
  }
  c->th.corr_valid = 0;
  c->thermo_ok = false;
  CK(cudaMemcpyAsync(c->scal, &t, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  c->have_state = true;
  return wait_stream(c);
}

dg_status dg_get_state(dg_ctx* c, double* u, int on_device, double* t) {
  if (!c || !u) return DG_EINVAL;
  if (!c->have_state) return DG_ESTATE;
  cudaSetDevice(c->dev);
  const int64_t n = c->K * c->nv * c->np;
  if (c->precision == DG_MIXED) {
    double* hp = on_device ? nullptr : (double*)pinned_device_ptr(u);
    double* dst = on_device ? u : (hp ? hp : c->stage64);
    launch_merge((const float*)c->u[c->cur], c->ulo, dst, n, c->stream);
    CK(cudaGetLastError());
    if (!on_device && !hp)
      CK(cudaMemcpyAsync(u, c->stage64, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  } else {
    CK(cudaMemcpyAsync(u, c->u[c->cur], sizeof(double) * n,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  }
  double tt = 0.0;
  CK(cudaMemcpyAsync(&tt, c->scal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  dg_status w = wait_stream(c);
  if (w != DG_OK) return w;
  if (t) *t = tt;
  return take_status(c, NULL);
}

dg_status dg_rhs(dg_ctx* c, const void* u, void* rhs, double t) {
  (void)t;
  if (!c || !u || !rhs || u == rhs) return DG_EINVAL;
  cudaSetDevice(c->dev);
  DgArgs a = base_args(c);
  a.u = u;
  a.out = rhs;
  a.mode = 0;
  CK(pre_rhs(c, a));
  CK(run_rhs(c, a));
  if (c->equations == DG_NAVIER_STOKES) {
    // keep the BR1 gradients of this input for dg_get_gradients (the stepping path
    // leaves the viscous fluxes in the buffer instead)
    DgArgs g = a;
    g.grad_mode = 1;
    CK(run_grad(c, g));
    c->grad_is_gradient = true;
  }
  return DG_OK;
}

dg_status dg_step_rk(dg_ctx* c, int nsteps, double cfl, double dt_fixed, double* t_inout) {
  if (!c || nsteps < 0 || (!(dt_fixed > 0.0) && !(cfl > 0.0))) return DG_EINVAL;
  if (!c->have_state) return DG_ESTATE;
  cudaSetDevice(c->dev);
  double A[5], B[5];
  rk_ck45(A, B);
  const bool cfl_mode = !(dt_fixed > 0.0);
  CK(cudaMemsetAsync(c->scal, 0, sizeof(double), c->stream));  // elapsed time
  DgArgs a = base_args(c);
  a.cfl = cfl;
  a.dt_fixed = dt_fixed;
  if (cfl_mode) {
    a.u = c->u[c->cur];
    // (a solve of this very state, e.g. the previous call's last wave-speed solve, stands)
    if (c->n_species > 0 && !(c->thermo_ok && c->thermo_u == a.u)) CK(run_thermo(c, a.u));
    CK(cudaMemsetAsync(c->lam + 2 * c->lam_slot, 0, 2 * sizeof(unsigned long long), c->stream));
    CK(run_lambda(c, a, c->lam_slot));
  }
  CK(run_step_dt(c, a, c->lam_slot, 0));
  if (nsteps > 0) c->grad_is_gradient = false;
  c->th.corr_valid = 0;  // the call's first source evaluation refreshes the corrections
  for (int step = 0; step < nsteps; ++step) {
    c->rk_step = step;
    for (int s = 0; s < 5; ++s) {
      DgArgs b = base_args(c);
      b.u = c->u[c->cur];
      b.out = c->u[c->cur ^ 1];
      b.du = c->du;
      b.ulo = c->ulo;
      b.ulo_out = c->ulo_alt;
      b.mode = 1;
      b.stage = s;
      b.rkA = A[s];
      b.rkB = B[s];
      b.cfl = cfl;
      b.dt_fixed = dt_fixed;
      b.lam_cur = c->lam_slot;
      b.want_lambda = (s == 4 && cfl_mode && c->n_species == 0) ? 1 : 0;
      CK(pre_rhs(c, b));
      c->thermo_ok = false;  // the stage writes the other state buffer
      CK(run_rhs(c, b));
      if (c->pos_eps > 0.0) CK(run_positivity(c, b));
      c->cur ^= 1;
      std::swap(c->ulo, c->ulo_alt);
    }
    if (cfl_mode) {
      if (c->n_species > 0) {
        // mixtures: wave speeds need the new temperature field
        DgArgs l = base_args(c);
        l.u = c->u[c->cur];
        CK(run_thermo(c, l.u));
        CK(run_lambda(c, l, c->lam_slot ^ 1));
      }
      c->lam_slot ^= 1;
    }
    // adds this step's dt to the elapsed time and sets the next step's dt
    CK(run_step_dt(c, a, c->lam_slot, 1));
  }
  dg_status w = wait_stream(c);
  if (w != DG_OK) return w;
  double el = 0.0;
  CK(cudaMemcpy(&el, c->scal, sizeof(double), cudaMemcpyDeviceToHost));
  if (t_inout) *t_inout += el;
  return take_status(c, NULL);
}

dg_status dg_diagnostics(dg_ctx* c, double out[8]) {
  if (!c || !out) return DG_EINVAL;
  if (!c->have_state) return DG_ESTATE;
  cudaSetDevice(c->dev);
  CK(upload_local_basis(c->N));
  double* dout = c->partial;  // reuse the tail of the partial buffer for the result
  const int nb = c->diag_blocks - 2;
  if (c->precision == DG_MIXED)
    diag_kernel<float><<<nb, 256, 0, c->stream>>>((const float*)c->u[c->cur], c->Ja64, c->J64,
                                                  c->K, c->dim, c->N, c->nsp, c->gamma,
                                                  c->n_species == 0, c->suth_s, c->suth_rt, c->partial);
  else
    diag_kernel<double><<<nb, 256, 0, c->stream>>>((const double*)c->u[c->cur], c->Ja64, c->J64,
                                                   c->K, c->dim, c->N, c->nsp, c->gamma,
                                                   c->n_species == 0, c->suth_s, c->suth_rt, c->partial);
  CK(cudaGetLastError());
  diag_final_kernel<<<1, 32, 0, c->stream>>>(c->partial, nb, dout + nb * 8);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, dout + nb * 8, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->stream));
  dg_status w = wait_stream(c);
  if (w != DG_OK) return w;
  return DG_OK;
}

dg_status dg_get_temperature(dg_ctx* c, double* T) {
  if (!c || !T || c->n_species == 0) return DG_EINVAL;
  if (!c->have_state) return DG_ESTATE;
  cudaSetDevice(c->dev);
  CK(run_thermo(c, c->u[c->cur]));
  CK(cudaMemcpyAsync(T, c->th.T, sizeof(double) * c->K * c->np, cudaMemcpyDeviceToHost, c->stream));
  dg_status w = wait_stream(c);
  if (w != DG_OK) return w;
  return take_status(c, NULL);
}

dg_status dg_set_surrogate(dg_ctx* c, int which, const float* params, const double* stats) {
  if (!c || c->n_species == 0 || (params && !stats)) return DG_EINVAL;
  if (which != DG_SURROGATE_TEMPERATURE && which != DG_SURROGATE_SOURCE) return DG_EINVAL;
  if (which == DG_SURROGATE_SOURCE && c->th.nr == 0) return DG_EINVAL;
  cudaSetDevice(c->dev);
  if (params) {
    const int std_off = which == DG_SURROGATE_TEMPERATURE ? 7 : DG_SRC_X_STD;
    for (int q = 0; q < 7; ++q)
      if (!(stats[std_off + q] > 0.0)) return DG_EINVAL;
    if (which == DG_SURROGATE_SOURCE) {
      for (int q = 0; q < 10; ++q)
        if (!(stats[DG_SRC_Y_STD + q] > 0.0)) return DG_EINVAL;
      if (!(stats[DG_SRC_OMEGA_REF] > 0.0) || !(stats[DG_SRC_JPI_REF] > 0.0) ||
          !(stats[DG_SRC_TOL_CHECK] >= 0.0) || !(stats[DG_SRC_TOL_MASS] >= 0.0) || !(stats[DG_SRC_FLOOR] >= 0.0))
        return DG_EINVAL;
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  c->thermo_ok = false;
  if (which == DG_SURROGATE_SOURCE) {
    CK(dg_chem_mlp_set(&c->th, params, stats));
    return DG_OK;
  }
  CK(dg_mlp_set(&c->th, params, stats));
  c->th.mode = params ? DG_THERMO_MLP : DG_THERMO_NEWTON;
  return DG_OK;
}

dg_status dg_set_source_refresh(dg_ctx* c, int period) {
  if (!c || period < 0 || c->n_species == 0 || c->th.nr == 0) return DG_EINVAL;
  cudaSetDevice(c->dev);
  CK(cudaStreamSynchronize(c->stream));
  if (period > 0 && !c->th.chem_corr)
    CK(cudaMalloc((void**)&c->th.chem_corr, sizeof(float) * 10 * c->K * c->np));
  if (period > 0 && !c->th.chem_trust) CK(cudaMalloc((void**)&c->th.chem_trust, (size_t)(c->K * c->np + 31) / 32));
  c->th.refresh_period = period;
  c->th.corr_valid = 0;
  return DG_OK;
}

dg_status dg_surrogate_stats(dg_ctx* c, int which, int64_t* out) {
  if (!c || !out || c->n_species == 0) return DG_EINVAL;
  if (which != DG_SURROGATE_TEMPERATURE && which != DG_SURROGATE_SOURCE) return DG_EINVAL;
  unsigned long long* dev = which == DG_SURROGATE_SOURCE ? c->th.chem_stats : c->th.mlp_stats;
  if (!dev) {
    out[0] = out[1] = 0;
    return DG_OK;
  }
  cudaSetDevice(c->dev);
  dg_status w = wait_stream(c);
  if (w != DG_OK) return w;
  unsigned long long h[2];
  CK(cudaMemcpy(h, dev, sizeof(h), cudaMemcpyDeviceToHost));
  CK(cudaMemset(dev, 0, sizeof(h)));
  out[0] = (int64_t)h[0];
  out[1] = (int64_t)h[1];
  return DG_OK;
}

dg_status dg_chem_sample(dg_ctx* c, int64_t n, uint64_t seed, float* X, double* targets) {
  if (!c || n < 1 || !X || !targets || c->n_species == 0 || c->th.nr == 0) return DG_EINVAL;
  if (!c->have_state) return DG_ESTATE;
  cudaSetDevice(c->dev);
  CK(run_thermo(c, c->u[c->cur]));
  CK(dg_chem_sample_dev(&c->th, c->u[c->cur], c->precision == DG_MIXED, n, seed, X, targets, c->stream));
  dg_status w = wait_stream(c);
  if (w != DG_OK) return w;
  return take_status(c, NULL);
}

dg_status dg_thermo_sample(dg_ctx* c, int64_t n, uint64_t seed, float* X, float* T) {
  if (!c || n < 1 || !X || !T || c->n_species == 0) return DG_EINVAL;
  if (!c->have_state) return DG_ESTATE;
  cudaSetDevice(c->dev);
  CK(run_thermo(c, c->u[c->cur]));
  CK(dg_mlp_sample(&c->th, c->u[c->cur], c->precision == DG_MIXED, n, seed, X, T, c->stream));
  dg_status w = wait_stream(c);
  if (w != DG_OK) return w;
  return take_status(c, NULL);
}

dg_status dg_get_alpha(dg_ctx* c, double* alpha) {
  if (!c || !alpha) return DG_EINVAL;
  if (!c->have_alpha) return DG_ESTATE;
  CK(cudaMemcpyAsync(alpha, c->alpha_used, sizeof(double) * c->K, cudaMemcpyDeviceToHost, c->stream));
  return wait_stream(c);
}

dg_status dg_get_source(dg_ctx* c, double* S, unsigned char* flags, int64_t* call) {
  if (!c || !S || c->n_species == 0 || c->th.nr == 0) return DG_EINVAL;
  if (!c->th.src_valid) return DG_ESTATE;
  cudaSetDevice(c->dev);
  dg_status w = wait_stream(c);
  if (w != DG_OK) return w;
  const int64_t n = c->K * 5 * c->np, ntiles = (c->K * c->np + 31) / 32;
  if (c->precision == DG_MIXED) {
    float* tmp = (float*)malloc(sizeof(float) * n);
    if (!tmp) return DG_ENOMEM;
    const cudaError_t e = cudaMemcpy(tmp, c->th.src, sizeof(float) * n, cudaMemcpyDeviceToHost);
    for (int64_t i = 0; e == cudaSuccess && i < n; ++i) S[i] = (double)tmp[i];
    free(tmp);
    CK(e);
  } else {
    CK(cudaMemcpy(S, c->th.src, sizeof(double) * n, cudaMemcpyDeviceToHost));
  }
  if (flags) {
    if (c->th.chem_mlp && c->th.chem_flags) CK(cudaMemcpy(flags, c->th.chem_flags, (size_t)ntiles, cudaMemcpyDeviceToHost));
    else memset(flags, 255, (size_t)ntiles);
  }
  if (call) *call = c->th.chem_calls > 0 ? (int64_t)c->th.chem_calls - 1 : -1;
  return DG_OK;
}

dg_status dg_get_metrics(dg_ctx* c, double* Ja, double* invJ, int on_device) {
  if (!c || !Ja || !invJ) return DG_EINVAL;
  cudaSetDevice(c->dev);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(Ja, c->Ja64, sizeof(double) * c->K * c->dim * c->dim * c->np, kind, c->stream));
  CK(cudaMemcpyAsync(invJ, c->invJ64, sizeof(double) * c->K * c->np, kind, c->stream));
  return wait_stream(c);
}

dg_status dg_get_gradients(dg_ctx* c, double* g) {
  if (!c || !g) return DG_EINVAL;
  if (!c->have_grad) return DG_ESTATE;
  cudaSetDevice(c->dev);
  if (!c->grad_is_gradient) {
    // after dg_step_rk: the gradients of the current state
    DgArgs a = base_args(c);
    a.u = c->u[c->cur];
    a.grad_mode = 1;
    if (c->n_species > 0) CK(run_thermo(c, a.u));
    CK(run_grad(c, a));
    c->grad_is_gradient = true;
  }
  const int64_t n = c->K * c->dim * (c->dim + 1) * c->np;
  if (c->precision == DG_MIXED) {
    double* tmp = NULL;
    CK(cudaMalloc((void**)&tmp, sizeof(double) * n));
    cvt_back_kernel<float><<<grid_for(n, 256), 256, 0, c->stream>>>((const float*)c->gradW, tmp, n);
    CK(cudaMemcpyAsync(g, tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    dg_status w = wait_stream(c);
    cudaFree(tmp);
    return w;
  }
  CK(cudaMemcpyAsync(g, c->gradW, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  return wait_stream(c);
}

dg_status dg_profile(dg_ctx* c, int enable) {
  if (!c) return DG_EINVAL;
  cudaSetDevice(c->dev);
  if (enable && !c->ev) {
    c->ev_cap = 8192;
    c->ev = (cudaEvent_t*)calloc(c->ev_cap, sizeof(cudaEvent_t));
    c->ev_kind = (int*)calloc(c->ev_cap / 2, sizeof(int));
    if (!c->ev || !c->ev_kind) return DG_ENOMEM;
    for (int i = 0; i < c->ev_cap; ++i) CK(cudaEventCreate(&c->ev[i]));
  }
  if (!enable && c->ev) prof_flush(c);
  c->prof = enable ? 1 : 0;
  return DG_OK;
}

dg_status dg_profile_read(dg_ctx* c, double* ms, int64_t* launches, int n) {
  if (!c || n < 0 || n > DG_PROF_KINDS) return DG_EINVAL;
  cudaSetDevice(c->dev);
  dg_status w = wait_stream(c);
  if (w != DG_OK) return w;
  if (c->ev) prof_flush(c);
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = c->prof_ms[i];
    if (launches) launches[i] = c->prof_n[i];
  }
  for (int i = 0; i < DG_PROF_KINDS; ++i) {
    c->prof_ms[i] = 0.0;
    c->prof_n[i] = 0;
  }
  return DG_OK;
}

dg_status dg_sync(dg_ctx* c) {
  if (!c) return DG_EINVAL;
  cudaSetDevice(c->dev);
  dg_status w = wait_stream(c);
  if (w != DG_OK) return w;
  dg_status s = take_status(c, NULL);
  if (s != DG_OK) cudaMemset(c->status, 0, sizeof(unsigned long long));
  return s;
}

int64_t dg_error_element(dg_ctx* c) {
  if (!c) return -1;
  int64_t e = -1;
  take_status(c, &e);
  return e;
}

}  // extern "C"

extern "C" dg_status dg_limiter_stats(dg_ctx* c, int64_t* out) {
  if (!c || !out) return DG_EINVAL;
  out[0] = 0;
  if (!c->pos_count) return DG_OK;
  cudaSetDevice(c->dev);
  dg_status w = wait_stream(c);
  if (w != DG_OK) return w;
  unsigned long long h = 0;
  CK(cudaMemcpy(&h, c->pos_count, sizeof(h), cudaMemcpyDeviceToHost));
  CK(cudaMemset(c->pos_count, 0, sizeof(h)));
  out[0] = (int64_t)h;
  return DG_OK;
}

extern "C" dg_status dg_limit_state(dg_ctx* c) {
  if (!c || !(c->pos_eps > 0.0)) return DG_EINVAL;
  if (!c->have_state) return DG_ESTATE;
  cudaSetDevice(c->dev);
  DgArgs b = base_args(c);
  b.out = c->u[c->cur];
  c->thermo_ok = false;
  CK(run_positivity(c, b));
  dg_status w = wait_stream(c);
  if (w != DG_OK) return w;
  return take_status(c, NULL);
}
