// Data preparation of the learned surrogates on the device: column statistics of sample
// arrays (optionally of their asinh image), standardisation, quantiles of absolute
// values, row gathers for minibatches, and the mean-squared error of the perceptron on a
// data set.  Every reduction is two-level with a fixed order (per-block partial results in
// a fixed tree, then one block over the partials), so results are deterministic.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "../../include/dg.h"
#include "dg_mlp.cuh"

namespace {

constexpr int RB = 256;     // threads of the reduction blocks
constexpr int MAXB = 1024;  // partial blocks

unsigned blocks_for(int64_t n) {
  int64_t b = (n + RB - 1) / RB;
  return (unsigned)(b < 1 ? 1 : (b > MAXB ? MAXB : b));
}

// value of column c of row i, through the asinh image when ref != null
__device__ __forceinline__ double col_val(const void* X, int is_f64, int64_t i, int d, int c, const double* ref) {
  const double v = is_f64 ? ((const double*)X)[i * d + c] : (double)((const float*)X)[i * d + c];
  return ref ? asinh(v / ref[c]) : v;
}

// per-block partials of column c: sum (pass 0) or sum of squared deviations from mean[c]
// (pass 1), and min / max; grid-stride over rows, fixed-tree block reduction
__global__ void col_partial_kernel(const void* X, int is_f64, int64_t n, int d, int c, const double* ref,
                                   const double* mean, double* part) {
  __shared__ double s_sum[RB], s_min[RB], s_max[RB];
  double sum = 0.0, mn = INFINITY, mx = -INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB) {
    const double v = col_val(X, is_f64, i, d, c, ref);
    if (mean) {
      const double dv = v - mean[c];
      sum += dv * dv;
    } else {
      sum += v;
    }
    mn = fmin(mn, v);
    mx = fmax(mx, v);
  }
  s_sum[threadIdx.x] = sum;
  s_min[threadIdx.x] = mn;
  s_max[threadIdx.x] = mx;
  __syncthreads();
  for (int h = RB / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s_sum[threadIdx.x] += s_sum[threadIdx.x + h];
      s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + h]);
      s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x + 0] = s_sum[0];
    part[3 * blockIdx.x + 1] = s_min[0];
    part[3 * blockIdx.x + 2] = s_max[0];
  }
}

// one block: combine nb partials in a fixed order into out[0..2] (sum, min, max)
__global__ void col_final_kernel(const double* part, int nb, double* out) {
  __shared__ double s_sum[RB], s_min[RB], s_max[RB];
  double sum = 0.0, mn = INFINITY, mx = -INFINITY;
  for (int b = threadIdx.x; b < nb; b += RB) {
    sum += part[3 * b];
    mn = fmin(mn, part[3 * b + 1]);
    mx = fmax(mx, part[3 * b + 2]);
  }
  s_sum[threadIdx.x] = sum;
  s_min[threadIdx.x] = mn;
  s_max[threadIdx.x] = mx;
  __syncthreads();
  for (int h = RB / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s_sum[threadIdx.x] += s_sum[threadIdx.x + h];
      s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + h]);
      s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s_sum[0];
    out[1] = s_min[0];
    out[2] = s_max[0];
  }
}

__global__ void standardize_kernel(const void* X, int is_f64, int64_t n, int d, const double* ref, const double* mean,
                                   const double* inv_std, float* out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * d; q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q % d);
    out[q] = (float)((col_val(X, is_f64, q / d, d, c, ref) - mean[c]) * inv_std[c]);
  }
}

// number of |Y[i][c]| (c0 <= c < c0 + nc) whose bit pattern is <= key (non-negative doubles
// order like their patterns), per-block partials
__global__ void count_le_kernel(const double* Y, int64_t n, int d, int c0, int nc, unsigned long long key,
                                unsigned long long* part) {
  __shared__ unsigned long long s[RB];
  unsigned long long cnt = 0;
  const int64_t m = n * nc;
  for (int64_t q = blockIdx.x * (int64_t)RB + threadIdx.x; q < m; q += (int64_t)gridDim.x * RB) {
    const double v = fabs(Y[(q / nc) * d + c0 + q % nc]);
    cnt += (unsigned long long)__double_as_longlong(v) <= key;
  }
  s[threadIdx.x] = cnt;
  __syncthreads();
  for (int h = RB / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void gather_rows_kernel(const float* X, int d, const int64_t* idx, int64_t m, float* out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m * d; q += (int64_t)gridDim.x * blockDim.x)
    out[q] = X[idx[q / d] * d + q % d];
}

// per-block partial sums of (y - t)^2 over n x no values
__global__ void sq_err_kernel(const float* y, const float* t, int64_t m, double* part) {
  __shared__ double s[RB];
  double sum = 0.0;
  for (int64_t q = blockIdx.x * (int64_t)RB + threadIdx.x; q < m; q += (int64_t)gridDim.x * RB) {
    const double e = (double)y[q] - (double)t[q];
    sum += e * e;
  }
  s[threadIdx.x] = sum;
  __syncthreads();
  for (int h = RB / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = s[0];
    part[3 * blockIdx.x + 1] = 0.0;
    part[3 * blockIdx.x + 2] = 0.0;
  }
}

// FP32 forward of the perceptron (dg_mlp.cu)
}  // namespace

cudaError_t dg_mlp_forward_f32_launch(const float* P, int no, const float* X, float* y, int64_t n, cudaStream_t s);

namespace {

dg_status copy_ref(const double* ref_host, int d, double** ref_dev) {
  *ref_dev = NULL;
  if (!ref_host) return DG_OK;
  for (int c = 0; c < d; ++c)
    if (!(ref_host[c] > 0.0)) return DG_EINVAL;
  if (cudaMalloc((void**)ref_dev, sizeof(double) * d) != cudaSuccess) return DG_ENOMEM;
  if (cudaMemcpy(*ref_dev, ref_host, sizeof(double) * d, cudaMemcpyHostToDevice) != cudaSuccess) return DG_ECUDA;
  return DG_OK;
}

}  // namespace

extern "C" {

dg_status dg_column_stats(const void* X, int is_f64, int64_t n, int d, const double* ref, double* out,
                          void* stream) {
  if (!X || !out || n < 2 || d < 1 || d > 64) return DG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  double *dref = NULL, *part = NULL, *res = NULL, *mean = NULL;
  dg_status r = copy_ref(ref, d, &dref);
  if (r != DG_OK) {
    cudaFree(dref);
    return r;
  }
  const unsigned nb = blocks_for(n);
  cudaError_t e = cudaMalloc((void**)&part, sizeof(double) * 3 * nb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&res, sizeof(double) * 3 * 2 * d);
  if (e == cudaSuccess) e = cudaMalloc((void**)&mean, sizeof(double) * d);
  double* h = (double*)malloc(sizeof(double) * 3 * 2 * d);
  double* hm = (double*)malloc(sizeof(double) * d);
  if (!h || !hm) e = cudaErrorMemoryAllocation;
  // pass 0: sums, min, max; then the means; pass 1: squared deviations from the means
  for (int c = 0; e == cudaSuccess && c < d; ++c) {
    col_partial_kernel<<<nb, RB, 0, st>>>(X, is_f64, n, d, c, dref, NULL, part);
    col_final_kernel<<<1, RB, 0, st>>>(part, (int)nb, res + 3 * c);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof(double) * 3 * d, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (int c = 0; e == cudaSuccess && c < d; ++c) hm[c] = h[3 * c] / (double)n;
  if (e == cudaSuccess) e = cudaMemcpy(mean, hm, sizeof(double) * d, cudaMemcpyHostToDevice);
  for (int c = 0; e == cudaSuccess && c < d; ++c) {
    col_partial_kernel<<<nb, RB, 0, st>>>(X, is_f64, n, d, c, dref, mean, part);
    col_final_kernel<<<1, RB, 0, st>>>(part, (int)nb, res + 3 * (d + c));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h + 3 * d, res + 3 * d, sizeof(double) * 3 * d, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    for (int c = 0; c < d; ++c) {
      out[c] = hm[c];                                          // mean
      out[d + c] = sqrt(h[3 * (d + c)] / (double)(n - 1));   // standard deviation (n - 1)
      out[2 * d + c] = h[3 * c + 1];                           // min
      out[3 * d + c] = h[3 * c + 2];                           // max
    }
  }
  cudaFree(part);
  cudaFree(res);
  cudaFree(mean);
  cudaFree(dref);
  free(h);
  free(hm);
  return e == cudaSuccess ? DG_OK : (e == cudaErrorMemoryAllocation ? DG_ENOMEM : DG_ECUDA);
}

dg_status dg_standardize(const void* X, int is_f64, int64_t n, int d, const double* ref, const double* mean,
                         const double* std_dev, float* out, void* stream) {
  if (!X || !mean || !std_dev || !out || n < 1 || d < 1 || d > 64) return DG_EINVAL;
  for (int c = 0; c < d; ++c)
    if (!(std_dev[c] > 0.0)) return DG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  double* dref = NULL;
  dg_status r = copy_ref(ref, d, &dref);
  if (r != DG_OK) {
    cudaFree(dref);
    return r;
  }
  double* ms = NULL;
  double* h = (double*)malloc(sizeof(double) * 2 * d);
  cudaError_t e = h ? cudaMalloc((void**)&ms, sizeof(double) * 2 * d) : cudaErrorMemoryAllocation;
  if (e == cudaSuccess) {
    for (int c = 0; c < d; ++c) {
      h[c] = mean[c];
      h[d + c] = 1.0 / std_dev[c];
    }
    e = cudaMemcpy(ms, h, sizeof(double) * 2 * d, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    int64_t g = (n * d + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    standardize_kernel<<<(unsigned)g, 256, 0, st>>>(X, is_f64, n, d, dref, ms, ms + d, out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(ms);
  cudaFree(dref);
  free(h);
  return e == cudaSuccess ? DG_OK : DG_ECUDA;
}

dg_status dg_abs_quantile(const double* Y, int64_t n, int d, int c0, int nc, double q, double* out, void* stream) {
  if (!Y || !out || n < 1 || d < 1 || c0 < 0 || nc < 1 || c0 + nc > d || !(q >= 0.0 && q <= 1.0)) return DG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t m = n * nc;
  const unsigned nb = blocks_for(m);
  unsigned long long *part = NULL, *hp = (unsigned long long*)malloc(sizeof(unsigned long long) * nb);
  cudaError_t e = hp ? cudaMalloc((void**)&part, sizeof(unsigned long long) * nb) : cudaErrorMemoryAllocation;
  // the k-th smallest |value| (0-based) by bisection on the bit pattern: the smallest key
  // with count(<= key) >= k + 1
  auto kth = [&](int64_t k, double* v) -> cudaError_t {
    unsigned long long lo = 0ull, hi = 0x7FF0000000000000ull;  // +0 .. +inf
    while (lo < hi) {
      const unsigned long long mid = lo + (hi - lo) / 2;
      count_le_kernel<<<nb, RB, 0, st>>>(Y, n, d, c0, nc, mid, part);
      cudaError_t e2 = cudaGetLastError();
      if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(hp, part, sizeof(unsigned long long) * nb, cudaMemcpyDeviceToHost, st);
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
      if (e2 != cudaSuccess) return e2;
      unsigned long long cnt = 0;
      for (unsigned b = 0; b < nb; ++b) cnt += hp[b];
      if (cnt >= (unsigned long long)(k + 1)) hi = mid;
      else lo = mid + 1;
    }
    long long bits = (long long)lo;
    memcpy(v, &bits, sizeof(double));
    return cudaSuccess;
  };
  // linear interpolation between the order statistics around position q (m - 1)
  const double pos = q * (double)(m - 1);
  const int64_t k = (int64_t)floor(pos);
  double v0 = 0.0, v1 = 0.0;
  if (e == cudaSuccess) e = kth(k, &v0);
  if (e == cudaSuccess) e = k + 1 < m ? kth(k + 1, &v1) : cudaSuccess;
  if (e == cudaSuccess) *out = k + 1 < m ? v0 + (pos - (double)k) * (v1 - v0) : v0;
  cudaFree(part);
  free(hp);
  return e == cudaSuccess ? DG_OK : DG_ECUDA;
}

dg_status dg_gather_rows(const float* X, int d, const int64_t* idx, int64_t m, float* out, void* stream) {
  if (!X || !idx || !out || d < 1 || m < 1) return DG_EINVAL;
  int64_t g = (m * d + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  gather_rows_kernel<<<(unsigned)g, 256, 0, (cudaStream_t)stream>>>(X, d, idx, m, out);
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_ECUDA;
}

dg_status dg_mlp_loss(const float* params, int n_out, const float* X, const float* t, int64_t n, double* loss,
                      void* stream) {
  if (!params || !X || !t || !loss || n < 1 || n_out < 1 || n_out > DG_MLP_NO_MAX) return DG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t m = n * n_out;
  const unsigned nb = blocks_for(m);
  float* y = NULL;
  double *part = NULL, *res = NULL;
  cudaError_t e = cudaMalloc((void**)&y, sizeof(float) * m);
  if (e == cudaSuccess) e = cudaMalloc((void**)&part, sizeof(double) * 3 * nb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&res, sizeof(double) * 3);
  if (e == cudaSuccess) e = dg_mlp_forward_f32_launch(params, n_out, X, y, n, st);
  if (e == cudaSuccess) {
    sq_err_kernel<<<nb, RB, 0, st>>>(y, t, m, part);
    col_final_kernel<<<1, RB, 0, st>>>(part, (int)nb, res);
    e = cudaGetLastError();
  }
  double h[3] = {0.0, 0.0, 0.0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) *loss = h[0] / (double)m;
  cudaFree(y);
  cudaFree(part);
  cudaFree(res);
  return e == cudaSuccess ? DG_OK : DG_ECUDA;
}

}  // extern "C"
