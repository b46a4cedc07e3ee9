// Arithmetic-peak microbenchmark: the denominator of the roofline for kernels bound by
// FP64 or FP32 arithmetic (the FP64 form, the temperature solve, the chemistry source).
// Every thread runs 8 independent chains of fused multiply-adds; the grid is 152 SMs x
// 8 CTAs of 256 threads; the result is 2 flops per FMA over the CUDA-event time.
#include <cuda_runtime.h>

#include "../../include/dg.h"

namespace {

template <typename T>
__global__ void fma_chains(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = x[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  if (s == (T)12345.678) out[0] = s;  // keeps the chains alive, never true in practice
}

}  // namespace

extern "C" dg_status dg_peak_flops(int precision, int iters, double* tflops) {
  if (!tflops || iters < 1 || (precision != DG_FP64 && precision != DG_MIXED)) return DG_EINVAL;
  const int grid = 152 * 8, block = 256;
  void* out = NULL;
  if (cudaMalloc(&out, 16) != cudaSuccess) return DG_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // warm-up launch, then the timed one
  for (int rep = 0; rep < 2; ++rep) {
    if (rep == 1) cudaEventRecord(e0);
    if (precision == DG_FP64)
      fma_chains<double><<<grid, block>>>((double*)out, iters, 0.999999, 1e-7);
    else
      fma_chains<float><<<grid, block>>>((float*)out, iters, 0.999999f, 1e-7f);
    if (rep == 1) cudaEventRecord(e1);
  }
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return DG_ECUDA;
  const double flops = 2.0 * 8.0 * (double)iters * grid * block;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return DG_OK;
}
