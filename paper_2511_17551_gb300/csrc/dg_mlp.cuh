// Device pieces shared by the learned surrogates (temperature: one output; chemistry
// source: ten outputs): the 7 -> 64 -> 64 -> NO perceptron with the tanh form of GELU,
// its BF16 weight image, and the tensor-core forward of a 16-row tile.
//
// Parameter vector (FP32 master copy, host and training layout): W1[64][7], b1[64],
// W2[64][64], b2[64], W3[NO][64], b3[NO].
//
// Tile forward (mlp16): one warp evaluates 16 rows with mma.sync m16n8k16 (BF16
// operands, FP32 accumulation).  Layer 1 is 8 MMAs against W1 zero-padded to K = 16,
// layer 2 is 32 MMAs; the FP32 accumulator fragments of a layer are exactly the A
// fragments of the next (two n-tiles of 8 = one k-block of 16), so activations never
// leave registers.  Layer 3 (NO outputs) is an FP32 dot product over the 64 hidden
// units, reduced across the 4 lanes that share a row.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define DG_MLP_NI 7
#define DG_MLP_NH 64
#define DG_MLP_NO_MAX 16

__host__ __device__ constexpr int dg_mlp_off_w3() { return DG_MLP_NH * DG_MLP_NI + DG_MLP_NH + DG_MLP_NH * DG_MLP_NH + DG_MLP_NH; }
__host__ __device__ constexpr int dg_mlp_off_b3(int no) { return dg_mlp_off_w3() + no * DG_MLP_NH; }
__host__ __device__ constexpr int dg_mlp_np(int no) { return dg_mlp_off_b3(no) + no; }

template <int NO>
struct __align__(16) DgMlpW {
  __nv_bfloat16 W1[DG_MLP_NH * 16];         // [j][k], k >= 7 zero
  __nv_bfloat16 W2[DG_MLP_NH * DG_MLP_NH];  // [j][i]
  float b1[DG_MLP_NH], b2[DG_MLP_NH];
  float W3[NO][DG_MLP_NH], b3[NO];
};

// BF16 image of an FP32 parameter vector (host side)
template <int NO>
inline void dg_mlp_pack(const float* p, DgMlpW<NO>* w) {
  const int NI = DG_MLP_NI, NH = DG_MLP_NH;
  for (int j = 0; j < NH; ++j) {
    for (int k = 0; k < 16; ++k) w->W1[j * 16 + k] = __float2bfloat16(k < NI ? p[j * NI + k] : 0.0f);
    for (int i = 0; i < NH; ++i) w->W2[j * NH + i] = __float2bfloat16(p[NH * NI + NH + j * NH + i]);
    w->b1[j] = p[NH * NI + j];
    w->b2[j] = p[NH * NI + NH + NH * NH + j];
    for (int o = 0; o < NO; ++o) w->W3[o][j] = p[dg_mlp_off_w3() + o * NH + j];
  }
  for (int o = 0; o < NO; ++o) w->b3[o] = p[dg_mlp_off_b3(NO) + o];
}

namespace dgmlp {

__device__ __forceinline__ float gelu_f(float x) {
  const float k = 0.7978845608028654f;  // sqrt(2/pi)
  return 0.5f * x * (1.0f + tanhf(k * (x + 0.044715f * x * x * x)));
}
// inference GELU: the hardware tanh approximation (tanh.approx.f32, relative error about
// 2^-11), below the BF16 rounding of the layer inputs
__device__ __forceinline__ float gelu_fast(float x) {
  const float k = 0.7978845608028654f;
  float z = k * (x + 0.044715f * x * x * x), t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(z));
  return 0.5f * x * (1.0f + t);
}
__device__ __forceinline__ float gelu_d_f(float x) {
  const float k = 0.7978845608028654f;
  float t = tanhf(k * (x + 0.044715f * x * x * x));
  return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * k * (1.0f + 3.0f * 0.044715f * x * x);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 16 rows of standardised features feat[16][17] (float, columns >= 7 zero) -> outputs
// y[o][row] for the calling warp.  Every lane of the warp must call it.
template <int NO>
__device__ __forceinline__ void mlp16(const DgMlpW<NO>& m, const float (*feat)[17], float (*y)[16]) {
  constexpr int NH = DG_MLP_NH;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t A[4];
  A[0] = pack_bf16(feat[g][2 * t], feat[g][2 * t + 1]);
  A[1] = pack_bf16(feat[g + 8][2 * t], feat[g + 8][2 * t + 1]);
  A[2] = pack_bf16(feat[g][2 * t + 8], feat[g][2 * t + 9]);
  A[3] = pack_bf16(feat[g + 8][2 * t + 8], feat[g + 8][2 * t + 9]);
  float h[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int col = 8 * nt + 2 * t;
    h[nt][0] = h[nt][2] = m.b1[col];
    h[nt][1] = h[nt][3] = m.b1[col + 1];
    const uint32_t* w = reinterpret_cast<const uint32_t*>(m.W1 + (8 * nt + g) * 16);
    mma_bf16(h[nt], A, w[t], w[t + 4]);
#pragma unroll
    for (int q = 0; q < 4; ++q) h[nt][q] = gelu_fast(h[nt][q]);
  }
  uint32_t A2[4][4];
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
    A2[kb][0] = pack_bf16(h[2 * kb][0], h[2 * kb][1]);
    A2[kb][1] = pack_bf16(h[2 * kb][2], h[2 * kb][3]);
    A2[kb][2] = pack_bf16(h[2 * kb + 1][0], h[2 * kb + 1][1]);
    A2[kb][3] = pack_bf16(h[2 * kb + 1][2], h[2 * kb + 1][3]);
  }
  float ya[NO], yb[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) ya[o] = yb[o] = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int col = 8 * nt + 2 * t;
    float o4[4] = {m.b2[col], m.b2[col + 1], m.b2[col], m.b2[col + 1]};
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
      const uint32_t* w = reinterpret_cast<const uint32_t*>(m.W2 + (8 * nt + g) * NH + 16 * kb);
      mma_bf16(o4, A2[kb], w[t], w[t + 4]);
    }
    const float q0 = gelu_fast(o4[0]), q1 = gelu_fast(o4[1]), q2 = gelu_fast(o4[2]), q3 = gelu_fast(o4[3]);
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      ya[o] += m.W3[o][col] * q0 + m.W3[o][col + 1] * q1;
      yb[o] += m.W3[o][col] * q2 + m.W3[o][col + 1] * q3;
    }
  }
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    ya[o] += __shfl_xor_sync(0xffffffffu, ya[o], 1);
    ya[o] += __shfl_xor_sync(0xffffffffu, ya[o], 2);
    yb[o] += __shfl_xor_sync(0xffffffffu, yb[o], 1);
    yb[o] += __shfl_xor_sync(0xffffffffu, yb[o], 2);
  }
  if (t == 0) {
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      y[o][g] = ya[o] + m.b3[o];
      y[o][g + 8] = yb[o] + m.b3[o];
    }
  }
}

// copy a weight image (any 16-byte-aligned struct) global -> shared, all threads of the CTA
template <typename W>
__device__ __forceinline__ void copy_to_smem(W& dst, const W* src) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(W) / 16); i += blockDim.x) d[i] = s[i];
}

}  // namespace dgmlp
