// Fifth-generation tensor-core (tcgen05) forward of the 7 -> 64 -> 64 -> NO perceptron:
// one CTA of four warps evaluates tiles of 128 rows.  Layers 1 and 2 are tcgen05.mma
// (kind::f16, BF16 operands from shared memory, FP32 accumulators in tensor memory);
// the epilogue of each reads its 32 rows per warp back with tcgen05.ld, adds the bias and
// applies GELU; the layer-2 epilogue also forms the NO outputs as FP32 dot products with
// W3 (as the warp-level path does), so the hidden units are rounded to BF16 only once.
//
// Shared-memory operands use the no-swizzle K-major canonical layout: core matrices of
// 8 rows x 16 bytes (8 BF16 of K), 128 bytes each; the two core matrices of a 16-wide K
// slice sit LBO = 128 bytes apart and consecutive 8-row groups SBO = (K/8) x 128 bytes
// apart, so element (row, k) of a [R][K] operand is at
//   (row/8) SBO + (k/8) 128 + (row%8) 16 + (k%8) 2 bytes.
// Tensor memory: 128 lanes (rows) x 128 columns, layer 1 in columns 0-63, layer 2 in
// 64-127.  Every wait on an mbarrier is bounded; on a timeout the kernel records it, waits
// once more (bounded) for its MMAs in flight, frees its tensor memory and returns.
#pragma once
#include "dg_mlp.cuh"

namespace dgtc5 {

constexpr int ROWS = 128;     // rows per tile (the MMA's M)
constexpr int THREADS = 128;  // four warps: one TMEM lane quarter each
constexpr uint32_t TMEM_COLS = 128;

template <int NO>
struct __align__(1024) Smem {
  __nv_bfloat16 X[ROWS * 16];                    // A of layer 1 [128][16], features zero padded
  __nv_bfloat16 H[ROWS * DG_MLP_NH];             // A of layer 2 [128][64]
  __nv_bfloat16 W1[DG_MLP_NH * 16];              // B of layer 1 [64][16]
  __nv_bfloat16 W2[DG_MLP_NH * DG_MLP_NH];       // B of layer 2 [64][64]
  float b1[DG_MLP_NH], b2[DG_MLP_NH];
  float W3[NO][DG_MLP_NH], b3[NO];
  unsigned long long bar;
  uint32_t tmem;
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) in a K-major canonical operand with K columns
__device__ __forceinline__ uint32_t canon(int row, int k, int K) {
  return (uint32_t)((row >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), descriptor
// version 1 (bits 46-47), base offset 0, no swizzle
__device__ __forceinline__ uint64_t sdesc(const void* p, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((su32(p) >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9 and
// 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// generic-proxy writes to shared memory made visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_smem_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ bool wait_parity(unsigned long long* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 16); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// weights from the FP32 parameter vector (layout of dg_mlp_np) into the canonical
// BF16 operands, biases and the FP32 output layer
template <int NO>
__device__ __forceinline__ void load_weights(Smem<NO>& s, const float* P) {
  constexpr int NI = DG_MLP_NI, NH = DG_MLP_NH;
  const int tid = threadIdx.x;
  for (int i = tid; i < NH * 16; i += THREADS) {
    const int j = i / 16, k = i % 16;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(s.W1) + canon(j, k, 16)) =
        __float2bfloat16(k < NI ? P[j * NI + k] : 0.0f);
  }
  for (int i = tid; i < NH * NH; i += THREADS) {
    const int j = i / NH, k = i % NH;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(s.W2) + canon(j, k, NH)) =
        __float2bfloat16(P[NH * NI + NH + j * NH + k]);
  }
  for (int j = tid; j < NH; j += THREADS) {
    s.b1[j] = P[NH * NI + j];
    s.b2[j] = P[NH * NI + NH + NH * NH + j];
  }
  for (int i = tid; i < NO * NH; i += THREADS) s.W3[i / NH][i % NH] = P[dg_mlp_off_w3() + i];
  if (tid < NO) s.b3[tid] = P[dg_mlp_off_b3(NO) + tid];
}

// the same from a packed BF16 weight image (dg_mlp_pack)
template <int NO>
__device__ __forceinline__ void load_weights(Smem<NO>& s, const DgMlpW<NO>& w) {
  constexpr int NH = DG_MLP_NH;
  const int tid = threadIdx.x;
  for (int i = tid; i < NH * 16; i += THREADS)
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(s.W1) + canon(i / 16, i % 16, 16)) = w.W1[i];
  for (int i = tid; i < NH * NH; i += THREADS)
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(s.W2) + canon(i / NH, i % NH, NH)) = w.W2[i];
  for (int j = tid; j < NH; j += THREADS) {
    s.b1[j] = w.b1[j];
    s.b2[j] = w.b2[j];
  }
  for (int i = tid; i < NO * NH; i += THREADS) s.W3[i / NH][i % NH] = w.W3[i / NH][i % NH];
  if (tid < NO) s.b3[tid] = w.b3[tid];
}

// The tile engine (after load_weights): for each 128-row tile of the CTA, thread t takes
// row = 128 tile + t.  prod(row, x) writes the row's 7 standardised features and returns a
// flag of its own; cons(row, out, flag, valid) gets the NO outputs, that flag and whether
// the launch's tensor-core waits all completed (when not, out is not valid).  Both are
// called by every thread of the CTA for every tile (rows >= n included), so consumers may
// use warp votes.  The engine allocates and frees the tensor memory and returns false
// after a timeout (the remaining tiles still reach cons with valid = false).
template <int NO, class Prod, class Cons>
__device__ __forceinline__ bool run_tiles(Smem<NO>& s, int64_t n, Prod prod, Cons cons) {
  constexpr int NH = DG_MLP_NH;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&s.tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&s.bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  fence_smem_async();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s.tmem;
  const uint32_t lane_base = (uint32_t)(32 * warp) << 16;  // this warp's TMEM lane quarter
  constexpr uint32_t ID_L = idesc_bf16(ROWS, NH);
  uint32_t parity = 0;
  bool ok = true;
  const int64_t tiles = (n + ROWS - 1) / ROWS;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t row = tile * ROWS + tid;
    float x[8];
    const bool flag = prod(row, x);
    if (ok) {
      // features -> A of layer 1 (this thread's row: K 0-7 and the zero padding 8-15)
      uint4 lo, hi = make_uint4(0u, 0u, 0u, 0u);
      lo.x = dgmlp::pack_bf16(x[0], x[1]);
      lo.y = dgmlp::pack_bf16(x[2], x[3]);
      lo.z = dgmlp::pack_bf16(x[4], x[5]);
      lo.w = dgmlp::pack_bf16(x[6], x[7]);
      unsigned char* xb = reinterpret_cast<unsigned char*>(s.X);
      *reinterpret_cast<uint4*>(xb + canon(tid, 0, 16)) = lo;
      *reinterpret_cast<uint4*>(xb + canon(tid, 8, 16)) = hi;
      fence_smem_async();
      fence_before();
      __syncthreads();
      fence_after();
      if (tid == 0) {
        mma(tmem, sdesc(s.X, 128, 256), sdesc(s.W1, 128, 256), ID_L, 0);
        commit(&s.bar);
      }
      // the wait's outcome made uniform across the CTA; the phase flips only on completion
      ok = __syncthreads_and(wait_parity(&s.bar, parity)) != 0;
      if (ok) parity ^= 1u;
      fence_after();
    }
    if (ok) {
      // layer-1 epilogue: bias, GELU, BF16 -> A of layer 2 (this thread's row)
      unsigned char* hb = reinterpret_cast<unsigned char*>(s.H);
      float v[NH / 16][16];
#pragma unroll
      for (int c = 0; c < NH / 16; ++c) ld16(tmem + lane_base + 16 * c, v[c]);
      ld_wait();
#pragma unroll
      for (int c = 0; c < NH / 16; ++c) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float g[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) g[q] = dgmlp::gelu_fast(v[c][8 * h + q] + s.b1[16 * c + 8 * h + q]);
          uint4 pk;
          pk.x = dgmlp::pack_bf16(g[0], g[1]);
          pk.y = dgmlp::pack_bf16(g[2], g[3]);
          pk.z = dgmlp::pack_bf16(g[4], g[5]);
          pk.w = dgmlp::pack_bf16(g[6], g[7]);
          *reinterpret_cast<uint4*>(hb + canon(tid, 16 * c + 8 * h, NH)) = pk;
        }
      }
      fence_smem_async();
      fence_before();
      __syncthreads();
      fence_after();
      if (tid == 0) {
#pragma unroll
        for (int kb = 0; kb < NH / 16; ++kb)
          mma(tmem + NH, sdesc(reinterpret_cast<unsigned char*>(s.H) + 256 * kb, 128, 1024),
              sdesc(reinterpret_cast<unsigned char*>(s.W2) + 256 * kb, 128, 1024), ID_L, kb > 0);
        commit(&s.bar);
      }
      ok = __syncthreads_and(wait_parity(&s.bar, parity)) != 0;
      if (ok) parity ^= 1u;
      fence_after();
    }
    // layer-2 epilogue: bias, GELU, then the NO outputs as FP32 dot products with W3
    float out[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) out[o] = s.b3[o];
    if (ok) {
      float v2[NH / 16][16];
#pragma unroll
      for (int c = 0; c < NH / 16; ++c) ld16(tmem + lane_base + NH + 16 * c, v2[c]);
      ld_wait();
#pragma unroll
      for (int c = 0; c < NH / 16; ++c) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float g = dgmlp::gelu_fast(v2[c][q] + s.b2[16 * c + q]);
#pragma unroll
          for (int o = 0; o < NO; ++o) out[o] += s.W3[o][16 * c + q] * g;
        }
      }
    }
    cons(row, out, flag, ok);
    fence_before();
    __syncthreads();  // the next tile rewrites X, H and the accumulators
    fence_after();
  }
  if (!ok)  // uniform: the MMAs of the phase that timed out may still run; one more bounded wait
    wait_parity(&s.bar, parity);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  return ok;
}

// y[n][NO] = network(X[n][7]) for standardised X.  *err is set to 1 when a bounded wait ran
// out (the outputs of that launch are then not valid).  Launch with THREADS threads and
// dynamic shared memory of at least sizeof(Smem<NO>) (more to limit resident CTAs).
template <int NO>
__global__ void __launch_bounds__(THREADS, 1) mlp_forward_tc5_kernel(const float* P, const float* X, float* y,
                                                                     int64_t n, unsigned* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Smem<NO>& s = *reinterpret_cast<Smem<NO>*>(smem_raw);
  load_weights<NO>(s, P);
  auto prod = [&](int64_t row, float* x) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (row < n && k < DG_MLP_NI) ? X[row * DG_MLP_NI + k] : 0.0f;
    return true;
  };
  auto cons = [&](int64_t row, const float* out, bool, bool valid) {
    if (row < n && valid)
#pragma unroll
      for (int o = 0; o < NO; ++o) y[row * NO + o] = out[o];
  };
  if (!run_tiles<NO>(s, n, prod, cons) && threadIdx.x == 0) atomicExch(err, 1u);
}

}  // namespace dgtc5
