// Kernels and launchers for one precision.  The including translation unit
// defines DG_REAL (double or float) and DG_PREFIX (namespace and function-name
// prefix, e.g. dg_f32), so profiles name kernels dg_f32::rhs_kernel<...>.
//
// The right-hand-side kernel comes in three flavours: FL = 1 fixes the production flux
// pair at compile time (Ranocha volume flux for one gas, Ducros for mixtures; LLF at
// interfaces and subcells, constant viscosity), FL = 2 + vf fixes another one-gas volume
// flux vf with LLF and constant viscosity (the split forms, emitted for 3D at N = 3), and
// FL = 0 switches on the runtime choice (every other pair, and Sutherland's law).
// A translation unit that defines DG_GENERIC_ONLY emits only the FL = 0 kernels (and
// its own basis table); one that also defines DG_SPLIT_ONLY emits only the FL = 2 + vf
// kernels; the main one emits everything else and forwards the other pairs to
// DG_SPLIT_RHS (where defined) or DG_GENERIC_RHS.  The split keeps register pressure of the
// compile-time kernels free of the unused branches and lets the parts compile in parallel.
#pragma once
#include <stdint.h>
#include "dg_kernels.cuh"

#ifdef DG_GENERIC_ONLY
#define DG_FL 0
#else
#define DG_FL 1
#endif

namespace DG_PREFIX {

using real = DG_REAL;
using namespace dgk;

__constant__ BasisTab<real> c_tab[DG_MAXN + 1];

// Scalars of one launch in the form precision (no double arithmetic or double->float
// conversion inside FP32 kernels).
struct KConst {
  real gamma, gm1, inv_gm1, mu, kap, visc, rkA, rkB;
  real pref, eref;  // pressure offset of the momentum fluxes and pref / (gamma - 1)
  real suth_s, suth_c1, suth_irt;  // Sutherland's law: s, 1 + s, 1 / rt_ref (s = 0: off)
};

inline KConst make_kconst(const DgArgs& a) {
  KConst k;
  k.gamma = (real)a.gamma;
  k.gm1 = (real)(a.gamma - 1.0);
  k.inv_gm1 = (real)(1.0 / (a.gamma - 1.0));
  k.mu = (real)a.mu;
  k.kap = (real)a.kappa_fac;
  k.visc = (real)a.visc_coef;
  k.rkA = (real)a.rkA;
  k.rkB = (real)a.rkB;
  k.pref = (real)a.pref;
  k.eref = (real)(a.pref / (a.gamma - 1.0));
  k.suth_s = (real)a.suth_s;
  k.suth_c1 = (real)(1.0 + a.suth_s);
  k.suth_irt = (real)(a.suth_rt > 0.0 ? 1.0 / a.suth_rt : 0.0);
  return k;
}

// elements per CTA: the largest count whose line threads fit in TPB threads
template <int DIM, int N, int TPB = 192>
constexpr int epb() {
  return Shape<DIM, N>::LINES >= TPB ? 1 : (TPB / Shape<DIM, N>::LINES > 24 ? 24 : TPB / Shape<DIM, N>::LINES);
}

// Shared-memory position of node n inside a per-variable block.  For power-of-two line
// lengths in 3D the i and j digits are XOR-ed with k: any two of (i, j, k) then fix the
// position mod N1^2, so the lines of every direction (and the nodes of every face) fall
// on distinct banks.  An involution; identity otherwise.
template <int DIM, int N>
struct Swizzle {
  static constexpr int N1 = N + 1;
  static constexpr bool ON = DIM == 3 && (N1 & (N1 - 1)) == 0;
  static __device__ __forceinline__ int at(int n) {
    if (!ON) return n;
    return n ^ ((n / (N1 * N1)) * (N1 + 1));
  }
};

// resident-CTA target of the one-gas kernels: 8 (measured with the aliased layout below:
// 9 and 10 CTAs of 96 threads cap the registers at 72 and 64, and the spills cost more than
// the extra warps give back)
#ifndef DG_RHS_CAP1
#define DG_RHS_CAP1 8
#endif
template <int DIM, int N, int NSP, bool NS, bool AL = true>
struct Layout {
  using S = Shape<DIM, N>;
  static constexpr int NV = NSP + DIM + 1;
  static constexpr int NP = S::NP;
  // CTA shape (measured): one gas 96-thread CTAs, up to 8 per SM; mixtures 192 threads
  static constexpr int EPB = epb<DIM, N, (NSP > 1 ? 192 : 96)>();
  static constexpr int NQ = DIM + 3;                // rho, v, p, beta(=rho/p)
  static constexpr int NFV = NS ? DIM * (DIM + 1) : 0;
  static constexpr int FACE_NODES = 2 * DIM * S::LPD;  // per element
  // Bank-conflict-free shared layout for power-of-two line lengths: nodes are swizzled
  // (swz), warps of the line and face phases take one direction (face) of two elements,
  // and in FP32 consecutive elements sit 16 words (mod 32) apart, so the two elements of
  // a warp fill complementary halves of the 32 banks.
  static constexpr bool SWZ = Swizzle<DIM, N>::ON;
  static constexpr bool UNI = SWZ && (EPB * S::LPD) % 32 == 0;
  static constexpr int padded(int w) { return (SWZ && sizeof(real) == 4) ? w + (48 - w % 32) % 32 : w; }
  // per-element strides (reals) and region offsets of one CTA
  static constexpr int SU = padded(NV * NP), SQ = padded(NQ * NP), SJA = padded(DIM * DIM * NP);
  // AL (the production flux pair's instances): the staged viscous fluxes of direction d sit in
  // the first DIM + 1 planes of direction d's block of the sums region (DIM blocks of NV
  // planes), which the line phase overwrites with the sums: each line reads the fluxes of
  // its own nodes in its own direction before it writes their sums, so the two need no
  // separate space, and the staged low part of the compensated energy sits in direction 0's
  // plane DIM + 1 (free until the line phase).  Otherwise (measured slower for the
  // compile-time split forms) the fluxes have a region of their own, planes [d][c], and the
  // low energy part sits at the start of the sums region, [e][node].
  static constexpr int SIJ = NP, SACC = padded(DIM * NV * NP);
  static constexpr int SFV = (AL || !NS) ? 0 : padded(NFV * NP);
  static constexpr int FVE = AL ? SACC : SFV;          // element stride of the fluxes
  static constexpr int FVD = AL ? NV : DIM + 1;        // planes per direction of the fluxes
  static __device__ __forceinline__ int fvp(int c) { return (c / (DIM + 1)) * FVD + c % (DIM + 1); }
  static __device__ __forceinline__ int elo(int e) { return AL ? e * SACC + (DIM + 1) * NP : e * NP; }
  static constexpr int SPC = NSP > 1 ? padded(2 * NP) : 0, SDU = NV * NP;
  static constexpr int U = 0;
  static constexpr int Q = U + EPB * SU;
  static constexpr int JA = Q + EPB * SQ;
  static constexpr int IJ = JA + EPB * SJA;
  static constexpr int ACC = IJ + EPB * SIJ;
  static constexpr int FV = ACC + EPB * SACC;
  static constexpr int PC = FV + EPB * SFV;          // mixtures: p, c per node
  static constexpr int DU = PC + EPB * SPC;           // prefetched RK register du
  // resident-CTA target (8 of the 96-thread CTAs for one gas; 3 for mixtures, whose
  // 9-variable line accumulators spill below ~110 registers a thread), lowered where shared
  // memory binds
  static constexpr int CAP = NSP > 1 ? 3 : DG_RHS_CAP1;
  static constexpr int ctas_of(size_t bytes) {
    return (int)((227 * 1024) / (bytes + 1024)) >= CAP ? CAP : (int)((227 * 1024) / (bytes + 1024));
  }
  // The residency and register targets below are taken on the footprint with the viscous
  // fluxes in a region of their own (RSV more reals): with the aliasing alone they would
  // rise for the larger instances (N = 7, FP64) and cut their registers into spills; only the
  // allocation shrinks.
  static constexpr int RSV = AL ? EPB * (NS ? padded(NFV * NP) : 0) : 0;
  // du is staged with the rest when that does not cost a resident CTA
  static constexpr bool PREFETCH_DU =
      ctas_of(sizeof(real) * (DU + RSV + EPB * SDU)) == ctas_of(sizeof(real) * (DU + RSV));
  static constexpr int TOTAL = DU + (PREFETCH_DU ? EPB * SDU : 0);
  static constexpr int THREADS = ((EPB * S::LINES + 31) / 32) * 32;
  static constexpr size_t SMEM = sizeof(real) * TOTAL;
  // CTAs per SM we ask the register allocator for (bounded by shared memory)
  static constexpr int MINB = ctas_of(SMEM + sizeof(real) * RSV) < 1 ? 1 : ctas_of(SMEM + sizeof(real) * RSV);
  // face nodes each thread takes in the interface phase
  static constexpr int FIT = (EPB * FACE_NODES + THREADS - 1) / THREADS;
};

// asynchronous global -> shared copies (cp.async): every copy of a phase is in flight at
// once and one wait retires them, instead of one memory round trip per loop iteration
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* dst, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Bulk copies by the TMA engine (cp.async.bulk, global -> shared), completed through one
// mbarrier that counts the bytes.  Both addresses must be 16-byte aligned and the size a
// multiple of 16; the callers check that at compile time (sizes, padded strides) and at run
// time (pointers), and use the per-thread cp.async path otherwise.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// waits for phase 0 of the barrier; bounded (at most 2^16 polls, each suspending for a
// short system-defined time), returns false when the limit ran out
__device__ __forceinline__ bool mbar_wait0(unsigned long long* bar) {
  for (int it = 0; it < (1 << 16); ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar))
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

__device__ __forceinline__ void stage_async(real* dst, const real* src, int n, int tid, int nth) {
  constexpr int V = 16 / sizeof(real);
  if ((((uintptr_t)dst | (uintptr_t)src) & 15) == 0 && (n % V) == 0) {
    for (int i = tid; i < n / V; i += nth) cp_async16(dst + i * V, src + i * V);
  } else {
    for (int i = tid; i < n; i += nth) cp_async_small<sizeof(real)>(dst + i, src + i);
  }
}

// stage ne elements of XV variable blocks into a region of element stride XS (a padded
// layout), 16-byte copies where both sides allow, element-wise otherwise
template <int XV, int XS, int NP>
__device__ __forceinline__ void stage_strided(real* dst, const real* src, int ne, int tid, int nth) {
  constexpr int V = 16 / sizeof(real);
  if (XS == XV * NP) {
    stage_async(dst, src, ne * XV * NP, tid, nth);
    return;
  }
  if ((XV * NP) % V == 0 && XS % V == 0 && (((uintptr_t)dst | (uintptr_t)src) & 15) == 0) {
    constexpr int PER = XV * NP / V;
    for (int i = tid; i < ne * PER; i += nth) {
      const int e = i / PER, r = i % PER;
      cp_async16(dst + e * XS + r * V, src + e * XV * NP + r * V);
    }
  } else {
    for (int i = tid; i < ne * XV * NP; i += nth) {
      const int e = i / (XV * NP), r = i % (XV * NP);
      cp_async_small<sizeof(real)>(dst + e * XS + r, src + i);
    }
  }
}

// stage one NP-block per element (source stride sstride reals between elements) into
// dst[e][NP], 16-byte copies when aligned
// W reals per element from a source element stride sstride to a destination stride dstride
template <int W>
__device__ __forceinline__ void stage_block(real* dst, int dstride, const real* src, int sstride, int ne, int tid,
                                            int nth) {
  constexpr int V = 16 / sizeof(real);
  if (W % V == 0 && (sstride % V) == 0 && (dstride % V) == 0 && (((uintptr_t)dst | (uintptr_t)src) & 15) == 0) {
    constexpr int PER = W / V;
    for (int i = tid; i < ne * PER; i += nth) {
      const int e = i / PER, r = i % PER;
      cp_async16(dst + e * dstride + r * V, src + (int64_t)e * sstride + r * V);
    }
  } else {
    for (int i = tid; i < ne * W; i += nth) {
      const int e = i / W, r = i % W;
      cp_async_small<sizeof(real)>(dst + e * dstride + r, src + (int64_t)e * sstride + r);
    }
  }
}

template <int NP>
__device__ __forceinline__ void stage_rows(real* dst, const real* src, int sstride, int ne, int tid, int nth) {
  constexpr int V = 16 / sizeof(real);
  if (NP % V == 0 && (sstride % V) == 0 && (((uintptr_t)dst | (uintptr_t)src) & 15) == 0) {
    constexpr int PER = NP / V;
    for (int i = tid; i < ne * PER; i += nth) {
      const int e = i / PER, r = i % PER;
      cp_async16(dst + e * NP + r * V, src + (int64_t)e * sstride + r * V);
    }
  } else {
    for (int i = tid; i < ne * NP; i += nth) {
      const int e = i / NP, r = i % NP;
      cp_async_small<sizeof(real)>(dst + e * NP + r, src + (int64_t)e * sstride + r);
    }
  }
}

// boundary / neighbour state at a face node.  Returns 1 when the face flux is the
// physical flux of the returned state (supersonic inflow / outflow).  For an interior
// face the neighbour's conserved state (and p, c for mixtures) arrives preloaded in nu/npc.
template <int DIM, int NSP, bool BND = true>
__device__ __forceinline__ int outer_state(const DgArgs& a, const KConst& kc, int nb, const real* nu,
                                           const real* npc, real nelo, const NodeState<real, DIM, NSP>& own,
                                           const real* n, NodeState<real, DIM, NSP>& x, bool& ok) {
  constexpr int NV = NSP + DIM + 1;
  if (!BND || nb >= 0) {  // BND = false: a mesh without boundary faces (every nb >= 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) x.u[k] = nu[k];
    ok = prim_from_cons<real, DIM, NSP>(x, kc.gamma, NSP > 1 ? npc[0] : real(0), NSP > 1 ? npc[1] : real(0),
                                        kc.pref, kc.eref, nelo);
    return 0;
  }
  int bc = -(nb + 1);
  int kind = a.bc_kind[bc];
  if (kind == DG_BC_INFLOW) {
    const real* bu = (const real*)a.bc_u;
#pragma unroll
    for (int k = 0; k < NV; ++k) x.u[k] = bu[bc * NV + k];
    real pe = 0, ce = 0;
    if (NSP > 1) {
      pe = ((const real*)a.bc_pc)[bc * 2 + 0];
      ce = ((const real*)a.bc_pc)[bc * 2 + 1];
    }
    ok = prim_from_cons<real, DIM, NSP>(x, kc.gamma, pe, ce, kc.pref, kc.eref);
    return 1;
  }
  x = own;
  if (kind == DG_BC_OUTFLOW) return 1;
  // slip and no-slip walls: mirror the normal velocity (no-slip enters through the viscous terms)
  real nn = 0, vn = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    nn += n[d] * n[d];
    vn += own.v[d] * n[d];
  }
  real s = real(2) * vn * RealOps<real>::rcp(nn);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    x.v[d] = own.v[d] - s * n[d];
    x.u[NSP + d] = own.rho * x.v[d];
  }
  return 0;
}

// ------------------------------------------------------------------ main RHS / RK kernel
// BND = false compiles the kernel for meshes without boundary faces (periodic or closed by
// connectivity): the interface code then carries no boundary-state branches.
template <int DIM, int N, int NSP, bool NS, int FL, bool BND = true>
// the runtime-choice kernel (FL = 0) carries more live branches: at most 5 CTAs per SM
// (up to 136 registers a thread at 96 threads) instead of 8, so that it does not spill;
// the split forms (FL >= 2) hold both nodes' conserved states per flux pair: at most 6
// (96 registers; at 7 the allocator is held to 80 and spills)
__global__ void __launch_bounds__(Layout<DIM, N, NSP, NS, FL == 1>::THREADS,
                                  (Layout<DIM, N, NSP, NS, FL == 1>::MINB > (FL == 1 ? DG_RHS_CAP1 : FL ? 6 : 5))
                                      ? (FL == 1 ? DG_RHS_CAP1 : FL ? 6 : 5)
                                      : Layout<DIM, N, NSP, NS, FL == 1>::MINB)
rhs_kernel(const DgArgs a, const KConst kc) {
  using S = Shape<DIM, N>;
  using L = Layout<DIM, N, NSP, NS, FL == 1>;
  constexpr int NV = L::NV, NP = L::NP, N1 = S::N1, EPB = L::EPB, NQ = L::NQ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* sm = reinterpret_cast<real*>(smem_raw);
  real* su = sm + L::U;
  real* sq = sm + L::Q;
  real* sja = sm + L::JA;
  real* sij = sm + L::IJ;
  real* sacc = sm + L::ACC;
  real* sfv = sm + (L::SFV ? L::FV : L::ACC);  // the sums region itself when aliased (AL)
  real* spc = sm + L::PC;
  real* sdu = sm + L::DU;
  __shared__ real s_alpha[EPB];
  __shared__ real s_dt;
  __shared__ unsigned long long s_lam[2];

  const int tid = threadIdx.x, nth = blockDim.x;
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int ne = (int)((a.K - e0) < EPB ? (a.K - e0) : EPB);
  const BasisTab<real>& B = c_tab[N];
  const bool read_du = a.mode == 1 && a.stage != 0;
  const int vf = FL == 0 ? a.vf : FL == 1 ? (NSP == 1 ? DG_VF_RANOCHA : DG_VF_DUCROS) : FL - 2;
  const int sf = FL ? DG_SF_LLF : a.sf;
  auto SW = [](int n) { return Swizzle<DIM, N>::at(n); };

  // ---- phase A: stage state, metric terms, 1/J, viscous fluxes (and du) asynchronously,
  // unswizzled: bulk copies by the TMA engine where sizes and addresses allow (one per
  // element and array, issued by the first warp), 16-byte cp.async otherwise.  The low
  // part of the compensated energy (FP32 state) goes to the accumulator region that the
  // line phase fills later: [e][node], unswizzled
  const bool have_elo = sizeof(real) == 4 && NSP == 1 && a.ulo != nullptr;
  constexpr int RS = sizeof(real);
  // (elements of fewer than 64 nodes stage faster by per-thread copies: measured on the 2D
  // N = 3 square cylinder)
  constexpr bool BULK_SHAPES = NP >= 64 && (NP * RS) % 16 == 0 && (L::SU * RS) % 16 == 0 && (L::SJA * RS) % 16 == 0 &&
                               (L::SIJ * RS) % 16 == 0 && (L::SFV * RS) % 16 == 0 && (L::SPC * RS) % 16 == 0 &&
                               (L::SDU * RS) % 16 == 0 && (L::ACC * RS) % 16 == 0 && (L::DU * RS) % 16 == 0 &&
                               (L::FV * RS) % 16 == 0 && (L::PC * RS) % 16 == 0 && (L::JA * RS) % 16 == 0 &&
                               (L::IJ * RS) % 16 == 0;
  const bool pre_du = L::PREFETCH_DU && read_du;
  const bool bulk = BULK_SHAPES && aligned16(a.u) && aligned16(a.Ja) && aligned16(a.invJ) &&
                    (!NS || aligned16(a.gradW)) && (!pre_du || aligned16(a.du)) &&
                    (!have_elo || aligned16(a.ulo)) && (NSP == 1 || aligned16(a.pc));
  __shared__ __align__(8) unsigned long long s_bar;
  if (bulk) {
    if (tid == 0) mbar_init(&s_bar);
    __syncthreads();
    if (tid < 32) {
      // total bytes first (one arrive with the expected count), then the copies
      const unsigned per_e = (unsigned)(RS * NP * (NV + DIM * DIM + 1 + (NSP > 1 ? 2 : 0) + (NS ? L::NFV : 0) +
                                                   (pre_du ? NV : 0) + (have_elo ? 1 : 0)));
      if (tid == 0) mbar_expect(&s_bar, per_e * (unsigned)ne);
      __syncwarp();
      // one copy per array when the shared-memory element stride equals the global block
      // (the CTA's elements are contiguous), one per element and array otherwise
      auto copy = [&](real* dst, int sstride, const real* src, int block, int e) {
        if (sstride == block) {
          if (e == 0) bulk_g2s(dst, src + e0 * block, (unsigned)(RS * block * ne), &s_bar);
        } else {
          bulk_g2s(dst + e * sstride, src + (e0 + e) * block, (unsigned)(RS * block), &s_bar);
        }
      };
      for (int j = tid; j < 8 * ne; j += 32) {
        const int e = j >> 3, kind = j & 7;
        if (kind == 0) copy(su, L::SU, (const real*)a.u, NV * NP, e);
        if (kind == 1) copy(sja, L::SJA, (const real*)a.Ja, DIM * DIM * NP, e);
        if (kind == 2) copy(sij, L::SIJ, (const real*)a.invJ, NP, e);
        if (kind == 3 && NSP > 1) copy(spc, L::SPC, (const real*)a.pc, 2 * NP, e);
        if (kind == 4 && NS) {
          if (L::FVD == DIM + 1) {
            copy(sfv, L::FVE, (const real*)a.gradW, L::NFV * NP, e);
          } else {
#pragma unroll
            for (int d = 0; d < DIM; ++d)
              bulk_g2s(sfv + e * L::FVE + d * L::FVD * NP,
                       (const real*)a.gradW + ((e0 + e) * L::NFV + d * (DIM + 1)) * NP, RS * (DIM + 1) * NP, &s_bar);
          }
        }
        if (kind == 5 && pre_du) copy(sdu, L::SDU, (const real*)a.du, NV * NP, e);
        if (kind == 6 && have_elo)  // rows at a source stride of NV NP: one per element
          bulk_g2s(sacc + L::elo(e), (const real*)a.ulo + (e0 + e) * NV * NP + (NSP + DIM) * NP, RS * NP, &s_bar);
      }
    }
  } else {
    stage_strided<NV, L::SU, NP>(su, (const real*)a.u + e0 * NV * NP, ne, tid, nth);
    stage_strided<DIM * DIM, L::SJA, NP>(sja, (const real*)a.Ja + e0 * DIM * DIM * NP, ne, tid, nth);
    stage_strided<1, L::SIJ, NP>(sij, (const real*)a.invJ + e0 * NP, ne, tid, nth);
    if (NSP > 1)
      stage_strided<2, (NSP > 1 ? L::SPC : 2 * NP), NP>(spc, (const real*)a.pc + e0 * 2 * NP, ne, tid, nth);
    if (NS)
#pragma unroll
      for (int d = 0; d < DIM; ++d)
        stage_block<(DIM + 1) * NP>(sfv + d * L::FVD * NP, L::FVE,
                                    (const real*)a.gradW + (e0 * L::NFV + d * (DIM + 1)) * NP, L::NFV * NP, ne, tid,
                                    nth);
    if (pre_du) stage_strided<NV, L::SDU, NP>(sdu, (const real*)a.du + e0 * NV * NP, ne, tid, nth);
    if (have_elo)
      stage_block<NP>(sacc + L::elo(0), L::elo(1) - L::elo(0), (const real*)a.ulo + e0 * NV * NP + (NSP + DIM) * NP,
                      NV * NP, ne, tid, nth);
  }
  // The line of this thread (phase B) and its neighbour traces at both end nodes (the
  // element's face nodes of faces 2d and 2d + 1): requested now, so that they arrive while
  // the element blocks are staged and the node phase runs, and consumed first thing in
  // the line phase (the registers are free again before its flux pairs).
  constexpr int NG = NS ? DIM + 1 : 1;
  int ln_e, ln_d, ln_m;
  if (L::UNI) {  // warp-uniform direction
    ln_d = tid / (EPB * S::LPD);
    ln_e = (tid / S::LPD) % EPB;
    ln_m = tid % S::LPD;
  } else {
    ln_e = tid / S::LINES;
    ln_d = (tid % S::LINES) / S::LPD;
    ln_m = tid % S::LPD;
  }
  const bool line_thread = tid < EPB * S::LINES && ln_e < ne;
  real pf_u[2][NV], pf_pc[2][2], pf_g[2][NG], pf_e[2];
  int pf_nb[2];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    pf_nb[side] = -1;
    pf_e[side] = real(0);
    if (line_thread) {
      const int nb = a.nbr[(e0 + ln_e) * 2 * DIM + 2 * ln_d + side];
      pf_nb[side] = nb;
      if (nb >= 0) {
        // the neighbour's node of this face: the other end of the same line there
        const int nnode = S::line_base(ln_d, ln_m) + (side ? 0 : N) * S::stride(ln_d);
        const real* gu = (const real*)a.u + (int64_t)nb * NV * NP + nnode;
#pragma unroll
        for (int k = 0; k < NV; ++k) pf_u[side][k] = gu[k * NP];
        if (have_elo) pf_e[side] = ((const real*)a.ulo)[(int64_t)nb * NV * NP + (NSP + DIM) * NP + nnode];
        if (NSP > 1) {
          const real* pc = (const real*)a.pc + (int64_t)nb * 2 * NP + nnode;
          pf_pc[side][0] = pc[0];
          pf_pc[side][1] = pc[NP];
        }
        if (NS) {
          // the neighbour's f^v . n: its contravariant viscous flux of direction d (the
          // partner face node sees the same face metric)
          const real* gn = (const real*)a.gradW + (int64_t)nb * L::NFV * NP + ln_d * (DIM + 1) * NP + nnode;
#pragma unroll
          for (int c = 0; c < NG; ++c) pf_g[side][c] = gn[c * NP];
        }
      }
    }
  }
  if (tid < EPB) {
    real al = 0;
    if (a.alpha_raw && tid < ne) {
      const real* ar = (const real*)a.alpha_raw;
      int64_t e = e0 + tid;
      al = ar[e];
      for (int f = 0; f < 2 * DIM; ++f) {
        int nb = a.nbr[e * 2 * DIM + f];
        if (nb >= 0) al = fmax(al, real(0.5) * ar[nb]);
      }
      if (a.alpha_used) a.alpha_used[e] = (double)al;
    }
    s_alpha[tid] = al;
  }
  if (tid == 0) {
    // the step's dt was reduced in FP64 by step_dt_kernel; the stage reads it
    if (a.mode == 1) s_dt = (real)a.scal[1];
    s_lam[0] = s_lam[1] = 0ull;
  }
  if (bulk) {
    if (!mbar_wait0(&s_bar)) latch_status(a.status, DG_ST_TIMEOUT, e0);
  } else {
    cp_async_wait_all();
  }
  __syncthreads();
  if (bulk && tid == 0) mbar_inval(&s_bar);
  // One thread per node: primitives (written swizzled), viscous fluxes, and the swizzled
  // rewrite of the metric terms, gradients -> contravariant viscous fluxes and p, c.  The
  // rewrite stays inside k-slabs of N1^2 nodes and nth is a multiple of N1^2, so one
  // barrier between the reads and the writes of a pass keeps it race-free.
  static_assert(!L::SWZ || (L::THREADS % (S::N1 * S::N1)) == 0, "swizzle slabs must not straddle passes");
  for (int i0 = 0; i0 < ne * NP; i0 += nth) {
    const int i = i0 + tid;
    const bool act = i < ne * NP;
    const int e = act ? i / NP : 0, n = i % NP, pn = SW(n);
    real jv[L::SWZ ? DIM * DIM : 1], fl[NS ? L::NFV : 1], pcv[2];
    if (act) {
      const real* uu = su + e * L::SU + n;
      real rho = 0;
#pragma unroll
      for (int k = 0; k < NSP; ++k) rho += uu[k * NP];
      real ir = RealOps<real>::rcp(rho), ke = 0;
      real* q = sq + e * L::SQ + pn;
      q[0] = rho;
      real vv[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        vv[d] = uu[(NSP + d) * NP] * ir;
        q[(1 + d) * NP] = vv[d];
        ke += uu[(NSP + d) * NP] * vv[d];
      }
      real p, pp;
      if (NSP == 1) {
        const real elo = have_elo ? sacc[L::elo(e) + n] : real(0);
        pp = kc.gm1 * (((uu[(NSP + DIM) * NP] - kc.eref) + elo) - real(0.5) * ke);
        p = pp + kc.pref;
      } else {
        pcv[0] = spc[e * L::SPC + n];
        pcv[1] = spc[e * L::SPC + NP + n];
        p = pcv[0];
        pp = p - kc.pref;
      }
      q[(1 + DIM) * NP] = pp;  // shifted pressure
      q[(2 + DIM) * NP] = rho * RealOps<real>::rcp(p);
      if (!(rho > real(0) && p > real(0) && isfinite(p)))
        latch_status(a.status, DG_ST_NONPHYS, e0 + e);
      const real* jn = sja + e * L::SJA + n;
      if (L::SWZ) {
#pragma unroll
        for (int c = 0; c < DIM * DIM; ++c) jv[c] = jn[c * NP];
      }
      if (NS) {
        // the contravariant viscous fluxes of the gradient kernel: slot (d, c) holds
        // sum_x Ja^d_x f^v_{x,c}, the flux along reference direction d (and, at a face of
        // direction d, the own f^v . n); rewritten at the swizzled position
        const real* gi = sfv + e * L::FVE + n;
#pragma unroll
        for (int c = 0; c < (NS ? L::NFV : 1); ++c) fl[c] = gi[L::fvp(c) * NP];
      }
    }
    if (L::SWZ) __syncthreads();
    if (act) {
      if (L::SWZ) {
        real* jo = sja + e * L::SJA + pn;
#pragma unroll
        for (int c = 0; c < DIM * DIM; ++c) jo[c * NP] = jv[c];
        if (NSP > 1) {
          spc[e * L::SPC + pn] = pcv[0];
          spc[e * L::SPC + NP + pn] = pcv[1];
        }
      }
      if (NS) {
        real* so = sfv + e * L::FVE + pn;
#pragma unroll
        for (int c = 0; c < (NS ? L::NFV : 1); ++c) so[L::fvp(c) * NP] = fl[c];
      }
    }
  }
  __syncthreads();

  // ---- phase B: one thread per line (THREADS >= EPB x LINES: at most one each): the volume
  // terms along the line, then the interface fluxes at its two end nodes.  The end nodes of
  // the lines of direction d are the element's face nodes of faces 2d and 2d + 1, so the
  // line thread lifts those fluxes onto its own sums in registers: no face pass, no second
  // barrier and no read-modify-write of the sums in shared memory.
  static_assert(L::THREADS >= EPB * S::LINES, "one line per thread");
  if (line_thread) {
    const int e = ln_e, d = ln_d, m = ln_m;
    {
    const int s = S::stride(d), base = S::line_base(d, m);
    const real* q = sq + e * L::SQ;
    const real* ja = sja + e * L::SJA + d * DIM * NP;  // Ja^d components at [c][node]
    const real* ue = su + e * L::SU;
    real acc[N1][NV];
#pragma unroll
    for (int i = 0; i < N1; ++i)
#pragma unroll
      for (int k = 0; k < NV; ++k) acc[i][k] = 0;
    // interface and boundary fluxes at the line's end nodes first (R5, R6: LLF / HLLC / EC,
    // the boundary states), lifted with -w_0^-1 (face 2d) and +w_N^-1 (face 2d + 1), and
    // the averaged viscous interface flux (R11) lifted as (Fv* - Fv).  One code instance
    // for both sides (a loop, not unrolled); the sums of the two end nodes take the lifted
    // terms by selects.
    const int64_t eg = e0 + e;
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
      const int f = 2 * d + side;
      const int rnode = base + (side ? N : 0) * s, node = SW(rnode);
      // the prefetched neighbour trace of this side (selects: one code instance, no
      // dynamically indexed registers)
      const int nb = side ? pf_nb[1] : pf_nb[0];
      real nbu[NV], nbpc[2], nbg[NG];
#pragma unroll
      for (int k = 0; k < NV; ++k) nbu[k] = side ? pf_u[1][k] : pf_u[0][k];
      const real nbe = side ? pf_e[1] : pf_e[0];
      if (NSP > 1) {
        nbpc[0] = side ? pf_pc[1][0] : pf_pc[0][0];
        nbpc[1] = side ? pf_pc[1][1] : pf_pc[0][1];
      }
      if (NS) {
#pragma unroll
        for (int c = 0; c < NG; ++c) nbg[c] = side ? pf_g[1][c] : pf_g[0][c];
      }
      const real iw = side ? B.iw[N] : -B.iw[0];
      NodeState<real, DIM, NSP> o;
#pragma unroll
      for (int k = 0; k < NV; ++k) o.u[k] = ue[k * NP + rnode];
      o.rho = q[node];
#pragma unroll
      for (int c = 0; c < DIM; ++c) o.v[c] = q[(1 + c) * NP + node];
      o.pp = q[(1 + DIM) * NP + node];
      o.p = o.pp + kc.pref;
      o.c = NSP == 1 ? RealOps<real>::sqrt_(kc.gamma * o.p * RealOps<real>::rcp(o.rho))
                     : spc[e * L::SPC + NP + node];
      real nface[DIM];
#pragma unroll
      for (int c = 0; c < DIM; ++c) nface[c] = ja[c * NP + node];
      NodeState<real, DIM, NSP> x;
      bool ok = true;
      real Fs[NV];
      int phys = outer_state<DIM, NSP, BND>(a, kc, nb, nbu, nbpc, nbe, o, nface, x, ok);
      if (!ok) latch_status(a.status, DG_ST_NONPHYS, nb >= 0 ? nb : eg);
      if (phys) phys_flux<real, DIM, NSP>(x, nface, Fs);
      else if (FL) llf_oriented<real, DIM, NSP>(o, x, side != 0, nface, Fs);  // the production pair: LLF
      else if (side) surface_flux<real, DIM, NSP>(sf, o, x, nface, kc.inv_gm1, kc.pref, Fs);
      else surface_flux<real, DIM, NSP>(sf, x, o, nface, kc.inv_gm1, kc.pref, Fs);
      const int bkind = (!BND || nb >= 0) ? 0 : a.bc_kind[-(nb + 1)];
      real vl[DIM + 1];
#pragma unroll
      for (int c = 0; c <= DIM; ++c) vl[c] = 0;
      const bool visc = NS && bkind != DG_BC_OUTFLOW;
      if (visc) {
        // viscous interface flux: mean of both sides' f^v . n, lifted as (Fv* - Fv).  At a
        // boundary the other side follows from the own flux (the flux is linear in the
        // interior gradient): m = sigma . n, h = q . n = Fv_E - m . v; inflow: the external
        // state's velocity and mu(T) (mean as at an interface); no-slip walls: Fv* = (m, h)
        // at zero velocity, h = 0 on an adiabatic wall (Fv* itself, not a mean)
        const bool wall = bkind == DG_BC_NOSLIP_ADIABATIC || bkind == DG_BC_ISOTHERMAL;
        const real* fvd = sfv + e * L::FVE + d * L::FVD * NP + node;
        real fx[DIM + 1];
        if (!BND || nb >= 0) {
#pragma unroll
          for (int c = 0; c <= DIM; ++c) fx[c] = nbg[c];
        } else {
          real h = fvd[DIM * NP];
#pragma unroll
          for (int c = 0; c < DIM; ++c) {
            fx[c] = fvd[c * NP];
            h -= fx[c] * o.v[c];
          }
          if (wall) {
            fx[DIM] = bkind == DG_BC_ISOTHERMAL ? h : real(0);
          } else {  // inflow
            real r = 1;
            if (!FL && kc.suth_s > real(0))
              r = sutherland_ratio(x.p * RealOps<real>::rcp(x.rho), kc.suth_s, kc.suth_c1, kc.suth_irt) *
                  RealOps<real>::rcp(sutherland_ratio(o.p * RealOps<real>::rcp(o.rho), kc.suth_s, kc.suth_c1,
                                                      kc.suth_irt));
            real w = 0;
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
              fx[c] *= r;
              w += fx[c] * x.v[c];
            }
            fx[DIM] = w + r * h;
          }
        }
#pragma unroll
        for (int c = 0; c <= DIM; ++c) vl[c] = wall ? fx[c] - fvd[c * NP] : real(0.5) * (fx[c] - fvd[c * NP]);
      }
      // the end node's sums take the lifted terms: + iw F*, then - iw (Fv* - Fv)
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        if (side) acc[N][k] += iw * Fs[k];
        else acc[0][k] += iw * Fs[k];
      }
      if (visc) {
#pragma unroll
        for (int c = 0; c <= DIM; ++c) {
          if (side) acc[N][NSP + c] -= iw * vl[c];
          else acc[0][NSP + c] -= iw * vl[c];
        }
      }
    }

    const real al = s_alpha[e];
    const real wdg = real(1) - al;
    // every two-point flux is linear in the normal: F(n_i + n_l) = 2 F((n_i + n_l) / 2)
    // exactly (a power-of-two scale), so the pair's mean normal is left unhalved and the
    // half goes into the coefficient
    const real hwdg = real(0.5) * wdg;

    // flux differencing: every symmetric pair once (split form, zero diagonal)
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      const int ri = base + i * s, ni = SW(ri);
      real vi[DIM], ui[NV];
#pragma unroll
      for (int c = 0; c < DIM; ++c) vi[c] = q[(1 + c) * NP + ni];
      if (NSP > 1 || vf != DG_VF_RANOCHA) {
#pragma unroll
        for (int k = 0; k < NV; ++k) ui[k] = ue[k * NP + ri];
      }
#pragma unroll
      for (int l = i + 1; l < N1; ++l) {
        const int rl = base + l * s, nl = SW(rl);
        real vl[DIM], ul[NV], nrm[DIM], F[NV];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          vl[c] = q[(1 + c) * NP + nl];
          nrm[c] = ja[c * NP + ni] + ja[c * NP + nl];
        }
        if (NSP > 1 || vf != DG_VF_RANOCHA) {
#pragma unroll
          for (int k = 0; k < NV; ++k) ul[k] = ue[k * NP + rl];
        }
        volume_flux<real, DIM, NSP>(vf, q[ni], vi, q[(1 + DIM) * NP + ni], q[(2 + DIM) * NP + ni], ui,
                                    q[nl], vl, q[(1 + DIM) * NP + nl], q[(2 + DIM) * NP + nl], ul,
                                    nrm, kc.inv_gm1, kc.pref, F);
        const real cil = hwdg * B.D2[i * N1 + l], cli = hwdg * B.D2[l * N1 + i];
        axpy<NV>(acc[i], cil, F);
        axpy<NV>(acc[l], cli, F);
      }
    }

    // subcell finite-volume part of blended elements
    if (al > real(0)) {
      real nh[DIM];
#pragma unroll
      for (int c = 0; c < DIM; ++c) nh[c] = ja[c * NP + SW(base)];
#pragma unroll
      for (int j = 1; j < N1; ++j) {
        // advance the subcell normal across subcell j-1: n += w_{j-1} (D Ja)_{j-1}
#pragma unroll
        for (int l = 0; l < N1; ++l) {
          const real cw = B.w[j - 1] * B.D[(j - 1) * N1 + l];
#pragma unroll
          for (int c = 0; c < DIM; ++c) nh[c] += cw * ja[c * NP + SW(base + l * s)];
        }
        NodeState<real, DIM, NSP> Lq, Rq;
        const int rl = base + (j - 1) * s, rr = base + j * s, nl = SW(rl), nr = SW(rr);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          Lq.u[k] = ue[k * NP + rl];
          Rq.u[k] = ue[k * NP + rr];
        }
        Lq.rho = q[nl];
        Rq.rho = q[nr];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          Lq.v[c] = q[(1 + c) * NP + nl];
          Rq.v[c] = q[(1 + c) * NP + nr];
        }
        Lq.pp = q[(1 + DIM) * NP + nl];
        Rq.pp = q[(1 + DIM) * NP + nr];
        Lq.p = Lq.pp + kc.pref;
        Rq.p = Rq.pp + kc.pref;
        if (NSP == 1) {
          Lq.c = RealOps<real>::sqrt_(kc.gamma * Lq.p * RealOps<real>::rcp(Lq.rho));
          Rq.c = RealOps<real>::sqrt_(kc.gamma * Rq.p * RealOps<real>::rcp(Rq.rho));
        } else {
          Lq.c = spc[e * L::SPC + NP + nl];
          Rq.c = spc[e * L::SPC + NP + nr];
        }
        real F[NV];
        surface_flux<real, DIM, NSP>(sf == DG_SF_EC ? DG_SF_LLF : sf, Lq, Rq, nh, kc.inv_gm1, kc.pref, F);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          acc[j - 1][k] += al * B.iw[j - 1] * F[k];
          acc[j][k] -= al * B.iw[j] * F[k];
        }
      }
    }

    if (NS) {
      // viscous volume term along the line: D Fv (enters the RHS with + sign), with the
      // contravariant flux of this direction read from shared memory
      const real* fvd = sfv + e * L::FVE + d * L::FVD * NP;
      real fl[N1][DIM + 1];
#pragma unroll
      for (int l = 0; l < N1; ++l)
#pragma unroll
        for (int c = 0; c <= DIM; ++c) fl[l][c] = fvd[c * NP + SW(base + l * s)];
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        real dsum[DIM + 1];
#pragma unroll
        for (int c = 0; c <= DIM; ++c) dsum[c] = 0;
#pragma unroll
        for (int l = 0; l < N1; ++l) axpy<DIM + 1>(dsum, B.D[i * N1 + l], fl[l]);
#pragma unroll
        for (int c = 0; c <= DIM; ++c) acc[i][NSP + c] -= dsum[c];
      }
    }

    real* sa = sacc + e * L::SACC + d * NV * NP;
#pragma unroll
    for (int i = 0; i < N1; ++i)
#pragma unroll
      for (int k = 0; k < NV; ++k) sa[k * NP + SW(base + i * s)] = acc[i][k];
    }
  }
  __syncthreads();

  // ---- phase C: one thread per node and pass.
  real lam_a = 0, lam_v = 0;
  constexpr int CIT = (EPB * NP + L::THREADS - 1) / L::THREADS;
  const bool comp = sizeof(real) == 4 && a.mode == 1 && a.ulo != nullptr && a.ulo_out != nullptr;
  // one node per pass (a loop, not unrolled: one code instance of the update)
#pragma unroll 1
  for (int it = 0; it < CIT; ++it) {
    const int i = tid + it * L::THREADS;
    if (i >= ne * NP) break;
    real lo_r[1][NV];
    if (comp) {
      const real* lp = (const real*)a.ulo + (e0 + i / NP) * NV * NP + i % NP;
#pragma unroll
      for (int k = 0; k < NV; ++k) lo_r[0][k] = lp[k * NP];
    }
    const int e = i / NP, node = i % NP, pn = SW(node);
    const real ij = sij[e * L::SIJ + node];
    const real* sa = sacc + e * L::SACC + pn;
    const int64_t gbase = (e0 + e) * NV * NP + node;
    if (a.mode == 0) {
      real* out = (real*)a.out;
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        real sum = 0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) sum += sa[(d * NV + k) * NP];
        real r = -ij * sum;
        if (NSP > 1 && k < NSP && a.src) r += ((const real*)a.src)[((e0 + e) * NSP + k) * NP + node];
        out[gbase + k * NP] = r;
      }
    } else {
      real* out = (real*)a.out;
      real* du = (real*)a.du;
      const real dt = s_dt;
      real un[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        real sum = 0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) sum += sa[(d * NV + k) * NP];
        real r = -ij * sum;
        if (NSP > 1 && k < NSP && a.src) r += ((const real*)a.src)[((e0 + e) * NSP + k) * NP + node];
        const real dold = !read_du ? real(0)
                          : (L::PREFETCH_DU ? sdu[e * L::SDU + k * NP + node] : du[gbase + k * NP]);
        real dn = kc.rkA * dold + dt * r;
        du[gbase + k * NP] = dn;
        const real hi = su[e * L::SU + k * NP + node];
        if (comp) {
          // compensated FP32 state: (hi, lo) += B dn by an exact TwoSum (Knuth), so the
          // rounding of every stage update is carried instead of lost
          const real inc = lo_r[0][k] + kc.rkB * dn;
          const real s2 = hi + inc;
          const real bb = s2 - hi;
          ((real*)a.ulo_out)[gbase + k * NP] = (hi - (s2 - bb)) + (inc - bb);
          un[k] = s2;
        } else {
          un[k] = hi + kc.rkB * dn;
        }
        out[gbase + k * NP] = un[k];
      }
      if (a.want_lambda && NSP == 1) {
        real rho = 0;
#pragma unroll
        for (int k = 0; k < NSP; ++k) rho += un[k];
        real ir = RealOps<real>::rcp(rho), ke = 0, v[DIM];
#pragma unroll
        for (int dd = 0; dd < DIM; ++dd) {
          v[dd] = un[NSP + dd] * ir;
          ke += un[NSP + dd] * v[dd];
        }
        real p = kc.gm1 * (un[NSP + DIM] - real(0.5) * ke);
        real c = RealOps<real>::sqrt_(kc.gamma * p * ir);
        real la = 0, lv = 0;
#pragma unroll
        for (int dd = 0; dd < DIM; ++dd) {
          real vn = 0, nn = 0;
#pragma unroll
          for (int cc = 0; cc < DIM; ++cc) {
            real jv = sja[e * L::SJA + (dd * DIM + cc) * NP + pn];
            vn += v[cc] * jv;
            nn += jv * jv;
          }
          la += fabs(vn) + c * RealOps<real>::sqrt_(nn);
          lv += nn;
        }
        la *= ij;
        lv *= ij * ij * kc.visc * ir;
        if (!FL && kc.suth_s > real(0)) lv *= sutherland_ratio(p * ir, kc.suth_s, kc.suth_c1, kc.suth_irt);
        if (!(p > real(0)) || !isfinite(la)) {
          latch_status(a.status, DG_ST_NONPHYS, e0 + e);
          la = real(0);
        }
        lam_a = fmax(lam_a, la);
        lam_v = fmax(lam_v, lv);
      }
    }
  }
  if (a.mode == 1 && a.want_lambda) {
    atomicMax(&s_lam[0], ordered_bits((double)lam_a));
    if (a.ns) atomicMax(&s_lam[1], ordered_bits((double)lam_v));
    __syncthreads();
    if (tid == 0) {
      atomicMax(&a.lam[2 * (a.lam_cur ^ 1) + 0], s_lam[0]);
      if (a.ns) atomicMax(&a.lam[2 * (a.lam_cur ^ 1) + 1], s_lam[1]);
    }
  }
}

// ------------------------------------------------------------------ time step (FP64)
// One thread: dt = cfl 2/((N+1) max lambda) (and the viscous bound) from the wave-speed
// maxima in slot `slot`, or dt_fixed; adds the previous step's dt to the elapsed time
// and clears the other slot for the coming step's reduction.
__global__ void step_dt_kernel(const DgArgs a, int slot, int advance_time) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (advance_time) a.scal[0] += a.scal[1];
  double dt = a.dt_fixed;
  if (!(dt > 0.0)) {
    const double la = __longlong_as_double((long long)a.lam[2 * slot + 0]);
    const double lv = __longlong_as_double((long long)a.lam[2 * slot + 1]);
    dt = a.cfl * 2.0 / ((a.N + 1) * la);
    if (a.ns && lv > 0.0) dt = fmin(dt, a.cfl * 4.0 / ((a.N + 1.0) * (a.N + 1.0) * lv));
  }
  a.scal[1] = dt;
  a.lam[2 * (slot ^ 1) + 0] = 0ull;
  a.lam[2 * (slot ^ 1) + 1] = 0ull;
}

// ------------------------------------------------------------------ positivity limiter
// Zhang-Shu limiter for one gas, one warp per element, applied to a stage's output state
// (u: form precision; ulo: the low part of the compensated FP32 state, or null).  With
// W_n = w_n / invJ_n and the element mean ubar (FP64 accumulation of hi + lo):
// density step rho <- rhobar + th1 (rho - rhobar), th1 = (rhobar - eps)/(rhobar - min rho);
// pressure step u <- ubar + th2 (u - ubar), th2 = min over nodes of the root t in (0, 1)
// of (E(t) - eps/(gamma-1)) rho(t) - |m(t)|^2/2 = 0.  Elements whose nodes are admissible
// are only read.  An inadmissible mean latches a non-physical status.
// FP64 passes for one element that may violate the bounds (whole warp)
template <int DIM, int N>
__device__ __forceinline__ void limit_element(const DgArgs& a, real* u, real* ulo, double eps,
                                              unsigned long long* nlim, int64_t k, int lane) {
  using S = Shape<DIM, N>;
  constexpr int NP = S::NP, N1 = S::N1, NV = DIM + 2;
  const BasisTab<real>& B = c_tab[N];
  const double g1 = a.gamma - 1.0;
  real* ue = u + k * NV * NP;
  real* le = ulo ? ulo + k * NV * NP : nullptr;
  const real* ij = (const real*)a.invJ + k * NP;
  auto val = [&](int v, int n) { return (double)ue[v * NP + n] + (le ? (double)le[v * NP + n] : 0.0); };
  auto weight = [&](int n) {
    double wq = (double)B.w[n % N1] * (double)B.w[(n / N1) % N1];
    if (DIM == 3) wq *= (double)B.w[n / (N1 * N1)];
    return wq / (double)ij[n];
  };
  auto pres = [&](const double* s) {
    double m2 = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) m2 += s[1 + d] * s[1 + d];
    return g1 * (s[1 + DIM] - 0.5 * m2 / s[0]);
  };
  // pass 1: mean, minima
  double acc[NV + 1], rmin = 1e300, pmin = 1e300;
#pragma unroll
  for (int v = 0; v <= NV; ++v) acc[v] = 0.0;
  for (int n = lane; n < NP; n += 32) {
    const double W = weight(n);
    double s[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      s[v] = val(v, n);
      acc[v] += W * s[v];
    }
    acc[NV] += W;
    rmin = fmin(rmin, s[0]);
    pmin = fmin(pmin, pres(s));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int v = 0; v <= NV; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
    rmin = fmin(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
    pmin = fmin(pmin, __shfl_xor_sync(0xffffffffu, pmin, o));
  }
  if (rmin >= eps && pmin >= eps) return;
  double ub[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) ub[v] = acc[v] / acc[NV];
  if (!(ub[0] > eps) || !(pres(ub) > eps)) {
    if (lane == 0) latch_status(a.status, DG_ST_NONPHYS, k);
    return;
  }
  auto put = [&](int v, int n, double x) {
    const real h = (real)x;
    ue[v * NP + n] = h;
    if (le) le[v * NP + n] = (real)(x - (double)h);
  };
  // pass 2: density
  if (rmin < eps) {
    const double th1 = (ub[0] - eps) / (ub[0] - rmin);
    for (int n = lane; n < NP; n += 32) put(0, n, ub[0] + th1 * (val(0, n) - ub[0]));
    __syncwarp();
  }
  // pass 3: pressure
  const double ep = eps / g1;
  double mb2 = 0.0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) mb2 += ub[1 + d] * ub[1 + d];
  const double c = (ub[1 + DIM] - ep) * ub[0] - 0.5 * mb2;
  double th2 = 1.0;
  for (int n = lane; n < NP; n += 32) {
    double s[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) s[v] = val(v, n);
    if (pres(s) >= eps) continue;
    const double dr = s[0] - ub[0], dE = s[1 + DIM] - ub[1 + DIM];
    double mdm = 0.0, dm2 = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const double dm = s[1 + d] - ub[1 + d];
      mdm += ub[1 + d] * dm;
      dm2 += dm * dm;
    }
    const double qa = dE * dr - 0.5 * dm2;
    const double qb = dE * ub[0] + (ub[1 + DIM] - ep) * dr - mdm;
    double t;
    if (fabs(qa) < 1e-14 * (fabs(qb) + fabs(c))) {
      t = -c / qb;
    } else {
      const double disc = fmax(0.0, qb * qb - 4.0 * qa * c);
      const double q = -0.5 * (qb + copysign(sqrt(disc), qb));
      const double t1 = q / qa, t2 = c / q;
      t = (t1 >= 0.0 && t1 <= 1.0) ? t1 : t2;
    }
    th2 = fmin(th2, fmin(1.0, fmax(0.0, t)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) th2 = fmin(th2, __shfl_xor_sync(0xffffffffu, th2, o));
  if (th2 < 1.0) {
    for (int n = lane; n < NP; n += 32)
#pragma unroll
      for (int v = 0; v < NV; ++v) put(v, n, ub[v] + th2 * (val(v, n) - ub[v]));
  }
  if (lane == 0 && nlim) atomicAdd(nlim, 1ull);
}

// FP64 passes for one element of a mixture (whole warp): partial densities toward their
// means by one common factor th1 until rho_s >= min(eps, mean rho_s); then every variable
// toward its mean by th2 until the internal energy reaches e(T_floor) at every node, i.e.
// g = (E - sum_s rho_s e_s(T_floor)) rho - |m|^2 / 2 >= 0, th2 the smallest root in [0, 1]
// of the quadratic g(ubar + t (u - ubar)); e_s(T_floor) per unit mass in a.pos_ef.
template <int DIM, int N, int NSP>
__device__ __forceinline__ void limit_element_mix(const DgArgs& a, real* u, real* ulo, double eps,
                                                  unsigned long long* nlim, int64_t k, int lane) {
  using S = Shape<DIM, N>;
  constexpr int NP = S::NP, N1 = S::N1, NV = NSP + DIM + 1;
  const BasisTab<real>& B = c_tab[N];
  real* ue = u + k * NV * NP;
  real* le = ulo ? ulo + k * NV * NP : nullptr;
  const real* ij = (const real*)a.invJ + k * NP;
  auto val = [&](int v, int n) { return (double)ue[v * NP + n] + (le ? (double)le[v * NP + n] : 0.0); };
  auto weight = [&](int n) {
    double wq = (double)B.w[n % N1] * (double)B.w[(n / N1) % N1];
    if (DIM == 3) wq *= (double)B.w[n / (N1 * N1)];
    return wq / (double)ij[n];
  };
  // g of a state and its two parts: E' = E - sum_s rho_s e_s(T_floor), rho
  auto gparts = [&](const double* x, double& Ep, double& r) {
    Ep = x[NSP + DIM];
    r = 0.0;
#pragma unroll
    for (int q = 0; q < NSP; ++q) {
      Ep -= x[q] * a.pos_ef[q];
      r += x[q];
    }
  };
  // pass 1: means and minima
  double acc[NV + 1], smin[NSP], gmin = 1e300;
#pragma unroll
  for (int v = 0; v <= NV; ++v) acc[v] = 0.0;
#pragma unroll
  for (int q = 0; q < NSP; ++q) smin[q] = 1e300;
  for (int n = lane; n < NP; n += 32) {
    const double W = weight(n);
    double x[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      x[v] = val(v, n);
      acc[v] += W * x[v];
    }
    acc[NV] += W;
#pragma unroll
    for (int q = 0; q < NSP; ++q) smin[q] = fmin(smin[q], x[q]);
    double Ep, r, m2 = 0.0;
    gparts(x, Ep, r);
#pragma unroll
    for (int d = 0; d < DIM; ++d) m2 += x[NSP + d] * x[NSP + d];
    gmin = fmin(gmin, r > 0.0 ? Ep * r - 0.5 * m2 : -1.0);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int v = 0; v <= NV; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
#pragma unroll
    for (int q = 0; q < NSP; ++q) smin[q] = fmin(smin[q], __shfl_xor_sync(0xffffffffu, smin[q], o));
    gmin = fmin(gmin, __shfl_xor_sync(0xffffffffu, gmin, o));
  }
  double ub[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) ub[v] = acc[v] / acc[NV];
  double th1 = 1.0;
  bool bad = false;
#pragma unroll
  for (int q = 0; q < NSP; ++q) {
    bad = bad || !(ub[q] >= 0.0);
    const double es = fmin(eps, ub[q]);
    if (smin[q] < es) th1 = fmin(th1, (ub[q] - es) / (ub[q] - smin[q]));
  }
  if (th1 >= 1.0 && gmin >= 0.0) return;
  double Ebar, rbar, mb2 = 0.0;
  gparts(ub, Ebar, rbar);
#pragma unroll
  for (int d = 0; d < DIM; ++d) mb2 += ub[NSP + d] * ub[NSP + d];
  const double c = Ebar * rbar - 0.5 * mb2;
  if (bad || !(rbar > 0.0) || !(c > 0.0)) {
    if (lane == 0) latch_status(a.status, DG_ST_NONPHYS, k);
    return;
  }
  auto put = [&](int v, int n, double x) {
    const real h = (real)x;
    ue[v * NP + n] = h;
    if (le) le[v * NP + n] = (real)(x - (double)h);
  };
  // pass 2: partial densities, one common factor
  if (th1 < 1.0) {
    for (int n = lane; n < NP; n += 32)
#pragma unroll
      for (int q = 0; q < NSP; ++q) put(q, n, ub[q] + th1 * (val(q, n) - ub[q]));
    __syncwarp();
  }
  // pass 3: temperature floor
  double th2 = 1.0;
  for (int n = lane; n < NP; n += 32) {
    double x[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = val(v, n);
    double Ep, r, m2 = 0.0, dr = 0.0, dE = x[NSP + DIM] - ub[NSP + DIM], mdm = 0.0, dm2 = 0.0;
    gparts(x, Ep, r);
#pragma unroll
    for (int q = 0; q < NSP; ++q) {
      dr += x[q] - ub[q];
      dE -= (x[q] - ub[q]) * a.pos_ef[q];
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const double dm = x[NSP + d] - ub[NSP + d];
      m2 += x[NSP + d] * x[NSP + d];
      mdm += ub[NSP + d] * dm;
      dm2 += dm * dm;
    }
    if (r > 0.0 && Ep * r - 0.5 * m2 >= 0.0) continue;
    const double qa = dE * dr - 0.5 * dm2;
    const double qb = dE * rbar + Ebar * dr - mdm;
    double t;
    if (fabs(qa) < 1e-14 * (fabs(qb) + fabs(c))) {
      t = -c / qb;
    } else {
      const double disc = fmax(0.0, qb * qb - 4.0 * qa * c);
      const double q = -0.5 * (qb + copysign(sqrt(disc), qb));
      const double t1 = q / qa, t2 = c / q;
      t = (t1 >= 0.0 && t1 <= 1.0) ? t1 : t2;
    }
    th2 = fmin(th2, fmin(1.0, fmax(0.0, t)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) th2 = fmin(th2, __shfl_xor_sync(0xffffffffu, th2, o));
  if (th2 < 1.0) {
    for (int n = lane; n < NP; n += 32)
#pragma unroll
      for (int v = 0; v < NV; ++v) put(v, n, ub[v] + th2 * (val(v, n) - ub[v]));
  }
  if (lane == 0 && nlim && (th1 < 1.0 || th2 < 1.0)) atomicAdd(nlim, 1ull);
}

// The limiter kernel: a warp screens EPW consecutive elements (about 128 nodes) in the
// form's precision with all loads in flight (margins cover the rounding of the check and
// the low part of the state), then runs the FP64 passes only for the flagged elements.
template <int DIM, int N, int NSP>
__global__ void __launch_bounds__(128) positivity_kernel(const DgArgs a, real* u, real* ulo, double eps,
                                                         unsigned long long* nlim) {
  using S = Shape<DIM, N>;
  constexpr int NP = S::NP, NV = NSP + DIM + 1;
  constexpr int EPW = NP >= 128 ? 1 : 128 / NP;
  static_assert(EPW <= 32, "flag mask");
  const int lane = threadIdx.x & 31;
  const int64_t k0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * EPW;
  if (k0 >= a.K) return;  // uniform per warp
  const int ch = (int)((a.K - k0) < EPW ? (a.K - k0) : EPW) * NP;
  const real tol = sizeof(real) == 4 ? real(1e-6) : real(1e-14);
  const real epsr = (real)eps, igm1 = (real)(1.0 / (a.gamma - 1.0));
  const real* ub = u + k0 * NV * NP;
  unsigned flag = 0;
#pragma unroll 4
  for (int n = lane; n < ch; n += 32) {
    const int el = n / NP, node = n - el * NP;
    const real* ue = ub + el * NV * NP + node;
    const real E = ue[(NSP + DIM) * NP];
    real m2 = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) m2 += ue[(NSP + d) * NP] * ue[(NSP + d) * NP];
    bool ok;
    if (NSP == 1) {
      // with r > 0: p >= eps + margin  <=>  r (E - (eps + margin)/(gamma-1)) >= |m|^2 / 2
      const real r = ue[0];
      const real pbound = (epsr + tol * fabs(E)) * igm1;
      ok = r >= epsr * (real(1) + tol) && r * (E - pbound) >= real(0.5) * m2;
    } else {
      // every partial density above the floor; E - sum rho_s e_s(T_floor), less a margin,
      // times rho above |m|^2 / 2
      real r = 0, Ep = E, mag = fabs(E);
      ok = true;
#pragma unroll
      for (int q = 0; q < NSP; ++q) {
        const real rq = ue[q * NP];
        ok = ok && rq >= epsr * (real(1) + tol);
        r += rq;
        const real t = rq * (real)a.pos_ef[q];
        Ep -= t;
        mag += fabs(t);
      }
      ok = ok && r * (Ep - tol * mag) >= real(0.5) * m2;
    }
    if (!ok) flag |= 1u << el;
  }
  flag = __reduce_or_sync(0xffffffffu, flag);
  while (flag) {
    const int el = __ffs(flag) - 1;
    flag &= flag - 1;
    if (NSP == 1) limit_element<DIM, N>(a, u, ulo, eps, nlim, k0 + el, lane);
    else limit_element_mix<DIM, N, NSP>(a, u, ulo, eps, nlim, k0 + el, lane);
  }
}

// ------------------------------------------------------------------ BR1 gradients
template <int DIM, int N, int NSP>
struct GLayout {
  using S = Shape<DIM, N>;
  static constexpr int NV = NSP + DIM + 1;
  static constexpr int NP = S::NP;
  static constexpr int EPB = epb<DIM, N>();
  static constexpr int NW = DIM + 1;
  // swizzled W and G blocks, direction-uniform line warps and (FP32) element strides of
  // 16 words mod 32, as in the right-hand-side kernel
  static constexpr bool SWZ = Swizzle<DIM, N>::ON;
  static constexpr bool UNI = SWZ && (EPB * S::LPD) % 32 == 0;
  static constexpr int padded(int w) { return (SWZ && sizeof(real) == 4) ? w + (48 - w % 32) % 32 : w; }
  static constexpr int SW = padded(NW * NP), SG = padded(DIM * NW * NP);
  static constexpr int W = 0;
  static constexpr int JA = W + EPB * SW;
  static constexpr int IJ = JA + EPB * DIM * DIM * NP;
  static constexpr int G = IJ + EPB * NP;
  static constexpr int TOTAL = G + EPB * SG;
  static constexpr int THREADS = ((EPB * S::LINES + 31) / 32) * 32;
  // resident CTAs the register allocator is asked for: what shared memory allows, <= 8
  static constexpr int BY_SMEM = (int)((227 * 1024) / (sizeof(real) * TOTAL + 1024));
  static constexpr int MINB = BY_SMEM >= 8 ? 8 : (BY_SMEM < 1 ? 1 : BY_SMEM);
};

template <int DIM, int N, int NSP>
__global__ void __launch_bounds__(GLayout<DIM, N, NSP>::THREADS, GLayout<DIM, N, NSP>::MINB)
gradient_kernel(const DgArgs a, const KConst kc) {
  using S = Shape<DIM, N>;
  using L = GLayout<DIM, N, NSP>;
  constexpr int NV = L::NV, NP = L::NP, N1 = S::N1, NW = L::NW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* sm = reinterpret_cast<real*>(smem_raw);
  real* sw = sm + L::W;
  real* sja = sm + L::JA;
  real* sij = sm + L::IJ;
  real* sg = sm + L::G;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int64_t e0 = (int64_t)blockIdx.x * L::EPB;
  const int ne = (int)((a.K - e0) < L::EPB ? (a.K - e0) : L::EPB);
  const BasisTab<real>& B = c_tab[N];
  const real* gu = (const real*)a.u;
  // the conserved state is staged in the gradient region, which is free until the line phase
  static_assert(L::TOTAL - L::G >= L::EPB * NV * NP, "gradient region too small for the state");
  // contiguous blocks of the CTA's elements: three TMA bulk copies where sizes and
  // addresses allow, 16-byte cp.async otherwise
  constexpr int RS = sizeof(real);
  constexpr bool BULK_SHAPES = (NP * RS) % 16 == 0 && (L::JA * RS) % 16 == 0 && (L::IJ * RS) % 16 == 0 &&
                               (L::G * RS) % 16 == 0;
  const bool bulk = BULK_SHAPES && aligned16(a.Ja) && aligned16(a.invJ) && aligned16(gu);
  __shared__ __align__(8) unsigned long long s_bar;
  if (bulk) {
    if (tid == 0) {
      mbar_init(&s_bar);
      mbar_expect(&s_bar, (unsigned)(RS * NP * ne * (DIM * DIM + 1 + NV)));
      bulk_g2s(sja, (const real*)a.Ja + e0 * DIM * DIM * NP, RS * ne * DIM * DIM * NP, &s_bar);
      bulk_g2s(sij, (const real*)a.invJ + e0 * NP, RS * ne * NP, &s_bar);
      bulk_g2s(sg, gu + e0 * NV * NP, RS * ne * NV * NP, &s_bar);
    }
    __syncthreads();  // the barrier is initialised before anyone polls it
    if (!mbar_wait0(&s_bar)) latch_status(a.status, DG_ST_TIMEOUT, e0);
  } else {
    stage_async(sja, (const real*)a.Ja + e0 * DIM * DIM * NP, ne * DIM * DIM * NP, tid, nth);
    stage_async(sij, (const real*)a.invJ + e0 * NP, ne * NP, tid, nth);
    stage_async(sg, gu + e0 * NV * NP, ne * NV * NP, tid, nth);
    cp_async_wait_all();
  }
  __syncthreads();
  if (bulk && tid == 0) mbar_inval(&s_bar);
  auto SWZ = [](int n) { return Swizzle<DIM, N>::at(n); };
  for (int i = tid; i < ne * NP; i += nth) {
    const int e = i / NP, node = i % NP, pn = SWZ(node);
    const real* uu = sg + e * NV * NP + node;
    real rho = 0;
#pragma unroll
    for (int k = 0; k < NSP; ++k) rho += uu[k * NP];
    real ir = RealOps<real>::rcp(rho), ke = 0;
    real vv[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      vv[d] = uu[(NSP + d) * NP] * ir;
      ke += uu[(NSP + d) * NP] * vv[d];
    }
    real p = kc.gm1 * (uu[(NSP + DIM) * NP] - real(0.5) * ke);
#pragma unroll
    for (int d = 0; d < DIM; ++d) sw[e * L::SW + d * NP + pn] = vv[d];
    sw[e * L::SW + DIM * NP + pn] = p * ir;
  }
  __syncthreads();
  for (int t = tid; t < L::EPB * S::LINES; t += nth) {
    int e, d, m;
    if (L::UNI) {  // warp-uniform direction
      d = t / (L::EPB * S::LPD);
      e = (t / S::LPD) % L::EPB;
      m = t % S::LPD;
    } else {
      e = t / S::LINES;
      d = (t % S::LINES) / S::LPD;
      m = t % S::LPD;
    }
    if (e >= ne) continue;
    const int s = S::stride(d), base = S::line_base(d, m);
    const int64_t eg = e0 + e;
    const real* w = sw + e * L::SW;
    real Wl[N1][NW];
#pragma unroll
    for (int i = 0; i < N1; ++i)
#pragma unroll
      for (int c = 0; c < NW; ++c) Wl[i][c] = w[c * NP + SWZ(base + i * s)];
    real G[N1][NW];
#pragma unroll
    for (int i = 0; i < N1; ++i)
#pragma unroll
      for (int c = 0; c < NW; ++c) {
        real acc = 0;
#pragma unroll
        for (int l = 0; l < N1; ++l) acc += B.D[i * N1 + l] * Wl[l][c];
        G[i][c] = acc;
      }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int f = 2 * d + side;
      const int nnode = base + (side ? 0 : N) * s;
      const int nb = a.nbr[eg * 2 * DIM + f];
      const int i = side ? N : 0;
      // boundary faces get their lifting from boundary_lift_kernel: here a valid address
      // (the own element) and a zero weight, without a branch
      const real* un = gu + (int64_t)(nb >= 0 ? nb : eg) * NV * NP + nnode;
      const real keep = nb >= 0 ? real(1) : real(0);
      real rn = 0;
#pragma unroll
      for (int k = 0; k < NSP; ++k) rn += un[k * NP];
      real irn = RealOps<real>::rcp(rn), ke = 0, Wn[NW];
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        Wn[c] = un[(NSP + c) * NP] * irn;
        ke += un[(NSP + c) * NP] * Wn[c];
      }
      Wn[DIM] = kc.gm1 * (un[(NSP + DIM) * NP] - real(0.5) * ke) * irn;
#pragma unroll
      for (int c = 0; c < NW; ++c) {
        real ws = real(0.5) * (Wl[i][c] + Wn[c]);
        if (side) G[N][c] += keep * B.iw[N] * (ws - Wl[N][c]);
        else G[0][c] -= keep * B.iw[0] * (ws - Wl[0][c]);
      }
    }
    real* g = sg + e * L::SG + d * NW * NP;
#pragma unroll
    for (int i = 0; i < N1; ++i)
#pragma unroll
      for (int c = 0; c < NW; ++c) g[c * NP + SWZ(base + i * s)] = G[i][c];
  }
  __syncthreads();
  // physical gradients G_x = (1/J) sum_d Ja^d_x Q_d; written as they are (grad_mode 1) or
  // turned into the contravariant viscous fluxes sum_x Ja^d_x f^v_x(G; v, mu(T)) that the
  // right-hand-side kernel consumes (grad_mode 0)
  real* out = (real*)a.gradW;
  for (int i = tid; i < ne * NP; i += nth) {
    const int e = i / NP, node = i % NP, pn = SWZ(node);
    const real ij = sij[e * NP + node];
    const real* jn = sja + e * DIM * DIM * NP + node;
    real G[DIM][NW];
#pragma unroll
    for (int x = 0; x < DIM; ++x)
#pragma unroll
      for (int c = 0; c < NW; ++c) {
        real acc = 0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) acc += jn[(d * DIM + x) * NP] * sg[e * L::SG + (d * NW + c) * NP + pn];
        G[x][c] = acc * ij;
      }
    real* o = out + (e0 + e) * DIM * NW * NP + node;
    if (a.grad_mode) {
#pragma unroll
      for (int x = 0; x < DIM; ++x)
#pragma unroll
        for (int c = 0; c < NW; ++c) o[(x * NW + c) * NP] = G[x][c];
      continue;
    }
    real vv[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) vv[c] = sw[e * L::SW + c * NP + pn];
    real mu_n = kc.mu, kap_n = kc.kap;
    if (kc.suth_s > real(0)) {
      const real r = sutherland_ratio(sw[e * L::SW + DIM * NP + pn], kc.suth_s, kc.suth_c1, kc.suth_irt);
      mu_n *= r;
      kap_n *= r;
    }
    real fv[DIM][DIM + 1];
    viscous_flux<real, DIM>(G, vv, mu_n, kap_n, fv);
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int c = 0; c < NW; ++c) {
        real acc = 0;
#pragma unroll
        for (int x = 0; x < DIM; ++x) acc += jn[(d * DIM + x) * NP] * fv[x][c];
        o[(d * NW + c) * NP] = acc;
      }
  }
}

// BR1 lifting at boundary faces (Eq. auxstrongf with the boundary value W* in place of
// the interface mean): adds dG = (1/J) sum_d Ja^d (+-1/w) (W* - W) to the gradient of every
// boundary face node (grad_mode 1), or f^v(dG) in contravariant form to its viscous fluxes
// (grad_mode 0: the flux is linear in the gradient); one thread per node, so that a node on several boundary faces (an
// edge or corner) sums its faces in one place.  Launched after gradient_kernel only for
// meshes with boundary faces.  W*: inflow (W + W_ext)/2, outflow W, no-slip walls
// (0, theta) or (0, theta_wall).
template <int DIM, int N, int NSP>
__global__ void boundary_lift_kernel(const DgArgs a, const KConst kc) {
  using S = Shape<DIM, N>;
  constexpr int NV = NSP + DIM + 1, NP = S::NP, N1 = S::N1, NW = DIM + 1;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.K * NP) return;
  const int64_t e = i / NP;
  const int node = (int)(i % NP);
  const int* nbr = a.nbr + e * 2 * DIM;
  bool any = false;
#pragma unroll
  for (int f = 0; f < 2 * DIM; ++f) {
    const int pos = (node / S::stride(f >> 1)) % N1;
    any |= nbr[f] < 0 && pos == ((f & 1) ? N : 0);
  }
  if (!any) return;
  const BasisTab<real>& B = c_tab[N];
  auto W_of = [&](const real* u, int64_t st, real* W) {
    real rho = 0;
#pragma unroll
    for (int k = 0; k < NSP; ++k) rho += u[k * st];
    const real ir = RealOps<real>::rcp(rho);
    real ke = 0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      W[c] = u[(NSP + c) * st] * ir;
      ke += u[(NSP + c) * st] * W[c];
    }
    W[DIM] = kc.gm1 * (u[(NSP + DIM) * st] - real(0.5) * ke) * ir;
  };
  real W[NW];
  W_of((const real*)a.u + e * NV * NP + node, NP, W);
  real dQ[DIM][NW];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
#pragma unroll
    for (int c = 0; c < NW; ++c) dQ[d][c] = real(0);
    const int pos = (node / S::stride(d)) % N1;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int nb = nbr[2 * d + side];
      if (nb >= 0 || pos != (side ? N : 0)) continue;
      const int bc = -(nb + 1), kind = a.bc_kind[bc];
      real We[NW], Ws[NW];
      W_of((const real*)a.bc_u + (int64_t)bc * NV, 1, We);
#pragma unroll
      for (int c = 0; c < NW; ++c) {
        if (kind == DG_BC_INFLOW) Ws[c] = real(0.5) * (W[c] + We[c]);
        else if (kind == DG_BC_NOSLIP_ADIABATIC) Ws[c] = c < DIM ? real(0) : W[c];
        else if (kind == DG_BC_ISOTHERMAL) Ws[c] = c < DIM ? real(0) : We[c];
        else Ws[c] = W[c];
        dQ[d][c] += side ? B.iw[N] * (Ws[c] - W[c]) : -B.iw[0] * (Ws[c] - W[c]);
      }
    }
  }
  const real ij = ((const real*)a.invJ)[e * NP + node];
  const real* ja = (const real*)a.Ja + e * DIM * DIM * NP + node;
  real* g = (real*)a.gradW + e * DIM * NW * NP + node;
  real dG[DIM][NW];
#pragma unroll
  for (int x = 0; x < DIM; ++x)
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      real acc = 0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) acc += ja[(d * DIM + x) * NP] * dQ[d][c];
      dG[x][c] = acc * ij;
    }
  if (a.grad_mode) {
#pragma unroll
    for (int x = 0; x < DIM; ++x)
#pragma unroll
      for (int c = 0; c < NW; ++c) g[(x * NW + c) * NP] += dG[x][c];
    return;
  }
  // the viscous flux is linear in the gradient: add f^v(dG; v, mu(T)) in contravariant form
  real mu_n = kc.mu, kap_n = kc.kap;
  if (kc.suth_s > real(0)) {
    const real r = sutherland_ratio(W[DIM], kc.suth_s, kc.suth_c1, kc.suth_irt);
    mu_n *= r;
    kap_n *= r;
  }
  real fv[DIM][DIM + 1];
  viscous_flux<real, DIM>(dG, W, mu_n, kap_n, fv);
#pragma unroll
  for (int d = 0; d < DIM; ++d)
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      real acc = 0;
#pragma unroll
      for (int x = 0; x < DIM; ++x) acc += ja[(d * DIM + x) * NP] * fv[x][c];
      g[(d * NW + c) * NP] += acc;
    }
}

// ------------------------------------------------------------------ wave speeds (dt)
template <int DIM, int NSP>
__global__ void lambda_kernel(const DgArgs a, const KConst kc, int slot) {
  __shared__ unsigned long long s_l[2];
  constexpr int NV = NSP + DIM + 1;
  const int np = a.np;
  const int64_t n = a.K * np;
  if (threadIdx.x == 0) s_l[0] = s_l[1] = 0ull;
  __syncthreads();
  real la_m = 0, lv_m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / np;
    const int node = (int)(i % np);
    const real* uu = (const real*)a.u + e * NV * np + node;
    real rho = 0;
    for (int k = 0; k < NSP; ++k) rho += uu[k * np];
    real ir = RealOps<real>::rcp(rho), ke = 0, v[DIM];
    for (int d = 0; d < DIM; ++d) {
      v[d] = uu[(NSP + d) * np] * ir;
      ke += uu[(NSP + d) * np] * v[d];
    }
    real c, p = 0;
    if (NSP == 1) {
      p = kc.gm1 * (uu[(NSP + DIM) * np] - real(0.5) * ke);
      c = RealOps<real>::sqrt_(kc.gamma * p * ir);
    } else {
      c = ((const real*)a.pc)[(e * 2 + 1) * np + node];
    }
    const real ij = ((const real*)a.invJ)[e * np + node];
    real la = 0, lv = 0;
    for (int d = 0; d < DIM; ++d) {
      real vn = 0, nn = 0;
      for (int x = 0; x < DIM; ++x) {
        real jv = ((const real*)a.Ja)[((e * DIM + d) * DIM + x) * np + node];
        vn += v[x] * jv;
        nn += jv * jv;
      }
      la += fabs(vn) + c * RealOps<real>::sqrt_(nn);
      lv += nn;
    }
    la *= ij;
    lv *= ij * ij * kc.visc * ir;
    if (NSP == 1 && kc.suth_s > real(0)) lv *= sutherland_ratio(p * ir, kc.suth_s, kc.suth_c1, kc.suth_irt);
    if (!isfinite(la)) la = real(0);
    la_m = fmax(la_m, la);
    lv_m = fmax(lv_m, lv);
  }
  atomicMax(&s_l[0], ordered_bits((double)la_m));
  atomicMax(&s_l[1], ordered_bits((double)lv_m));
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicMax(&a.lam[2 * slot + 0], s_l[0]);
    if (a.ns) atomicMax(&a.lam[2 * slot + 1], s_l[1]);
  }
}

// ------------------------------------------------------------------ shock indicator
// Hennemann-Gassner modal energy of rho*p (or of p).  The indicator quantity of every node
// is formed during coalesced loads into shared memory; the tensor-product transform to
// orthonormal Legendre modes runs line by line in place, and the energies of all modes, of
// the modes up to degree N-1 and of the two highest degrees are summed directly (no
// cancellation).  Small elements (NP <= 64): one thread per element on a padded row of the
// CTA's block; larger ones: one warp per element (lines across lanes, warp reduction).
template <int DIM, int N>
struct IndShape {
  static constexpr int NP = Shape<DIM, N>::NP;
  static constexpr bool WARP = NP > 64;
  static constexpr int EPC = WARP ? 4 : (sizeof(real) == 8 ? 64 : 128);  // elements per CTA
  static constexpr int THREADS = WARP ? EPC * 32 : EPC;
  static constexpr int ROW = WARP ? NP : NP + 1;  // padded rows: conflict-free per-thread access
};

template <int DIM, int N>
__device__ __forceinline__ real indicator_alpha(real Et, real E1, real Eh1, real Eh2, real alpha_max) {
  const BasisTab<real>& B = c_tab[N];
  const real fr1 = Et > real(0) ? Eh1 / Et : real(0);
  const real fr2 = E1 > real(0) ? Eh2 / E1 : real(0);
  const real E = fmax(fr1, fr2);
  const real thr = B.thr;
  const real sp = real(9.21024036697585);  // ln((1 - 1e-4) / 1e-4)
  real al = real(1) / (real(1) + exp(-(sp / thr) * (E - thr)));
  if (al < real(1e-3)) al = real(0);
  if (al > alpha_max) al = alpha_max;
  return al;
}

template <int DIM, int N, int NSP>
__global__ void __launch_bounds__(IndShape<DIM, N>::THREADS) indicator_kernel(const DgArgs a, const KConst kc,
                                                                              real alpha_max, real* alpha_raw) {
  using S = Shape<DIM, N>;
  using I = IndShape<DIM, N>;
  constexpr int NP = S::NP, N1 = S::N1, NV = NSP + DIM + 1, ROW = I::ROW;
  __shared__ real sf[I::EPC * ROW];
  const BasisTab<real>& B = c_tab[N];
  const int tid = threadIdx.x;
  const int64_t e0 = (int64_t)blockIdx.x * I::EPC;
  const int ne = (int)((a.K - e0) < I::EPC ? (a.K - e0) : I::EPC);
  const real* ub = (const real*)a.u + e0 * NV * NP;
  // indicator quantity of every node of the CTA's elements (coalesced: nodes of a variable
  // block are contiguous)
  for (int i = tid; i < ne * NP; i += I::THREADS) {
    const int el = i / NP, node = i - el * NP;
    const real* uu = ub + el * NV * NP + node;
    real rho = 0;
#pragma unroll
    for (int k = 0; k < NSP; ++k) rho += uu[k * NP];
    real p;
    if (NSP == 1) {
      real ke = 0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) ke += uu[(NSP + d) * NP] * uu[(NSP + d) * NP];
      p = kc.gm1 * (uu[(NSP + DIM) * NP] - real(0.5) * ke * RealOps<real>::rcp(rho));
    } else {
      p = ((const real*)a.pc)[((e0 + el) * 2) * NP + node];
    }
    sf[el * ROW + node] = a.ind_var ? p : rho * p;
  }
  __syncthreads();
  // worker: a thread (small elements) or a warp (large ones) per element
  const int lane = I::WARP ? (tid & 31) : 0, step = I::WARP ? 32 : 1;
  const int el = I::WARP ? (tid >> 5) : tid;
  if (el >= ne) return;
  real* f = sf + el * ROW;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int s = S::stride(d);
#pragma unroll 1
    for (int m = lane; m < S::LPD; m += step) {
      const int base = S::line_base(d, m);
      real x[N1];
#pragma unroll
      for (int l = 0; l < N1; ++l) x[l] = f[base + l * s];
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        real acc = 0;
#pragma unroll
        for (int l = 0; l < N1; ++l) acc += B.Vinv[i * N1 + l] * x[l];
        f[base + i * s] = acc;
      }
    }
    if (I::WARP) __syncwarp();
  }
  real Et = 0, E1 = 0, Eh1 = 0, Eh2 = 0;
#pragma unroll 4
  for (int node = lane; node < NP; node += step) {
    int mx = node % N1;
    if (DIM >= 2) mx = max(mx, (node / N1) % N1);
    if (DIM == 3) mx = max(mx, node / (N1 * N1));
    const real e2 = f[node] * f[node];
    Et += e2;
    if (mx <= N - 1) E1 += e2;
    if (mx == N) Eh1 += e2;
    if (mx == N - 1) Eh2 += e2;
  }
  if (I::WARP) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      Et += __shfl_xor_sync(0xffffffffu, Et, o);
      E1 += __shfl_xor_sync(0xffffffffu, E1, o);
      Eh1 += __shfl_xor_sync(0xffffffffu, Eh1, o);
      Eh2 += __shfl_xor_sync(0xffffffffu, Eh2, o);
    }
    if (lane != 0) return;
  }
  alpha_raw[e0 + el] = indicator_alpha<DIM, N>(Et, E1, Eh1, Eh2, alpha_max);
}

// opt in to more than the default 48 KB (dynamic + static) of shared memory
template <typename KernelT>
cudaError_t set_smem(KernelT k, size_t bytes) {
  if (bytes + 1024 <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int DIM, int N, int NSP, bool NS, int FL, bool BND>
cudaError_t launch_rhs_b(const DgArgs& a, cudaStream_t st) {
  using L = Layout<DIM, N, NSP, NS, FL == 1>;
  auto k = rhs_kernel<DIM, N, NSP, NS, FL, BND>;
  cudaError_t err = set_smem(k, L::SMEM);
  if (err != cudaSuccess) return err;
  const int64_t grid = (a.K + L::EPB - 1) / L::EPB;
  k<<<(unsigned)grid, L::THREADS, L::SMEM, st>>>(a, make_kconst(a));
  return cudaGetLastError();
}

// the production pair of a one-gas 3D mesh without boundary faces runs the kernel
// compiled without boundary code (measured 5-7 % faster on the periodic Taylor-Green box)
template <int DIM, int N, int NSP, bool NS, int FL = DG_FL>
cudaError_t launch_rhs_t(const DgArgs& a, cudaStream_t st) {
  if constexpr (FL == 1 && DIM == 3 && NSP == 1) {
    if (!a.has_bnd) return launch_rhs_b<DIM, N, NSP, NS, FL, false>(a, st);
  }
  return launch_rhs_b<DIM, N, NSP, NS, FL, true>(a, st);
}

#ifndef DG_GENERIC_ONLY
template <int DIM, int N, int NSP>
cudaError_t launch_grad_t(const DgArgs& a, cudaStream_t st) {
  using L = GLayout<DIM, N, NSP>;
  const size_t smem = sizeof(real) * L::TOTAL;
  auto k = gradient_kernel<DIM, N, NSP>;
  cudaError_t err = set_smem(k, smem);
  if (err != cudaSuccess) return err;
  const int64_t grid = (a.K + L::EPB - 1) / L::EPB;
  k<<<(unsigned)grid, L::THREADS, smem, st>>>(a, make_kconst(a));
  err = cudaGetLastError();
  if (err != cudaSuccess || !a.has_bnd) return err;
  const int64_t nn = a.K * Shape<DIM, N>::NP;
  boundary_lift_kernel<DIM, N, NSP><<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(a, make_kconst(a));
  return cudaGetLastError();
}

template <int DIM, int N, int NSP>
cudaError_t launch_pos_t(const DgArgs& a, void* u, void* ulo, double eps, unsigned long long* nlim,
                         cudaStream_t st) {
  constexpr int NP = Shape<DIM, N>::NP, EPW = NP >= 128 ? 1 : 128 / NP;
  const int64_t warps = (a.K + EPW - 1) / EPW;
  const int64_t grid = (warps * 32 + 127) / 128;
  positivity_kernel<DIM, N, NSP><<<(unsigned)grid, 128, 0, st>>>(a, (real*)u, (real*)ulo, eps, nlim);
  return cudaGetLastError();
}

template <int DIM, int N, int NSP>
cudaError_t launch_ind_t(const DgArgs& a, double amax, void* out, cudaStream_t st) {
  using I = IndShape<DIM, N>;
  const int64_t grid = (a.K + I::EPC - 1) / I::EPC;
  indicator_kernel<DIM, N, NSP><<<(unsigned)grid, I::THREADS, 0, st>>>(a, make_kconst(a), (real)amax, (real*)out);
  return cudaGetLastError();
}
#endif  // DG_GENERIC_ONLY

}  // namespace DG_PREFIX

#define DG_CAT2(a, b) a##b
#define DG_CAT(a, b) DG_CAT2(a, b)

// dispatch on (dim, N, nsp, ns)
#define DG_DISPATCH_N(MACRO, DIM, NSP, ...)             \
  switch (a.N) {                                        \
    case 2: return MACRO(DIM, 2, NSP, __VA_ARGS__);     \
    case 3: return MACRO(DIM, 3, NSP, __VA_ARGS__);     \
    case 4: return MACRO(DIM, 4, NSP, __VA_ARGS__);     \
    case 7: return MACRO(DIM, 7, NSP, __VA_ARGS__);     \
    default: return cudaErrorInvalidValue;              \
  }
#define DG_DISPATCH_N_MIX(MACRO, DIM, NSP, ...)         \
  switch (a.N) {                                        \
    case 3: return MACRO(DIM, 3, NSP, __VA_ARGS__);     \
    case 4: return MACRO(DIM, 4, NSP, __VA_ARGS__);     \
    default: return cudaErrorInvalidValue;              \
  }

#define DG_RHS_CALL(DIM, N, NSP, NS) DG_PREFIX::launch_rhs_t<DIM, N, NSP, NS>(a, st)
#define DG_GRAD_CALL(DIM, N, NSP, X) DG_PREFIX::launch_grad_t<DIM, N, NSP>(a, st)
#define DG_IND_CALL(DIM, N, NSP, X) DG_PREFIX::launch_ind_t<DIM, N, NSP>(a, amax, out, st)
#define DG_POS_CALL(DIM, N, NSP, X) DG_PREFIX::launch_pos_t<DIM, N, NSP>(a, u, ulo, eps, nlim, st)

#ifdef DG_SPLIT_ONLY
// the compile-time split forms: one-gas 3D at N = 3, LLF, constant viscosity
#define DG_SPLIT_CALL(VF)                                                                        \
  return a.ns ? DG_PREFIX::launch_rhs_t<3, 3, 1, true, 2 + (VF)>(a, st)                          \
              : DG_PREFIX::launch_rhs_t<3, 3, 1, false, 2 + (VF)>(a, st)
cudaError_t DG_CAT(DG_PREFIX, _rhs)(const DgArgs& a, cudaStream_t st) {
  if (!(a.dim == 3 && a.nsp == 1 && a.N == 3 && a.sf == DG_SF_LLF && !(a.suth_s > 0.0)))
    return cudaErrorInvalidValue;
  switch (a.vf) {
    case DG_VF_DUCROS: DG_SPLIT_CALL(DG_VF_DUCROS);
    case DG_VF_CENTRAL: DG_SPLIT_CALL(DG_VF_CENTRAL);
    case DG_VF_KG: DG_SPLIT_CALL(DG_VF_KG);
    case DG_VF_PIROZZOLI: DG_SPLIT_CALL(DG_VF_PIROZZOLI);
    case DG_VF_MORINISHI: DG_SPLIT_CALL(DG_VF_MORINISHI);
    default: return cudaErrorInvalidValue;
  }
}
#else
cudaError_t DG_CAT(DG_PREFIX, _rhs)(const DgArgs& a, cudaStream_t st) {
#ifndef DG_GENERIC_ONLY
  const bool production = a.sf == DG_SF_LLF && a.vf == (a.nsp == 1 ? DG_VF_RANOCHA : DG_VF_DUCROS) &&
                          !(a.suth_s > 0.0);
#ifdef DG_SPLIT_RHS
  const bool split = a.dim == 3 && a.nsp == 1 && a.N == 3 && a.sf == DG_SF_LLF && !(a.suth_s > 0.0) &&
                     a.vf != DG_VF_RANOCHA;
  if (split) return DG_SPLIT_RHS(a, st);
#endif
  if (!production) return DG_GENERIC_RHS(a, st);
#endif
  if (a.dim == 3 && a.nsp == 1 && a.ns) { DG_DISPATCH_N(DG_RHS_CALL, 3, 1, true) }
  if (a.dim == 3 && a.nsp == 1) { DG_DISPATCH_N(DG_RHS_CALL, 3, 1, false) }
  if (a.dim == 2 && a.nsp == 1) { DG_DISPATCH_N(DG_RHS_CALL, 2, 1, false) }
  if (a.dim == 3 && a.nsp == 5) { DG_DISPATCH_N_MIX(DG_RHS_CALL, 3, 5, false) }
  return cudaErrorInvalidValue;
}
#endif  // DG_SPLIT_ONLY

#ifndef DG_GENERIC_ONLY
cudaError_t DG_CAT(DG_PREFIX, _gradients)(const DgArgs& a, cudaStream_t st) {
  if (a.dim == 3 && a.nsp == 1) { DG_DISPATCH_N(DG_GRAD_CALL, 3, 1, 0) }
  return cudaErrorInvalidValue;
}

cudaError_t DG_CAT(DG_PREFIX, _indicator)(const DgArgs& a, double amax, void* out, cudaStream_t st) {
  if (a.dim == 2 && a.nsp == 1) { DG_DISPATCH_N(DG_IND_CALL, 2, 1, 0) }
  if (a.dim == 3 && a.nsp == 1) { DG_DISPATCH_N(DG_IND_CALL, 3, 1, 0) }
  if (a.dim == 3 && a.nsp == 5) { DG_DISPATCH_N_MIX(DG_IND_CALL, 3, 5, 0) }
  return cudaErrorInvalidValue;
}

cudaError_t DG_CAT(DG_PREFIX, _positivity)(const DgArgs& a, void* u, void* ulo, double eps,
                                          unsigned long long* nlim, cudaStream_t st) {
  if (a.dim == 3 && a.nsp == 1) { DG_DISPATCH_N(DG_POS_CALL, 3, 1, 0) }
  if (a.dim == 2 && a.nsp == 1) { DG_DISPATCH_N(DG_POS_CALL, 2, 1, 0) }
  if (a.dim == 3 && a.nsp == 5) { DG_DISPATCH_N_MIX(DG_POS_CALL, 3, 5, 0) }
  return cudaErrorInvalidValue;
}

cudaError_t DG_CAT(DG_PREFIX, _lambda)(const DgArgs& a, int slot, cudaStream_t st) {
  const int bs = 256;
  int64_t n = a.K * a.np;
  int64_t grid = (n + bs - 1) / bs;
  if (grid > 152 * 16) grid = 152 * 16;
  const DG_PREFIX::KConst kc = DG_PREFIX::make_kconst(a);
  if (a.dim == 3 && a.nsp == 1) DG_PREFIX::lambda_kernel<3, 1><<<(unsigned)grid, bs, 0, st>>>(a, kc, slot);
  else if (a.dim == 2 && a.nsp == 1) DG_PREFIX::lambda_kernel<2, 1><<<(unsigned)grid, bs, 0, st>>>(a, kc, slot);
  else if (a.dim == 3 && a.nsp == 5) DG_PREFIX::lambda_kernel<3, 5><<<(unsigned)grid, bs, 0, st>>>(a, kc, slot);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t DG_CAT(DG_PREFIX, _step_dt)(const DgArgs& a, int slot, int advance_time, cudaStream_t st) {
  DG_PREFIX::step_dt_kernel<<<1, 32, 0, st>>>(a, slot, advance_time);
  return cudaGetLastError();
}

#endif  // DG_GENERIC_ONLY

cudaError_t DG_CAT(DG_PREFIX, _upload_basis)() {
  using DG_PREFIX::real;
  dgk::BasisTab<real> tab[DG_MAXN + 1];
  memset(tab, 0, sizeof(tab));
  for (int N = 1; N <= DG_MAXN; ++N) {
    DgHostBasis b;
    if (dg_host_basis(N, &b)) return cudaErrorInvalidValue;
    const int n1 = N + 1;
    for (int i = 0; i < n1; ++i) {
      tab[N].w[i] = (real)b.w[i];
      tab[N].iw[i] = (real)(1.0 / b.w[i]);
      for (int j = 0; j < n1; ++j) {
        tab[N].D[i * n1 + j] = (real)b.D[i * n1 + j];
        tab[N].D2[i * n1 + j] = i == j ? (real)0 : (real)(2.0 * b.D[i * n1 + j]);
        tab[N].Vinv[i * n1 + j] = (real)b.Vinv[i * n1 + j];
      }
    }
    tab[N].thr = (real)(0.5 * pow(10.0, -1.8 * pow(N + 1.0, 0.25)));
  }
  cudaError_t err = cudaMemcpyToSymbol(DG_PREFIX::c_tab, tab, sizeof(tab));
#ifndef DG_GENERIC_ONLY
  if (err == cudaSuccess) err = DG_GENERIC_UPLOAD();
#ifdef DG_SPLIT_UPLOAD
  if (err == cudaSuccess) err = DG_SPLIT_UPLOAD();
#endif
#endif
  return err;
}
