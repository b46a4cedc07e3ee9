// Right-hand-side kernels of the entropy-stable DGSEM (H3PC, arXiv 2511.17551),
// templated on precision, dimension, degree and number of species.  Included by
// one translation unit per precision (dg_rhs_f64.cu, dg_rhs_f32.cu).
//
// Design (one CTA = EPB elements, all of its data staged in shared memory):
//   phase A  coalesced (16-byte) copy of the elements' conserved state, metric
//            terms and 1/J into shared memory; per-node primitives (rho, v, p,
//            rho/p) computed once; for Navier-Stokes, the viscous fluxes f^v_x.
//   phase B1 one thread per grid line (direction d, line m): every symmetric pair
//            (i < l) of the line is evaluated ONCE with the two-point flux and
//            added to both end points with 2 D_il and 2 D_li in registers (split
//            form with zero diagonal, Eqs. fluxdiff / fluxdiffcons, so no self-flux
//            is ever formed), plus the subcell FV fluxes of blended elements
//            (Eq. fluxes_discrete_with_fv) and the BR1 viscous volume term (Eq.
//            auxstrongf); each line stores its N+1 node sums once.
//   phase B2 one thread per face node: interface flux from the neighbour's trace
//            (Eqs. riemann_problem1-3) or the boundary state, lifted onto the face
//            node, plus the averaged viscous interface flux.
//   phase C  one thread per node: sum the DIM line contributions in a fixed
//            order, scale by -1/J, and either store du/dt or apply the
//            2N-storage Runge-Kutta update (and the wave-speed maximum of the
//            new state for the next step's dt).
// No atomics touch floating-point sums: results are deterministic.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include "dg_internal.h"
#include "../../include/dg.h"

namespace dgk {

template <typename real>
struct BasisTab {
  real D[(DG_MAXN + 1) * (DG_MAXN + 1)];
  real D2[(DG_MAXN + 1) * (DG_MAXN + 1)];  // 2 D with zero diagonal
  real w[DG_MAXN + 1];
  real iw[DG_MAXN + 1];
  real Vinv[(DG_MAXN + 1) * (DG_MAXN + 1)];
  real thr;                                 // indicator threshold 0.5 10^(-1.8 (N+1)^(1/4))
};

template <typename real> struct RealOps;
template <> struct RealOps<double> {
  static __device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double log_(double x) { return log(x); }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static constexpr double ln_eps = 1e-4;
};
template <> struct RealOps<float> {
  // single MUFU reciprocal / reciprocal square root (<= 2 ulp): the mixed form's
  // error budget (1e-5) is far above FP32 rounding
  static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
  static __device__ __forceinline__ float sqrt_(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
  static __device__ __forceinline__ float log_(float x) { return logf(x); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
  // the artanh series truncated after f^6 has relative error f^8/9: 1.1e-9 at 1e-2
  static constexpr float ln_eps = 1e-2f;
};

// logarithmic mean L(x,y) = (y-x)/ln(y/x): artanh series for nearly equal
// arguments, closed form otherwise
template <typename real>
__device__ __forceinline__ real ln_mean(real x, real y) {
  real s = x + y, d = y - x;
  real rs = RealOps<real>::rcp(s);
  real f = d * rs, f2 = f * f;
  if (f2 < RealOps<real>::ln_eps) {
    if (sizeof(real) == 8) {
      // L = (s/2) / (1 + x), x = f2 (1/3 + f2 (1/5 + f2/7)) <= 3.4e-5: the geometric series
      // to x^3 is exact to FP64 rounding (x^4 < 2e-18) and needs no second reciprocal
      const real x = f2 * (real(1.0 / 3.0) + f2 * (real(1.0 / 5.0) + f2 * real(1.0 / 7.0)));
      return real(0.5) * s * (real(1) - x * (real(1) - x * (real(1) - x)));
    }
    real poly = real(2) + f2 * (real(2.0 / 3.0) + f2 * (real(2.0 / 5.0) + f2 * real(2.0 / 7.0)));
    return s * RealOps<real>::rcp(poly);
  }
  return RealOps<real>::div(d, RealOps<real>::log_(RealOps<real>::div(y, x)));
}

// 1 / L(x,y)
template <typename real>
__device__ __forceinline__ real inv_ln_mean(real x, real y) {
  real s = x + y, d = y - x;
  real rs = RealOps<real>::rcp(s);
  real f = d * rs, f2 = f * f;
  if (f2 < RealOps<real>::ln_eps) {
    real poly = real(2) + f2 * (real(2.0 / 3.0) + f2 * (real(2.0 / 5.0) + f2 * real(2.0 / 7.0)));
    return poly * rs;
  }
  return RealOps<real>::div(RealOps<real>::log_(RealOps<real>::div(y, x)), d);
}

// Single precision: L(xr, yr) and 1 / L(xb, yb) together, the two near-equal series in
// the lanes of the packed FP32 operations of sm_100 (same roundings as ln_mean and
// inv_ln_mean); the closed forms one at a time when either pair is not near-equal.
__device__ __forceinline__ void ln_mean_pair(float xr, float yr, float xb, float yb, float& Lr, float& iLb) {
  const float2 x = make_float2(xr, xb), y = make_float2(yr, yb);
  const float2 s = __fadd2_rn(x, y);
  const float2 d = __ffma2_rn(x, make_float2(-1.f, -1.f), y);  // y - x
  const float2 rs = make_float2(RealOps<float>::rcp(s.x), RealOps<float>::rcp(s.y));
  const float2 f = __fmul2_rn(d, rs);
  const float2 f2 = __fmul2_rn(f, f);
  if (f2.x < RealOps<float>::ln_eps && f2.y < RealOps<float>::ln_eps) {
    float2 poly = __ffma2_rn(f2, make_float2(2.f / 7.f, 2.f / 7.f), make_float2(2.f / 5.f, 2.f / 5.f));
    poly = __ffma2_rn(f2, poly, make_float2(2.f / 3.f, 2.f / 3.f));
    poly = __ffma2_rn(f2, poly, make_float2(2.f, 2.f));
    Lr = s.x * RealOps<float>::rcp(poly.x);
    iLb = poly.y * rs.y;
    return;
  }
  Lr = ln_mean(xr, yr);
  iLb = inv_ln_mean(xb, yb);
}

__device__ __forceinline__ void latch_status(unsigned long long* st, unsigned long long code,
                                             int64_t elem) {
  unsigned long long v = (code << 56) | (unsigned long long)(elem & 0x00ffffffffffffffll);
  atomicCAS(st, 0ull, v);
}

__device__ __forceinline__ unsigned long long ordered_bits(double x) {
  return (unsigned long long)__double_as_longlong(x);  // x >= 0: order preserved
}

template <int DIM, int N>
struct Shape {
  static constexpr int N1 = N + 1;
  static constexpr int NP = DIM == 3 ? N1 * N1 * N1 : N1 * N1;
  static constexpr int LPD = DIM == 3 ? N1 * N1 : N1;  // lines per direction
  static constexpr int LINES = DIM * LPD;
  static __device__ __forceinline__ int stride(int d) { return d == 0 ? 1 : (d == 1 ? N1 : N1 * N1); }
  static __device__ __forceinline__ int line_base(int d, int m) {
    if (DIM == 2) return d == 0 ? m * N1 : m;
    if (d == 0) return m * N1;
    if (d == 1) return (m % N1) + (m / N1) * N1 * N1;
    return m;
  }
};

// ---------------------------------------------------------------- pointwise physics
// Node state in registers (one gas: NSP = 1).  p is the pressure, pp = p - p_ref the
// shifted pressure that the momentum components of every flux use: a constant pressure
// contributes nothing to the discrete right-hand side (free-stream preservation), so the
// shift is exact in arithmetic and keeps low-Mach pressure fluctuations in FP32.
template <typename real, int DIM, int NSP>
struct NodeState {
  static constexpr int NV = NSP + DIM + 1;
  real u[NV];
  real rho, v[DIM], p, c, pp;
};

// pref, eref = pref / (gamma - 1): pressure offset; elo: low part of the compensated
// energy (0 when the state is not compensated).  pp = (gamma - 1)((E - eref) + elo - ke/2),
// E - eref exact near the reference (Sterbenz).
template <typename real, int DIM, int NSP>
__device__ __forceinline__ bool prim_from_cons(NodeState<real, DIM, NSP>& s, real gamma,
                                               real p_ext, real c_ext, real pref = real(0),
                                               real eref = real(0), real elo = real(0)) {
  real rho = 0;
#pragma unroll
  for (int k = 0; k < NSP; ++k) rho += s.u[k];
  s.rho = rho;
  real ir = RealOps<real>::rcp(rho);
  real ke = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    s.v[d] = s.u[NSP + d] * ir;
    ke += s.u[NSP + d] * s.v[d];
  }
  if (NSP == 1) {
    s.pp = (gamma - real(1)) * (((s.u[NSP + DIM] - eref) + elo) - real(0.5) * ke);
    s.p = s.pp + pref;
    s.c = RealOps<real>::sqrt_(gamma * s.p * ir);
  } else {
    s.p = p_ext;
    s.pp = p_ext - pref;
    s.c = c_ext;
  }
  return rho > real(0) && s.p > real(0) && isfinite(s.p);
}

template <typename real, int DIM, int NSP>
__device__ __forceinline__ void phys_flux(const NodeState<real, DIM, NSP>& s, const real* n,
                                          real* f) {
  real vn = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) vn += s.v[d] * n[d];
#pragma unroll
  for (int k = 0; k < NSP; ++k) f[k] = s.u[k] * vn;
#pragma unroll
  for (int d = 0; d < DIM; ++d) f[NSP + d] = s.u[NSP + d] * vn + s.pp * n[d];
  f[NSP + DIM] = (s.u[NSP + DIM] + s.p) * vn;
}

// interface flux in the +n orientation between left state L and right state R
template <typename real, int DIM, int NSP>
__device__ __forceinline__ void surface_flux(int sf, const NodeState<real, DIM, NSP>& L,
                                             const NodeState<real, DIM, NSP>& R, const real* n,
                                             real inv_gm1, real pref, real* f);

// two-point volume flux F#(L, R; n); pL, pR are shifted pressures p - pref (momentum
// components), bL, bR = rho / p of the full pressures
template <typename real, int DIM, int NSP>
__device__ __forceinline__ void volume_flux(int vf, real rL, const real* vL, real pL, real bL,
                                            const real* uL, real rR, const real* vR, real pR,
                                            real bR, const real* uR, const real* n,
                                            real inv_gm1, real pref, real* f) {
  constexpr int NV = NSP + DIM + 1;
  real vnL = 0, vnR = 0;
  if constexpr (sizeof(real) == 4) {
    float2 vn = make_float2(0.f, 0.f);
#pragma unroll
    for (int d = 0; d < DIM; ++d) vn = __ffma2_rn(make_float2(vL[d], vR[d]), make_float2(n[d], n[d]), vn);
    vnL = vn.x;
    vnR = vn.y;
  } else {
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      vnL += vL[d] * n[d];
      vnR += vR[d] * n[d];
    }
  }
  if (NSP == 1 && vf == DG_VF_RANOCHA) {
    real rho_m, ib;  // L(rho), 1 / L(rho/p)
    if constexpr (sizeof(real) == 4) {
      ln_mean_pair(rL, rR, bL, bR, rho_m, ib);
    } else {
      rho_m = ln_mean(rL, rR);
      ib = inv_ln_mean(bL, bR);
    }
    real vv = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) vv += vL[d] * vR[d];
    real frho = rho_m * real(0.5) * (vnL + vnR);
    real pa = real(0.5) * (pL + pR);
    f[0] = frho;
#pragma unroll
    for (int d = 0; d < DIM; ++d) f[1 + d] = frho * real(0.5) * (vL[d] + vR[d]) + pa * n[d];
    f[1 + DIM] = frho * (real(0.5) * vv + ib * inv_gm1) + real(0.5) * ((pL + pref) * vnR + (pR + pref) * vnL);
  } else if (NSP == 1 && (vf == DG_VF_KG || vf == DG_VF_PIROZZOLI)) {
    // Kennedy-Gruber / Pirozzoli split forms as products of arithmetic means
    const real frho = real(0.25) * (rL + rR) * (vnL + vnR);
    const real irL = RealOps<real>::rcp(rL), irR = RealOps<real>::rcp(rR);
    f[0] = frho;
#pragma unroll
    for (int d = 0; d < DIM; ++d) f[1 + d] = frho * real(0.5) * (vL[d] + vR[d]) + real(0.5) * (pL + pR) * n[d];
    if (vf == DG_VF_KG)
      f[1 + DIM] = frho * real(0.5) * (uL[1 + DIM] * irL + uR[1 + DIM] * irR) +
                   real(0.25) * ((pL + pref) + (pR + pref)) * (vnL + vnR);
    else
      f[1 + DIM] = frho * real(0.5) * ((uL[1 + DIM] + (pL + pref)) * irL + (uR[1 + DIM] + (pR + pref)) * irR);
  } else if (NSP == 1 && vf == DG_VF_MORINISHI) {
    // Morinishi: mass and enthalpy in divergence form, skew-symmetric momentum, kinetic
    // energy f_rho v_L.v_R / 2
    real frho = 0, vv = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      frho += (uL[1 + d] + uR[1 + d]) * n[d];
      vv += vL[d] * vR[d];
    }
    frho *= real(0.5);
    f[0] = frho;
#pragma unroll
    for (int d = 0; d < DIM; ++d) f[1 + d] = frho * real(0.5) * (vL[d] + vR[d]) + real(0.5) * (pL + pR) * n[d];
    f[1 + DIM] = (real(1) + inv_gm1) * real(0.5) * ((pL + pref) * vnL + (pR + pref) * vnR) + frho * real(0.5) * vv;
  } else if (vf == DG_VF_DUCROS) {
    real vn = real(0.5) * (vnL + vnR);
    real pa = real(0.5) * (pL + pR);
#pragma unroll
    for (int k = 0; k < NSP; ++k) f[k] = real(0.5) * (uL[k] + uR[k]) * vn;
#pragma unroll
    for (int d = 0; d < DIM; ++d) f[NSP + d] = real(0.5) * (uL[NSP + d] + uR[NSP + d]) * vn + pa * n[d];
    f[NSP + DIM] = real(0.5) * (uL[NSP + DIM] + (pL + pref) + uR[NSP + DIM] + (pR + pref)) * vn;
  } else {  // central
#pragma unroll
    for (int k = 0; k < NSP; ++k) f[k] = real(0.5) * (uL[k] * vnL + uR[k] * vnR);
#pragma unroll
    for (int d = 0; d < DIM; ++d)
      f[NSP + d] = real(0.5) * (uL[NSP + d] * vnL + pL * n[d] + uR[NSP + d] * vnR + pR * n[d]);
    f[NSP + DIM] = real(0.5) * ((uL[NSP + DIM] + (pL + pref)) * vnL + (uR[NSP + DIM] + (pR + pref)) * vnR);
  }
  (void)NV;
}

// LLF flux between the own state o and the other side's state x for either orientation
// with one code instance: F(L, R) with (L, R) = (o, x) when own_left, (x, o) otherwise;
// bit for bit the same as surface_flux(DG_SF_LLF, L, R, ...) (the mean and the maximum
// are symmetric, the jump only changes sign)
template <typename real, int DIM, int NSP>
__device__ __forceinline__ void llf_oriented(const NodeState<real, DIM, NSP>& o, const NodeState<real, DIM, NSP>& x,
                                             bool own_left, const real* n, real* f) {
  constexpr int NV = NSP + DIM + 1;
  real nn = 0, vno = 0, vnx = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    nn += n[d] * n[d];
    vno += o.v[d] * n[d];
    vnx += x.v[d] * n[d];
  }
  nn = RealOps<real>::sqrt_(nn);
  real fo[NV], fx[NV];
  phys_flux<real, DIM, NSP>(o, n, fo);
  phys_flux<real, DIM, NSP>(x, n, fx);
  const real lam = fmax(fabs(vno) + o.c * nn, fabs(vnx) + x.c * nn);
  const real hl = own_left ? real(0.5) * lam : real(-0.5) * lam;
#pragma unroll
  for (int k = 0; k < NV; ++k) f[k] = real(0.5) * (fo[k] + fx[k]) - hl * (x.u[k] - o.u[k]);
}

template <typename real, int DIM, int NSP>
__device__ __forceinline__ void surface_flux(int sf, const NodeState<real, DIM, NSP>& L,
                                             const NodeState<real, DIM, NSP>& R, const real* n,
                                             real inv_gm1, real pref, real* f) {
  constexpr int NV = NSP + DIM + 1;
  if (sf == DG_SF_EC) {
    real bL = L.rho * RealOps<real>::rcp(L.p), bR = R.rho * RealOps<real>::rcp(R.p);
    volume_flux<real, DIM, NSP>(NSP == 1 ? DG_VF_RANOCHA : DG_VF_DUCROS, L.rho, L.v, L.pp, bL, L.u,
                                R.rho, R.v, R.pp, bR, R.u, n, inv_gm1, pref, f);
    return;
  }
  real nn = 0, vnL = 0, vnR = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    nn += n[d] * n[d];
    vnL += L.v[d] * n[d];
    vnR += R.v[d] * n[d];
  }
  nn = RealOps<real>::sqrt_(nn);
  real fL[NV], fR[NV];
  phys_flux<real, DIM, NSP>(L, n, fL);
  phys_flux<real, DIM, NSP>(R, n, fR);
  if (sf == DG_SF_LLF) {
    real lam = fmax(fabs(vnL) + L.c * nn, fabs(vnR) + R.c * nn);
#pragma unroll
    for (int k = 0; k < NV; ++k) f[k] = real(0.5) * (fL[k] + fR[k]) - real(0.5) * lam * (R.u[k] - L.u[k]);
    return;
  }
  // HLLC along n/|n| with Davis speed estimates, scaled by |n|
  real inn = RealOps<real>::rcp(nn);
  real uLn = vnL * inn, uRn = vnR * inn;
  real SL = fmin(uLn - L.c, uRn - R.c);
  real SR = fmax(uLn + L.c, uRn + R.c);
  if (SL >= real(0)) {
#pragma unroll
    for (int k = 0; k < NV; ++k) f[k] = fL[k];
    return;
  }
  if (SR <= real(0)) {
#pragma unroll
    for (int k = 0; k < NV; ++k) f[k] = fR[k];
    return;
  }
  if (sf == DG_SF_HLL) {
    // HLL with the same Davis speeds (one intermediate state), scaled by |n|
    const real iden = RealOps<real>::rcp(SR - SL);
#pragma unroll
    for (int k = 0; k < NV; ++k) f[k] = (SR * fL[k] - SL * fR[k] + nn * SL * SR * (R.u[k] - L.u[k])) * iden;
    return;
  }
  real Ss = RealOps<real>::div(R.p - L.p + L.rho * uLn * (SL - uLn) - R.rho * uRn * (SR - uRn),
                               L.rho * (SL - uLn) - R.rho * (SR - uRn));
  const bool left = Ss >= real(0);
  const NodeState<real, DIM, NSP>& K = left ? L : R;
  const real* fK = left ? fL : fR;
  real SK = left ? SL : SR, unK = left ? uLn : uRn;
  real fac = RealOps<real>::div(SK - unK, SK - Ss);
  real us[NV];
#pragma unroll
  for (int k = 0; k < NSP; ++k) us[k] = K.u[k] * fac;
#pragma unroll
  for (int d = 0; d < DIM; ++d) us[NSP + d] = K.rho * fac * (K.v[d] + (Ss - unK) * n[d] * inn);
  us[NSP + DIM] = K.rho * fac *
                  (RealOps<real>::div(K.u[NSP + DIM], K.rho) +
                   (Ss - unK) * (Ss + RealOps<real>::div(K.p, K.rho * (SK - unK))));
#pragma unroll
  for (int k = 0; k < NV; ++k) f[k] = fK[k] + nn * SK * (us[k] - K.u[k]);
}

// physical viscous flux f^v_x (x = physical direction) for one gas; c = 0..DIM-1
// momentum, c = DIM energy (the density component is zero).  g[x][a] = d(W_a)/dx_x with
// W = (v_1..v_DIM, theta = p / rho).
// a[k] += c x[k] for k < M: two at a time with the packed FP32 FMA of sm_100 (__ffma2_rn,
// per component the same rounding as fmaf) in single precision, one at a time otherwise
template <int M, typename real>
__device__ __forceinline__ void axpy(real* a, real c, const real* x) {
  if constexpr (sizeof(real) == 4) {
    const float2 cc = make_float2(c, c);
#pragma unroll
    for (int k = 0; k + 1 < M; k += 2) {
      const float2 r = __ffma2_rn(cc, make_float2(x[k], x[k + 1]), make_float2(a[k], a[k + 1]));
      a[k] = r.x;
      a[k + 1] = r.y;
    }
    if (M % 2) a[M - 1] = fmaf(c, x[M - 1], a[M - 1]);
  } else {
#pragma unroll
    for (int k = 0; k < M; ++k) a[k] = fma(c, x[k], a[k]);
  }
}

// mu(T) / mu by Sutherland's law (Eq. sutherland): c1 th^1.5 / (th + s) with
// th = (p / rho) / rt_ref, c1 = 1 + s, irt = 1 / rt_ref
template <typename real>
__device__ __forceinline__ real sutherland_ratio(real p_over_rho, real s, real c1, real irt) {
  const real th = p_over_rho * irt;
  return c1 * th * RealOps<real>::sqrt_(th) * RealOps<real>::rcp(th + s);
}

template <typename real, int DIM>
__device__ __forceinline__ void viscous_flux(const real (*g)[DIM + 1], const real* v, real mu,
                                             real kap, real (*fv)[DIM + 1]) {
  real div = 0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) div += g[a][a];
#pragma unroll
  for (int x = 0; x < DIM; ++x) {
    real work = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      real sig = mu * (g[x][a] + g[a][x]);
      if (a == x) sig -= real(2.0 / 3.0) * mu * div;
      fv[x][a] = sig;
      work += v[a] * sig;
    }
    fv[x][DIM] = work + kap * g[x][DIM];
  }
}

}  // namespace dgk
