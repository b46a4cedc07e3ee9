"""Plain FP64 CPU oracle of the entropy-stable DGSEM (arXiv 2511.17551).

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the GPU library and its
Python binding never do.  It compiles the C sources in this directory with gcc
(``build()``) and exposes them through ctypes with numpy marshalling.
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")
_SRCS = ["or_basis.c", "or_geometry.c", "or_physics.c", "or_rhs.c", "or_thermo_chem.c",
         "or_mlp.c"]

EULER, NAVIER_STOKES = 0, 1
VF_RANOCHA, VF_DUCROS, VF_CENTRAL, VF_KG, VF_PIROZZOLI, VF_MORINISHI = 0, 1, 2, 3, 4, 5
SF_LLF, SF_HLLC, SF_EC, SF_HLL = 0, 1, 2, 3
BC_INFLOW, BC_OUTFLOW, BC_SLIP_WALL = 1, 2, 3


def build(force=False):
    """Compile liboracle.so (gcc, -O2, OpenMP over elements)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS if os.path.exists(os.path.join(_HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "oracle.h")])
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


class Problem(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("N", C.c_int), ("K", C.c_int64),
        ("n_species", C.c_int), ("equations", C.c_int),
        ("volume_flux", C.c_int), ("surface_flux", C.c_int),
        ("gamma", C.c_double), ("mu", C.c_double), ("Pr", C.c_double),
        ("alpha_max", C.c_double),
        ("nbr_elem", C.c_void_p), ("nbr_face", C.c_void_p),
        ("n_bc", C.c_int), ("bc_kind", C.c_void_p), ("bc_prim", C.c_void_p),
        ("species", C.c_void_p), ("Ja", C.c_void_p), ("J", C.c_void_p),
        ("alpha_override", C.c_double),
        ("n_reactions", C.c_int), ("reactions", C.c_void_p), ("chem_dt", C.c_double),
        ("positivity_eps", C.c_double),
        ("sutherland_s", C.c_double), ("sutherland_rt", C.c_double), ("indicator_var", C.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        d, i, vp = C.c_double, C.c_int, C.c_void_p
        sig = {
            "or_lgl": (i, [i, vp, vp]),
            "or_dmat": (None, [i, vp, vp]),
            "or_vandermonde_legendre": (None, [i, vp, vp]),
            "or_geometry": (i, [i, i, C.c_int64, vp, vp, vp]),
            "or_rhs": (i, [vp, vp, vp, vp, vp]),
            "or_indicator": (i, [vp, vp, vp]),
            "or_max_dt": (d, [vp, vp, d]),
            "or_step_rk": (i, [vp, vp, i, d, d, vp]),
            "or_diagnostics": (i, [vp, vp, vp]),
            "or_prim_to_cons_field": (i, [vp, vp, vp]),
            "or_ck45": (None, [vp, vp, vp]),
            "or_ln_mean": (d, [d, d]),
            "or_nv": (i, [i, i]),
            "or_flux_pair": (i, [vp, vp, vp, vp, i, vp]),
            "or_entropy_vars_u": (i, [vp, vp, vp]),
            "or_mixture_eval": (i, [i, vp, i, vp, vp, vp, vp]),
            "or_temperature_field": (i, [vp, vp, vp]),
            "or_mlp_nparams": (i, []),
            "or_mlp_nparams_n": (i, [i]),
            "or_mlp_forward_n": (i, [vp, i, i, vp, vp]),
            "or_mlp_forward_sd_n": (i, [vp, i, i, vp, d, d, d, d, vp, vp, vp]),
            "or_mlp_loss_grad_n": (d, [vp, i, i, vp, vp, vp]),
            "or_chem_eval": (i, [vp, i, vp, i, vp, vp, d, vp, vp, vp]),
            "or_gelu": (d, [d]),
            "or_gelu_d": (d, [d]),
            "or_mlp_forward": (None, [vp, i, vp, vp]),
            "or_mlp_loss_grad": (d, [vp, i, vp, vp, vp]),
            "or_adam_step": (None, [vp, vp, vp, vp, i, i, d, d, d, d]),
            "or_mixture_temperature": (i, [i, vp, i, vp, vp, vp, vp, vp]),
            "or_positivity": (i, [vp, vp, d, vp]),
            "or_set_threads": (i, [i]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


def set_threads(n):
    """OpenMP threads of the oracle's element loops (n <= 0: query); returns the count."""
    return lib().or_set_threads(int(n))


def lgl(N):
    x = np.zeros(N + 1)
    w = np.zeros(N + 1)
    if lib().or_lgl(N, _p(x), _p(w)):
        raise ValueError("bad N")
    return x, w


def dmat(N):
    x, _ = lgl(N)
    D = np.zeros((N + 1, N + 1))
    lib().or_dmat(N, _p(x), _p(D))
    return D


def vandermonde(N):
    x, _ = lgl(N)
    V = np.zeros((N + 1, N + 1))
    lib().or_vandermonde_legendre(N, _p(x), _p(V))
    return V


def geometry(dim, N, xyz):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    K = xyz.shape[0]
    np_ = (N + 1) ** dim
    Ja = np.zeros((K, dim, dim, np_))
    J = np.zeros((K, np_))
    rc = lib().or_geometry(dim, N, K, _p(xyz), _p(Ja), _p(J))
    if rc:
        raise ValueError("or_geometry failed (%d)" % rc)
    return Ja, J


class Oracle:
    """Holds one problem (mesh + physics) and its metric terms."""

    def __init__(self, dim, N, xyz, nbr_elem, nbr_face, *, n_species=0, equations=EULER,
                 volume_flux=VF_RANOCHA, surface_flux=SF_LLF, gamma=1.4, mu=0.0, Pr=0.72,
                 alpha_max=0.0, bc_kind=None, bc_prim=None, species=None,
                 alpha_override=-1.0, reactions=None, chem_dt=0.0, positivity_eps=0.0,
                 sutherland_s=0.0, sutherland_rt=1.0, indicator_variable=0):
        self.dim, self.N = dim, N
        self.np = (N + 1) ** dim
        self.nv = lib().or_nv(dim, n_species)
        self.Ja, self.J = geometry(dim, N, xyz)
        self.K = self.J.shape[0]
        self.nbr_elem = np.ascontiguousarray(nbr_elem, dtype=np.int64)
        self.nbr_face = np.ascontiguousarray(nbr_face, dtype=np.int8)
        self.bc_kind = np.ascontiguousarray(bc_kind if bc_kind is not None else [0],
                                            dtype=np.int32)
        self.bc_prim = np.ascontiguousarray(
            bc_prim if bc_prim is not None else np.zeros((1, self.nv)), dtype=np.float64)
        self.species = (np.ascontiguousarray(species, dtype=np.float64)
                        if species is not None else None)
        self.reactions = (np.ascontiguousarray(reactions, dtype=np.float64)
                          if reactions is not None else None)
        self.P = Problem(dim=dim, N=N, K=self.K, n_species=n_species, equations=equations,
                         volume_flux=volume_flux, surface_flux=surface_flux, gamma=gamma,
                         mu=mu, Pr=Pr, alpha_max=alpha_max,
                         nbr_elem=_p(self.nbr_elem), nbr_face=_p(self.nbr_face),
                         n_bc=len(self.bc_kind) if bc_kind is not None else 0,
                         bc_kind=_p(self.bc_kind), bc_prim=_p(self.bc_prim),
                         species=_p(self.species), Ja=_p(self.Ja), J=_p(self.J),
                         alpha_override=alpha_override,
                         n_reactions=0 if reactions is None else len(self.reactions),
                         reactions=_p(self.reactions), chem_dt=chem_dt,
                         positivity_eps=positivity_eps, sutherland_s=sutherland_s,
                         sutherland_rt=sutherland_rt, indicator_var=indicator_variable)

    def _ref(self):
        return C.byref(self.P)

    def _field(self, u, copy=False):
        """u as a C-contiguous float64 [K][nv][np] array (shape checked: the C side trusts it)."""
        u = np.array(u, dtype=np.float64, copy=True, order="C") if copy else \
            np.ascontiguousarray(u, dtype=np.float64)
        if u.shape != (self.K, self.nv, self.np):
            raise ValueError("state shape %s, expected %s" % (u.shape, (self.K, self.nv, self.np)))
        return u

    def prim_to_cons(self, w):
        w = self._field(w)
        u = np.zeros_like(w)
        if lib().or_prim_to_cons_field(self._ref(), _p(w), _p(u)):
            raise ValueError("non-physical primitive state")
        return u

    def rhs(self, u, want_alpha=False, want_grad=False):
        u = self._field(u)
        r = np.zeros_like(u)
        a = np.zeros(self.K) if want_alpha else None
        g = (np.zeros((self.K, self.dim, self.dim + 1, self.np)) if want_grad else None)
        rc = lib().or_rhs(self._ref(), _p(u), _p(r), _p(a), _p(g))
        if rc:
            raise ValueError("or_rhs failed (%d)" % rc)
        out = [r]
        if want_alpha:
            out.append(a)
        if want_grad:
            out.append(g)
        return out[0] if len(out) == 1 else tuple(out)

    def indicator(self, u):
        u = self._field(u)
        a = np.zeros(self.K)
        lib().or_indicator(self._ref(), _p(u), _p(a))
        return a

    def max_dt(self, u, cfl):
        u = self._field(u)
        return lib().or_max_dt(self._ref(), _p(u), cfl)

    def step_rk(self, u, nsteps, cfl=0.5, dt_fixed=0.0, t=0.0):
        u = self._field(u, copy=True)
        tt = C.c_double(t)
        rc = lib().or_step_rk(self._ref(), _p(u), nsteps, cfl, dt_fixed, C.byref(tt))
        if rc:
            raise ValueError("or_step_rk failed (%d)" % rc)
        return u, tt.value

    def flux_pair(self, uL, uR, n, which):
        """which = 0 volume flux, 1 surface flux, 2 physical flux of uL."""
        uL = np.ascontiguousarray(uL, dtype=np.float64)
        uR = np.ascontiguousarray(uR, dtype=np.float64)
        n3 = np.zeros(3)
        n3[:len(n)] = n
        f = np.zeros(self.nv)
        if lib().or_flux_pair(self._ref(), _p(uL), _p(uR), _p(n3), which, _p(f)):
            raise ValueError("non-physical state")
        return f

    def entropy_vars(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        w = np.zeros(self.nv)
        if lib().or_entropy_vars_u(self._ref(), _p(u), _p(w)):
            raise ValueError("non-physical state")
        return w

    def temperature(self, u):
        u = self._field(u)
        T = np.zeros((self.K, self.np))
        if lib().or_temperature_field(self._ref(), _p(u), _p(T)):
            raise ValueError("temperature solve failed")
        return T

    def positivity(self, u, eps):
        """Zhang-Shu limited copy of u and the number of elements changed."""
        u = self._field(u, copy=True)
        n = C.c_int(0)
        rc = lib().or_positivity(self._ref(), _p(u), eps, C.byref(n))
        if rc:
            raise ValueError("an element mean is not admissible")
        return u, n.value

    def diagnostics(self, u):
        u = self._field(u)
        out = np.zeros(8)
        lib().or_diagnostics(self._ref(), _p(u), _p(out))
        return out


def mixture_eval(species, Y, T):
    """e(T) and cv(T) of mixtures with mass fractions Y [n][ns]."""
    species = np.ascontiguousarray(species, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    e = np.zeros(len(T))
    cv = np.zeros(len(T))
    lib().or_mixture_eval(species.shape[0], _p(species), len(T), _p(Y), _p(T), _p(e), _p(cv))
    return e, cv


def mixture_temperature(species, Y, e, T0=None):
    """Newton T(e) per state; returns (T, iterations, failed)."""
    species = np.ascontiguousarray(species, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    T0 = None if T0 is None else np.ascontiguousarray(T0, dtype=np.float64)
    T = np.zeros(len(e))
    it = np.zeros(len(e), dtype=np.int32)
    bad = lib().or_mixture_temperature(species.shape[0], _p(species), len(e), _p(Y), _p(e),
                                       _p(T0), _p(T), _p(it))
    return T, it, bool(bad)


def chem_eval(species, reactions, rhos, T, dt=0.0):
    """omega, diagonal Jacobian and point-implicit source for states rhos [n][5], T [n]."""
    species = np.ascontiguousarray(species, dtype=np.float64)
    reactions = np.ascontiguousarray(reactions, dtype=np.float64)
    rhos = np.ascontiguousarray(rhos, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    n = len(T)
    om, jd, S = np.zeros((n, 5)), np.zeros((n, 5)), np.zeros((n, 5))
    lib().or_chem_eval(_p(species), len(reactions), _p(reactions), n, _p(rhos), _p(T), dt, _p(om),
                       _p(jd), _p(S))
    return om, jd, S


def mlp_nparams(n_out=1):
    return lib().or_mlp_nparams_n(n_out)


def mlp_forward(params, X, n_out=1):
    """Outputs [n] for one output, [n][n_out] otherwise."""
    params = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    y = np.zeros((X.shape[0], n_out))
    if lib().or_mlp_forward_n(_p(params), n_out, X.shape[0], _p(X), _p(y)):
        raise ValueError("n_out out of range")
    return y[:, 0] if n_out == 1 else y


def mlp_loss_grad(params, X, t, n_out=1):
    params = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    g = np.zeros_like(params)
    loss = lib().or_mlp_loss_grad_n(_p(params), n_out, X.shape[0], _p(X), _p(t), _p(g))
    if loss < 0:
        raise ValueError("n_out out of range")
    return loss, g


# unit roundoff of BF16 (8-bit significand, round to nearest)
BF16_U = 2.0 ** -8
# bound on the absolute error of the GPU's hardware tanh approximation (tanh.approx.f32):
# measured on a GB300 over 2^24 arguments in [-12, 12], 8.0e-6 = 2^-16.9; taken as 2^-16
TANH_APPROX_EPS = 2.0 ** -16


def mlp_forward_sd(params, X, n_out=1, u=BF16_U, eps_t=TANH_APPROX_EPS, x_rel=0.0, u_flip=0.0,
                   want_flip=False):
    """Exact FP64 outputs [n][n_out] and the standard deviation of the GPU's difference from
    a reference under the first-order rounding model of or_mlp_forward_sd_n (u = BF16_U:
    the reference is the exact network; u = 0, u_flip = BF16_U: the reference is the BF16
    emulation mlp_forward_bf16, and want_flip adds the largest effect of one hidden unit
    rounding to its neighbouring BF16 value)."""
    params = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    y = np.zeros((X.shape[0], n_out))
    sd = np.zeros((X.shape[0], n_out))
    fl = np.zeros((X.shape[0], n_out)) if want_flip else None
    if lib().or_mlp_forward_sd_n(_p(params), n_out, X.shape[0], _p(X), u, u_flip, eps_t, x_rel, _p(y),
                                 _p(sd), _p(fl)):
        raise ValueError("n_out out of range")
    return (y, sd, fl) if want_flip else (y, sd)


def bf16(x):
    """Round to BF16 (round to nearest, ties to even) via the FP32 bit pattern; returns
    float32 values."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _gelu32(z):
    k = np.float32(np.sqrt(2.0 / np.pi))
    arg = (k * (z + np.float32(0.044715) * z * z * z)).astype(np.float32)
    t = np.tanh(arg.astype(np.float64)).astype(np.float32)
    return (np.float32(0.5) * z * (np.float32(1.0) + t)).astype(np.float32)


def mlp_forward_bf16(params, Xn32, n_out, want_flip=False, eps_t=TANH_APPROX_EPS):
    """The network evaluated with the GPU's roundings, for decisions in the kernel's
    precision: FP32 standardised inputs Xn32 [n][7], inputs, W1, W2 and the first hidden
    layer's activations rounded to BF16, each sum rounded once to FP32 (exact products of
    BF16 values summed in FP64), GELU in FP32 with the tanh of FP64 rounded to FP32, the
    output layer in FP32 with FP32 weights.  Returns float64 [n][n_out].

    want_flip: also returns, per output, the effect of the first hidden units that may
    round to the other BF16 neighbour on the GPU: a unit whose FP32 activation lies within
    d of a rounding boundary, d bounding the GPU's difference before rounding (its FP32 sum
    of 8 terms, the tanh approximation's eps_t, the GELU's FP32 operations), contributes
    the first-order effect of one BF16 spacing on each output,
    sum_j |W3_oj| |gelu'(z2_j)| |W2_ji| spacing_i."""
    NI_, NH_ = 7, 64
    p32 = np.asarray(params, dtype=np.float32)
    W1 = bf16(p32[:NH_ * NI_].reshape(NH_, NI_)).astype(np.float64)
    b1 = p32[NH_ * NI_:NH_ * NI_ + NH_]
    o = NH_ * NI_ + NH_
    W2 = bf16(p32[o:o + NH_ * NH_].reshape(NH_, NH_)).astype(np.float64)
    b2 = p32[o + NH_ * NH_:o + NH_ * NH_ + NH_]
    o3 = o + NH_ * NH_ + NH_
    W3 = p32[o3:o3 + n_out * NH_].reshape(n_out, NH_).astype(np.float64)
    b3 = p32[o3 + n_out * NH_:o3 + n_out * NH_ + n_out]
    xb = bf16(np.asarray(Xn32, dtype=np.float32)).astype(np.float64)
    z1 = ((xb @ W1.T).astype(np.float32) + b1).astype(np.float32)
    a1f = _gelu32(z1)
    a1 = bf16(a1f).astype(np.float64)
    z2 = ((a1 @ W2.T).astype(np.float32) + b2).astype(np.float32)
    a2 = _gelu32(z2).astype(np.float64)
    y = ((a2 @ W3.T).astype(np.float32) + b3).astype(np.float64)
    if not want_flip:
        return y
    u32 = 2.0 ** -24
    z1d = z1.astype(np.float64)
    mag1 = np.abs(xb) @ np.abs(W1.T) + np.abs(b1.astype(np.float64))
    gd1 = np.abs(_gelu_d_np(z1d))
    d = gd1 * 10 * u32 * mag1 + 0.5 * np.abs(z1d) * eps_t + 6 * u32 * np.abs(a1f.astype(np.float64))
    # distance of the FP32 activation to the nearest BF16 rounding boundary (the midpoints
    # between neighbouring BF16 values), and the BF16 spacing there
    lo = bf16(a1f).astype(np.float64)
    b = np.ascontiguousarray(bf16(a1f)).view(np.uint32).astype(np.int64)
    # neighbouring BF16 values: the next and previous 16-bit patterns (BF16 is the top half
    # of the FP32 pattern)
    up = (b + (1 << 16)).astype(np.uint32).view(np.float32).astype(np.float64)
    dn = (b - (1 << 16)).astype(np.uint32).view(np.float32).astype(np.float64)
    dist = np.minimum(np.abs(a1f - 0.5 * (lo + up)), np.abs(a1f - 0.5 * (lo + dn)))
    spacing = np.maximum(np.abs(up - lo), np.abs(lo - dn))
    near = dist <= d
    gd2 = np.abs(_gelu_d_np(z2.astype(np.float64)))
    flip = np.zeros((xb.shape[0], n_out))
    for r in np.nonzero(near.any(axis=1))[0]:
        units = np.nonzero(near[r])[0]
        # effect of unit i on output o: sum_j |W3_oj| |gelu'(z2_j)| |W2_ji| spacing_i
        eff = (np.abs(W3) * gd2[r][None, :]) @ np.abs(W2[:, units]) * spacing[r, units][None, :]
        flip[r] = eff.sum(axis=1)
    return y, flip


def _gelu_d_np(x):
    """Derivative of the tanh form of GELU (vectorised; the same formula as or_gelu_d)."""
    k = np.sqrt(2.0 / np.pi)
    t = np.tanh(k * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * k * (1.0 + 3.0 * 0.044715 * x * x)


_M64 = (1 << 64) - 1


def splitmix64(x):
    """Steele, Lea & Flood's SplitMix64 output function of the state increment x (one step
    from state x): z = x + 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds (30, 27)
    and a final xor-shift (31).  Python integers, vectorised over a sequence."""
    out = []
    for v in np.atleast_1d(x):
        z = (int(v) + 0x9E3779B97F4A7C15) & _M64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        out.append(z ^ (z >> 31))
    return out


def chem_surrogate_correction(params, stats, rhos, T, dt=0.0, *, species, reactions, lam=8.0, x_rel=0.0,
                              network="fp64", plain_rel=1e-10):
    """Step 9 of reading R18s (plain correction) at a refresh state rhos [n][5], T [n] with
    the running step dt: the plain rates minus the network's decoded rates, c_omega =
    omega - omega^ and c_jpi = jpi - jpi' (jpi = max(0, -d omega_s / d rho_s) of the plain
    source, jpi' the decoded value before its clamp at 0), with the bounds of the GPU's
    difference from them (the network's rounding bound at this state, and the FP32 storage
    of the corrections); and the full check of every node: the uncorrected learned source
    (steps 2 and 5) against the plain source with the sampled check's test (step 6), a
    32-node tile trusted when all of its nodes pass (trust_ambiguous where a margin lies
    within the bound).  plain_rel: the relative difference allowed between the GPU's plain
    rates at this state and the oracle's (1e-10 for an FP64 state; larger where the GPU's
    temperature differs, as in the mixed form).  Returns the dict that
    chem_surrogate_source takes as `correction`."""
    st = np.asarray(stats, dtype=np.float64)
    d = chem_surrogate_source(params, stats, rhos, T, dt, lam=lam, x_rel=x_rel, network=network)
    om_p, jd, S_p = chem_eval(species, reactions, rhos, T, dt)
    jpi_p = np.maximum(0.0, -jd)
    c_om = om_p - d["omega_net"]
    c_j = jpi_p - d["jpi_raw"]
    u32 = 2.0 ** -24
    n = len(T)
    scale = np.abs(S_p).sum(axis=1)
    thr = st[50] * scale + st[52]
    m = thr[:, None] - np.abs(d["S_learned"] - S_p)
    node_ok = np.all(m >= 0.0, axis=1) & np.isfinite(d["S_learned"]).all(axis=1)
    node_amb = np.any(np.abs(m) <= d["bound"] + max(plain_rel, 1e-10) * scale[:, None] + u32 * thr[:, None],
                      axis=1)
    ntiles = (n + 31) // 32
    pad = ntiles * 32 - n
    trust = np.concatenate([node_ok, np.ones(pad, dtype=bool)]).reshape(ntiles, 32).all(axis=1)
    trust_amb = np.concatenate([node_amb, np.zeros(pad, dtype=bool)]).reshape(ntiles, 32).any(axis=1)
    # the plain rates' own difference: relative to the node's largest rate (the rates are
    # sums of forward and backward terms that cancel near equilibrium)
    om_scale = np.abs(om_p).max(axis=1, keepdims=True)
    j_scale = jpi_p.max(axis=1, keepdims=True)
    return {"c_omega": c_om, "c_jpi": c_j,
            "B_omega": d["B_omega"] + u32 * np.abs(c_om) + plain_rel * (np.abs(om_p) + om_scale),
            "B_jpi": d["B_jpi"] + u32 * np.abs(c_j) + plain_rel * (jpi_p + j_scale),
            "trust": trust, "trust_ambiguous": trust_amb}


def chem_surrogate_source(params, stats, rhos, T, dt=0.0, *, species=None, reactions=None, call=None,
                          lam=8.0, x_rel=0.0, network="fp64", correction=None):
    """The learned chemistry source by the acceptance rule of reading R18s, in FP64.

    params: ten-output perceptron (FP32 values); stats: the statistics vector of the C
    interface (feature mean 0:7, std 7:14; target mean 14:24, std 24:34; omega_ref 34,
    jpi_ref 35; trust box lo 36:43, hi 43:50; tau_c 50, tau_m 51, floor 52); rhos [n][5]
    species densities, T [n] temperatures of the nodes in element-major order; dt the
    point-implicit step.

    Steps (R18s): features x = (Y_1..Y_5, ln rho, T); network on (x - mean)/std; decode
    omega = omega_ref sinh(z), jpi = max(0, jpi_ref sinh(z')) with z = mean + std y; trust
    box in FP32; mass balance |sum omega| <= tau_m sum|omega| + floor (finite); projection
    omega_s -= |omega_s| sum(omega) / sum|omega|; S = omega / (1 + dt jpi); positivity
    rho_s + dt S_s >= 0 in FP32 (reported in mass_ok and, alone, in positive).  With species,
    reactions and the call counter given: the sampled check of every 32-node tile against
    the plain source (chem_eval) at node 32 t + splitmix64(call 1099511628211 + t) mod n_t,
    and the per-tile decision.

    network = "fp64" evaluates the network exactly (the definition) and bounds the GPU's
    difference by its BF16 roundings; network = "bf16" evaluates it with the GPU's own
    roundings (mlp_forward_bf16: decisions in the kernel's precision) and bounds only what
    remains (FP32 sum order, the tanh approximation, the rare BF16 rounding of a hidden
    unit to the neighbouring value).  The bound is lam standard deviations of the
    first-order model, carried through decode, projection and the point-implicit factor;
    per tile, the result says whether any decision lies within that bound of its
    threshold (ambiguous: the GPU may decide either way).  x_rel: relative error of the
    raw features of the GPU's input state (0 for an FP64 state).  correction (the dict of
    chem_surrogate_correction at a refresh state, step 9): the decoded rates become
    omega^ + c_omega and max(0, jpi' + c_jpi) before the tests, and the bound adds the
    correction's own."""
    st = np.asarray(stats, dtype=np.float64)
    rhos = np.asarray(rhos, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    n = len(T)
    u32 = 2.0 ** -24
    rho = rhos.sum(axis=1)
    x = np.column_stack([rhos / rho[:, None], np.log(rho), T])
    # 1. trust box, decided in FP32
    x32 = x.astype(np.float32)
    lo32, hi32 = st[36:43].astype(np.float32), st[43:50].astype(np.float32)
    inside = np.all((x32 >= lo32) & (x32 <= hi32), axis=1)
    ulp = np.spacing(np.abs(x32)).astype(np.float64)
    box_amb = np.any((np.abs(x32.astype(np.float64) - lo32) <= ulp) |
                     (np.abs(x32.astype(np.float64) - hi32) <= ulp), axis=1)
    # 2. network and decode, with the rounding bound
    if network == "bf16":
        # standardisation as the kernel does it: FP32 features, FP32 mean and 1/std
        xn32 = ((x32 - st[0:7].astype(np.float32)) * (1.0 / st[7:14]).astype(np.float32)).astype(np.float32)
        _, sd = mlp_forward_sd(params, xn32.astype(np.float64), 10, u=0.0, x_rel=x_rel)
        y, fl = mlp_forward_bf16(params, xn32, 10, want_flip=True)
        # the hidden units that may round to the other BF16 neighbour, as worst-case jumps
        sd = sd + fl / lam
    else:
        y, sd = mlp_forward_sd(params, (x - st[0:7]) / st[7:14], 10, x_rel=x_rel)
    z = st[14:24] + st[24:34] * y
    Bz = lam * np.abs(st[24:34]) * sd + 4 * u32 * (np.abs(st[14:24]) + np.abs(st[24:34] * y))
    om = st[34] * np.sinh(z[:, :5])
    jp_raw = st[35] * np.sinh(z[:, 5:])
    Bom = st[34] * np.cosh(np.abs(z[:, :5]) + Bz[:, :5]) * Bz[:, :5] + 8 * u32 * np.abs(om)
    Bjp = st[35] * np.cosh(np.abs(z[:, 5:]) + Bz[:, 5:]) * Bz[:, 5:] + 8 * u32 * np.abs(jp_raw)
    net = {"omega_net": om, "jpi_raw": jp_raw, "B_omega": Bom, "B_jpi": Bjp}
    if correction is not None:
        # step 9: the stored plain-minus-network differences, added in FP32 on the GPU
        c_om, c_j = correction["c_omega"], correction["c_jpi"]
        Bom = Bom + correction["B_omega"] + 2 * u32 * (np.abs(om) + np.abs(c_om))
        Bjp = Bjp + correction["B_jpi"] + 2 * u32 * (np.abs(jp_raw) + np.abs(c_j))
        om = om + c_om
        jp_raw = jp_raw + c_j
    jpi = np.maximum(0.0, jp_raw)
    # 3. mass balance
    tau_c, tau_m, floor = st[50], st[51], st[52]
    msum = om.sum(axis=1)
    asum = np.abs(om).sum(axis=1)
    finite = np.isfinite(asum)
    margin = tau_m * asum + floor - np.abs(msum)
    unc = (1.0 + tau_m) * (Bom.sum(axis=1) + 6 * u32 * asum) + u32 * floor
    mass_ok = finite & (margin >= 0.0)
    mass_amb = np.abs(margin) <= unc
    # 4. projection and the point-implicit factor
    f = np.divide(msum, asum, out=np.zeros_like(msum), where=asum > 0)
    om_t = om - np.abs(om) * f[:, None]
    den = 1.0 + dt * jpi
    S_l = om_t / den
    dA = Bom.sum(axis=1)
    Bomt = (1.0 + np.abs(f))[:, None] * (Bom + np.abs(om) * np.divide(
        dA, asum, out=np.zeros_like(dA), where=asum > 0)[:, None]) + 4 * u32 * np.abs(om) * (1 + np.abs(f))[:, None]
    bound = Bomt / den + np.abs(S_l) * dt * Bjp / den + 4 * u32 * np.abs(S_l)
    # 5b. positivity of the learned update, decided in FP32: rho_s + dt S_s >= 0
    dt32 = np.float32(dt)
    pos_val = (rhos.astype(np.float32) + dt32 * S_l.astype(np.float32)).astype(np.float64)
    pos_ok = np.all(pos_val >= 0.0, axis=1)
    pos_amb = np.any(np.abs(pos_val) <= dt * bound + 4 * u32 * np.abs(rhos), axis=1)
    mass_ok = mass_ok & pos_ok
    mass_amb = mass_amb | pos_amb
    out = {"S_learned": S_l, "bound": bound, "inside": inside, "mass_ok": mass_ok, "positive": pos_ok,
           "omega": om, "jpi": jpi, "x": x}
    out.update(net)
    if call is None:
        return out
    # 5. sampled check per 32-node tile and the decisions
    _, _, S_p = chem_eval(species, reactions, rhos, T, dt)
    ntiles = (n + 31) // 32
    flag = np.zeros(ntiles, dtype=np.int8)
    amb = np.zeros(ntiles, dtype=bool)
    sampled = np.zeros(ntiles, dtype=np.int64)
    node_ok = inside & mass_ok
    node_amb = box_amb | mass_amb
    trust = np.ones(ntiles, dtype=bool) if correction is None else correction["trust"]
    trust_amb = np.zeros(ntiles, dtype=bool) if correction is None else correction["trust_ambiguous"]
    hashes = splitmix64([(int(call) * 1099511628211 + t) & _M64 for t in range(ntiles)])
    for t in range(ntiles):
        a, b = 32 * t, min(n, 32 * t + 32)
        i = a + int(hashes[t] % (b - a))
        sampled[t] = i
        amb[t] = bool(node_amb[a:b].any()) or bool(trust_amb[t])
        if not trust[t]:
            flag[t] = 4  # step 9: the network missed the plain source at the last refresh
            continue
        if not node_ok[a:b].all():
            flag[t] = 1
            continue
        thr = tau_c * np.abs(S_p[i]).sum() + floor
        m = thr - np.abs(S_l[i] - S_p[i])
        if (m < 0.0).any():
            flag[t] = 2
        amb[t] |= bool((np.abs(m) <= bound[i] + 1e-10 * np.abs(S_p[i]).sum() + u32 * thr).any())
    acc_node = np.repeat(flag == 0, 32)[:n]
    out.update({"S_plain": S_p, "S": np.where(acc_node[:, None], S_l, S_p), "tile_flag": flag,
                "tile_ambiguous": amb, "sampled_node": sampled})
    return out


def adam_step(params, m, v, g, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays."""
    lib().or_adam_step(_p(params), _p(m), _p(v), _p(np.ascontiguousarray(g)), len(params), step,
                       lr, b1, b2, eps)


def gelu(x):
    return lib().or_gelu(float(x))


def gelu_d(x):
    return lib().or_gelu_d(float(x))


def ck45():
    A, B, c = np.zeros(5), np.zeros(5), np.zeros(5)
    lib().or_ck45(_p(A), _p(B), _p(c))
    return A, B, c


def ln_mean(x, y):
    return lib().or_ln_mean(float(x), float(y))
