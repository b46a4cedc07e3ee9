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
            "or_mlp_loss_grad_n": (d, [vp, i, i, vp, vp, vp]),
            "or_chem_eval": (i, [vp, i, vp, i, vp, vp, d, vp, vp, vp]),
            "or_gelu": (d, [d]),
            "or_gelu_d": (d, [d]),
            "or_mlp_forward": (None, [vp, i, vp, vp]),
            "or_mlp_loss_grad": (d, [vp, i, vp, vp, vp]),
            "or_adam_step": (None, [vp, vp, vp, vp, i, i, d, d, d, d]),
            "or_mixture_temperature": (i, [i, vp, i, vp, vp, vp, vp, vp]),
            "or_positivity": (i, [vp, vp, d, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


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


def chem_surrogate_source(params, stats, rhos, T, dt=0.0):
    """FP64 evaluation of the learned chemistry source at nodes (rhos [n][5] species
    densities, T [n]) with the ten-output perceptron and the statistics vector of the
    C interface (offsets: feature mean 0, std 7; target mean 14, std 24; omega_ref 34,
    jpi_ref 35; box lo 36, hi 43; tolerances 50 (check), 51 (mass), floor 52).

    Steps: raw features x = (Y_1..Y_5, ln rho, T); network on (x - mean)/std; decode
    omega_s = omega_ref sinh(mu_s + sd_s y_s), jpi_s = max(0, jpi_ref sinh(mu_{5+s} +
    sd_{5+s} y_{5+s})); node accepted when x lies in the box and |sum omega| <=
    tol_mass sum|omega| + floor; projection omega_s -= |omega_s| sum(omega)/sum|omega|;
    S_s = omega_s / (1 + dt jpi_s).  Returns (S [n][5], accepted [n] bool, omega raw
    [n][5], jpi [n][5])."""
    st = np.asarray(stats, dtype=np.float64)
    rhos = np.asarray(rhos, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    rho = rhos.sum(axis=1)
    x = np.column_stack([rhos / rho[:, None], np.log(rho), T])
    y = mlp_forward(params, (x - st[0:7]) / st[7:14], 10)
    z = st[14:24] + st[24:34] * y
    om = st[34] * np.sinh(z[:, :5])
    jpi = np.maximum(0.0, st[35] * np.sinh(z[:, 5:]))
    msum = om.sum(axis=1)
    asum = np.abs(om).sum(axis=1)
    inside = np.all((x >= st[36:43]) & (x <= st[43:50]), axis=1)
    accepted = inside & (np.abs(msum) <= st[51] * asum + st[52])
    frac = np.divide(msum, asum, out=np.zeros_like(msum), where=asum > 0)
    S = (om - np.abs(om) * frac[:, None]) / (1.0 + dt * jpi)
    return S, accepted, om, jpi


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
