"""GB300-native entropy-stable DGSEM (arXiv 2511.17551) -- Python binding of libdg.

A thin ctypes layer over the C ABI declared in ``include/dg.h``: the functions
below carry the same names and only marshal arguments.  Every step of the
right-hand side and of the Runge-Kutta stepping runs in the CUDA kernels of
``libdg.so``; there is no CPU fallback.  Importing this module does not need a
GPU; creating a context does, and fails with DgError(DG_ECUDA) without one.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = [
    "DgError", "lib", "dg_lgl_nodes", "dg_init_mesh", "dg_set_state", "dg_set_state_primitive",
    "dg_get_state", "dg_rhs", "dg_step_rk", "dg_diagnostics", "dg_get_alpha", "dg_get_gradients",
    "dg_sync", "dg_destroy", "dg_error_element", "dg_profile", "dg_profile_read", "Solver",
    "EXPORTED",
]

DG_OK, DG_EINVAL, DG_ENOMEM, DG_ECUDA, DG_ENONPHYS, DG_ENEWTON, DG_ETIMEOUT, DG_ESTATE = range(8)
DG_EULER, DG_NAVIER_STOKES = 0, 1
DG_VF_RANOCHA, DG_VF_DUCROS, DG_VF_CENTRAL, DG_VF_KG, DG_VF_PIROZZOLI, DG_VF_MORINISHI = 0, 1, 2, 3, 4, 5
DG_SF_LLF, DG_SF_HLLC, DG_SF_EC, DG_SF_HLL = 0, 1, 2, 3
DG_FP64, DG_MIXED = 0, 1
DG_THERMO_NEWTON, DG_THERMO_MLP = 0, 1
DG_BC_INFLOW, DG_BC_OUTFLOW, DG_BC_SLIP_WALL, DG_BC_NOSLIP_ADIABATIC, DG_BC_ISOTHERMAL = 1, 2, 3, 4, 5

# every symbol declared in include/dg.h
EXPORTED = [
    "dg_lgl_nodes", "dg_init_mesh", "dg_set_state", "dg_set_state_primitive", "dg_get_state",
    "dg_rhs", "dg_step_rk", "dg_diagnostics", "dg_get_alpha", "dg_get_gradients", "dg_sync",
    "dg_error_element", "dg_status_string", "dg_destroy", "dg_profile", "dg_profile_read",
    "dg_rhs_ns_noalloc", "dg_get_temperature", "dg_set_surrogate", "dg_surrogate_stats",
    "dg_thermo_sample", "dg_mlp_nparams", "dg_mlp_workspace_bytes", "dg_mlp_grad",
    "dg_mlp_train_step", "dg_mlp_forward", "dg_peak_flops", "dg_chem_sample", "dg_limiter_stats", "dg_limit_state",
    "dg_noalloc_status", "dg_get_metrics", "dg_get_source", "dg_column_stats", "dg_standardize",
    "dg_abs_quantile", "dg_gather_rows", "dg_mlp_loss", "dg_set_source_refresh",
]
PROF_KINDS = ["rhs", "gradients", "indicator", "lambda", "thermo", "mlp", "chem", "other", "limiter"]


class DgError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = lib().dg_status_string(code).decode()
        super().__init__("%s: %s (%d)" % (where, msg, code))


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("N", C.c_int), ("K", C.c_int64),
                ("node_xyz", C.c_void_p), ("nbr_elem", C.c_void_p),
                ("nbr_face", C.c_void_p), ("nbr_orient", C.c_void_p)]


class PhysicsDesc(C.Structure):
    _fields_ = [("equations", C.c_int), ("n_species", C.c_int), ("gamma", C.c_double),
                ("mu", C.c_double), ("Pr", C.c_double), ("species", C.c_void_p),
                ("volume_flux", C.c_int), ("surface_flux", C.c_int),
                ("alpha_max", C.c_double), ("precision", C.c_int), ("thermo", C.c_int),
                ("n_bc", C.c_int), ("bc_kind", C.c_void_p), ("bc_prim", C.c_void_p),
                ("stream", C.c_void_p), ("reactions", C.c_void_p), ("n_reactions", C.c_int),
                ("p_ref", C.c_double), ("positivity_eps", C.c_double),
                ("sutherland_s", C.c_double), ("sutherland_rt", C.c_double),
                ("indicator_variable", C.c_int)]


_lib = None


def lib():
    """Load libdg.so (building it in-tree when missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        i, d, vp, i64 = C.c_int, C.c_double, C.c_void_p, C.c_int64
        sig = {
            "dg_lgl_nodes": (i, [i, vp, vp]),
            "dg_init_mesh": (i, [vp, vp, vp]),
            "dg_set_state": (i, [vp, vp, i, d]),
            "dg_set_state_primitive": (i, [vp, vp, i, d]),
            "dg_get_state": (i, [vp, vp, i, vp]),
            "dg_rhs": (i, [vp, vp, vp, d]),
            "dg_step_rk": (i, [vp, i, d, d, vp]),
            "dg_diagnostics": (i, [vp, vp]),
            "dg_get_alpha": (i, [vp, vp]),
            "dg_get_gradients": (i, [vp, vp]),
            "dg_get_metrics": (i, [vp, vp, vp, i]),
            "dg_get_source": (i, [vp, vp, vp, vp]),
            "dg_column_stats": (i, [vp, i, i64, i, vp, vp, vp]),
            "dg_standardize": (i, [vp, i, i64, i, vp, vp, vp, vp, vp]),
            "dg_abs_quantile": (i, [vp, i64, i, i, i, d, vp, vp]),
            "dg_gather_rows": (i, [vp, i, vp, i64, vp, vp]),
            "dg_mlp_loss": (i, [vp, i, vp, vp, i64, vp, vp]),
            "dg_noalloc_status": (i, [vp, vp]),
            "dg_sync": (i, [vp]),
            "dg_error_element": (i64, [vp]),
            "dg_status_string": (C.c_char_p, [i]),
            "dg_destroy": (None, [vp]),
            "dg_profile": (i, [vp, i]),
            "dg_profile_read": (i, [vp, vp, vp, i]),
            "dg_rhs_ns_noalloc": (i, [i, i64, vp, vp, vp, d, d, d, i, i, vp, vp, vp]),
            "dg_get_temperature": (i, [vp, vp]),
            "dg_set_surrogate": (i, [vp, i, vp, vp]),
            "dg_surrogate_stats": (i, [vp, i, vp]),
            "dg_set_source_refresh": (i, [vp, i]),
            "dg_chem_sample": (i, [vp, i64, C.c_uint64, vp, vp]),
            "dg_limiter_stats": (i, [vp, vp]),
            "dg_limit_state": (i, [vp]),
            "dg_thermo_sample": (i, [vp, i64, C.c_uint64, vp, vp]),
            "dg_mlp_nparams": (i, [i]),
            "dg_mlp_workspace_bytes": (C.c_size_t, [i, i]),
            "dg_mlp_grad": (i, [vp, i, vp, vp, i, vp, vp, vp, C.c_size_t, vp]),
            "dg_mlp_train_step": (i, [vp, i, vp, vp, vp, vp, i, i, C.c_float, vp, vp, C.c_size_t,
                                      vp]),
            "dg_mlp_forward": (i, [vp, i, vp, vp, i64, i, vp]),
            "dg_peak_flops": (i, [i, i, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _check(code, where):
    if code != DG_OK:
        raise DgError(code, where)


def _ptr(a):
    """Address of a numpy array or of a torch tensor (device or host)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _on_device(a):
    return int(bool(getattr(a, "is_cuda", False)))


# ----------------------------------------------------------------- C-ABI mirrors
def dg_lgl_nodes(N):
    x = np.zeros(N + 1)
    w = np.zeros(N + 1)
    _check(lib().dg_lgl_nodes(N, _ptr(x), _ptr(w)), "dg_lgl_nodes")
    return x, w


def dg_init_mesh(mesh, phys):
    ctx = C.c_void_p()
    _check(lib().dg_init_mesh(C.byref(mesh), C.byref(phys), C.byref(ctx)), "dg_init_mesh")
    return ctx


def dg_set_state(ctx, u, t=0.0):
    _check(lib().dg_set_state(ctx, _ptr(u), _on_device(u), t), "dg_set_state")


def dg_set_state_primitive(ctx, w, t=0.0):
    _check(lib().dg_set_state_primitive(ctx, _ptr(w), _on_device(w), t), "dg_set_state_primitive")


def dg_get_state(ctx, u):
    t = C.c_double()
    _check(lib().dg_get_state(ctx, _ptr(u), _on_device(u), C.byref(t)), "dg_get_state")
    return t.value


def dg_rhs(ctx, u, rhs, t=0.0):
    _check(lib().dg_rhs(ctx, _ptr(u), _ptr(rhs), t), "dg_rhs")


def dg_step_rk(ctx, nsteps, cfl=0.5, dt_fixed=0.0, t=0.0):
    tt = C.c_double(t)
    _check(lib().dg_step_rk(ctx, nsteps, cfl, dt_fixed, C.byref(tt)), "dg_step_rk")
    return tt.value


def dg_diagnostics(ctx):
    out = np.zeros(8)
    _check(lib().dg_diagnostics(ctx, _ptr(out)), "dg_diagnostics")
    return out


def dg_get_temperature(ctx, shape):
    T = np.zeros(shape)
    _check(lib().dg_get_temperature(ctx, _ptr(T)), "dg_get_temperature")
    return T


DG_SURROGATE_TEMPERATURE = 0
DG_SURROGATE_SOURCE = 1
DG_SRC_NSTATS = 53


def dg_set_surrogate(ctx, params=None, stats=None, which=DG_SURROGATE_TEMPERATURE):
    """params: host float32 [P] (or None to switch the surrogate off); stats: float64
    [16] (temperature) or [DG_SRC_NSTATS] (source)."""
    p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
    s = None if stats is None else np.ascontiguousarray(stats, dtype=np.float64)
    _check(lib().dg_set_surrogate(ctx, which, _ptr(p), _ptr(s)), "dg_set_surrogate")


def dg_set_source_refresh(ctx, period):
    """Plain correction of the learned source: refresh every `period` RK steps (0: off)."""
    _check(lib().dg_set_source_refresh(ctx, int(period)), "dg_set_source_refresh")


def dg_surrogate_stats(ctx, which=DG_SURROGATE_TEMPERATURE):
    out = np.zeros(2, dtype=np.int64)
    _check(lib().dg_surrogate_stats(ctx, which, _ptr(out)), "dg_surrogate_stats")
    return int(out[0]), int(out[1])


def dg_thermo_sample(ctx, X, T, seed=0):
    """X: device float32 tensor [n][7], T: device float32 [n]."""
    _check(lib().dg_thermo_sample(ctx, T.shape[0], seed, _ptr(X), _ptr(T)), "dg_thermo_sample")


def dg_chem_sample(ctx, X, targets, seed=0):
    """X: device float32 [n][7] (Y_1..Y_5, ln rho, T); targets: device float64 [n][10]
    (omega_1..5, jpi_1..5) of the plain source."""
    _check(lib().dg_chem_sample(ctx, targets.shape[0], seed, _ptr(X), _ptr(targets)), "dg_chem_sample")


def _n_out(t):
    return 1 if t.dim() == 1 else t.shape[1]


def dg_mlp_nparams(n_out=1):
    return lib().dg_mlp_nparams(n_out)


def dg_mlp_workspace_bytes(batch, n_out=1):
    return lib().dg_mlp_workspace_bytes(batch, n_out)


def dg_mlp_grad(params, X, t, grad, loss, workspace, stream=None):
    """t: [batch] (one output) or [batch][n_out] standardised targets (device float32)."""
    _check(lib().dg_mlp_grad(_ptr(params), _n_out(t), _ptr(X), _ptr(t), t.shape[0], _ptr(grad), _ptr(loss),
                             _ptr(workspace), workspace.numel() * workspace.element_size(), stream),
           "dg_mlp_grad")


def dg_mlp_train_step(params, m, v, X, t, step, lr, loss, workspace, stream=None):
    _check(lib().dg_mlp_train_step(_ptr(params), _n_out(t), _ptr(m), _ptr(v), _ptr(X), _ptr(t), t.shape[0],
                                   step, lr, _ptr(loss), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), stream),
           "dg_mlp_train_step")


def dg_mlp_forward(params, X, y, tensor_cores=1, stream=None):
    """y: [n] (one output) or [n][n_out] device float32."""
    _check(lib().dg_mlp_forward(_ptr(params), _n_out(y), _ptr(X), _ptr(y), y.shape[0],
                                int(tensor_cores), stream), "dg_mlp_forward")


def dg_limit_state(ctx):
    _check(lib().dg_limit_state(ctx), "dg_limit_state")


def dg_limiter_stats(ctx):
    """Elements changed by the positivity limiter since the last call."""
    out = np.zeros(1, dtype=np.int64)
    _check(lib().dg_limiter_stats(ctx, _ptr(out)), "dg_limiter_stats")
    return int(out[0])


def dg_peak_flops(precision, iters=20000):
    """Measured FMA peak of the device in TFLOP/s (DG_FP64 or DG_MIXED = FP32)."""
    t = C.c_double()
    _check(lib().dg_peak_flops(precision, iters, C.byref(t)), "dg_peak_flops")
    return t.value


def dg_get_alpha(ctx, K):
    a = np.zeros(K)
    _check(lib().dg_get_alpha(ctx, _ptr(a)), "dg_get_alpha")
    return a


def dg_get_gradients(ctx, shape):
    g = np.zeros(shape)
    _check(lib().dg_get_gradients(ctx, _ptr(g)), "dg_get_gradients")
    return g


def dg_get_metrics(ctx, Ja, invJ):
    """FP64 metric terms of the context into caller buffers Ja [K][dim][dim][np] and
    invJ [K][np] (numpy arrays or CUDA tensors, both on the same side)."""
    _check(lib().dg_get_metrics(ctx, _ptr(Ja), _ptr(invJ), _on_device(Ja)), "dg_get_metrics")


def dg_get_source(ctx, shape):
    """(S [K][5][np] FP64, tile flags uint8, call index) of the last source evaluation."""
    K, _, npn = shape
    S = np.zeros((K, 5, npn))
    flags = np.zeros((K * npn + 31) // 32, dtype=np.uint8)
    call = C.c_int64(-1)
    _check(lib().dg_get_source(ctx, _ptr(S), _ptr(flags), C.byref(call)), "dg_get_source")
    return S, flags, call.value


def _dev_f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def dg_column_stats(X, ref=None, stream=None):
    """Per-column (mean, std, min, max) of a device array X [n][d] (FP32 or FP64), of
    asinh(X / ref) when ref [d] is given; four float64 arrays."""
    n, d = X.shape
    out = np.zeros(4 * d)
    r = _dev_f64(ref)
    _check(lib().dg_column_stats(_ptr(X), int(X.element_size() == 8), n, d, _ptr(r), _ptr(out), stream),
           "dg_column_stats")
    return out[:d], out[d:2 * d], out[2 * d:3 * d], out[3 * d:]


def dg_standardize(X, mean, std, out, ref=None, stream=None):
    """out [n][d] FP32 = ((asinh(X / ref) or X) - mean) / std, on the device."""
    n, d = X.shape
    m, s, r = _dev_f64(mean), _dev_f64(std), _dev_f64(ref)
    _check(lib().dg_standardize(_ptr(X), int(X.element_size() == 8), n, d, _ptr(r), _ptr(m), _ptr(s), _ptr(out),
                                stream), "dg_standardize")


def dg_abs_quantile(Y, c0, nc, q, stream=None):
    """q-quantile of |Y[:, c0:c0+nc]| (FP64 device array), linear interpolation."""
    n, d = Y.shape
    out = C.c_double(0.0)
    _check(lib().dg_abs_quantile(_ptr(Y), n, d, c0, nc, float(q), C.byref(out), stream), "dg_abs_quantile")
    return out.value


def dg_gather_rows(X, idx, out, stream=None):
    """out[r] = X[idx[r]] (FP32 rows, int64 indices; device arrays)."""
    _check(lib().dg_gather_rows(_ptr(X), X.shape[1], _ptr(idx), idx.shape[0], _ptr(out), stream), "dg_gather_rows")


def dg_mlp_loss(params, X, t, stream=None):
    """Mean squared error of the FP32 network on (X, t) (device arrays)."""
    loss = C.c_double(0.0)
    n_out = 1 if t.dim() == 1 else t.shape[1]
    _check(lib().dg_mlp_loss(_ptr(params), n_out, _ptr(X), _ptr(t), X.shape[0], C.byref(loss), stream),
           "dg_mlp_loss")
    return loss.value


def dg_sync(ctx):
    _check(lib().dg_sync(ctx), "dg_sync")


def dg_error_element(ctx):
    return lib().dg_error_element(ctx)


def dg_profile(ctx, enable):
    _check(lib().dg_profile(ctx, int(enable)), "dg_profile")


def dg_profile_read(ctx):
    """{kind: (milliseconds, launches)} since the last read."""
    n = len(PROF_KINDS)
    ms = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    _check(lib().dg_profile_read(ctx, _ptr(ms), _ptr(cnt), n), "dg_profile_read")
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PROF_KINDS)}


def dg_rhs_ns_noalloc(N, K, nbr, Ja, invJ, gamma, mu, Pr, volume_flux, surface_flux, u, rhs,
                      stream=None):
    """Allocation-free Navier-Stokes right-hand side: every argument is a caller-owned
    device tensor; the gradient scratch is libdg's static device array."""
    _check(lib().dg_rhs_ns_noalloc(N, K, _ptr(nbr), _ptr(Ja), _ptr(invJ), gamma, mu, Pr,
                                   volume_flux, surface_flux, _ptr(u), _ptr(rhs), stream),
           "dg_rhs_ns_noalloc")


def dg_noalloc_status(stream=None):
    """(code, raw status word) latched by the last dg_rhs_ns_noalloc call on the current
    device, after the stream's queued work: code DG_OK, DG_EINVAL or DG_ENONPHYS."""
    w = C.c_uint64(0)
    code = lib().dg_noalloc_status(stream, C.byref(w))
    if code not in (DG_OK, DG_EINVAL, DG_ENONPHYS):
        raise DgError(code, "dg_noalloc_status")
    return code, int(w.value)


def dg_destroy(ctx):
    if ctx:
        lib().dg_destroy(ctx)


# ----------------------------------------------------------------- convenience holder
class Solver:
    """Owns one libdg context and the host arrays its descriptors point at."""

    def __init__(self, dim, N, xyz, nbr_elem, nbr_face, *, n_species=0, equations=DG_EULER,
                 gamma=1.4, mu=0.0, Pr=0.72, species=None, volume_flux=DG_VF_RANOCHA,
                 surface_flux=DG_SF_LLF, alpha_max=0.0, precision=DG_FP64,
                 thermo=DG_THERMO_NEWTON, bc_kind=None, bc_prim=None, stream=None,
                 reactions=None, p_ref=0.0, positivity_eps=0.0, sutherland_s=0.0,
                 sutherland_rt=1.0, indicator_variable=0):
        self.dim, self.N = dim, N
        self.np = (N + 1) ** dim
        self.nsp = max(1, n_species)
        self.nv = self.nsp + dim + 1
        self.precision = precision
        self._xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.K = self._xyz.shape[0]
        self._nbr = np.ascontiguousarray(nbr_elem, dtype=np.int64)
        self._face = np.ascontiguousarray(nbr_face, dtype=np.int8)
        self._species = (np.ascontiguousarray(species, dtype=np.float64)
                         if species is not None else None)
        self._bck = np.ascontiguousarray(bc_kind if bc_kind is not None else [1], dtype=np.int32)
        self._bcp = np.ascontiguousarray(bc_prim if bc_prim is not None else np.zeros((1, self.nv)),
                                         dtype=np.float64)
        self._reac = (np.ascontiguousarray(reactions, dtype=np.float64)
                      if reactions is not None else None)
        mesh = MeshDesc(dim=dim, N=N, K=self.K, node_xyz=_ptr(self._xyz), nbr_elem=_ptr(self._nbr),
                        nbr_face=_ptr(self._face), nbr_orient=None)
        phys = PhysicsDesc(equations=equations, n_species=n_species, gamma=gamma, mu=mu, Pr=Pr,
                           species=_ptr(self._species), volume_flux=volume_flux,
                           surface_flux=surface_flux, alpha_max=alpha_max, precision=precision,
                           thermo=thermo, n_bc=len(self._bck) if bc_kind is not None else 0,
                           bc_kind=_ptr(self._bck), bc_prim=_ptr(self._bcp), stream=stream,
                           reactions=_ptr(self._reac),
                           n_reactions=0 if reactions is None else len(self._reac), p_ref=p_ref,
                           positivity_eps=positivity_eps, sutherland_s=sutherland_s,
                           sutherland_rt=sutherland_rt, indicator_variable=indicator_variable)
        self.ctx = dg_init_mesh(mesh, phys)

    @property
    def shape(self):
        return (self.K, self.nv, self.np)

    def set_state(self, u, t=0.0):
        dg_set_state(self.ctx, np.ascontiguousarray(u, dtype=np.float64) if isinstance(u, np.ndarray) else u, t)

    def set_primitive(self, w, t=0.0):
        dg_set_state_primitive(self.ctx, np.ascontiguousarray(w, dtype=np.float64) if isinstance(w, np.ndarray) else w, t)

    def get_state(self):
        u = np.zeros(self.shape)
        t = dg_get_state(self.ctx, u)
        return u, t

    def step(self, nsteps, cfl=0.5, dt_fixed=0.0, t=0.0):
        return dg_step_rk(self.ctx, nsteps, cfl, dt_fixed, t)

    def diagnostics(self):
        return dg_diagnostics(self.ctx)

    def close(self):
        if self.ctx:
            dg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
