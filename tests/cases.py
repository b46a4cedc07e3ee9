"""Workload builders shared by the oracle pins and the GPU parity tests.

Each builder takes the caller's own LGL node set (``xi``) so that the oracle
side and the library side each place nodes with their own basis.
"""
import numpy as np

import workloads as W

GAMMA = 1.4


def tgv(xi, n_el, warp=0.0, mach=0.1, shape=None):
    shape = shape or (n_el,) * 3
    xyz, nbr, face = W.box_mesh(shape, xi, (-np.pi,) * 3, (np.pi,) * 3, periodic=True,
                                warp=warp)
    return xyz, nbr, face, W.tgv_primitive(xyz, GAMMA, mach)


def supersonic_tgv(xi, n_el, warp=0.0, shape=None, mach=1.25):
    shape = shape or (n_el,) * 3
    xyz, nbr, face = W.box_mesh(shape, xi, (-np.pi,) * 3, (np.pi,) * 3, periodic=True,
                                warp=warp)
    return xyz, nbr, face, W.supersonic_tgv_primitive(xyz, GAMMA, mach)


def tgv_p0(mach=0.1):
    """Mean pressure of the Taylor-Green state, p0 = 1 / (gamma Ma^2)."""
    return 1.0 / (GAMMA * mach * mach)


def vortex(xi, n_el, t=0.0):
    xyz, nbr, face = W.box_mesh((n_el, n_el), xi, (-5.0, -5.0), (5.0, 5.0), periodic=True)
    return xyz, nbr, face, W.vortex_primitive(xyz, t=t, gamma=GAMMA)


def perturbed_state(w, seed, amp=0.05):
    """Random smooth-free perturbation of a primitive state (parity stress cases)."""
    rng = np.random.default_rng(seed)
    w = w.copy()
    w *= 1.0 + amp * rng.uniform(-1, 1, size=w.shape)
    return w


def square_cylinder_small(xi, seed=3):
    """A 24 x 12 cut of the square-cylinder workload with the same boundary kinds."""
    lo = (-1.2, -0.6)
    h = 0.1
    nx, ny = 24, 12
    xyz, nbr, face = W.box_mesh((nx, ny), xi, lo, (lo[0] + nx * h, lo[1] + ny * h),
                                periodic=False, bc_ids=[0, 1, 0, 0])
    k = np.arange(nx * ny)
    ix, iy = k % nx, k // nx
    solid = (ix >= 8) & (ix < 12) & (iy >= 4) & (iy < 8)
    return W._compact_and_shuffle(xyz, nbr, face, ~solid, 2, seed)


def mach3_freestream(gamma=GAMMA, mach=3.0):
    return np.array([1.0, 1.0, 0.0, 1.0 / (gamma * mach * mach)])


# ---------------------------------------------------------------- matched problem pairs
def field_errors(a, ref, nsp, dim):
    """Relative L2 error per conserved field (R19 reading): momentum components are
    normalised by the norm of the whole momentum block."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    nv = a.shape[1]
    out = []
    mom = np.linalg.norm(ref[:, nsp:nsp + dim])
    for v in range(nv):
        den = mom if nsp <= v < nsp + dim else np.linalg.norm(ref[:, v])
        out.append(np.linalg.norm(a[:, v] - ref[:, v]) / max(den, 1e-300))
    return np.array(out)


class Pair:
    """The same workload built twice: once on the oracle's nodes, once on libdg's."""

    def __init__(self, builder, dim, N, precision=0, **kw):
        import oracle
        import paper_2511_17551_gb300 as dg
        self.dim, self.N = dim, N
        xo, _ = oracle.lgl(N)
        xg, _ = dg.dg_lgl_nodes(N)
        self.mesh_o = builder(xo)
        self.mesh_g = builder(xg)
        okw = dict(kw)
        gkw = dict(kw)
        okw.pop("p_ref", None)  # an offset the oracle does not need (exact in arithmetic)
        for k in ("equations", "volume_flux", "surface_flux"):
            pass
        self.orc = oracle.Oracle(dim, N, *self.mesh_o[:3], **okw)
        gkw.pop("alpha_override", None)
        self.gpu = dg.Solver(dim, N, *self.mesh_g[:3], precision=precision, **gkw)
        self.K = self.orc.K
        self.nv = self.orc.nv

    def close(self):
        self.gpu.close()


# ---------------------------------------------------------------- mixture workloads
MIX_RHO, MIX_T = 0.1, 300.0
MIX_U = 2000.0  # nominal Mach 5 for the seeded mixture at 300 K


def mixture_ogrid(xi, nr=3, nth=4, nz=2, u_inf=MIX_U, seed=7, hot=None):
    """Half O-grid around a cylinder (R = 0.5 m), inflow on the outer arc, outflow at the
    ends, slip wall on the body, periodic span; seeded Dirichlet mass-fraction field."""
    import workloads as W
    xyz, nbr, face = W.ogrid_mesh(xi, nr, nth, nz)
    w = W.mixture_primitive(xyz, rho=MIX_RHO, vel=(u_inf, 0.0, 0.0), T=MIX_T, seed=seed, hot=hot)
    return xyz, nbr, face, w


def mixture_bc(w):
    fs = w[0, :, 0].copy()
    return [1, 2, 3], np.stack([fs, fs, fs])


def mixture_perturbed(w, seed):
    rng = np.random.default_rng(seed)
    w = w.copy()
    w[:, :5] *= 1 + 0.05 * rng.uniform(-1, 1, size=w[:, :5].shape)
    w[:, 5:8] += 100.0 * rng.normal(size=w[:, 5:8].shape)
    w[:, 8] *= 1 + 0.3 * rng.uniform(-1, 1, size=w[:, 8].shape)
    return w


def rounding_floor(orc, u, eps=2.0 ** -24, seed=5):
    """The oracle's own sensitivity of its right-hand side to a rounding of the state:
    relative L2 per field (R19) of rhs(u (1 + eps s)) - rhs(u) with seeded signs s = +-1.
    eps = 2^-24 is one FP32 unit in the last place, the rounding floor of any right-hand
    side computed from an FP32 state; eps = 2^-53 the FP64 one."""
    sgn = np.random.default_rng(seed).choice([-1.0, 1.0], size=u.shape)
    r0 = orc.rhs(u)
    return field_errors(orc.rhs(u * (1.0 + eps * sgn)), r0, orc.nv - orc.dim - 1, orc.dim)


def step_floor(orc, u0, nsteps, dt, eps=2.0 ** -53, seed=5, nsp=None):
    """The oracle's own sensitivity of nsteps CK45 steps (and whatever limiter or blending
    the problem carries) to a rounding of the initial state: relative L2 per field of the
    end states from u0 and from u0 (1 + eps s), s = +-1 seeded."""
    sgn = np.random.default_rng(seed).choice([-1.0, 1.0], size=u0.shape)
    a, _ = orc.step_rk(u0, nsteps, dt_fixed=dt)
    b, _ = orc.step_rk(u0 * (1.0 + eps * sgn), nsteps, dt_fixed=dt)
    nsp = orc.nv - orc.dim - 1 if nsp is None else nsp
    return field_errors(b, a, nsp, orc.dim)


def fp64_bar(floor):
    """The FP64 parity bar of a case: 1e-12 relative L2, or 16 times the oracle's own one-ulp
    floor of that case where rounding amplification puts the floor above 1e-12 / 16."""
    return np.maximum(1e-12, 16.0 * np.asarray(floor))
