"""Seeded synthetic workloads (meshes, initial states, species data).

This module produces problem INPUTS only: node coordinates at caller-supplied
reference points, face connectivity, primitive initial states and seeded
tables of species/reaction constants.  It contains none of the method's
arithmetic (no basis, metric, flux, thermodynamic or time-stepping code), so
the oracle and the GPU library can both consume what it returns while sharing
no code with each other.  Each caller passes its OWN one-dimensional LGL node
set in ``xi``; the two sets agree to rounding.

Layouts: xyz [K][dim][np] (node index x fastest), nbr_elem/nbr_face [K][2dim]
(faces -x,+x,-y,+y,-z,+z; boundary faces hold -(bc_id+1)), primitive states
[K][nv][np] with (rho, v, p) for a single gas and (rho_1..rho_ns, v, T) for a
mixture.
"""
import numpy as np

__all__ = [
    "box_mesh", "tgv_primitive", "vortex_primitive", "square_cylinder_mesh",
    "freestream_primitive", "ogrid_mesh", "species_table", "mixture_primitive",
    "reaction_table", "splitmix64_permutation", "tgv_config", "config_sizes",
]


def _ref_points(xi, dim):
    n1 = len(xi)
    idx = np.indices((n1,) * dim).reshape(dim, -1)[::-1]  # idx[0] = x index (fastest)
    return [np.asarray(xi)[idx[d]] for d in range(dim)]


def box_mesh(shape, xi, lo, hi, periodic=True, warp=0.0, bc_ids=None):
    """Structured box of len(shape) in {2,3} dims, element (ix,iy[,iz]) -> k = ix + nx*(iy + ny*iz).

    Node positions x = lo + (i + (1+xi)/2) h (bitwise equal on shared faces).
    ``warp`` > 0 adds warp*sin(x)sin(y)sin(z) to every coordinate (3D; the
    TGV curved mesh).  ``periodic`` is a bool or a per-direction tuple;
    non-periodic sides get bc ids ``bc_ids[face]`` (face = 2*dir + side).
    """
    dim = len(shape)
    if isinstance(periodic, bool):
        periodic = (periodic,) * dim
    shape = tuple(int(s) for s in shape)
    K = int(np.prod(shape))
    n1 = len(xi)
    npn = n1 ** dim
    ref = _ref_points(xi, dim)
    eidx = np.indices(shape[::-1]).reshape(dim, -1)[::-1]  # eidx[0] = ix fastest
    h = [(hi[d] - lo[d]) / shape[d] for d in range(dim)]
    xyz = np.empty((K, dim, npn))
    for d in range(dim):
        xyz[:, d, :] = lo[d] + (eidx[d][:, None] + (1.0 + ref[d][None, :]) / 2.0) * h[d]
    if warp:
        assert dim == 3
        s = warp * np.sin(xyz[:, 0]) * np.sin(xyz[:, 1]) * np.sin(xyz[:, 2])
        xyz = xyz + s[:, None, :]
    nbr = np.empty((K, 2 * dim), dtype=np.int64)
    strides = [int(np.prod(shape[:d])) for d in range(dim)]
    for d in range(dim):
        for side in (0, 1):
            f = 2 * d + side
            step = 1 if side else -1
            j = eidx[d] + step
            inside = (j >= 0) & (j < shape[d])
            jw = j % shape[d]
            kk = np.arange(K) + (jw - eidx[d]) * strides[d]
            if periodic[d]:
                nbr[:, f] = kk
            else:
                bc = bc_ids[f] if bc_ids is not None else 0
                nbr[:, f] = np.where(inside, kk, -(bc + 1))
    face = np.tile(np.array([f ^ 1 for f in range(2 * dim)], dtype=np.int8), (K, 1))
    return xyz, nbr, face


def tgv_primitive(xyz, gamma=1.4, mach=0.1):
    """Taylor-Green vortex on [-pi,pi]^3: rho=1, U0=1, p0 = 1/(gamma Ma^2)."""
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    p0 = 1.0 / (gamma * mach * mach)
    w = np.empty((xyz.shape[0], 5, xyz.shape[2]))
    w[:, 0] = 1.0
    w[:, 1] = np.sin(x) * np.cos(y) * np.cos(z)
    w[:, 2] = -np.cos(x) * np.sin(y) * np.cos(z)
    w[:, 3] = 0.0
    w[:, 4] = p0 + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    return w


SUTHERLAND_S = 0.4042   # S / T_o of the supersonic TGV's Sutherland law (Eq. sutherland)


def supersonic_tgv_primitive(xyz, gamma=1.4, mach=1.25):
    """Supersonic Taylor-Green vortex on [-pi,pi]^3 in units rho_o = L = U_o = 1: the
    subsonic field with p_o = 1/(gamma M^2) and the perturbation rho_o U_o^2 / 16 (...)
    (the dimensionally consistent reading), uniform temperature T = T_o, so that
    rho = p / (R T_o) = p / p_o."""
    w = tgv_primitive(xyz, gamma=gamma, mach=mach)
    p0 = 1.0 / (gamma * mach * mach)
    w[:, 0] = w[:, 4] / p0
    return w


def channel_primitive(xyz, p0):
    """Wall-bounded channel 0 <= y <= 1 (walls at y = 0 and 1): a parabolic streamwise
    profile 4y(1-y) with peak 1, zero at both walls, a small wall-normal and spanwise
    perturbation, rho = 1, uniform pressure p0."""
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    w = np.empty((xyz.shape[0], 5, xyz.shape[2]))
    w[:, 0] = 1.0 + 0.01 * np.sin(0.5 * np.pi * x)
    w[:, 1] = 4.0 * y * (1.0 - y)
    w[:, 2] = 0.01 * np.sin(0.5 * np.pi * x) * np.sin(np.pi * y)
    w[:, 3] = 0.01 * np.cos(np.pi * z) * np.sin(np.pi * y)
    w[:, 4] = p0
    return w


def supersonic_tgv_physics(gamma=1.4, mach=1.25, reynolds=1600.0):
    """Physics keywords of the supersonic TGV in the same units: mu_o = rho_o L U_o / Re at
    T_o, Sutherland's law with s = S / T_o and the reference p/rho = p_o / rho_o."""
    return dict(mu=1.0 / reynolds, Pr=0.72, gamma=gamma, sutherland_s=SUTHERLAND_S,
                sutherland_rt=1.0 / (gamma * mach * mach), indicator_variable=1)


def vortex_primitive(xyz, t=0.0, gamma=1.4, eps=5.0, period=10.0):
    """Shu isentropic vortex (2D), advected with v_inf = (1,1) on a periodic square."""
    x = xyz[:, 0] - t
    y = xyz[:, 1] - t
    x = (x + period / 2) % period - period / 2
    y = (y + period / 2) % period - period / 2
    r2 = x * x + y * y
    dT = -(gamma - 1.0) * eps * eps / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = (1.0 + dT) ** (1.0 / (gamma - 1.0))
    dv = eps / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    w = np.empty((xyz.shape[0], 4, xyz.shape[2]))
    w[:, 0] = rho
    w[:, 1] = 1.0 - dv * y
    w[:, 2] = 1.0 + dv * x
    w[:, 3] = rho ** gamma
    return w


def splitmix64_permutation(n, seed):
    """Fisher-Yates shuffle driven by splitmix64 (published generator)."""
    mask = (1 << 64) - 1
    state = seed & mask
    perm = np.arange(n, dtype=np.int64)
    for i in range(n - 1, 0, -1):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        z ^= z >> 31
        j = z % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return perm


def _compact_and_shuffle(xyz, nbr, face, keep, removed_bc, seed):
    K = xyz.shape[0]
    new_id = -np.ones(K, dtype=np.int64)
    new_id[keep] = np.arange(int(keep.sum()))
    xyz, nbr, face = xyz[keep], nbr[keep], face[keep]
    inner = nbr >= 0
    mapped = np.where(inner, new_id[np.maximum(nbr, 0)], nbr)
    mapped = np.where(inner & (mapped < 0), -(removed_bc + 1), mapped)
    nbr = mapped
    if seed is not None:
        Kn = xyz.shape[0]
        perm = splitmix64_permutation(Kn, seed)  # new position of old element e is perm[e]
        inv = np.empty(Kn, dtype=np.int64)
        inv[perm] = np.arange(Kn)
        xyz = xyz[inv]
        face = face[inv]
        nbr = nbr[inv]
        nbr = np.where(nbr >= 0, perm[np.maximum(nbr, 0)], nbr)
    return xyz, nbr, face


def square_cylinder_mesh(xi, nx=512, ny=256, h=0.1, seed=20251117):
    """Mach-3 square cylinder (2D): [-10.5,40.7]x[-12.8,12.8], unit square removed.

    bc 0: supersonic inflow (left, top, bottom), bc 1: outflow (right),
    bc 2: slip wall (cylinder).  Elements shuffled by a seeded permutation.
    """
    lo = (-10.5, -12.8)
    hi = (lo[0] + nx * h, lo[1] + ny * h)
    xyz, nbr, face = box_mesh((nx, ny), xi, lo, hi, periodic=False, bc_ids=[0, 1, 0, 0])
    ix0 = int(round((-0.5 - lo[0]) / h))
    iy0 = int(round((-0.5 - lo[1]) / h))
    nc = int(round(1.0 / h))
    k = np.arange(nx * ny)
    ix, iy = k % nx, k // nx
    solid = (ix >= ix0) & (ix < ix0 + nc) & (iy >= iy0) & (iy < iy0 + nc)
    return _compact_and_shuffle(xyz, nbr, face, ~solid, 2, seed)


def freestream_primitive(K, npn, state):
    state = np.asarray(state, dtype=np.float64)
    return np.broadcast_to(state[None, :, None], (K, len(state), npn)).copy()


def ogrid_mesh(xi, nr, nth, nz, R=0.5, Rout_over_R=6.0, Lz=None, theta0=0.5 * np.pi,
               theta1=1.5 * np.pi):
    """Half O-grid around a cylinder of radius R (upstream half, x <= 0), z periodic.

    xi -> r (bc 2 slip wall at r=R, bc 0 inflow at the outer arc),
    eta -> theta (bc 1 outflow at both ends), zeta -> z (periodic).
    """
    Lz = Lz if Lz is not None else 2.0 * R
    xyz, nbr, face = box_mesh((nr, nth, nz), xi, (R, theta0, 0.0), (R * Rout_over_R, theta1, Lz),
                              periodic=(False, False, True), bc_ids=[2, 0, 1, 1, 0, 0])
    r, th = xyz[:, 0].copy(), xyz[:, 1].copy()
    xyz[:, 0] = r * np.cos(th)
    xyz[:, 1] = r * np.sin(th)
    return xyz, nbr, face


def species_table(seed=5, ns=5):
    """Five seeded species {A, B, A2, B2, AB} with [W (kg/mol), a1..a7].

    Atom masses a, b ~ U[14,16] g/mol; cp/R = c0 + c1 tau + .. + c4 tau^4 with
    tau = T/1000 K, c0 ~ U[2.5,3.5], c_k ~ U[0,1]*(0.2, 0.02, 1e-3, 3e-5)
    (all >= 0: cp > 0 and increasing on 200..1e4 K); a7 ~ U[0,20].  Formation
    constants a6 (K): atoms U[2e4, 5e4], molecules U[-1e4, 1e4], so that the
    molecules are bound (dissociation is endothermic, dH/R in 3e4..1.1e5 K).
    """
    rng = np.random.default_rng(seed)
    a, b = rng.uniform(14.0, 16.0, size=2)
    W = np.array([a, b, 2 * a, 2 * b, a + b])[:ns] * 1e-3
    tab = np.zeros((ns, 8))
    tab[:, 0] = W
    c0 = rng.uniform(2.5, 3.5, size=ns)
    ck = rng.uniform(0.0, 1.0, size=(ns, 4)) * np.array([0.2, 0.02, 1e-3, 3e-5])
    tab[:, 1] = c0
    tab[:, 2] = ck[:, 0] / 1e3
    tab[:, 3] = ck[:, 1] / 1e6
    tab[:, 4] = ck[:, 2] / 1e9
    tab[:, 5] = ck[:, 3] / 1e12
    a6 = rng.uniform(-1e4, 1e4, size=5)
    a6[:2] = rng.uniform(2e4, 5e4, size=2)  # atoms A, B
    tab[:, 6] = a6[:ns]
    tab[:, 7] = rng.uniform(0.0, 20.0, size=ns)
    return tab


def mixture_primitive(xyz, rho, vel, T, seed=7, ns=5, hot=None, cylinder=None):
    """(rho_s, v, T) with Y from a smooth seeded Dirichlet field.

    Y_s ~ b_s (1 + 0.5 sin(k_s . x + phi_s)), normalised, b ~ Dirichlet(1..1).
    ``hot`` = (radius, T_hot): nodes closer than radius to the z axis get T_hot.
    ``cylinder`` = R: the velocity is the incompressible potential flow past a cylinder of
    radius R on the z axis (free stream vel[0] along x), tangent to the body at r = R.
    """
    rng = np.random.default_rng(seed)
    b = rng.dirichlet(np.ones(ns))
    kvec = rng.uniform(-2.0, 2.0, size=(ns, 3))
    phi = rng.uniform(0.0, 2 * np.pi, size=ns)
    K, dim, npn = xyz.shape
    arg = np.einsum("sd,kdn->skn", kvec[:, :dim], xyz) + phi[:, None, None]
    Yr = b[:, None, None] * (1.0 + 0.5 * np.sin(arg))
    Y = Yr / Yr.sum(axis=0, keepdims=True)
    w = np.empty((K, ns + dim + 1, npn))
    for s in range(ns):
        w[:, s] = rho * Y[s]
    for d in range(dim):
        w[:, ns + d] = vel[d]
    if cylinder is not None:
        R = cylinder
        x, y = xyz[:, 0], xyz[:, 1]
        r2 = np.maximum(x * x + y * y, 1e-300)
        U = vel[0]
        # u - i v = U (1 - R^2 / z^2) with z = x + i y
        zr2 = (x * x - y * y) / (r2 * r2)
        zi2 = -2 * x * y / (r2 * r2)
        w[:, ns + 0] = U * (1.0 - R * R * zr2)
        w[:, ns + 1] = U * R * R * zi2
    w[:, ns + dim] = T
    if hot is not None:
        # smooth hot layer around the z axis: T + (T_hot - T) exp(-(r / rad)^4)
        rad, Th = hot
        r = np.sqrt(xyz[:, 0] ** 2 + xyz[:, 1] ** 2)
        w[:, ns + dim] = T + (Th - T) * np.exp(-(r / rad) ** 4)
    return w


def reaction_table(seed=11, nr=17, n_third=4, species=None):
    """Seeded element-balanced mechanism over species {A,B,A2,B2,AB}.

    Rows: [nu_f(5), nu_b(5), third_body_flag, eff(5), A, beta, theta].
    beta U[-1.5,0.5]; A = 10^U[9,12] / 5000^beta, so that the rate constant at 5000 K is
    1e9..1e12 cm^3/(mol s) (chemical time scales near the flow step; A within [1e9, 1e22]);
    third-body efficiencies U[0.2,22].  Activation temperature theta = max(0, dH_r/R) +
    U[0, 1e4] K for dissociations and + U[1e4, 3e4] K for exchanges (capped at 1.2e5 K),
    dH_r/R = sum_s dnu_s a6_s from the species' formation constants, so the backward
    activation theta - dH/R is never negative (no recombination rate that grows without
    bound as T falls).
    """
    sp = species if species is not None else species_table()
    A_, B_, A2, B2, AB = range(5)
    pool = []
    for X2, prods in ((A2, (A_, A_)), (B2, (B_, B_)), (AB, (A_, B_))):
        for M in range(5):
            pool.append(((X2, M), prods + (M,), 0))
        pool.append(((X2,), prods, 1))
    pool += [((A2, B_), (AB, A_), 0), ((B2, A_), (AB, B_), 0), ((A2, B2), (AB, AB), 0)]
    rng = np.random.default_rng(seed)
    third = [i for i, p in enumerate(pool) if p[2] == 1]
    other = [i for i, p in enumerate(pool) if p[2] == 0]
    nt = min(n_third, len(third))
    pick = list(rng.choice(third, size=nt, replace=False)) + list(
        rng.choice(other, size=nr - nt, replace=False))
    rows = np.zeros((nr, 19))
    for r, i in enumerate(pick):
        reac, prod, tb = pool[i]
        for s in reac:
            rows[r, s] += 1
        for s in prod:
            rows[r, 5 + s] += 1
        rows[r, 10] = tb
        rows[r, 11:16] = rng.uniform(0.2, 22.0, size=5) if tb else 0.0
        beta = rng.uniform(-1.5, 0.5)
        rows[r, 16] = min(1e22, max(1e9, 10.0 ** rng.uniform(9.0, 12.0) / 5000.0 ** beta))
        rows[r, 17] = beta
        dnu = rows[r, 5:10] - rows[r, 0:5]
        dH = float(dnu @ sp[:, 6])
        margin = rng.uniform(0.0, 1e4) if dnu.sum() > 0 else rng.uniform(1e4, 3e4)
        rows[r, 18] = min(1.2e5, max(0.0, dH) + margin)
    return rows


def tgv_config(xi, n_el, warp=0.0):
    """TGV workload on [-pi,pi]^3 with n_el^3 elements (x fastest)."""
    return box_mesh((n_el,) * 3, xi, (-np.pi,) * 3, (np.pi,) * 3, periodic=True, warp=warp)


def config_sizes():
    """Element count, degree and dimension of the five synthetic workloads."""
    return {
        "tgv_euler_4^3_N3": dict(K=64, N=3, dim=3, nv=5),
        "tgv_ns_32^3_N3": dict(K=32768, N=3, dim=3, nv=5),
        "tgv_ns_16^3_N7": dict(K=4096, N=7, dim=3, nv=5),
        "square_cylinder_512x256_N3": dict(K=130972, N=3, dim=2, nv=4),
        "mixture_24^3_N4": dict(K=13824, N=4, dim=3, nv=9),
        "reacting_48x48x16_N4": dict(K=36864, N=4, dim=3, nv=9),
    }
