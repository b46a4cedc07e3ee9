"""Pins of the oracle's semi-discrete operator (Eqs. strong_form, fluxes_discrete_strong,
differencing, fluxdiffcons, DGvec, fluxes_discrete_with_fv, auxil, auxstrongf)."""
import numpy as np
import pytest

import cases
import workloads as W


def _quad_weights(orc, o):
    _, w = orc.lgl(o.N)
    idx = np.indices((o.N + 1,) * o.dim).reshape(o.dim, -1)
    wq = np.prod(w[idx], axis=0)
    return wq[None, :] * o.J  # [K][np]


def _tgv_oracle(orc, n_el, N, warp=0.1, **kw):
    x, _ = orc.lgl(N)
    xyz, nbr, face, w = cases.tgv(x, n_el, warp=warp)
    o = orc.Oracle(3, N, xyz, nbr, face, **kw)
    return o, o.prim_to_cons(w)


@pytest.mark.parametrize("N", [2, 3])
@pytest.mark.parametrize("sf", [0, 1, 2])
def test_free_stream_preservation_warped(orc, N, sf):
    o, u = _tgv_oracle(orc, 3, N, surface_flux=sf)
    const = np.array([1.1, 0.3, -0.2, 0.5, 80.0])
    u[:] = const[None, :, None]
    r = o.rhs(u)
    scale = np.abs(const).max() * np.abs(o.Ja).max() / o.J.min() * N ** 2
    assert np.abs(r).max() < 1e-13 * scale


@pytest.mark.parametrize("sf", [0, 1, 2])
def test_conservation_periodic(orc, sf):
    o, u = _tgv_oracle(orc, 3, 3, surface_flux=sf)
    u = o.prim_to_cons(cases.perturbed_state(
        cases.tgv(orc.lgl(3)[0], 3, warp=0.1)[3], seed=1))
    r = o.rhs(u)
    M = _quad_weights(orc, o)
    for v in range(5):
        tot = np.sum(M * r[:, v])
        scale = np.sum(M * np.abs(r[:, v]))
        assert abs(tot) < 1e-13 * scale


@pytest.mark.parametrize("warp", [0.0, 0.1])
def test_discrete_entropy_conservation(orc, warp):
    """EC volume + EC surface flux on a periodic mesh: sum J w (w(u) . du/dt) = 0;
    with LLF at the faces the same sum is negative."""
    x, _ = orc.lgl(3)
    xyz, nbr, face, w = cases.tgv(x, 3, warp=warp, mach=0.5)
    w = cases.perturbed_state(w, seed=2, amp=0.1)
    M = None
    for sf, expect in ((2, "zero"), (0, "neg")):
        o = orc.Oracle(3, 3, xyz, nbr, face, surface_flux=sf)
        u = o.prim_to_cons(w)
        r = o.rhs(u)
        M = _quad_weights(orc, o)
        wv = np.stack([np.stack([o.entropy_vars(u[k, :, n]) for n in range(o.np)], 1)
                       for k in range(o.K)], 0)
        prod = np.sum(wv * r, axis=1)
        tot = np.sum(M * prod)
        scale = np.sum(M * np.sum(np.abs(wv * r), axis=1))
        if expect == "zero":
            assert abs(tot) < 1e-13 * scale
        else:
            assert tot < -1e-6 * scale


def test_central_flux_equals_standard_dgsem(orc):
    """With the central two-point flux and a central face flux the split operator must
    equal the textbook strong-form DGSEM  -(1/J)[D F + M^{-1} B (F* - F)] (R2 pin)."""
    N = 3
    x, wq = orc.lgl(N)
    D = orc.dmat(N)
    xyz, nbr, face = W.box_mesh((3, 2), x, (0, 0), (3.0, 1.0), periodic=True)
    w = np.empty((6, 4, 16))
    rng = np.random.default_rng(3)
    w[:, 0] = 1 + 0.2 * rng.uniform(size=(6, 16))
    w[:, 1:3] = 0.3 * rng.normal(size=(6, 2, 16))
    w[:, 3] = 1 + 0.2 * rng.uniform(size=(6, 16))
    o = orc.Oracle(2, N, xyz, nbr, face, volume_flux=2, surface_flux=2)
    u = o.prim_to_cons(w)
    r = o.rhs(u)
    g = 1.4
    h = np.array([1.0, 0.5]) / 2  # dx/dxi per direction
    n1 = N + 1
    ref = np.zeros_like(u)
    uu = u.reshape(6, 4, n1, n1)  # [k][v][j][i]
    rho = uu[:, 0]
    v = uu[:, 1:3] / rho[:, None]
    p = (g - 1) * (uu[:, 3] - 0.5 * rho * (v ** 2).sum(1))
    for d in range(2):
        # physical flux in x_d times the contravariant metric (J/h_d)
        Jd = h[0] * h[1] / h[d]
        F = np.stack([uu[:, 1 + d], uu[:, 1 + d] * v[:, 0] + (d == 0) * p,
                      uu[:, 1 + d] * v[:, 1] + (d == 1) * p, (uu[:, 3] + p) * v[:, d]], 1) * Jd
        ax = 3 - d  # i is the last axis
        dF = np.moveaxis(np.tensordot(D, np.moveaxis(F, ax, 0), axes=(1, 0)), 0, ax)
        lift = np.zeros_like(F)
        for side in (0, 1):
            f = 2 * d + side
            nb = nbr[:, f]
            Fn = F[nb]
            own = np.take(F, N if side else 0, axis=ax)
            oth = np.take(Fn, 0 if side else N, axis=ax)
            Fs = 0.5 * (own + oth)
            sl = [slice(None)] * 4
            sl[ax] = N if side else 0
            lift[tuple(sl)] += (Fs - own) / wq[N if side else 0] * (1 if side else -1)
        ref += -(dF + lift).reshape(6, 4, -1)
    ref /= h[0] * h[1]
    assert np.allclose(r, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def _vortex_error(orc, n_el, N, t_end, cfl=0.1):
    x, _ = orc.lgl(N)
    xyz, nbr, face, w0 = cases.vortex(x, n_el)
    o = orc.Oracle(2, N, xyz, nbr, face, surface_flux=0)
    u = o.prim_to_cons(w0)
    dt0 = o.max_dt(u, cfl)
    nsteps = int(np.ceil(t_end / dt0))
    u, t = o.step_rk(u, nsteps, dt_fixed=t_end / nsteps)
    ue = o.prim_to_cons(W.vortex_primitive(xyz, t=t))
    M = _quad_weights(orc, o)
    return np.sqrt(np.sum(M * (u[:, 0] - ue[:, 0]) ** 2))


@pytest.mark.parametrize("N,meshes", [(2, (8, 16, 32)), (3, (16, 32, 64)), (4, (8, 16, 32))])
def test_isentropic_vortex_convergence(orc, N, meshes):
    """Observed order on h, h/2, h/4: about N+1 for odd N once asymptotic (3.8 at N=3),
    N + 0.1..0.5 for even N (collocated split-form DGSEM loses up to half an order there).
    Any dropped or mis-signed term drops the order to <= 1."""
    errs = [_vortex_error(orc, n, N, 0.5) for n in meshes]
    eoc = np.log2(errs[1] / errs[2])
    lo = N + 0.5 if N % 2 else N
    assert lo <= eoc <= N + 1.6, (errs, eoc)


def test_rk_temporal_order(orc):
    """CK45 on a fixed mesh: halving dt divides the error by ~16."""
    N = 3
    x, _ = orc.lgl(N)
    xyz, nbr, face, w0 = cases.vortex(x, 4)
    o = orc.Oracle(2, N, xyz, nbr, face)
    u0 = o.prim_to_cons(w0)
    T = 0.4
    ref, _ = o.step_rk(u0, 256, dt_fixed=T / 256)
    e = []
    for n in (8, 16):
        u, _ = o.step_rk(u0, n, dt_fixed=T / n)
        e.append(np.abs(u - ref).max())
    assert 13 < e[0] / e[1] < 19, e


def test_ck45_order_conditions(orc):
    A, B, c = orc.ck45()
    s = 5
    # convert the 2N-storage scheme to Butcher form: stage increments are combinations of k_j
    coef = np.zeros((s, s))  # du_i = sum_j coef[i, j] dt k_j
    a = np.zeros((s, s))
    b = np.zeros(s)
    ucoef = np.zeros(s)  # u_i - u_0 = sum_j ucoef_j dt k_j (running)
    run = np.zeros(s)
    for i in range(s):
        a[i] = run
        prev = coef[i - 1] if i else np.zeros(s)
        coef[i] = A[i] * prev
        coef[i, i] += 1.0
        run = run + B[i] * coef[i]
    b = run
    cc = a.sum(1)
    assert np.allclose(cc, c, atol=1e-12)
    conds = [(b.sum(), 1), (b @ cc, 1 / 2), (b @ cc ** 2, 1 / 3), (b @ (a @ cc), 1 / 6),
             (b @ cc ** 3, 1 / 4), (b @ (cc * (a @ cc)), 1 / 8), (b @ (a @ cc ** 2), 1 / 12),
             (b @ (a @ (a @ cc)), 1 / 24)]
    for got, want in conds:
        assert abs(got - want) < 1e-11


def test_tgv_closed_forms(orc):
    """KE0 = 1/8 and enstrophy0 = 3/8 (TGV definitions); spectral convergence."""
    o, u = _tgv_oracle(orc, 4, 7, warp=0.0)
    d = o.diagnostics(u)
    assert abs(d[0] - 1 / 8) < 1e-6
    assert abs(d[1] - 3 / 8) < 1e-5
    assert abs(d[5] - (2 * np.pi) ** 3) < 1e-10
    o, u = _tgv_oracle(orc, 4, 7, warp=0.1)
    d = o.diagnostics(u)
    assert abs(d[5] - (2 * np.pi) ** 3) < 1e-9


def test_tgv_viscous_dissipation_sign_and_size(orc):
    """d(KE)/dt from the viscous part alone equals -2 mu * enstrophy0 = -3 mu / 4
    (incompressible limit of Eq. TGV_SD with rho = 1): fixes the sign of BR1."""
    N, n_el = 4, 4
    mu = 0.01
    x, _ = orc.lgl(N)
    xyz, nbr, face, w = cases.tgv(x, n_el, warp=0.1)
    oe = orc.Oracle(3, N, xyz, nbr, face, equations=0)
    on = orc.Oracle(3, N, xyz, nbr, face, equations=1, mu=mu, Pr=0.72)
    u = oe.prim_to_cons(w)
    rv = on.rhs(u) - oe.rhs(u)
    M = _quad_weights(orc, oe)
    rho = u[:, 0]
    v = u[:, 1:4] / rho[:, None]
    dke = np.sum(M * (np.sum(v * rv[:, 1:4], 1) - 0.5 * np.sum(v * v, 1) * rv[:, 0]))
    dke /= (2 * np.pi) ** 3
    assert abs(dke / (-0.75 * mu) - 1) < 0.02, dke


def test_br1_discrete_gauss_theorem(orc):
    """Per element, sum J w dW/dx = face integral of W* n_x for discontinuous data."""
    N = 3
    x, wq = orc.lgl(N)
    xyz, nbr, face = W.box_mesh((2, 2, 3), x, (0, 0, 0), (2.0, 1.0, 1.5), periodic=True)
    rng = np.random.default_rng(9)
    K, np_ = xyz.shape[0], (N + 1) ** 3
    w = np.empty((K, 5, np_))
    w[:, 0] = 1 + 0.3 * rng.uniform(size=(K, np_))
    w[:, 1:4] = rng.normal(size=(K, 3, np_))
    w[:, 4] = 1 + 0.3 * rng.uniform(size=(K, np_))
    o = orc.Oracle(3, N, xyz, nbr, face, equations=1, mu=1e-3)
    u = o.prim_to_cons(w)
    _, G = o.rhs(u, want_grad=True)
    Wf = np.concatenate([w[:, 1:4], (w[:, 4] / w[:, 0])[:, None]], 1)  # (v, theta)
    M = _quad_weights(orc, o)
    n1 = N + 1
    h = np.array([1.0, 0.5, 0.5]) / 2
    for k in range(K):
        for xdir in range(3):
            lhs = np.sum(M[k][None] * G[k, xdir], axis=1)
            Wk = Wf[k].reshape(4, n1, n1, n1)
            rhs = np.zeros(4)
            for side in (0, 1):
                fnb = nbr[k, 2 * xdir + side]
                Wn = Wf[fnb].reshape(4, n1, n1, n1)
                ax = 3 - xdir
                own = np.take(Wk, N if side else 0, axis=ax)
                oth = np.take(Wn, 0 if side else N, axis=ax)
                ws = 0.5 * (own + oth)
                area = np.prod(h) / h[xdir]
                face_w = np.outer(wq, wq)
                rhs += (1 if side else -1) * area * np.sum(ws * face_w[None], axis=(1, 2))
            assert np.allclose(lhs, rhs, atol=1e-12)


def _cyl_oracle(orc, N=3, **kw):
    x, _ = orc.lgl(N)
    xyz, nbr, face = cases.square_cylinder_small(x)
    fs = cases.mach3_freestream()
    bc_kind = [orc.BC_INFLOW, orc.BC_OUTFLOW, orc.BC_SLIP_WALL]
    bc_prim = np.stack([fs, fs, fs])
    o = orc.Oracle(2, N, xyz, nbr, face, bc_kind=bc_kind, bc_prim=bc_prim, **kw)
    return o, xyz, nbr, face, fs


def _blast_state(orc, o, xyz, fs):
    """Freestream with a pressure/density bump: smooth in most elements, steep in some."""
    w = W.freestream_primitive(xyz.shape[0], xyz.shape[2], fs)
    r2 = (xyz[:, 0] - 0.3) ** 2 + (xyz[:, 1] - 0.15) ** 2
    w[:, 0] *= 1 + 2.0 * (r2 < 0.05)
    w[:, 3] *= 1 + 4.0 * (r2 < 0.05)
    return o.prim_to_cons(w)


def test_blending_alpha0_equals_split_form(orc):
    """alpha = 0 through the subcell-flux path equals the direct split form (Eq. differencing)."""
    o0, xyz, nbr, face, fs = _cyl_oracle(orc)
    oa, *_ = _cyl_oracle(orc, alpha_override=0.0)
    u = _blast_state(orc, o0, xyz, fs)
    r0, ra = o0.rhs(u), oa.rhs(u)
    assert np.allclose(ra, r0, rtol=1e-12, atol=1e-12 * np.abs(r0).max())


def test_blending_alpha1_is_first_order_fv(orc):
    """alpha = 1 equals a first-order FV scheme on subcells of width w_i h/2, written here
    by assembling the oracle's own face and two-point-free LLF fluxes."""
    N = 3
    o1, xyz, nbr, face, fs = _cyl_oracle(orc, N=N, alpha_override=1.0)
    u = _blast_state(orc, o1, xyz, fs)
    r1 = o1.rhs(u)
    o0, *_ = _cyl_oracle(orc, N=N)  # supplies the face fluxes (alpha-independent)
    x, wq = orc.lgl(N)
    n1 = N + 1
    h = 0.1
    # face-flux part: the DG operator with the volume term removed = the alpha=1 operator minus
    # its FV interior part; build the FV interior part independently
    fv = np.zeros_like(u)
    uu = u.reshape(u.shape[0], 4, n1, n1)
    for k in range(u.shape[0]):
        for d in range(2):
            n = np.zeros(2)
            n[d] = h / 2  # Ja^d on a Cartesian square element of side h
            ax = 2 - d
            for j in range(1, n1):
                a = np.take(uu[k], j - 1, axis=ax)
                b = np.take(uu[k], j, axis=ax)
                for m in range(n1):
                    F = o1.flux_pair(a[:, m], b[:, m], n, 1)
                    idx_l = [slice(None), m, j - 1] if d == 0 else [slice(None), j - 1, m]
                    idx_r = [slice(None), m, j] if d == 0 else [slice(None), j, m]
                    tmp = fv[k].reshape(4, n1, n1)
                    tmp[tuple(idx_l)] -= F / wq[j - 1]
                    tmp[tuple(idx_r)] += F / wq[j]
    # r1 = -(1/J)[FV interior + face terms]; the face terms alone come from alpha=1 with u
    # replaced by a per-element constant... instead compare differences of two states that
    # share face traces: the interior FV part must match exactly.
    oz, *_ = _cyl_oracle(orc, N=N, alpha_override=1.0)
    J = (h / 2) ** 2
    face_part = r1 + (-fv.reshape(u.shape)) / J  # r1 = -(fv + face)/J  ->  -face/J
    # face_part must vanish at every node not on the element boundary
    interior = np.ones((n1, n1), bool)
    interior[0, :] = interior[-1, :] = interior[:, 0] = interior[:, -1] = False
    assert np.abs(face_part.reshape(-1, 4, n1, n1)[:, :, interior]).max() < \
        1e-12 * np.abs(r1).max()


def test_blending_is_linear_in_alpha(orc):
    o0, xyz, nbr, face, fs = _cyl_oracle(orc, alpha_override=0.0)
    o1, *_ = _cyl_oracle(orc, alpha_override=1.0)
    oh, *_ = _cyl_oracle(orc, alpha_override=0.3)
    u = _blast_state(orc, o0, xyz, fs)
    r0, r1, rh = o0.rhs(u), o1.rhs(u), oh.rhs(u)
    assert np.allclose(rh, 0.7 * r0 + 0.3 * r1, rtol=1e-12, atol=1e-12 * np.abs(r0).max())


def test_indicator_special_cases(orc):
    N = 3
    x, _ = orc.lgl(N)
    xyz, nbr, face = W.box_mesh((3, 1), x, (0, 0), (3.0, 1.0), periodic=True)
    o = orc.Oracle(2, N, xyz, nbr, face, alpha_max=0.5)
    K, np_ = 3, 16
    w = np.empty((K, 4, np_))
    w[:, 1:3] = 0.0
    # rho * p of degree <= N-2 = 1 in each element: rho = 1, p linear in the element
    X = xyz[:, 0] - (np.arange(K)[:, None] + 0.5)
    w[:, 0] = 1.0
    w[:, 3] = 2.0 + X + 0.3 * xyz[:, 1]
    a = o.indicator(o.prim_to_cons(w))
    assert np.all(a == 0.0)
    # element 1 carries (almost) only its highest mode: alpha = alpha_max there,
    # neighbours get half of it by smoothing
    V = orc.vandermonde(N)
    mode = np.outer(V[:, N], V[:, 0]).T.reshape(-1)  # P_N in x, constant in y (node x fastest)
    w[:, 3] = 2.0
    w[1, 3] = 2.0 + 0.5 * mode / np.abs(mode).max()
    w[1, 0] = 1.0
    a = o.indicator(o.prim_to_cons(w))
    assert a[1] == 0.5
    assert a[0] == 0.25 and a[2] == 0.25


def test_permutation_invariance(orc):
    """Shuffling element order permutes the RHS and changes nothing else (bitwise)."""
    N = 2
    x, _ = orc.lgl(N)
    fs = cases.mach3_freestream()
    xyz0, nbr0, face0 = cases.square_cylinder_small(x, seed=None)
    xyz1, nbr1, face1 = cases.square_cylinder_small(x, seed=3)
    kw = dict(bc_kind=[1, 2, 3], bc_prim=np.stack([fs] * 3), alpha_max=0.5)
    o0 = orc.Oracle(2, N, xyz0, nbr0, face0, **kw)
    o1 = orc.Oracle(2, N, xyz1, nbr1, face1, **kw)
    u0 = _blast_state(orc, o0, xyz0, fs)
    perm = W.splitmix64_permutation(xyz0.shape[0], 3)
    u1 = np.empty_like(u0)
    u1[perm] = u0
    r0, r1 = o0.rhs(u0), o1.rhs(u1)
    assert np.array_equal(r1[perm], r0)


def test_time_step_closed_form(orc):
    N = 3
    x, _ = orc.lgl(N)
    xyz, nbr, face = W.box_mesh((2, 2, 2), x, (0, 0, 0), (1.0, 1.0, 1.0), periodic=True)
    o = orc.Oracle(3, N, xyz, nbr, face)
    g, rho, vel, p = 1.4, 1.3, np.array([0.5, -0.2, 0.1]), 2.0
    w = np.broadcast_to(np.array([rho, *vel, p])[None, :, None], (8, 5, 64)).copy()
    u = o.prim_to_cons(w)
    c = np.sqrt(g * p / rho)
    lam = np.sum(np.abs(vel) + c) / 0.25  # h/2 = 0.25 per direction
    assert abs(o.max_dt(u, 0.5) - 0.5 * 2 / (4 * lam)) < 1e-14


@pytest.mark.parametrize("vf,sf", [(3, 0), (4, 3), (3, 3), (5, 0), (5, 1)])
def test_free_stream_and_conservation_other_split_forms(orc, vf, sf):
    """Kennedy-Gruber / Pirozzoli volume fluxes with LLF / HLL faces: free stream preserved
    on the warped mesh, total mass / momentum / energy conserved on the periodic box."""
    o, u = _tgv_oracle(orc, 3, 3, volume_flux=vf, surface_flux=sf)
    const = np.array([1.1, 0.3, -0.2, 0.5, 80.0])
    r = o.rhs(np.broadcast_to(const[None, :, None], u.shape).copy())
    scale = np.abs(const).max() * np.abs(o.Ja).max() / o.J.min() * 9
    assert np.abs(r).max() < 1e-13 * scale
    u = o.prim_to_cons(cases.perturbed_state(cases.tgv(orc.lgl(3)[0], 3, warp=0.1)[3], 4))
    r = o.rhs(u)
    x, w = orc.lgl(3)
    W = np.einsum("i,j,k->kji", w, w, w).reshape(-1)[None, :] * o.J
    tot = np.einsum("kn,kvn->v", W, r)
    assert np.abs(tot).max() < 1e-12 * np.abs(np.einsum("kn,kvn->v", W, np.abs(r))).max()
