"""Pins of the oracle's two-point and interface fluxes (Eqs. conssymm, fluxdiff,
riemann_problem1-3) and of the logarithmic mean."""
import mpmath
import numpy as np
import pytest

import workloads as W


def _orc1(orc, dim=3, **kw):
    N = 1
    x, _ = orc.lgl(N)
    shape = (1,) * dim
    xyz, nbr, face = W.box_mesh(shape, x, (0,) * dim, (1,) * dim)
    return orc.Oracle(dim, N, xyz, nbr, face, **kw)


def _state(rng, dim, g=1.4):
    rho = rng.uniform(0.5, 2.0)
    v = rng.normal(size=dim)
    p = rng.uniform(0.5, 3.0)
    return np.concatenate([[rho], rho * v, [p / (g - 1) + 0.5 * rho * v @ v]])


def _prim(u, g=1.4):
    dim = len(u) - 2
    rho = u[0]
    v = u[1:1 + dim] / rho
    p = (g - 1) * (u[-1] - 0.5 * rho * v @ v)
    return rho, v, p


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("vf", [0, 1, 2, 3, 4, 5])
def test_volume_flux_consistency_and_symmetry(orc, dim, vf):
    o = _orc1(orc, dim, volume_flux=vf)
    rng = np.random.default_rng(vf + 10 * dim)
    for _ in range(20):
        uL, uR = _state(rng, dim), _state(rng, dim)
        n = rng.normal(size=dim)
        f = o.flux_pair(uL, uL, n, 2)
        assert np.allclose(o.flux_pair(uL, uL, n, 0), f, rtol=1e-14, atol=1e-14)
        assert np.allclose(o.flux_pair(uL, uR, n, 0), o.flux_pair(uR, uL, n, 0),
                           rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_physical_flux_textbook(orc, dim):
    o = _orc1(orc, dim)
    rng = np.random.default_rng(3)
    u = _state(rng, dim)
    n = rng.normal(size=dim)
    rho, v, p = _prim(u)
    vn = v @ n
    ref = np.concatenate([[rho * vn], rho * v * vn + p * n, [(u[-1] + p) * vn]])
    assert np.allclose(o.flux_pair(u, u, n, 2), ref, rtol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_ranocha_tadmor_entropy_conservation(orc, dim):
    """(w_R - w_L) . F#(u_L,u_R) = psi_R - psi_L with psi = rho v.n (Tadmor's condition for
    the entropy S = -rho s/(gamma-1)); a dropped or mis-signed term breaks it."""
    o = _orc1(orc, dim, volume_flux=0)
    rng = np.random.default_rng(4)
    for close in (False, True):
        for _ in range(50):
            uL = _state(rng, dim)
            uR = uL * (1 + 1e-3 * rng.normal(size=uL.size)) if close else _state(rng, dim)
            n = rng.normal(size=dim)
            F = o.flux_pair(uL, uR, n, 0)
            wL, wR = o.entropy_vars(uL), o.entropy_vars(uR)
            psiL, psiR = uL[1:1 + dim] @ n, uR[1:1 + dim] @ n
            lhs = (wR - wL) @ F
            scale = np.abs(wR - wL) @ np.abs(F) + abs(psiR) + abs(psiL)
            assert abs(lhs - (psiR - psiL)) < 1e-12 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_entropy_variables_are_gradient_of_entropy(orc, dim):
    o = _orc1(orc, dim)
    rng = np.random.default_rng(5)
    u = _state(rng, dim)
    g = 1.4

    def S(uu):
        rho, v, p = _prim(uu)
        return -rho * (np.log(p) - g * np.log(rho)) / (g - 1)

    w = o.entropy_vars(u)
    h = 1e-6
    for i in range(u.size):
        e = np.zeros_like(u)
        e[i] = h * max(1, abs(u[i]))
        fd = (S(u + e) - S(u - e)) / (2 * e[i])
        assert abs(fd - w[i]) < 1e-7 * max(1, abs(w[i]))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("sf", [0, 1, 3])
def test_surface_flux_consistency_and_dissipation(orc, dim, sf):
    o = _orc1(orc, dim, surface_flux=sf)
    rng = np.random.default_rng(6 + sf)
    for _ in range(50):
        uL, uR = _state(rng, dim), _state(rng, dim)
        n = rng.normal(size=dim)
        assert np.allclose(o.flux_pair(uL, uL, n, 1), o.flux_pair(uL, uL, n, 2),
                           rtol=1e-13, atol=1e-13)
        if sf == 0:  # LLF produces entropy: (w_R - w_L).F* - (psi_R - psi_L) <= 0
            F = o.flux_pair(uL, uR, n, 1)
            wL, wR = o.entropy_vars(uL), o.entropy_vars(uR)
            psiL, psiR = uL[1:1 + dim] @ n, uR[1:1 + dim] @ n
            assert (wR - wL) @ F - (psiR - psiL) <= 1e-12 * (np.abs(wR - wL) @ np.abs(F))


def test_hllc_resolves_stationary_contact(orc):
    """A pure density jump at rest: HLLC returns the exact flux (0, p n, 0); LLF does not."""
    g = 1.4
    n = np.array([0.3, -1.2, 0.5])
    p = 1.7
    uL = np.array([1.0, 0, 0, 0, p / (g - 1)])
    uR = np.array([0.125, 0, 0, 0, p / (g - 1)])
    exact = np.concatenate([[0], p * n, [0]])
    hllc = _orc1(orc, 3, surface_flux=1).flux_pair(uL, uR, n, 1)
    llf = _orc1(orc, 3, surface_flux=0).flux_pair(uL, uR, n, 1)
    assert np.allclose(hllc, exact, atol=1e-14)
    assert np.abs(llf - exact).max() > 0.1


def test_hllc_upwinds_supersonic_flow(orc):
    o = _orc1(orc, 2, surface_flux=1)
    g = 1.4
    uL = np.array([1.0, 3.0, 0.0, 1.0 / (g - 1) + 4.5])  # u = 3 > c ~ 1.18
    uR = np.array([0.5, 1.0, 0.2, 0.4 / (g - 1) + 1.04])
    n = np.array([2.0, 0.0])
    assert np.allclose(o.flux_pair(uL, uR, n, 1), o.flux_pair(uL, uL, n, 2), rtol=1e-14)
    assert np.allclose(o.flux_pair(uR, uL, -n, 1), o.flux_pair(uL, uL, -n, 2), rtol=1e-14)


def test_ln_mean_branches(orc):
    mpmath.mp.dps = 40
    rng = np.random.default_rng(7)
    for _ in range(200):
        x = rng.uniform(0.1, 10)
        y = x * np.exp(rng.normal() * rng.choice([1e-6, 1e-3, 1e-2, 0.3, 2]))
        exact = (mpmath.mpf(y) - mpmath.mpf(x)) / mpmath.log(mpmath.mpf(y) / mpmath.mpf(x))
        assert abs(orc.ln_mean(x, y) - float(exact)) < 4e-15 * float(exact)
    assert orc.ln_mean(2.5, 2.5) == 2.5
    # both branches agree at the switch point |x-y|^2/(x+y)^2 = 1e-4
    x = 1.0
    y = (1 + 1e-2) / (1 - 1e-2)
    lo, hi = orc.ln_mean(x, y * (1 - 1e-9)), orc.ln_mean(x, y * (1 + 1e-9))
    assert abs(hi - lo) < 1e-8 * lo


@pytest.mark.parametrize("vf", [0, 3, 4])
def test_kinetic_energy_preserving_momentum(orc, vf):
    """Ranocha, Kennedy-Gruber and Pirozzoli fluxes share the kinetic-energy-preserving
    momentum flux f_rho {{v}} + {{p}} n; KG and Pirozzoli carry f_rho = {{rho}} {{v.n}}."""
    o = _orc1(orc, 3, volume_flux=vf)
    rng = np.random.default_rng(30 + vf)
    for _ in range(20):
        uL, uR = _state(rng, 3), _state(rng, 3)
        n = rng.normal(size=3)
        f = o.flux_pair(uL, uR, n, 0)
        (rL, vL, pL), (rR, vR, pR) = _prim(uL), _prim(uR)
        assert np.allclose(f[1:4], f[0] * 0.5 * (vL + vR) + 0.5 * (pL + pR) * n, rtol=1e-13, atol=1e-13)
        if vf:
            assert abs(f[0] - 0.5 * (rL + rR) * 0.5 * (vL + vR) @ n) < 1e-13 * (1 + abs(f[0]))
            h = (lambda u, r, p: (u[-1] + p) / r)
            e = (lambda u, r: u[-1] / r)
            fe = (f[0] * 0.5 * (e(uL, rL) + e(uR, rR)) + 0.5 * (pL + pR) * 0.5 * (vL + vR) @ n if vf == 3
                  else f[0] * 0.5 * (h(uL, rL, pL) + h(uR, rR, pR)))
            assert abs(f[4] - fe) < 1e-13 * (1 + abs(fe))


def test_hll_stationary_contact_and_upwinding(orc):
    """HLL with the Davis speeds: for a density jump at rest the speeds are -+c_max|n| and
    HLL reduces to LLF, mass flux -c_max |n| (rho_R - rho_L) / 2; supersonic flow upwinds."""
    g = 1.4
    n = np.array([0.3, -1.2, 0.5])
    p = 1.7
    uL = np.array([1.0, 0, 0, 0, p / (g - 1)])
    uR = np.array([0.125, 0, 0, 0, p / (g - 1)])
    hll = _orc1(orc, 3, surface_flux=3).flux_pair(uL, uR, n, 1)
    llf = _orc1(orc, 3, surface_flux=0).flux_pair(uL, uR, n, 1)
    cmax = np.sqrt(g * p / 0.125)
    assert np.allclose(hll, llf, rtol=1e-13, atol=1e-13)
    assert abs(hll[0] + 0.5 * cmax * np.linalg.norm(n) * (0.125 - 1.0)) < 1e-13
    o = _orc1(orc, 2, surface_flux=3)
    uL = np.array([1.0, 3.0, 0.0, 1.0 / (g - 1) + 4.5])
    uR = np.array([0.5, 1.0, 0.2, 0.4 / (g - 1) + 1.04])
    n2 = np.array([2.0, 0.0])
    assert np.allclose(o.flux_pair(uL, uR, n2, 1), o.flux_pair(uL, uL, n2, 2), rtol=1e-14)


def _split_form_derivative(vf, U, n, D, g=1.4):
    """The split-form derivative each named two-point flux stands for (Gassner, Winters and
    Kopriva's product-rule splittings): with constant metrics n, flux differencing
    2 sum_l D_il F#(U_i, U_l) equals, for every D with zero row sums,
      {{a}}{{b}}      ->  (D(ab) + a Db + b Da) / 2
      {{a}}{{b}}{{c}} ->  (D(abc) + a D(bc) + b D(ac) + c D(ab) + ab Dc + ac Db + bc Da) / 4
      {{a}}           ->  Da,   {{a}}  v_L.v_R / 2 with a = rho v.n  ->  (a v.Dv + v.D(a v)) / 2.
    Written here from the splittings, not from the two-point formulas."""
    dim = U.shape[1] - 2
    rho, m, E = U[:, 0], U[:, 1:1 + dim], U[:, -1]
    v = m / rho[:, None]
    p = (g - 1) * (E - 0.5 * rho * (v * v).sum(1))
    vn = v @ n
    s2 = lambda a, b: 0.5 * (D @ (a * b) + a * (D @ b) + b * (D @ a))
    s3 = lambda a, b, c: 0.25 * (D @ (a * b * c) + a * (D @ (b * c)) + b * (D @ (a * c)) + c * (D @ (a * b))
                                 + a * b * (D @ c) + a * c * (D @ b) + b * c * (D @ a))
    out = np.zeros_like(U)
    if vf == 1:      # Ducros: every conserved quantity times v.n, pressure in divergence form
        out[:, 0] = s2(rho, vn)
        for d in range(dim):
            out[:, 1 + d] = s2(m[:, d], vn) + (D @ p) * n[d]
        out[:, -1] = s2(E + p, vn)
    elif vf == 2:    # standard DG: the divergence of the flux
        out[:, 0] = D @ (rho * vn)
        for d in range(dim):
            out[:, 1 + d] = D @ (m[:, d] * vn + p * n[d])
        out[:, -1] = D @ ((E + p) * vn)
    elif vf in (3, 4):  # Kennedy-Gruber / Pirozzoli: cubic splits of rho (v.n) phi
        out[:, 0] = s2(rho, vn)
        for d in range(dim):
            out[:, 1 + d] = s3(rho, vn, v[:, d]) + (D @ p) * n[d]
        out[:, -1] = s3(rho, vn, E / rho) + s2(p, vn) if vf == 3 else s3(rho, vn, (E + p) / rho)
    elif vf == 5:    # Morinishi: mass and enthalpy in divergence form, skew momentum and KE
        mn = m @ n
        out[:, 0] = D @ mn
        for d in range(dim):
            out[:, 1 + d] = s2(mn, v[:, d]) + (D @ p) * n[d]
        ke = 0.5 * ((mn[:, None] * v) * (D @ v)).sum(1) + 0.5 * (v * (D @ (mn[:, None] * v))).sum(1)
        out[:, -1] = g / (g - 1) * (D @ (p * vn)) + ke
    return out


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("vf", [1, 2, 3, 4, 5])
def test_two_point_flux_is_its_split_form(orc, dim, vf):
    """Flux differencing with each two-point flux reproduces its split-form derivative
    (Eq. fluxdiffcons with the forms listed beside it) on a line of random states."""
    o = _orc1(orc, dim, volume_flux=vf)
    rng = np.random.default_rng(70 + vf + 10 * dim)
    n_pts = 6
    U = np.array([_state(rng, dim) for _ in range(n_pts)])
    D = rng.normal(size=(n_pts, n_pts))
    D -= D.mean(1, keepdims=True)   # zero row sums: the only property the identity uses
    n = rng.normal(size=dim)
    fd = np.zeros_like(U)
    for i in range(n_pts):
        for l in range(n_pts):
            fd[i] += 2 * D[i, l] * o.flux_pair(U[i], U[l], n, 0)
    ref = _split_form_derivative(vf, U, n, D)
    assert np.allclose(fd, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
