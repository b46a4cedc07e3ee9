"""Pins of the supersonic Taylor-Green ingredients in the oracle: Sutherland's law
(Eq. sutherland) in the viscous fluxes and the viscous time step, the mu(T)-weighted
dissipation integrals of Eqs. TGV_SD and TGV_DD, the shock indicator on pressure, and the
initial state.  Sutherland's law is evaluated here in its textbook dimensional form,
mu / mu_ref = (T / T_ref)^(3/2) (T_ref + S) / (T + S) with T_ref = 273.15 K, S = 110.4 K
(whose ratio S / T_ref = 0.4042 is the constant the paper prints)."""
import numpy as np
import pytest

import cases
import workloads as W

T_REF, S_K = 273.15, 110.4
S_RATIO = S_K / T_REF


def _textbook_mu_ratio(theta):
    T = theta * T_REF
    return (T / T_REF) ** 1.5 * (T_REF + S_K) / (T + S_K)


def _mesh(orc, N, n_el, warp=0.1):
    x, _ = orc.lgl(N)
    return x, W.box_mesh((n_el,) * 3, x, (-np.pi,) * 3, (np.pi,) * 3, periodic=True, warp=warp)


def _uniform_theta_state(orc, x, xyz, theta, rt, seed=5):
    """TGV velocities, a rough positive density and p = theta rt rho (uniform p/rho)."""
    w = cases.perturbed_state(W.tgv_primitive(xyz, 1.4, 0.5), seed, amp=0.1)
    w[:, 4] = theta * rt * w[:, 0]
    return w


def test_paper_constant_is_the_textbook_ratio():
    assert abs(S_RATIO - W.SUTHERLAND_S) < 1e-4
    assert _textbook_mu_ratio(1.0) == 1.0


@pytest.mark.parametrize("theta", [1.0, 1.7, 0.6])
def test_uniform_temperature_equals_constant_viscosity(orc, theta):
    """With p/rho uniform, the Sutherland RHS is the constant-viscosity RHS at mu(T)."""
    N, mu, rt = 3, 0.02, 0.4
    x, (xyz, nbr, face) = _mesh(orc, N, 3)
    w = _uniform_theta_state(orc, x, xyz, theta, rt)
    os_ = orc.Oracle(3, N, xyz, nbr, face, equations=1, mu=mu, Pr=0.72,
                     sutherland_s=S_RATIO, sutherland_rt=rt)
    oc = orc.Oracle(3, N, xyz, nbr, face, equations=1, mu=mu * _textbook_mu_ratio(theta), Pr=0.72)
    u = os_.prim_to_cons(w)
    rs, rc = os_.rhs(u), oc.rhs(u)
    err = cases.field_errors(rs, rc, 1, 3)
    assert err.max() < 1e-13, err
    ds, dc = os_.diagnostics(u), oc.diagnostics(u)
    ratio = _textbook_mu_ratio(theta)
    # the weighted integrals carry mu(T)/mu: the constant-viscosity oracle has mu(T)/mu = 1
    assert abs(ds[6] / dc[6] - ratio) < 1e-13 and abs(ds[7] / dc[7] - ratio) < 1e-13
    assert np.allclose(ds[:6], dc[:6], rtol=1e-15, atol=0)


def test_viscous_time_step_takes_the_node_viscosity(orc):
    """On a Cartesian box sum_i |Ja^i|^2 / J^2 = 3 / (h/2)^2; with the viscous bound
    dominating, dt = cfl 4 / ((N+1)^2 max_node gamma mu(T)/(Pr rho) 3/(h/2)^2), here with
    a temperature that varies from node to node."""
    N, n_el, mu, rt, cfl, g, Pr = 3, 2, 3.0, 0.5, 0.4, 1.4, 0.72
    x, (xyz, nbr, face) = _mesh(orc, N, n_el, warp=0.0)
    w = _uniform_theta_state(orc, x, xyz, 1.0, rt)
    w[:, 1:4] *= 1e-3
    rng = np.random.default_rng(2)
    w[:, 4] = rt * w[:, 0] * rng.uniform(0.5, 2.0, size=w[:, 0].shape)
    o = orc.Oracle(3, N, xyz, nbr, face, equations=1, mu=mu, Pr=Pr,
                   sutherland_s=S_RATIO, sutherland_rt=rt)
    u = o.prim_to_cons(w)
    h2 = np.pi / n_el
    lamv = np.max(g * mu * _textbook_mu_ratio(w[:, 4] / (w[:, 0] * rt)) / (Pr * w[:, 0])) * 3 / h2 ** 2
    c = np.sqrt(g * w[:, 4] / w[:, 0])
    lam_a = np.max(np.sum(np.abs(w[:, 1:4]), 1) + 3 * c) / h2
    dt_v = cfl * 4 / ((N + 1) ** 2 * lamv)
    assert dt_v < cfl * 2 / ((N + 1) * lam_a)     # the viscous bound is the one taken
    assert abs(o.max_dt(u, cfl) / dt_v - 1) < 1e-13


def test_dissipation_integrals_closed_forms(orc):
    """Constant viscosity: for the TGV field (rho = 1, divergence free) int|omega|^2/|Omega|
    = 3/4 = 2 x the mass-weighted enstrophy and int (div v)^2 ~ 0; for the potential flow
    v = a (sin x, sin y, sin z) (curl free), int (div v)^2 / |Omega| = 3 a^2 / 2."""
    N = 7
    x, (xyz, nbr, face) = _mesh(orc, N, 4, warp=0.0)
    o = orc.Oracle(3, N, xyz, nbr, face, equations=1, mu=0.01)
    w = W.tgv_primitive(xyz, 1.4, 0.1)
    d = o.diagnostics(o.prim_to_cons(w))
    assert abs(d[7] - 0.75) < 1e-5 and abs(d[7] - 2 * d[1]) < 1e-14
    assert d[6] < 1e-9
    a = 0.3
    w[:, 1:4] = a * np.sin(xyz)
    d = o.diagnostics(o.prim_to_cons(w))
    assert abs(d[6] - 1.5 * a * a) < 1e-6 and d[7] < 1e-9


def test_pressure_indicator(orc):
    """rho = 1: the indicator on p equals the one on rho p bit for bit; p constant with a
    rough density: the pressure indicator sees nothing while rho p does."""
    N = 3
    x, (xyz, nbr, face) = _mesh(orc, N, 3, warp=0.1)
    o_rp = orc.Oracle(3, N, xyz, nbr, face, alpha_max=0.5)
    o_p = orc.Oracle(3, N, xyz, nbr, face, alpha_max=0.5, indicator_variable=1)
    w = cases.perturbed_state(W.tgv_primitive(xyz, 1.4, 0.3), 3, amp=0.3)
    w[:, 0] = 1.0
    u = o_p.prim_to_cons(w)
    a_p = o_p.indicator(u)
    assert np.array_equal(a_p, o_rp.indicator(u)) and a_p.max() > 0
    w = cases.perturbed_state(W.tgv_primitive(xyz, 1.4, 0.3), 4, amp=0.3)
    w[:, 4] = 2.0
    u = o_p.prim_to_cons(w)
    assert np.all(o_p.indicator(u) == 0.0) and o_rp.indicator(u).max() > 0


def test_supersonic_tgv_initial_state(orc):
    """Uniform temperature (p / rho = p_o), U_o / c_o = M = 1.25, mean pressure p_o."""
    x, (xyz, nbr, face) = _mesh(orc, 4, 2, warp=0.0)
    w = W.supersonic_tgv_primitive(xyz)
    phys = W.supersonic_tgv_physics()
    p0 = phys["sutherland_rt"]
    assert np.allclose(w[:, 4] / w[:, 0], p0, rtol=1e-15)
    assert abs(1.0 / np.sqrt(1.4 * p0) - 1.25) < 1e-14
    # the perturbation (cos 2x + cos 2y)(cos 2z + 2) / 16 spans [-3/8, 3/8], reached at nodes
    assert abs(w[:, 4].min() - (p0 - 0.375)) < 1e-14 and abs(w[:, 4].max() - (p0 + 0.375)) < 1e-14


def test_conservation_with_sutherland_and_limiter_state(orc):
    """Periodic supersonic TGV with Sutherland's law and pressure-indicator blending:
    mass, momentum and energy are conserved by the RHS."""
    N = 3
    x, (xyz, nbr, face) = _mesh(orc, N, 3, warp=0.1)
    o = orc.Oracle(3, N, xyz, nbr, face, equations=1, alpha_max=0.5, **W.supersonic_tgv_physics())
    w = cases.perturbed_state(W.supersonic_tgv_primitive(xyz), 6, amp=0.1)
    u = o.prim_to_cons(w)
    r, a = o.rhs(u, want_alpha=True)
    assert a.max() > 0
    xq, wq = orc.lgl(N)
    M = np.einsum("i,j,k->kji", wq, wq, wq).reshape(-1)[None, :] * o.J
    tot = np.einsum("kn,kvn->v", M, r)
    assert np.abs(tot).max() < 1e-12 * np.einsum("kn,kvn->v", M, np.abs(r)).max()
