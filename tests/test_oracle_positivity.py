"""Pins of the oracle's Zhang-Shu positivity limiter: admissible states untouched, element
means preserved, the critical node lands exactly on the bound, the pressure scaling factor
equals an independent bisection on p(ubar + t (u - ubar)) = eps, inadmissible means refused."""
import numpy as np
import pytest

import cases

GAMMA = 1.4


def _problem(orc_mod, warp=0.1):
    xo, _ = orc_mod.lgl(3)
    xyz, nbr, face, w = cases.tgv(xo, 2, warp=warp)
    o = orc_mod.Oracle(3, 3, xyz, nbr, face)
    return o, o.prim_to_cons(w)


def _weights(o, xo_w):
    w3 = np.einsum("i,j,k->kji", xo_w, xo_w, xo_w).reshape(-1)  # node = i + 4 j + 16 k
    return w3[None, :] * o.J


def _pressure(u):
    return (GAMMA - 1.0) * (u[:, 4] - 0.5 * (u[:, 1] ** 2 + u[:, 2] ** 2 + u[:, 3] ** 2) / u[:, 0])


def _means(o, u):
    import oracle
    _, w = oracle.lgl(3)
    W = _weights(o, w)
    return np.einsum("kn,kvn->kv", W, u) / W.sum(1)[:, None]


def test_admissible_state_is_untouched():
    import oracle
    o, u = _problem(oracle)
    v, n = o.positivity(u, 1e-10)
    assert n == 0 and np.array_equal(v, u)


def test_negative_density_is_lifted_to_the_bound_keeping_the_mean():
    import oracle
    o, u = _problem(oracle)
    u = u.copy()
    # density below the bound at one node of element 3, at rest, positive energy: only the
    # density step acts
    eps = 1e-6
    u[3, 0, 5] = 1e-9
    u[3, 1:4, 5] = 0.0
    v, n = o.positivity(u, eps)
    assert n == 1
    assert np.allclose(_means(o, v), _means(o, u), rtol=1e-13, atol=1e-13)
    assert abs(v[3, 0].min() - eps) < 1e-14          # the critical node sits on the bound
    assert np.array_equal(v[np.arange(8) != 3], u[np.arange(8) != 3])
    assert _pressure(v).min() >= eps * (1 - 1e-9)


def test_negative_pressure_scaling_matches_bisection():
    import oracle
    o, u = _problem(oracle)
    u = u.copy()
    k, node = 6, 21
    u[k, 4, node] -= 1.3 * _pressure(u)[k, node] / (GAMMA - 1.0)   # p -> -0.3 p there
    eps = 1e-3
    v, n = o.positivity(u, eps)
    assert n == 1
    ubar = _means(o, u)[k]
    # independent root of p(ubar + t (u_i - ubar)) = eps by bisection
    d = u[k, :, node] - ubar
    lo, hi = 0.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        s = ubar + mid * d
        p = (GAMMA - 1.0) * (s[4] - 0.5 * (s[1] ** 2 + s[2] ** 2 + s[3] ** 2) / s[0])
        lo, hi = (mid, hi) if p > eps else (lo, mid)
    theta = 0.5 * (lo + hi)
    expect = ubar[:, None] + theta * (u[k] - ubar[:, None])
    assert np.allclose(v[k], expect, rtol=1e-12, atol=1e-12)
    assert abs(_pressure(v)[k].min() - eps) < 1e-10
    assert np.allclose(_means(o, v), _means(o, u), rtol=1e-13, atol=1e-13)


def test_inadmissible_mean_is_refused():
    import oracle
    o, u = _problem(oracle)
    u = u.copy()
    u[2, 0] = -1.0
    with pytest.raises(ValueError):
        o.positivity(u, 1e-8)


def test_both_steps_leave_an_admissible_element_with_the_same_mean():
    import oracle
    o, u = _problem(oracle)
    u = u.copy()
    u[3, 0, 5] = -0.2           # negative density, momentum kept: both steps act
    eps = 1e-6
    v, n = o.positivity(u, eps)
    assert n == 1
    assert np.allclose(_means(o, v), _means(o, u), rtol=1e-13, atol=1e-13)
    assert v[:, 0].min() >= eps * (1 - 1e-12)
    assert _pressure(v).min() >= eps * (1 - 1e-9)
    # the pressure bound is the active one: some node sits on it
    assert abs(_pressure(v)[3].min() - eps) < 1e-9


# ---------------------------------------------------------------- mixtures
T_FLOOR = 200.0


def _mix_problem(orc_mod, seed=7):
    import workloads as W
    x, _ = orc_mod.lgl(3)
    xyz, nbr, face = W.box_mesh((3, 2, 2), x, (-np.pi,) * 3, (np.pi,) * 3, periodic=True, warp=0.1)
    sp = W.species_table()
    w = W.mixture_primitive(xyz, rho=0.1, vel=(300.0, -50.0, 20.0), T=1500.0, seed=seed)
    o = orc_mod.Oracle(3, 3, xyz, nbr, face, n_species=5, volume_flux=orc_mod.VF_DUCROS, species=sp)
    return o, sp, w


def _energy_at(sp, rs, T):
    """rho e(T) of a node with partial densities rs (the e_s(T) of the species table)."""
    RU = 8.314462618
    e = 0.0
    for s in range(len(rs)):
        a = sp[s, 1:]
        h = a[0] * T + a[1] * T ** 2 / 2 + a[2] * T ** 3 / 3 + a[3] * T ** 4 / 4 + a[4] * T ** 5 / 5 + a[5]
        e += rs[s] * RU / sp[s, 0] * (h - T)
    return e


def _mix_means(o, u):
    import oracle
    _, w = oracle.lgl(3)
    Wt = _weights(o, w)
    return np.einsum("kn,kvn->kv", Wt, u) / Wt.sum(1)[:, None]


def test_mixture_admissible_state_is_untouched():
    import oracle
    o, sp, w = _mix_problem(oracle)
    u = o.prim_to_cons(w)
    v, n = o.positivity(u, 1e-8)
    assert n == 0 and np.array_equal(v, u)


def test_mixture_negative_partial_density_is_lifted_keeping_the_means():
    """A negative partial density at one node: all species of the element move toward their
    means by one factor, the critical species lands on the floor, the means are kept."""
    import oracle
    o, sp, w = _mix_problem(oracle)
    u = o.prim_to_cons(w)
    k, node, s = 2, 17, 3
    u[k, s, node] = -0.2 * u[k, s].mean()
    eps = 1e-6
    v, n = o.positivity(u, eps)
    assert n == 1
    assert v[:, :5].min() >= eps * (1 - 1e-12) - 1e-18
    assert abs(v[k, s, node] - eps) < 1e-12 * abs(u[k, s].mean())
    assert np.allclose(_mix_means(o, v), _mix_means(o, u), rtol=1e-13, atol=1e-14)
    others = [kk for kk in range(u.shape[0]) if kk != k]
    assert np.array_equal(v[others], u[others])
    # one common factor for the species; momentum and energy untouched by this step
    th = (v[k, :5] - _mix_means(o, u)[k, :5, None]) / (u[k, :5] - _mix_means(o, u)[k, :5, None])
    assert np.allclose(th, th[0, 0], rtol=1e-9) and np.array_equal(v[k, 5:], u[k, 5:])


def _excess(sp, uu):
    """rho (e - e(T_floor)) at every node of uu [..., 9, np] (rho e from the conserved state;
    e(T) written out from the species table here): >= 0 exactly when T >= T_floor."""
    rs = uu[..., :5, :]
    rho = rs.sum(-2)
    m2 = (uu[..., 5:8, :] ** 2).sum(-2)
    rho_e = uu[..., 8, :] - 0.5 * m2 / rho
    ef = np.array([_energy_at(sp, np.eye(5)[s], T_FLOOR) for s in range(5)])
    return rho_e - np.tensordot(ef, rs, axes=([0], [-2]))


def test_mixture_temperature_floor_matches_bisection():
    """A node below the temperature floor (150 K): the element moves toward its mean by the
    factor at which that node's internal energy reaches e(T_floor), found here by bisection;
    afterwards no node lies below the floor."""
    import oracle
    o, sp, w = _mix_problem(oracle)
    u = o.prim_to_cons(w)
    k, node = 5, 30
    rs, m = u[k, :5, node], u[k, 5:8, node]
    u[k, 8, node] = _energy_at(sp, rs, 150.0) + 0.5 * (m @ m) / rs.sum()
    assert _excess(sp, u[k])[node] < 0
    v, n = o.positivity(u, 1e-8)
    assert n == 1
    scale = np.abs(u[k, 8]).max()
    assert _excess(sp, v).min() > -1e-12 * scale
    assert abs(_excess(sp, v[k])[node]) < 1e-10 * scale     # the critical node on the floor
    ubar = _mix_means(o, u)[k]
    lo, hi = 0.0, 1.0   # excess(0) > 0, excess(1) < 0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        uu = ubar[:, None] + mid * (u[k] - ubar[:, None])
        if _excess(sp, uu)[node] >= 0:
            lo = mid
        else:
            hi = mid
    th = (v[k, 8, node] - ubar[8]) / (u[k, 8, node] - ubar[8])
    assert abs(th - lo) < 1e-9
    assert np.allclose(_mix_means(o, v), _mix_means(o, u), rtol=1e-13, atol=1e-14)


def test_mixture_inadmissible_mean_is_refused():
    import oracle
    o, sp, w = _mix_problem(oracle)
    u = o.prim_to_cons(w)
    k = 1
    for node in range(u.shape[2]):   # the whole element below the floor
        rs, m = u[k, :5, node], u[k, 5:8, node]
        u[k, 8, node] = _energy_at(sp, rs, 150.0) + 0.5 * (m @ m) / rs.sum()
    with pytest.raises(ValueError):
        o.positivity(u, 1e-8)
