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
