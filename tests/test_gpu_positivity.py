"""The Zhang-Shu positivity limiter on the GPU against the oracle: one application to a
state with planted violations (density-only and pressure) and CK45 steps of a 2D double
rarefaction in which the limiter holds the density bound every step."""
import numpy as np
import pytest

import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_17551_gb300 as dg
    dg.lib()
    return dg


def _planted(u):
    u = u.copy()
    u[3, 0, 5] = 1e-9            # density below the bound, at rest: density step only
    u[3, 1:4, 5] = 0.0
    p = 0.4 * (u[6, 4] - 0.5 * (u[6, 1] ** 2 + u[6, 2] ** 2 + u[6, 3] ** 2) / u[6, 0])
    u[6, 4, 21] -= 1.3 * p[21] / 0.4   # negative pressure: pressure step
    u[1, 0, 40] = -0.2           # negative density with momentum: both steps
    return u


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 2e-6)])
def test_limit_state_matches_oracle(dg, precision, tol):
    eps = 1e-6
    p = cases.Pair(lambda x: cases.tgv(x, 2, warp=0.1), 3, 3, precision=precision, positivity_eps=eps)
    try:
        u_o = _planted(p.orc.prim_to_cons(p.mesh_o[3]))
        v_o, n_o = p.orc.positivity(u_o, eps)
        assert n_o == 3
        p.gpu.set_state(u_o)
        dg.dg_limit_state(p.gpu.ctx)
        v_g, _ = p.gpu.get_state()
        assert dg.dg_limiter_stats(p.gpu.ctx) == 3
        err = cases.field_errors(v_g, v_o, 1, 3)
        assert err.max() < tol, err
        # bounds hold on the GPU state
        pr = 0.4 * (v_g[:, 4] - 0.5 * (v_g[:, 1] ** 2 + v_g[:, 2] ** 2 + v_g[:, 3] ** 2) / v_g[:, 0])
        assert v_g[:, 0].min() >= eps * (1 - 1e-6) and pr.min() >= eps * (1 - 1e-3)
    finally:
        p.close()


def _rarefaction(x, U=3.0):
    import workloads as W
    xyz, nbr, face = W.box_mesh((8, 4), x, (-1.0, -0.5), (1.0, 0.5), periodic=True)
    w = np.zeros((xyz.shape[0], 4, 16))
    w[:, 0] = 1.0
    w[:, 1] = np.where(xyz[:, 0, :] > 0, U, -U)
    w[:, 3] = 1.0 / 1.4
    return xyz, nbr, face, w


@pytest.mark.parametrize("precision,tol", [(0, None), (1, 1e-5)])
def test_rk_with_limiter_matches_oracle(dg, precision, tol):
    eps = 0.17  # above the flow's own minima: the limiter acts in the expansion
    p = cases.Pair(_rarefaction, 2, 3, precision=precision, alpha_max=0.5, positivity_eps=eps)
    try:
        u_o = p.orc.prim_to_cons(p.mesh_o[3])
        dt = 0.3 * p.orc.max_dt(u_o, 0.5)
        p.gpu.set_primitive(p.mesh_g[3])
        p.gpu.step(10, dt_fixed=dt)
        u_g, _ = p.gpu.get_state()
        assert dg.dg_limiter_stats(p.gpu.ctx) > 0
        u_r, _ = p.orc.step_rk(u_o, 10, dt_fixed=dt)
        if tol is None:  # FP64: 1e-12 or the oracle's own one-ulp floor of these 10 steps
            tol = cases.fp64_bar(cases.step_floor(p.orc, u_o, 10, dt))
        assert abs(u_r[:, 0].min() - eps) < 1e-12          # the oracle holds the bound
        err = cases.field_errors(u_g, u_r, 1, 2)
        print("limiter steps error", err, "bar", tol)
        assert np.all(err < tol), (err, tol)
        assert u_g[:, 0].min() >= eps * (1 - 1e-6)
    finally:
        p.close()


def _mix_box(x):
    import workloads as W
    xyz, nbr, face = W.box_mesh((3, 2, 2), x, (-np.pi,) * 3, (np.pi,) * 3, periodic=True, warp=0.1)
    w = W.mixture_primitive(xyz, rho=0.1, vel=(300.0, -50.0, 20.0), T=1500.0, seed=7)
    return xyz, nbr, face, w


def _mix_pair(dg, precision, eps):
    import workloads as W
    return cases.Pair(_mix_box, 3, 3, precision=precision, n_species=5, volume_flux=1,
                      species=W.species_table(), positivity_eps=eps)


def _energy_at(sp, rs, T):
    RU = 8.314462618
    e = 0.0
    for s in range(len(rs)):
        a = sp[s, 1:]
        h = a[0] * T + a[1] * T ** 2 / 2 + a[2] * T ** 3 / 3 + a[3] * T ** 4 / 4 + a[4] * T ** 5 / 5 + a[5]
        e += rs[s] * RU / sp[s, 0] * (h - T)
    return e


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 2e-6)])
def test_mixture_limit_state_matches_oracle(dg, precision, tol):
    """A negative partial density and a node below the temperature floor, in two elements:
    the GPU limiter gives the oracle's state and counts the two elements."""
    import workloads as W
    sp = W.species_table()
    eps = 1e-6
    p = _mix_pair(dg, precision, eps)
    try:
        u = p.orc.prim_to_cons(p.mesh_o[3])
        u[2, 3, 17] = -0.2 * u[2, 3].mean()
        rs, m = u[5, :5, 30], u[5, 5:8, 30]
        u[5, 8, 30] = _energy_at(sp, rs, 150.0) + 0.5 * (m @ m) / rs.sum()
        v_o, n_o = p.orc.positivity(u, eps)
        assert n_o == 2
        p.gpu.set_state(u)
        dg.dg_limit_state(p.gpu.ctx)
        v_g, _ = p.gpu.get_state()
        assert dg.dg_limiter_stats(p.gpu.ctx) == 2
        err = cases.field_errors(v_g, v_o, 5, 3)
        assert err.max() < tol, err
    finally:
        p.close()


@pytest.mark.parametrize("precision,tol", [(0, None), (1, 1e-5)])
def test_mixture_rk_with_limiter_matches_oracle(dg, precision, tol):
    """Three CK45 steps of the frozen mixture with a partial-density floor above the
    smallest partial densities of the state, so that the limiter acts in every stage."""
    p0 = _mix_pair(dg, 0, 0.0)
    u0 = p0.orc.prim_to_cons(p0.mesh_o[3])
    p0.close()
    eps = 1.5 * u0[:, :5].min()
    p = _mix_pair(dg, precision, eps)
    try:
        u_o = p.orc.prim_to_cons(p.mesh_o[3])
        dt = 0.3 * p.orc.max_dt(u_o, 0.5)
        p.gpu.set_primitive(p.mesh_g[3])
        p.gpu.step(3, dt_fixed=dt)
        u_g, _ = p.gpu.get_state()
        assert dg.dg_limiter_stats(p.gpu.ctx) > 0
        u_r, _ = p.orc.step_rk(u_o, 3, dt_fixed=dt)
        err = cases.field_errors(u_g, u_r, 5, 3)
        if tol is None:  # FP64: 1e-12 or the oracle's own one-ulp floor of these 3 steps
            tol = cases.fp64_bar(cases.step_floor(p.orc, u_o, 3, dt))
        print("mixture limiter steps error", err, "bar", tol)
        assert np.all(err < tol), (err, tol)
    finally:
        p.close()
