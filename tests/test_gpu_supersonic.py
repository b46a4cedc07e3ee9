"""The supersonic Taylor-Green ingredients on the GPU against the oracle: Sutherland's law
(Eq. sutherland) in the viscous fluxes and the viscous time step, the pressure shock
indicator with subcell blending, the mu(T)-weighted dissipation integrals (Eqs. TGV_SD,
TGV_DD), and CK45 steps with the positivity limiter on top."""
import numpy as np
import pytest

import cases
import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def dg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_17551_gb300 as dg
    dg.lib()
    return dg


def _builder(shape, warp=0.1):
    return lambda x: cases.supersonic_tgv(x, None, warp=warp, shape=shape)


def _pair(dg, precision, shape=(3, 3, 5), N=3, alpha_max=0.5, **kw):
    phys = dict(W.supersonic_tgv_physics())
    phys.update(kw)
    return cases.Pair(_builder(shape), 3, N, precision=precision, equations=1,
                      alpha_max=alpha_max, **phys)


def _rhs_pair(dg, pair, w_o, w_g):
    import torch
    u_o = pair.orc.prim_to_cons(w_o)
    r_o, a_o = pair.orc.rhs(u_o, want_alpha=True)
    pair.gpu.set_primitive(w_g)
    dt = torch.float32 if pair.gpu.precision == dg.DG_MIXED else torch.float64
    u_d = torch.empty(pair.gpu.shape, dtype=torch.float64, device="cuda")
    dg.dg_get_state(pair.gpu.ctx, u_d)
    u_d = u_d.to(dt)
    r_d = torch.empty_like(u_d)
    dg.dg_rhs(pair.gpu.ctx, u_d, r_d)
    dg.dg_sync(pair.gpu.ctx)
    return r_d.double().cpu().numpy(), r_o, a_o


def _rough(w, seed, amp=0.15):
    """A rough perturbation (p and rho independently) so that blending and a varying
    temperature are both exercised."""
    return cases.perturbed_state(w, seed=seed, amp=amp)


@pytest.mark.parametrize("precision,tol,atol_a", [(0, FP64_TOL, 1e-14), (1, 2e-4, 1e-4)])
@pytest.mark.parametrize("N,shape", [(3, (3, 3, 5)), (4, (2, 3, 3))])
def test_rhs_sutherland_pressure_indicator(dg, precision, tol, atol_a, N, shape):
    p = _pair(dg, precision, shape=shape, N=N)
    try:
        r_g, r_o, a_o = _rhs_pair(dg, p, _rough(p.mesh_o[3], 8), _rough(p.mesh_g[3], 8))
        a_g = dg.dg_get_alpha(p.gpu.ctx, p.K)
        assert (a_o > 0).sum() > 3
        assert np.allclose(a_g, a_o, rtol=1e-12, atol=atol_a)
        err = cases.field_errors(r_g, r_o, 1, 3)
        assert err.max() < tol, err
    finally:
        p.close()


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, 2e-4)])
def test_rhs_sutherland_without_blending(dg, precision, tol):
    """Sutherland's law alone (no blending), Pirozzoli volume flux and HLLC faces."""
    p = _pair(dg, precision, alpha_max=0.0, volume_flux=4, surface_flux=1)
    try:
        r_g, r_o, _ = _rhs_pair(dg, p, _rough(p.mesh_o[3], 9, 0.05), _rough(p.mesh_g[3], 9, 0.05))
        err = cases.field_errors(r_g, r_o, 1, 3)
        assert err.max() < tol, err
    finally:
        p.close()


def test_viscous_time_step_and_integrals(dg):
    """The device time step (viscous bound with mu(T) dominating at a large viscosity) and
    the dissipation integrals match the oracle's."""
    p = _pair(dg, 0, alpha_max=0.0, mu=0.5)
    try:
        w_o, w_g = _rough(p.mesh_o[3], 10), _rough(p.mesh_g[3], 10)
        u_o = p.orc.prim_to_cons(w_o)
        p.gpu.set_primitive(w_g)
        d_g = p.gpu.diagnostics()
        d_o = p.orc.diagnostics(u_o)
        assert d_o[6] > 0 and d_o[7] > 0
        assert np.allclose(d_g, d_o, rtol=1e-12, atol=1e-14), (d_g, d_o)
        dt_g = p.gpu.step(1, cfl=0.5)
        dt_o = p.orc.max_dt(u_o, 0.5)
        assert abs(dt_g / dt_o - 1) < 1e-12, (dt_g, dt_o)
    finally:
        p.close()


@pytest.mark.parametrize("precision,tol", [(0, None), (1, 1e-5)])
def test_rk_supersonic_tgv_with_limiter(dg, precision, tol):
    """Ten CK45 steps of the supersonic TGV on the warped box: Sutherland's law, pressure
    indicator blending and the positivity limiter (a bound above the initial minimum
    pressure p_o - 3/8 = 0.0821, so that it acts)."""
    eps = 0.09
    p = _pair(dg, precision, positivity_eps=eps)
    try:
        u_o = p.orc.prim_to_cons(p.mesh_o[3])
        dt = 0.5 * p.orc.max_dt(u_o, 0.5)
        p.gpu.set_primitive(p.mesh_g[3])
        p.gpu.step(10, dt_fixed=dt)
        u_g, _ = p.gpu.get_state()
        assert dg.dg_limiter_stats(p.gpu.ctx) > 0
        u_r, _ = p.orc.step_rk(u_o, 10, dt_fixed=dt)
        err = cases.field_errors(u_g, u_r, 1, 3)
        if tol is None:  # FP64: 1e-12 or the oracle's own one-ulp floor of these 10 steps
            tol = cases.fp64_bar(cases.step_floor(p.orc, u_o, 10, dt))
        print("supersonic limiter steps error", err, "bar", tol)
        assert np.all(err < tol), (err, tol)
    finally:
        p.close()
