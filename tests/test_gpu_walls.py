"""Navier-Stokes boundaries on the GPU against the oracle: no-slip adiabatic and isothermal
walls, supersonic inflow and outflow (BR1 boundary values and boundary viscous fluxes), in
a channel, in a closed box whose edge and corner nodes lie on several walls, with
Sutherland's law, and over CK45 steps."""
import numpy as np
import pytest

import cases
import workloads as W

pytestmark = pytest.mark.gpu

INFLOW, OUTFLOW, NOSLIP, ISOTHERMAL = 1, 2, 4, 5
FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def dg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_17551_gb300 as dg
    dg.lib()
    return dg


def _channel_builder(shape=(3, 4, 2), H=1.5):
    """Periodic in x and z, walls / inflow / outflow at y = 0 (bc id 0) and y = H (id 1);
    a shear flow with a rough perturbation."""
    def build(x):
        xyz, nbr, face = W.box_mesh(shape, x, (0.0, 0.0, 0.0), (2.0, H, 1.0),
                                    periodic=(True, False, True), bc_ids=[9, 9, 0, 1, 9, 9])
        K, _, npn = xyz.shape
        w = np.empty((K, 5, npn))
        w[:, 0] = 1.0 + 0.2 * np.sin(np.pi * xyz[:, 0])
        w[:, 1] = 0.5 * xyz[:, 1] / H
        w[:, 2] = 0.05 * np.sin(np.pi * xyz[:, 0]) * np.sin(np.pi * xyz[:, 1] / H)
        w[:, 3] = 0.02
        w[:, 4] = 1.0 + 0.1 * np.cos(np.pi * xyz[:, 2])
        return xyz, nbr, face, w
    return build


def _box_builder(n=3):
    def build(x):
        xyz, nbr, face = W.box_mesh((n, n, n), x, (-np.pi,) * 3, (np.pi,) * 3, periodic=False,
                                    bc_ids=[0, 0, 1, 1, 0, 0], warp=0.1)
        return xyz, nbr, face, W.tgv_primitive(xyz, 1.4, 0.3)
    return build


WALL = [1.0, 0.0, 0.0, 0.0, 1.2]      # isothermal walls: theta_wall = p / rho = 1.2
INFLOW_STATE = [1.1, 0.3, 0.4, 0.0, 1.0]

CASES = {
    "channel_noslip_isothermal": dict(builder=_channel_builder(), kinds=[NOSLIP, ISOTHERMAL],
                                      prims=[WALL, WALL], kw={}),
    "channel_inflow_outflow": dict(builder=_channel_builder(), kinds=[INFLOW, OUTFLOW],
                                   prims=[INFLOW_STATE, INFLOW_STATE], kw={}),
    "channel_noslip_outflow_hllc": dict(builder=_channel_builder(), kinds=[NOSLIP, OUTFLOW],
                                        prims=[WALL, WALL], kw=dict(surface_flux=1)),
    "box_adiabatic_isothermal": dict(builder=_box_builder(), kinds=[NOSLIP, ISOTHERMAL],
                                     prims=[WALL, WALL], kw={}),
    "box_walls_sutherland_kg": dict(builder=_box_builder(), kinds=[ISOTHERMAL, NOSLIP],
                                    prims=[WALL, WALL],
                                    kw=dict(sutherland_s=W.SUTHERLAND_S, sutherland_rt=0.9,
                                            volume_flux=3)),
}


def _pair(dg, name, precision):
    c = CASES[name]
    return cases.Pair(c["builder"], 3, 3, precision=precision, equations=1, mu=0.02, Pr=0.72,
                      bc_kind=c["kinds"], bc_prim=np.array(c["prims"], dtype=float), **c["kw"])


def _rhs_pair(dg, pair, w_o, w_g):
    import torch
    u_o = pair.orc.prim_to_cons(w_o)
    r_o, g_o = pair.orc.rhs(u_o, want_grad=True)
    pair.gpu.set_primitive(w_g)
    dt = torch.float32 if pair.gpu.precision == dg.DG_MIXED else torch.float64
    u_d = torch.empty(pair.gpu.shape, dtype=torch.float64, device="cuda")
    dg.dg_get_state(pair.gpu.ctx, u_d)
    u_d = u_d.to(dt)
    r_d = torch.empty_like(u_d)
    dg.dg_rhs(pair.gpu.ctx, u_d, r_d)
    dg.dg_sync(pair.gpu.ctx)
    g_g = dg.dg_get_gradients(pair.gpu.ctx, g_o.shape)
    return r_d.double().cpu().numpy(), r_o, g_g, g_o


@pytest.mark.parametrize("name", sorted(CASES))
def test_rhs_and_gradients_fp64(dg, name):
    p = _pair(dg, name, dg.DG_FP64)
    try:
        w_o = cases.perturbed_state(p.mesh_o[3], 5, amp=0.05)
        w_g = cases.perturbed_state(p.mesh_g[3], 5, amp=0.05)
        r_g, r_o, g_g, g_o = _rhs_pair(dg, p, w_o, w_g)
        gerr = np.linalg.norm(g_g - g_o) / np.linalg.norm(g_o)
        assert gerr < FP64_TOL, gerr
        err = cases.field_errors(r_g, r_o, 1, 3)
        assert err.max() < FP64_TOL, err
    finally:
        p.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_rhs_mixed(dg, name):
    p = _pair(dg, name, dg.DG_MIXED)
    try:
        w_o = cases.perturbed_state(p.mesh_o[3], 5, amp=0.05)
        w_g = cases.perturbed_state(p.mesh_g[3], 5, amp=0.05)
        r_g, r_o, _, _ = _rhs_pair(dg, p, w_o, w_g)
        err = cases.field_errors(r_g, r_o, 1, 3)
        assert err.max() < 2e-4, err
    finally:
        p.close()


@pytest.mark.parametrize("precision,tol", [(0, None), (1, 1e-5)])
def test_rk_closed_box(dg, precision, tol):
    """Ten CK45 steps in the closed box (adiabatic and isothermal walls): the state matches
    the oracle's; mass stays constant in both."""
    p = _pair(dg, "box_adiabatic_isothermal", precision)
    try:
        u_o = p.orc.prim_to_cons(p.mesh_o[3])
        dt = p.orc.max_dt(u_o, 0.4)
        p.gpu.set_primitive(p.mesh_g[3])
        m0 = p.gpu.diagnostics()[3]
        p.gpu.step(10, dt_fixed=dt)
        u_g, _ = p.gpu.get_state()
        assert abs(p.gpu.diagnostics()[3] / m0 - 1) < (1e-14 if precision == 0 else 1e-6)
        u_r, _ = p.orc.step_rk(u_o, 10, dt_fixed=dt)
        err = cases.field_errors(u_g, u_r, 1, 3)
        if tol is None:  # FP64: 1e-12 or the oracle's own one-ulp floor of these 10 steps
            tol = cases.fp64_bar(cases.step_floor(p.orc, u_o, 10, dt))
        print("closed box steps error", err, "bar", tol)
        assert np.all(err < tol), (err, tol)
    finally:
        p.close()


def test_slip_wall_rejected_for_navier_stokes(dg):
    c = CASES["channel_inflow_outflow"]
    with pytest.raises(dg.DgError) as ei:
        cases.Pair(c["builder"], 3, 3, precision=0, equations=1, mu=0.02, Pr=0.72,
                   bc_kind=[3, 2], bc_prim=np.array(c["prims"], dtype=float))
    assert ei.value.code == dg.DG_EINVAL
