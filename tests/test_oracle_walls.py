"""Pins of the oracle's viscous boundary conditions (no-slip adiabatic and isothermal walls,
supersonic inflow and outflow for Navier-Stokes): steady states, the Couette shear whose
only right-hand side is viscous heating, exact mass and energy conservation in a closed
adiabatic box, the wall heat flux of an isothermal wall from the BR1 lifting, and the BR1
boundary values seen in the gradients."""
import numpy as np
import pytest

import workloads as W

INFLOW, OUTFLOW, SLIP, NOSLIP, ISOTHERMAL = 1, 2, 3, 4, 5
G_, PR = 1.4, 0.72


def _channel(orc, N, kinds, prims, shape=(2, 3, 2), H=1.5, warp=0.0):
    """Periodic in x and z, bounded in y in [0, H]: bc id 0 at y = 0, id 1 at y = H."""
    x, _ = orc.lgl(N)
    xyz, nbr, face = W.box_mesh(shape, x, (0.0, 0.0, 0.0), (2.0, H, 1.0),
                                periodic=(True, False, True), bc_ids=[9, 9, 0, 1, 9, 9], warp=warp)
    return x, xyz, nbr, face, dict(bc_kind=list(kinds), bc_prim=np.array(prims, dtype=float))


def _state(xyz, rho=1.0, vel=(0.0, 0.0, 0.0), p=1.0):
    K, _, npn = xyz.shape
    w = np.empty((K, 5, npn))
    w[:, 0] = rho
    for d in range(3):
        w[:, 1 + d] = vel[d]
    w[:, 4] = p
    return w


def _weights(orc, o, N):
    _, wq = orc.lgl(N)
    return np.einsum("i,j,k->kji", wq, wq, wq).reshape(-1)[None, :] * o.J


@pytest.mark.parametrize("kinds", [(NOSLIP, NOSLIP), (ISOTHERMAL, ISOTHERMAL), (INFLOW, OUTFLOW),
                                   (NOSLIP, OUTFLOW)])
def test_rest_state_is_steady(orc, kinds):
    """Fluid at rest at uniform temperature (isothermal walls at that temperature, inflow
    state equal to it): the right-hand side vanishes."""
    N = 3
    rest = [1.3, 0.0, 0.0, 0.0, 0.9]
    x, xyz, nbr, face, bc = _channel(orc, N, kinds, [rest, rest])
    o = orc.Oracle(3, N, xyz, nbr, face, equations=1, mu=0.05, Pr=PR, **bc)
    u = o.prim_to_cons(_state(xyz, 1.3, p=0.9))
    assert np.abs(o.rhs(u)).max() < 1e-13


@pytest.mark.parametrize("wall", [NOSLIP, ISOTHERMAL])
def test_couette_shear_heats_uniformly(orc, wall):
    """u = U y / H over a no-slip wall at y = 0 (outflow at y = H), uniform rho and p: the
    shear stress mu U / H is uniform, so momentum does not change and the energy grows at
    the viscous heating rate mu (U / H)^2 everywhere, wall nodes included."""
    N, H, U, mu, p0 = 3, 1.5, 0.4, 0.03, 1.0
    wall_state = [1.0, 0.0, 0.0, 0.0, p0]      # isothermal wall at the fluid's temperature
    x, xyz, nbr, face, bc = _channel(orc, N, (wall, OUTFLOW), [wall_state, wall_state], H=H)
    o = orc.Oracle(3, N, xyz, nbr, face, equations=1, mu=mu, Pr=PR, **bc)
    w = _state(xyz, 1.0, p=p0)
    w[:, 1] = U * xyz[:, 1] / H
    r = o.rhs(o.prim_to_cons(w))
    assert np.abs(r[:, :4]).max() < 1e-13
    assert np.abs(r[:, 4] - mu * (U / H) ** 2).max() < 1e-13


def test_closed_adiabatic_box_conserves_mass_and_energy(orc):
    """All six sides no-slip adiabatic walls, a rough flow on the warped box: total mass and
    total energy are conserved to rounding (no mass or energy crosses an adiabatic wall)."""
    N = 3
    x, _ = orc.lgl(N)
    xyz, nbr, face = W.box_mesh((3, 3, 3), x, (-np.pi,) * 3, (np.pi,) * 3, periodic=False,
                                bc_ids=[0] * 6, warp=0.1)
    o = orc.Oracle(3, N, xyz, nbr, face, equations=1, mu=0.02, Pr=PR,
                   bc_kind=[NOSLIP], bc_prim=np.array([[1.0, 0, 0, 0, 1.0]]))
    w = W.tgv_primitive(xyz, G_, 0.3)
    w *= 1 + 0.05 * np.random.default_rng(1).uniform(-1, 1, size=w.shape)
    r = o.rhs(o.prim_to_cons(w))
    M = _weights(orc, o, N)
    tot = np.einsum("kn,kvn->v", M, r)
    scale = np.einsum("kn,kvn->v", M, np.abs(r))
    assert abs(tot[0]) < 1e-12 * scale[0] and abs(tot[4]) < 1e-12 * scale[4]
    assert abs(tot[1]) > 1e-6 * scale[1]        # momentum is not conserved: wall forces


def test_isothermal_wall_heat_flux(orc):
    """Fluid at rest at theta = p/rho between two isothermal walls at theta_w: BR1 lifts the
    jump theta_w - theta into the wall-node gradient, d theta/dn = (2/h)(theta_w - theta)/w_0,
    so the total energy grows at 2 kappa A (2/h)(theta_w - theta)/w_0 (A the wall area,
    kappa = mu gamma / ((gamma - 1) Pr), w_0 = 2 / (N (N+1))); mass and momentum stay."""
    N, H, mu = 3, 1.5, 0.05
    shape = (2, 3, 2)
    p, rho, th_w = 0.8, 1.0, 1.1
    wall = [1.0, 0.0, 0.0, 0.0, th_w]          # T_wall from the bc state's p / rho
    x, xyz, nbr, face, bc = _channel(orc, N, (ISOTHERMAL, ISOTHERMAL), [wall, wall], shape=shape, H=H)
    o = orc.Oracle(3, N, xyz, nbr, face, equations=1, mu=mu, Pr=PR, **bc)
    r = o.rhs(o.prim_to_cons(_state(xyz, rho, p=p)))
    M = _weights(orc, o, N)
    tot = np.einsum("kn,kvn->v", M, r)
    h = H / shape[1]
    w0 = 2.0 / (N * (N + 1))
    kappa = mu * G_ / ((G_ - 1) * PR)
    expect = 2 * kappa * (2.0 * 1.0) * (2 / h) * (th_w - p / rho) / w0
    assert abs(tot[4] / expect - 1) < 1e-12
    assert np.abs(tot[:4]).max() < 1e-12 * abs(expect)
    # an adiabatic wall passes no heat
    bc["bc_kind"] = [NOSLIP, NOSLIP]
    o2 = orc.Oracle(3, N, xyz, nbr, face, equations=1, mu=mu, Pr=PR, **bc)
    assert np.abs(o2.rhs(o2.prim_to_cons(_state(xyz, rho, p=p)))).max() < 1e-13


def test_boundary_values_in_the_gradients(orc):
    """Uniform slip velocity U and temperature theta: the BR1 gradient is zero except at
    wall nodes, where it is (2/h) (W* - W) / w_0 times the outward sign: no-slip W* = 0 for
    the velocity, theta_w on the isothermal wall (y = 0), theta on the adiabatic one (y = H);
    at a supersonic inflow W* is the mean of interior and external values."""
    N, H = 3, 1.5
    shape = (2, 3, 2)
    U, p, th_w = 0.3, 0.9, 1.2
    h = H / shape[1]
    w0 = 2.0 / (N * (N + 1))
    x, xyz, nbr, face, bc = _channel(orc, N, (ISOTHERMAL, NOSLIP),
                                     [[1.0, 0, 0, 0, th_w], [1.0, 0, 0, 0, 1.0]], shape=shape, H=H)
    o = orc.Oracle(3, N, xyz, nbr, face, equations=1, mu=0.01, Pr=PR, **bc)
    u = o.prim_to_cons(_state(xyz, 1.0, vel=(U, 0, 0), p=p))
    _, g = o.rhs(u, want_grad=True)                      # [K][x][c][node], c = (u, v, w, theta)
    y = xyz[:, 1]
    bottom, top = np.abs(y) < 1e-14, np.abs(y - H) < 1e-14
    dudy, dthdy = g[:, 1, 0], g[:, 1, 3]
    lift = (2 / h) / w0
    assert np.allclose(dudy[bottom], lift * U, rtol=1e-13)        # -(0 - U) at the lower side
    assert np.allclose(dudy[top], -lift * U, rtol=1e-13)          # +(0 - U) at the upper side
    assert np.allclose(dthdy[bottom], -lift * (th_w - p), rtol=1e-13)
    assert np.abs(dthdy[top]).max() < 1e-13
    inner = ~(bottom | top)
    assert np.abs(g[np.broadcast_to(inner[:, None, None, :], g.shape)]).max() < 1e-12
    # supersonic inflow at y = 0 with an external state of other velocity and temperature
    ext = [1.0, 0.5, 0.0, 0.0, 1.4]
    x, xyz, nbr, face, bc = _channel(orc, N, (INFLOW, OUTFLOW), [ext, ext], shape=shape, H=H)
    o = orc.Oracle(3, N, xyz, nbr, face, equations=1, mu=0.01, Pr=PR, **bc)
    _, g = o.rhs(o.prim_to_cons(_state(xyz, 1.0, vel=(U, 0, 0), p=p)), want_grad=True)
    assert np.allclose(g[:, 1, 0][bottom], -lift * 0.5 * (0.5 - U), rtol=1e-13)
    assert np.allclose(g[:, 1, 3][bottom], -lift * 0.5 * (1.4 - p), rtol=1e-13)
    assert np.abs(g[:, 1, 0][top]).max() < 1e-13


def test_navier_stokes_slip_wall_is_rejected(orc):
    x, xyz, nbr, face, bc = _channel(orc, 2, (SLIP, OUTFLOW), [[1.0, 0, 0, 0, 1.0]] * 2)
    o = orc.Oracle(3, 2, xyz, nbr, face, equations=1, mu=0.01, Pr=PR, **bc)
    with pytest.raises(ValueError):
        o.rhs(o.prim_to_cons(_state(xyz)))
