"""Parity at the full bench sizes: the Navier-Stokes Taylor-Green workload on 32^3 curved
elements at N = 3 and on 16^3 at N = 7 (10.5 M DOF each), with the flux pair, viscosity and
pressure offset p0 the bench runs (the compile-time production kernel), against the FP64
oracle on the same seeded inputs, on every node.

* One right-hand side of a seeded perturbed state (the small cases' stress input) and of
  the Taylor-Green state itself: FP64 form 1e-12 relative L2 per field (the stress input)
  and within 16 times the oracle's FP64 rounding floor (the Taylor-Green state, where the
  Mach-0.1 pressure cancels to gradients of order 0.1); mixed form within 16 times the
  oracle's FP32 rounding floor per field (its own right-hand side moved by one FP32 unit
  of every state value); node by node, the stress input's largest error of a field within
  1e-10 (FP64) / 2e-3 (mixed) of that field's largest value.
* The increment u_n - u_0 of 16 CK45 steps (the bench's parity run) against the oracle's
  increment, per field, within 16 times the oracle's own increment floor of the form's
  precision (its increment moved by one unit in the last place of every initial state
  value; FP64: at least 1e-12).  The density barely changes over these steps (the initial
  velocity field is solenoidal), so its increment sits on that floor: 1.5e-9 in FP64.
* One CK45 step of the Taylor-Green state with the oracle's CFL-0.5 step (the stage-fused
  update the bench times): FP64 form 1e-12, mixed form 1e-6 relative L2 per field (the
  compensated FP32 state stays within 1e-7 of the oracle over the bench's 16 steps).

Measured on GB300 for the stress right-hand side: FP64 1.9e-13 (N = 7) and 3.1e-14
(N = 3), the largest at N = 7 set by the rounding of the metric terms.
"""
import numpy as np
import pytest

import cases

pytestmark = pytest.mark.gpu

MU = 1.0 / 1600.0
SHAPES = [(3, 32), (7, 16)]


@pytest.fixture(scope="module")
def dg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_17551_gb300 as dg
    dg.lib()
    return dg


def _pair(dg, N, n_el, precision):
    return cases.Pair(lambda x: cases.tgv(x, n_el, warp=0.1), 3, N, precision=precision,
                      equations=1, mu=MU, Pr=0.72, p_ref=cases.tgv_p0())


def _max_rel(a, ref):
    """Largest node error of each field over that field's largest magnitude."""
    nv = ref.shape[1]
    return np.array([np.abs(a[:, v] - ref[:, v]).max() / max(np.abs(ref[:, v]).max(), 1e-300)
                     for v in range(nv)])


@pytest.mark.parametrize("N,n_el", SHAPES)
@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_full_size_rhs(dg, N, n_el, form):
    import torch
    precision = dg.DG_FP64 if form == "fp64" else dg.DG_MIXED
    p = _pair(dg, N, n_el, precision)
    try:
        w_o = cases.perturbed_state(p.mesh_o[3], seed=11, amp=0.05)
        w_g = cases.perturbed_state(p.mesh_g[3], seed=11, amp=0.05)
        r_o = p.orc.rhs(p.orc.prim_to_cons(w_o))
        p.gpu.set_primitive(w_g)
        dt = torch.float32 if precision == dg.DG_MIXED else torch.float64
        u_d = torch.empty(p.gpu.shape, dtype=torch.float64, device="cuda")
        dg.dg_get_state(p.gpu.ctx, u_d)
        u_d = u_d.to(dt)
        r_d = torch.empty_like(u_d)
        dg.dg_rhs(p.gpu.ctx, u_d, r_d)
        dg.dg_sync(p.gpu.ctx)
        r_g = r_d.double().cpu().numpy()
        assert np.isfinite(r_g).all()
        l2 = cases.field_errors(r_g, r_o, 1, 3)
        mx = _max_rel(r_g, r_o)
        if form == "fp64":
            assert l2.max() < 1e-12, l2
            assert mx.max() < 1e-10, mx
        else:
            floor = cases.rounding_floor(p.orc, p.orc.prim_to_cons(w_o))
            assert np.all(l2 <= 16.0 * floor), (l2, floor)
            assert mx.max() < 2e-3, mx
    finally:
        p.close()


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_full_size_taylor_green_rhs_and_increment(dg, form):
    """The bench's own parity quantities at 32^3, N = 3: the right-hand side of the
    Taylor-Green state and the increment of 16 CK45 steps at the oracle's CFL-0.5 step,
    each against the oracle per field, with bars in units of the oracle's own rounding
    floor of the form's precision."""
    import torch
    precision = dg.DG_FP64 if form == "fp64" else dg.DG_MIXED
    p = _pair(dg, 3, 32, precision)
    try:
        eps = 2.0 ** -53 if form == "fp64" else 2.0 ** -24
        u0 = p.orc.prim_to_cons(p.mesh_o[3])
        r_o = p.orc.rhs(u0)
        floor = cases.rounding_floor(p.orc, u0, eps=eps)
        p.gpu.set_primitive(p.mesh_g[3])
        u_d = torch.empty(p.gpu.shape, dtype=torch.float64, device="cuda")
        dg.dg_get_state(p.gpu.ctx, u_d)
        u0_g = u_d.cpu().numpy()
        u_d = u_d.to(torch.float32 if form == "mixed" else torch.float64)
        r_d = torch.empty_like(u_d)
        dg.dg_rhs(p.gpu.ctx, u_d, r_d)
        dg.dg_sync(p.gpu.ctx)
        err = cases.field_errors(r_d.double().cpu().numpy(), r_o, 1, 3)
        print(form, "rhs error", err, "floor", floor)
        assert np.all(err <= 16.0 * floor), (err, floor)
        # increments of 16 steps
        n, dt = 16, p.orc.max_dt(u0, 0.5)
        u_n, _ = p.orc.step_rk(u0, n, dt_fixed=dt)
        p.gpu.step(n, dt_fixed=dt)
        u_g = p.gpu.get_state()[0]
        inc = cases.field_errors(u_g - u0_g, u_n - u0, 1, 3)
        sgn = np.random.default_rng(5).choice([-1.0, 1.0], size=u0.shape)
        u0p = u0 * (1.0 + eps * sgn)
        u_np, _ = p.orc.step_rk(u0p, n, dt_fixed=dt)
        inc_floor = cases.field_errors(u_np - u0p, u_n - u0, 1, 3)
        print(form, "increment error", inc, "increment floor", inc_floor)
        if form == "fp64":
            bar = cases.fp64_bar(inc_floor)
            assert np.all(inc < bar), (inc, bar)
        else:
            assert np.all(inc <= 16.0 * inc_floor), (inc, inc_floor)
    finally:
        p.close()


@pytest.mark.parametrize("N,n_el", SHAPES)
@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_full_size_ck45_step(dg, N, n_el, form):
    precision = dg.DG_FP64 if form == "fp64" else dg.DG_MIXED
    p = _pair(dg, N, n_el, precision)
    try:
        u0 = p.orc.prim_to_cons(p.mesh_o[3])
        dt = p.orc.max_dt(u0, 0.5)
        u_o, _ = p.orc.step_rk(u0, 1, dt_fixed=dt)
        p.gpu.set_primitive(p.mesh_g[3])
        p.gpu.step(1, dt_fixed=dt)
        u_g = p.gpu.get_state()[0]
        err = cases.field_errors(u_g, u_o, 1, 3)
        assert err.max() < (1e-12 if form == "fp64" else 1e-6), err
    finally:
        p.close()
