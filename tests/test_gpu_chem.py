"""GPU parity of the reacting mixture (finite-rate FP64 source with point-implicit scaling)
against the oracle on a cylinder O-grid with a hot region near the body."""
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


def _pair(dg, precision, N=3):
    import workloads as W
    sp = W.species_table()
    R = W.reaction_table()

    def builder(x):
        return cases.mixture_ogrid(x, hot=(1.2, 2500.0))

    import oracle
    xo, _ = oracle.lgl(N)
    w0 = builder(xo)[3]
    kinds, bcp = cases.mixture_bc(w0)
    return cases.Pair(builder, 3, N, precision=precision, n_species=5, species=sp, reactions=R,
                      volume_flux=1, surface_flux=0, bc_kind=kinds, bc_prim=bcp)


def test_reacting_rhs_fp64(dg):
    import torch
    p = _pair(dg, 0)
    try:
        u_o = p.orc.prim_to_cons(p.mesh_o[3])
        r_o = p.orc.rhs(u_o)
        p.gpu.set_primitive(p.mesh_g[3])
        u_d = torch.empty(p.gpu.shape, dtype=torch.float64, device="cuda")
        dg.dg_get_state(p.gpu.ctx, u_d)
        r_d = torch.empty_like(u_d)
        dg.dg_rhs(p.gpu.ctx, u_d, r_d)
        dg.dg_sync(p.gpu.ctx)
        r_g = r_d.cpu().numpy()
        # chemistry must be active: the species rows carry a source far above rounding
        assert np.abs(r_o[:, :5]).max() > 1.0
        err = cases.field_errors(r_g, r_o, 5, 3)
        bar = cases.fp64_bar(cases.rounding_floor(p.orc, u_o))
        print("reacting rhs fp64 error", err, "bar", bar)
        assert np.all(err < bar), (err, bar)
    finally:
        p.close()


@pytest.mark.parametrize("precision,tol", [(0, None), (1, 1e-5)])
def test_reacting_rk_steps(dg, precision, tol):
    p = _pair(dg, precision)
    try:
        u_o = p.orc.prim_to_cons(p.mesh_o[3])
        dt = 0.1 * p.orc.max_dt(u_o, 0.5)  # stiff hot-layer chemistry
        p.gpu.set_primitive(p.mesh_g[3])
        p.gpu.step(3, dt_fixed=dt)
        u_g, _ = p.gpu.get_state()
        u_r, _ = p.orc.step_rk(u_o, 3, dt_fixed=dt)
        err = cases.field_errors(u_g, u_r, 5, 3)
        bar = cases.fp64_bar(cases.step_floor(p.orc, u_o, 3, dt)) if tol is None else tol
        print("reacting 3 steps error", err, "bar", bar)
        assert np.all(err < bar), (err, bar)
        # species mass is exchanged, total mass is not created
        assert np.allclose(u_g[:, :5].sum(1), u_r[:, :5].sum(1), rtol=1e-5 if precision else 1e-11)
    finally:
        p.close()
