"""Long Navier-Stokes Taylor-Green runs: kinetic-energy and enstrophy histories (the
domain averages of Eqs. TGV_KE / TGV_SD) every 10 steps over 1000 Carpenter-Kennedy RK45
steps.  At 8^3 elements the FP64 and mixed GPU forms are compared with the oracle's own
1000-step run; at the full 32^3 (N = 3) and 16^3 (N = 7) shapes, where 1000 oracle steps
would take tens of minutes, the mixed form is compared with the FP64 GPU form, which the
8^3 comparison (and the right-hand-side parity tests) tie to the oracle."""
import numpy as np
import pytest

import cases

pytestmark = pytest.mark.gpu

MU = 1.0 / 1600.0


@pytest.fixture(scope="module")
def dg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_17551_gb300 as dg
    dg.lib()
    return dg


def _gpu_history(dg, N, n_el, precision, steps, every, dt, final_state=False):
    x, _ = dg.dg_lgl_nodes(N)
    xyz, nbr, face, w = cases.tgv(x, n_el, warp=0.1)
    s = dg.Solver(3, N, xyz, nbr, face, equations=dg.DG_NAVIER_STOKES, mu=MU, Pr=0.72,
                  precision=precision, p_ref=cases.tgv_p0())
    try:
        s.set_primitive(w)
        h = [s.diagnostics()[:2]]
        for _ in range(steps // every):
            s.step(every, dt_fixed=dt)
            h.append(s.diagnostics()[:2])
        if final_state:
            return np.array(h), s.get_state()[0]
        return np.array(h)
    finally:
        s.close()


def _dt(N, n_el, cfl=0.5):
    """One fixed step for all forms: the oracle's CFL step of the initial state."""
    import oracle
    xo, _ = oracle.lgl(N)
    xyz, nbr, face, w = cases.tgv(xo, n_el, warp=0.1)
    o = oracle.Oracle(3, N, xyz, nbr, face, equations=1, mu=MU, Pr=0.72)
    return o, o.prim_to_cons(w), o.max_dt(o.prim_to_cons(w), cfl)


def test_history_8cubed_matches_oracle(dg):
    o, u, dt = _dt(3, 8)
    h_o = [o.diagnostics(u)[:2]]
    for _ in range(100):
        u, _ = o.step_rk(u, 10, dt_fixed=dt)
        h_o.append(o.diagnostics(u)[:2])
    h_o = np.array(h_o)
    h64 = _gpu_history(dg, 3, 8, dg.DG_FP64, 1000, 10, dt)
    h32 = _gpu_history(dg, 3, 8, dg.DG_MIXED, 1000, 10, dt)
    # the flow evolves: kinetic energy decays, enstrophy grows (early TGV)
    assert h_o[-1, 0] < h_o[0, 0] and h_o[-1, 1] > h_o[0, 1]
    assert np.abs(h64 / h_o - 1).max() < 1e-11
    assert np.abs(h32 / h_o - 1).max() < 1e-5


@pytest.mark.parametrize("N,n_el,steps", [(3, 32, 1000), (7, 16, 1000)])
def test_history_full_size_mixed_vs_fp64(dg, N, n_el, steps):
    # one fixed step for both forms: the FP64 form's CFL-0.5 step of the initial state
    x, _ = dg.dg_lgl_nodes(N)
    xyz, nbr, face, w = cases.tgv(x, n_el, warp=0.1)
    s = dg.Solver(3, N, xyz, nbr, face, equations=dg.DG_NAVIER_STOKES, mu=MU, Pr=0.72,
                  precision=dg.DG_FP64)
    try:
        s.set_primitive(w)
        dt = s.step(1, 0.5)
    finally:
        s.close()
    h64, u64 = _gpu_history(dg, N, n_el, dg.DG_FP64, steps, 10, dt, final_state=True)
    h32, u32 = _gpu_history(dg, N, n_el, dg.DG_MIXED, steps, 10, dt, final_state=True)
    # discrete initial averages converge spectrally to KE0 = 1/8, enstrophy0 = 3/8
    assert abs(h64[0, 0] - 0.125) < 1e-4 and abs(h64[0, 1] - 0.375) < 2e-3
    assert h64[-1, 0] < h64[0, 0]
    # the mixed form's bar on conserved variables after 1000 steps
    err = cases.field_errors(u32, u64, 1, 3)
    assert err.max() < 1e-5, err
    # the quadratic averages integrate the FP32 rounding of 5000 stage updates of the
    # FP32 state: measured 1.05e-5 (KE) at 32^3, N = 3
    assert np.abs(h32 / h64 - 1).max() < 3e-5


def test_mixed_steps_reproduce_bit_for_bit(dg):
    """The same 20 CFL steps of the mixed form (compensated state, 32^3 elements: many CTA
    waves per launch) from the same state give the same bits twice: no kernel of an RK
    stage reads data that another CTA of the same launch writes (the state and its
    compensation part are both ping-ponged)."""
    x, _ = dg.dg_lgl_nodes(3)
    xyz, nbr, face, w = cases.tgv(x, 32, warp=0.1)
    s = dg.Solver(3, 3, xyz, nbr, face, equations=dg.DG_NAVIER_STOKES, mu=MU, Pr=0.72,
                  precision=dg.DG_MIXED, p_ref=cases.tgv_p0())
    try:
        runs = []
        for _ in range(2):
            s.set_primitive(w)
            t = s.step(20, 0.5)
            u, _ = s.get_state()
            runs.append((t, u))
        assert runs[0][0] == runs[1][0]
        assert np.array_equal(runs[0][1], runs[1][1])
    finally:
        s.close()
