"""The allocation-free Navier-Stokes right-hand side (dg_rhs_ns_noalloc) against dg_rhs.

Callers that may not allocate device memory (a framework that owns all device memory,
or a loop that cannot afford cudaMalloc's synchronisation) use dg_rhs_ns_noalloc; its
scratch is a static device array shared by all calls.  Every degree it accepts
(N = 2, 3, 4, 7) runs here on the curved (warped) Taylor-Green mesh, with the production
flux pair and with a pair that the runtime-choice kernels serve, two calls in a row, each
against dg_rhs of a context on the same mesh (whose metric terms the call takes) and
against the FP64 oracle.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import cases

pytestmark = pytest.mark.gpu

MU, PR, GAMMA = 0.01, 0.72, 1.4
# elements per direction for each degree (the scratch holds K (N+1)^3 12 doubles)
SIZES = {2: 4, 3: 4, 4: 4, 7: 3}


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_17551_gb300 as dg
    dg.lib()
    return dg, torch


def _case(dg, torch, N, vf, sf):
    n_el = SIZES[N]
    x, _ = dg.dg_lgl_nodes(N)
    xyz, nbr, face, w0 = cases.tgv(x, n_el, warp=0.1)
    s = dg.Solver(3, N, xyz, nbr, face, equations=dg.DG_NAVIER_STOKES, mu=MU, Pr=PR,
                  precision=dg.DG_FP64, volume_flux=vf, surface_flux=sf)
    Ja = torch.empty((s.K, 3, 3, s.np), dtype=torch.float64, device="cuda")
    invJ = torch.empty((s.K, s.np), dtype=torch.float64, device="cuda")
    dg.dg_get_metrics(s.ctx, Ja, invJ)
    nbr_d = torch.from_numpy(np.ascontiguousarray(nbr, dtype=np.int32)).cuda()
    return s, w0, Ja, invJ, nbr_d


@pytest.mark.parametrize("N,vf,sf", [(2, 0, 0), (3, 0, 0), (4, 0, 0), (7, 0, 0), (3, 3, 3), (7, 3, 3)])
def test_noalloc_rhs_matches_context_rhs_twice(env, N, vf, sf):
    dg, torch = env
    s, w0, Ja, invJ, nbr_d = _case(dg, torch, N, vf, sf)
    stream = torch.cuda.current_stream().cuda_stream
    try:
        for seed in (1, 2):  # two calls in a row, on different states
            s.set_primitive(cases.perturbed_state(w0, seed=seed))
            u = torch.empty(s.shape, dtype=torch.float64, device="cuda")
            dg.dg_get_state(s.ctx, u)
            ref = torch.empty_like(u)
            dg.dg_rhs(s.ctx, u, ref)
            dg.dg_sync(s.ctx)
            out = torch.full_like(u, float("nan"))
            dg.dg_rhs_ns_noalloc(N, s.K, nbr_d, Ja, invJ, GAMMA, MU, PR, vf, sf, u, out, stream)
            code, word = dg.dg_noalloc_status(stream)
            assert (code, word) == (dg.DG_OK, 0)
            err = cases.field_errors(out.cpu().numpy(), ref.cpu().numpy(), 1, 3)
            assert err.max() < 1e-12, err
    finally:
        s.close()


@pytest.mark.parametrize("N", [2, 4, 7])
def test_noalloc_rhs_matches_oracle(env, N):
    """The same call against the FP64 oracle on the warped mesh (FP64 bar 1e-12)."""
    dg, torch = env
    import oracle
    s, w0, Ja, invJ, nbr_d = _case(dg, torch, N, 0, 0)
    try:
        xo, _ = oracle.lgl(N)
        xyz_o, nbr_o, face_o, w_o = cases.tgv(xo, SIZES[N], warp=0.1)
        o = oracle.Oracle(3, N, xyz_o, nbr_o, face_o, equations=oracle.NAVIER_STOKES, mu=MU, Pr=PR)
        u_o = o.prim_to_cons(cases.perturbed_state(w_o, seed=3))
        r_o = o.rhs(u_o)
        u = torch.from_numpy(u_o).cuda()
        out = torch.full_like(u, float("nan"))
        stream = torch.cuda.current_stream().cuda_stream
        dg.dg_rhs_ns_noalloc(N, s.K, nbr_d, Ja, invJ, GAMMA, MU, PR, 0, 0, u, out, stream)
        assert dg.dg_noalloc_status(stream)[0] == dg.DG_OK
        err = cases.field_errors(out.cpu().numpy(), r_o, 1, 3)
        assert err.max() < 1e-12, err
    finally:
        s.close()


def test_noalloc_status_and_limits(env):
    """A non-physical state (negative density planted on the host) is latched and read
    back by dg_noalloc_status; the next clean call clears it; sizes beyond the static
    scratch are rejected before any work is queued."""
    dg, torch = env
    N = 3
    s, w0, Ja, invJ, nbr_d = _case(dg, torch, N, 0, 0)
    stream = torch.cuda.current_stream().cuda_stream
    try:
        s.set_primitive(w0)
        u = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        dg.dg_get_state(s.ctx, u)
        bad = u.clone()
        bad[5, 0, 7] = -1.0
        out = torch.empty_like(u)
        dg.dg_rhs_ns_noalloc(N, s.K, nbr_d, Ja, invJ, GAMMA, MU, PR, 0, 0, bad, out, stream)
        code, word = dg.dg_noalloc_status(stream)
        assert code == dg.DG_ENONPHYS
        assert word >> 56 == dg.DG_ENONPHYS
        dg.dg_rhs_ns_noalloc(N, s.K, nbr_d, Ja, invJ, GAMMA, MU, PR, 0, 0, u, out, stream)
        assert dg.dg_noalloc_status(stream) == (dg.DG_OK, 0)
        with pytest.raises(dg.DgError) as ei:
            dg.dg_rhs_ns_noalloc(N, 10 ** 6, nbr_d, Ja, invJ, GAMMA, MU, PR, 0, 0, u, out, stream)
        assert ei.value.code == dg.DG_EINVAL
    finally:
        s.close()
