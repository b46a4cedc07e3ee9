"""The allocation-free Navier-Stokes right-hand side (dg_rhs_ns_noalloc) against dg_rhs.

Callers that may not allocate device memory (a framework that owns all device memory,
or a loop that cannot afford cudaMalloc's synchronisation) use dg_rhs_ns_noalloc; its
scratch is a static device array shared by all calls.  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import cases

pytestmark = pytest.mark.gpu


def test_noalloc_rhs_matches_context_rhs_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_17551_gb300 as dg
    import workloads as W
    N, n_el, mu, Pr, g = 3, 4, 0.01, 0.72, 1.4
    x, _ = dg.dg_lgl_nodes(N)
    xyz, nbr, face, w0 = cases.tgv(x, n_el, warp=0.0)
    s = dg.Solver(3, N, xyz, nbr, face, equations=dg.DG_NAVIER_STOKES, mu=mu, Pr=Pr,
                  precision=dg.DG_FP64)
    K, npn = s.K, s.np
    # Cartesian periodic box: the metric terms are those of the affine map
    h = 2 * np.pi / n_el / 2
    Ja = torch.zeros((K, 3, 3, npn), dtype=torch.float64, device="cuda")
    for i in range(3):
        Ja[:, i, i, :] = h * h
    invJ = torch.full((K, npn), 1.0 / h ** 3, dtype=torch.float64, device="cuda")
    nbr_d = torch.from_numpy(nbr.astype(np.int32)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (1, 2):  # two calls in a row, on different states
        s.set_primitive(cases.perturbed_state(w0, seed=seed))
        u = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        dg.dg_get_state(s.ctx, u)
        ref = torch.empty_like(u)
        dg.dg_rhs(s.ctx, u, ref)
        dg.dg_sync(s.ctx)
        out = torch.full_like(u, float("nan"))
        dg.dg_rhs_ns_noalloc(N, K, nbr_d, Ja, invJ, g, mu, Pr, dg.DG_VF_RANOCHA, dg.DG_SF_LLF,
                             u, out, stream)
        torch.cuda.synchronize()
        err = cases.field_errors(out.cpu().numpy(), ref.cpu().numpy(), 1, 3)
        assert err.max() < 1e-12, err
    # sizes beyond the static scratch are rejected
    with pytest.raises(dg.DgError) as ei:
        dg.dg_rhs_ns_noalloc(N, 10 ** 6, nbr_d, Ja, invJ, g, mu, Pr, 0, 0, u, out, stream)
    assert ei.value.code == dg.DG_EINVAL
    s.close()
