"""The learned temperature surrogate on the GPU: gradients of the project's own training
kernels against the FP64 oracle, the BF16 tensor-core forward pass, Adam, and a network
trained on data produced by the plain solver (accuracy after the FP64 polish, fallback,
and what it saves over the plain Newton solve)."""
import numpy as np
import pytest

import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_2511_17551_gb300 as dg
    dg.lib()
    return dg, oracle, torch


def _rand(oracle, seed, scale=0.3, n=300):
    rng = np.random.default_rng(seed)
    p = (scale * rng.normal(size=oracle.mlp_nparams())).astype(np.float32)
    X = rng.normal(size=(n, 7)).astype(np.float32)
    t = rng.normal(size=n).astype(np.float32)
    return p, X, t


def test_gradient_fp32_matches_oracle(env):
    dg, oracle, torch = env
    p, X, t = _rand(oracle, 1)
    loss_o, g_o = oracle.mlp_loss_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    P, Xd, td = (torch.from_numpy(a).cuda() for a in (p, X, t))
    grad = torch.empty_like(P)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(dg.dg_mlp_workspace_bytes(len(t)) // 4 + 1, dtype=torch.float32, device="cuda")
    dg.dg_mlp_grad(P, Xd, td, grad, loss, ws)
    torch.cuda.synchronize()
    g = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_o) / np.linalg.norm(g_o) < 1e-5
    assert abs(loss.item() / loss_o - 1) < 1e-5


def test_forward_fp32_and_tensor_cores(env):
    dg, oracle, torch = env
    p, X, _ = _rand(oracle, 2, n=1000)
    y_o = oracle.mlp_forward(p.astype(np.float64), X.astype(np.float64))
    P, Xd = torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda()
    y32 = torch.empty(1000, dtype=torch.float32, device="cuda")
    ytc = torch.empty_like(y32)
    dg.dg_mlp_forward(P, Xd, y32, tensor_cores=0)
    dg.dg_mlp_forward(P, Xd, ytc, tensor_cores=1)
    torch.cuda.synchronize()
    y32, ytc = y32.cpu().numpy(), ytc.cpu().numpy()
    assert np.linalg.norm(y32 - y_o) / np.linalg.norm(y_o) < 1e-5
    # BF16 operands (8 significant bits), FP32 accumulation: ~1e-2 relative
    assert np.linalg.norm(ytc - y_o) / np.linalg.norm(y_o) < 3e-2


@pytest.mark.parametrize("n_out", [1, 10])
def test_forward_tcgen05_matches_oracle_and_warp_mma(env, n_out):
    """The tcgen05 forward (128-row tiles, tensor-memory accumulators) against the oracle's
    FP64 network and the warp-level BF16 path, on a ragged row count that spans many tiles
    and several tiles per CTA."""
    dg, oracle, torch = env
    rng = np.random.default_rng(40 + n_out)
    n = 1_000_003
    p = (0.3 * rng.normal(size=oracle.mlp_nparams(n_out))).astype(np.float32)
    X = rng.normal(size=(n, 7)).astype(np.float32)
    P, Xd = torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda()
    shape = (n,) if n_out == 1 else (n, n_out)
    y5 = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    y1 = torch.empty_like(y5)
    dg.dg_mlp_forward(P, Xd, y5, tensor_cores=2)
    dg.dg_mlp_forward(P, Xd, y1, tensor_cores=1)
    torch.cuda.synchronize()
    y5, y1 = y5.cpu().numpy().reshape(n, n_out), y1.cpu().numpy().reshape(n, n_out)
    assert np.all(np.isfinite(y5))
    sample = np.r_[0:2000, n - 2000:n]             # the oracle on a sample, the ragged tail included
    y_o = oracle.mlp_forward(p.astype(np.float64), X[sample].astype(np.float64), n_out).reshape(-1, n_out)
    assert np.linalg.norm(y5[sample] - y_o) / np.linalg.norm(y_o) < 3e-2
    # same BF16 roundings of inputs, weights and hidden units; only the summation order of
    # the FP32 accumulation differs
    assert np.linalg.norm(y5 - y1) / np.linalg.norm(y1) < 5e-3


def test_adam_step_matches_oracle(env):
    dg, oracle, torch = env
    p, X, t = _rand(oracle, 3)
    po = p.astype(np.float64)
    m_o = np.zeros_like(po)
    v_o = np.zeros_like(po)
    for step in (1, 2):
        _, g_o = oracle.mlp_loss_grad(po, X.astype(np.float64), t.astype(np.float64))
        oracle.adam_step(po, m_o, v_o, g_o, step, lr=1e-3)
    P, Xd, td = (torch.from_numpy(a).cuda() for a in (p, X, t))
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    ws = torch.empty(dg.dg_mlp_workspace_bytes(len(t)) // 4 + 1, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    for step in (1, 2):
        dg.dg_mlp_train_step(P, m, v, Xd, td, step, 1e-3, loss, ws)
    torch.cuda.synchronize()
    # updates are ~lr per step; FP32 gradients give ~1e-5 relative differences in the moments
    d = P.cpu().numpy().astype(np.float64) - p
    d_o = po - p
    assert np.linalg.norm(d - d_o) / np.linalg.norm(d_o) < 1e-3


@pytest.fixture(scope="module")
def trained(env):
    """Plain-solver data on the mixture O-grid, a short training run."""
    dg, oracle, torch = env
    import workloads as W
    from paper_2511_17551_gb300 import surrogate as S
    x, _ = dg.dg_lgl_nodes(3)
    xyz, nbr, face, w = cases.mixture_ogrid(x, nr=4, nth=6, nz=2)
    kinds, bcp = cases.mixture_bc(w)
    s = dg.Solver(3, 3, xyz, nbr, face, n_species=5, species=W.species_table(), volume_flux=1,
                  surface_flux=0, bc_kind=kinds, bc_prim=bcp, precision=dg.DG_MIXED)
    s.set_primitive(cases.mixture_perturbed(w, 5))
    X, T = S.collect(s.ctx, 60000, 6, 2)
    params, stats, hist = S.train(X, T, epochs=25, batch=1024, lr=3e-3)
    s.close()
    return params, stats, hist, (xyz, nbr, face, w, kinds, bcp)


def test_training_converges(env, trained):
    params, stats, hist, _ = trained
    assert hist[-1][2] < 0.05 * hist[0][2] or hist[-1][2] < 1e-3


def test_surrogate_temperature_accuracy_and_fallback(env, trained):
    """Mixed form with the surrogate: T within 1e-4 (relative) of the oracle's Newton T;
    accepted nodes dominate; the forced-failure case routes every node to the fallback
    and reproduces the plain result."""
    dg, oracle, torch = env
    import workloads as W
    params, stats, _, (xyz, nbr, face, w, kinds, bcp) = trained
    s = dg.Solver(3, 3, xyz, nbr, face, n_species=5, species=W.species_table(), volume_flux=1,
                  surface_flux=0, bc_kind=kinds, bc_prim=bcp, precision=dg.DG_MIXED)
    try:
        wp = cases.mixture_perturbed(w, 5)
        s.set_primitive(wp)
        dg.dg_set_surrogate(s.ctx, params, stats)
        T_s = dg.dg_get_temperature(s.ctx, (s.K, s.np))
        acc, fb = dg.dg_surrogate_stats(s.ctx)
        xo, _ = oracle.lgl(3)
        xyz_o, _, _, w_o = cases.mixture_ogrid(xo, nr=4, nth=6, nz=2)
        o = oracle.Oracle(3, 3, xyz_o, nbr, face, n_species=5, species=W.species_table(),
                          volume_flux=1, bc_kind=kinds, bc_prim=bcp)
        T_o = o.temperature(o.prim_to_cons(cases.mixture_perturbed(w_o, 5)))
        assert np.abs(T_s / T_o - 1).max() < 1e-4
        assert acc + fb == s.K * s.np and acc > 0.25 * (acc + fb)
        # wrong weights: every node falls back; the fallback's full FP64 Newton solve and the
        # mixed form's plain solve (FP32 Newton, FP64 residual with FP32-rounded temperature
        # coefficients: about 2e-7 relative) agree within the latter's accuracy
        dg.dg_set_surrogate(s.ctx, None)
        T_plain = dg.dg_get_temperature(s.ctx, (s.K, s.np))
        bad = params.copy()
        bad[-1] += 50.0
        dg.dg_set_surrogate(s.ctx, bad, stats)
        T_b = dg.dg_get_temperature(s.ctx, (s.K, s.np))
        acc, fb = dg.dg_surrogate_stats(s.ctx)
        assert acc == 0 and fb == s.K * s.np
        assert np.abs(T_b / T_plain - 1).max() < 1e-6
    finally:
        s.close()


def test_surrogate_rk_steps_match_oracle(env, trained):
    dg, oracle, torch = env
    import workloads as W
    params, stats, _, (xyz, nbr, face, w, kinds, bcp) = trained
    s = dg.Solver(3, 3, xyz, nbr, face, n_species=5, species=W.species_table(), volume_flux=1,
                  surface_flux=0, bc_kind=kinds, bc_prim=bcp, precision=dg.DG_MIXED)
    try:
        s.set_primitive(w)
        dg.dg_set_surrogate(s.ctx, params, stats)
        xo, _ = oracle.lgl(3)
        xyz_o, _, _, w_o = cases.mixture_ogrid(xo, nr=4, nth=6, nz=2)
        o = oracle.Oracle(3, 3, xyz_o, nbr, face, n_species=5, species=W.species_table(),
                          volume_flux=1, bc_kind=kinds, bc_prim=bcp)
        u_o = o.prim_to_cons(w_o)
        dt = 0.2 * o.max_dt(u_o, 0.5)
        s.step(3, dt_fixed=dt)
        u_g, _ = s.get_state()
        u_r, _ = o.step_rk(u_o, 3, dt_fixed=dt)
        err = cases.field_errors(u_g, u_r, 5, 3)
        assert err.max() < 1e-5, err
        T_g = dg.dg_get_temperature(s.ctx, (s.K, s.np))
        assert np.abs(T_g / o.temperature(u_r) - 1).max() < 1e-4
    finally:
        s.close()
