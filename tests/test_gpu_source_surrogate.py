"""The learned chemistry source on the GPU: ten-output training / forward kernels against
the FP64 oracle; the learned source against the oracle's evaluation of the same network
(decode, projection, point-implicit terms); rejected tiles reproduce the plain FP64
source bit for bit; and a network trained on data of the plain reacting run."""
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


def test_ten_output_gradient_and_forward_match_oracle(env):
    dg, oracle, torch = env
    rng = np.random.default_rng(21)
    p = (0.3 * rng.normal(size=oracle.mlp_nparams(10))).astype(np.float32)
    X = rng.normal(size=(300, 7)).astype(np.float32)
    t = rng.normal(size=(300, 10)).astype(np.float32)
    loss_o, g_o = oracle.mlp_loss_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64), 10)
    P, Xd, td = (torch.from_numpy(a).cuda() for a in (p, X, t))
    grad = torch.empty_like(P)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(dg.dg_mlp_workspace_bytes(300, 10) // 4 + 1, dtype=torch.float32, device="cuda")
    dg.dg_mlp_grad(P, Xd, td, grad, loss, ws)
    y32 = torch.empty((300, 10), dtype=torch.float32, device="cuda")
    ytc = torch.empty_like(y32)
    dg.dg_mlp_forward(P, Xd, y32, tensor_cores=0)
    dg.dg_mlp_forward(P, Xd, ytc, tensor_cores=1)
    torch.cuda.synchronize()
    g = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_o) / np.linalg.norm(g_o) < 1e-5
    assert abs(loss.item() / loss_o - 1) < 1e-5
    y_o = oracle.mlp_forward(p.astype(np.float64), X.astype(np.float64), 10)
    assert np.linalg.norm(y32.cpu().numpy() - y_o) / np.linalg.norm(y_o) < 1e-5
    # BF16 operands, FP32 accumulation
    assert np.linalg.norm(ytc.cpu().numpy() - y_o) / np.linalg.norm(y_o) < 3e-2


def _reacting(dg, precision=0, N=3):
    import workloads as W
    x, _ = dg.dg_lgl_nodes(N)
    xyz, nbr, face, w = cases.mixture_ogrid(x, hot=(1.2, 2500.0))
    kinds, bcp = cases.mixture_bc(w)
    s = dg.Solver(3, N, xyz, nbr, face, n_species=5, species=W.species_table(), volume_flux=1,
                  surface_flux=0, bc_kind=kinds, bc_prim=bcp, precision=precision,
                  reactions=W.reaction_table())
    s.set_primitive(w)
    s.w0 = w
    return s


def _rhs(dg, torch, s):
    """Right-hand side of the initial state.  Setting the state again re-seeds the
    temperature cache, so repeated evaluations start the Newton solve identically."""
    s.set_primitive(s.w0)
    u = torch.empty(s.shape, dtype=torch.float64, device="cuda")
    dg.dg_get_state(s.ctx, u)
    r = torch.empty_like(u)
    dg.dg_rhs(s.ctx, u, r)
    dg.dg_sync(s.ctx)
    return u.cpu().numpy(), r.cpu().numpy()


def _stats(w_ref=1e2, j_ref=1e3, lo=-1e30, hi=1e30, tol_check=1e30, tol_mass=1e30, floor=0.0):
    st = np.zeros(53)
    st[0:7] = [0.2, 0.2, 0.2, 0.2, 0.2, np.log(0.1), 1500.0]
    st[7:14] = [0.1, 0.1, 0.1, 0.1, 0.1, 1.0, 1000.0]
    st[14:24] = 0.0
    st[24:34] = 1.0
    st[34], st[35] = w_ref, j_ref
    st[36:43], st[43:50] = lo, hi
    st[50], st[51], st[52] = tol_check, tol_mass, floor
    return st


def _plain_source(oracle, u, T, dt=0.0):
    import workloads as W
    rhos = u[:, :5, :].transpose(0, 2, 1).reshape(-1, 5)
    _, _, S = oracle.chem_eval(W.species_table(), W.reaction_table(), rhos, T.reshape(-1), dt)
    return rhos, S


def test_rejected_tiles_reproduce_the_plain_source_bitwise(env):
    dg, oracle, torch = env
    s = _reacting(dg)
    try:
        _, r_plain = _rhs(dg, torch, s)
        n = s.K * s.np
        p = (0.3 * np.random.default_rng(3).normal(size=dg.dg_mlp_nparams(10))).astype(np.float32)
        # an empty trust box rejects every tile
        dg.dg_set_surrogate(s.ctx, p, _stats(lo=1e30, hi=-1e30), which=dg.DG_SURROGATE_SOURCE)
        _, r_box = _rhs(dg, torch, s)
        acc, fb = dg.dg_surrogate_stats(s.ctx, dg.DG_SURROGATE_SOURCE)
        assert (acc, fb) == (0, n)
        assert np.array_equal(r_box, r_plain)
        # a zero tolerance at the sampled node rejects every tile whose sample is off
        dg.dg_set_surrogate(s.ctx, p, _stats(tol_check=0.0), which=dg.DG_SURROGATE_SOURCE)
        _, r_chk = _rhs(dg, torch, s)
        acc, fb = dg.dg_surrogate_stats(s.ctx, dg.DG_SURROGATE_SOURCE)
        assert (acc, fb) == (0, n)
        assert np.array_equal(r_chk, r_plain)
        # switched off again: plain
        dg.dg_set_surrogate(s.ctx, None, which=dg.DG_SURROGATE_SOURCE)
        _, r_off = _rhs(dg, torch, s)
        assert np.array_equal(r_off, r_plain)
    finally:
        s.close()


def test_accepted_source_matches_the_oracle_surrogate(env):
    """Everything accepted: the species rows of the right-hand side move by exactly
    S_learned - S_plain; S_learned against the oracle's FP64 evaluation of the same
    network (BF16 hidden layers on the GPU), compared in the asinh image."""
    dg, oracle, torch = env
    s = _reacting(dg)
    try:
        u, r_plain = _rhs(dg, torch, s)
        T = dg.dg_get_temperature(s.ctx, (s.K, s.np))
        p = (0.1 * np.random.default_rng(4).normal(size=dg.dg_mlp_nparams(10))).astype(np.float32)
        st = _stats()
        dg.dg_set_surrogate(s.ctx, p, st, which=dg.DG_SURROGATE_SOURCE)
        _, r_mlp = _rhs(dg, torch, s)
        acc, fb = dg.dg_surrogate_stats(s.ctx, dg.DG_SURROGATE_SOURCE)
        assert (acc, fb) == (s.K * s.np, 0)
        rhos, S_plain = _plain_source(oracle, u, T)
        dS = (r_mlp - r_plain)[:, :5, :].transpose(0, 2, 1).reshape(-1, 5)
        S_gpu = S_plain + dS
        S_o, ok_o, _, _ = oracle.chem_surrogate_source(p.astype(np.float64), st, rhos, T.reshape(-1))
        assert ok_o.all()
        err = np.abs(np.arcsinh(S_gpu / st[34]) - np.arcsinh(S_o / st[34]))
        assert err.max() < 0.05, err.max()
        # projected rates conserve mass
        assert np.abs(S_gpu.sum(1)).max() <= 1e-5 * np.abs(S_gpu).sum(1).max()
    finally:
        s.close()


@pytest.fixture(scope="module")
def trained_source(env):
    """Plain reacting run on the O-grid (FP64), 24 states x 2000 samples, short training."""
    dg, oracle, torch = env
    from paper_2511_17551_gb300 import surrogate as S
    s = _reacting(dg)
    try:
        import workloads as W
        xo, _ = oracle.lgl(3)
        xyz_o, nbr, face, w_o = cases.mixture_ogrid(xo, hot=(1.2, 2500.0))
        kinds, bcp = cases.mixture_bc(w_o)
        o = oracle.Oracle(3, 3, xyz_o, nbr, face, n_species=5, species=W.species_table(), volume_flux=1,
                          bc_kind=kinds, bc_prim=bcp, reactions=W.reaction_table())
        dt = 0.1 * o.max_dt(o.prim_to_cons(w_o), 0.5)
        X, Y = S.collect_source(s.ctx, 48000, 24, 1, dt_fixed=dt)
        params, stats, hist = S.train_source(X, Y, epochs=150, batch=2048, lr=3e-3)
        return params, stats, hist, dt
    finally:
        s.close()


def test_trained_source_surrogate(env, trained_source):
    """A network trained on the plain run: training converges, most tiles are accepted on
    the initial state, and the accepted source is within the acceptance tolerance of the
    oracle's plain source at 95 % of the nodes."""
    dg, oracle, torch = env
    params, stats, hist, dt = trained_source
    assert hist[-1][2] < 0.2 * hist[0][2]
    s = _reacting(dg)
    try:
        u, _ = _rhs(dg, torch, s)
        T = dg.dg_get_temperature(s.ctx, (s.K, s.np))
        dg.dg_set_surrogate(s.ctx, params, stats, which=dg.DG_SURROGATE_SOURCE)
        _, r_mlp = _rhs(dg, torch, s)
        acc, fb = dg.dg_surrogate_stats(s.ctx, dg.DG_SURROGATE_SOURCE)
        assert acc + fb == s.K * s.np
        assert acc > 0
        dg.dg_set_surrogate(s.ctx, None, which=dg.DG_SURROGATE_SOURCE)
        _, r_plain = _rhs(dg, torch, s)
        rhos, S_plain = _plain_source(oracle, u, T)
        dS = (r_mlp - r_plain)[:, :5, :].transpose(0, 2, 1).reshape(-1, 5)
        bound = stats[50] * np.abs(S_plain).sum(1) + stats[52]
        frac_within = np.mean(np.all(np.abs(dS) <= 2.0 * bound[:, None], axis=1))
        assert frac_within > 0.95, (frac_within, acc, fb)
        # RK steps with the learned source stay close to the plain FP64 run
        s.set_primitive(s.w0)
        dg.dg_set_surrogate(s.ctx, params, stats, which=dg.DG_SURROGATE_SOURCE)
        s.step(3, dt_fixed=dt)
        u_l, _ = s.get_state()
        dg.dg_set_surrogate(s.ctx, None, which=dg.DG_SURROGATE_SOURCE)
        s.set_primitive(s.w0)
        s.step(3, dt_fixed=dt)
        u_p, _ = s.get_state()
        # the species increments of the learned run against those of the plain run: the
        # accepted sources carry up to tol_check of the local rates (plus the floor), so
        # the increments differ by a fraction of that order
        u0 = np.zeros_like(u_p)
        s.set_primitive(s.w0)
        u0, _ = s.get_state()
        inc = np.linalg.norm((u_p - u0)[:, :5, :].transpose(1, 0, 2).reshape(5, -1), axis=1)
        dif = np.linalg.norm((u_l - u_p)[:, :5, :].transpose(1, 0, 2).reshape(5, -1), axis=1)
        ratio = dif / inc
        assert ratio.max() < 0.25, (ratio, acc, fb)
        # momentum and energy are not touched by the source beyond the coupling
        err = cases.field_errors(u_l, u_p, 5, 3)
        assert err[5:].max() < 1e-3, err
    finally:
        s.close()
