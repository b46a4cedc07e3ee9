"""The learned surrogates' data preparation in libdg against numpy (column statistics,
standardisation with and without the asinh map, quantiles of absolute values, row
gathers) and the oracle (mean-squared error of the network)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_17551_gb300 as dg
    dg.lib()
    return dg, torch


def test_column_stats_and_standardize(env):
    dg, torch = env
    rng = np.random.default_rng(31)
    X = rng.normal(size=(100_003, 7)) * np.array([1, 2, 3, 0.1, 1e3, 5, 1e-2]) + np.arange(7)
    for dtype in (np.float32, np.float64):
        Xd = torch.from_numpy(X.astype(dtype)).cuda()
        Xh = X.astype(dtype).astype(np.float64)
        mean, std, lo, hi = dg.dg_column_stats(Xd)
        assert np.allclose(mean, Xh.mean(0), rtol=1e-12, atol=1e-12)
        assert np.allclose(std, Xh.std(0, ddof=1), rtol=1e-12)
        assert np.array_equal(lo, Xh.min(0)) and np.array_equal(hi, Xh.max(0))
        out = torch.empty(X.shape, dtype=torch.float32, device="cuda")
        dg.dg_standardize(Xd, mean, std, out)
        ref = ((Xh - mean) / std).astype(np.float32)
        assert np.allclose(out.cpu().numpy(), ref, rtol=1e-6, atol=1e-6)
    # the asinh image of signed rates, per-column reference scales
    Y = rng.normal(size=(50_000, 10)) * 10.0 ** rng.uniform(-3, 6, size=(50_000, 10))
    refs = np.array([3.0] * 5 + [0.5] * 5)
    Yd = torch.from_numpy(Y).cuda()
    mz, sz, lz, hz = dg.dg_column_stats(Yd, ref=refs)
    Z = np.arcsinh(Y / refs)
    assert np.allclose(mz, Z.mean(0), rtol=1e-11, atol=1e-12)
    assert np.allclose(sz, Z.std(0, ddof=1), rtol=1e-11)
    out = torch.empty(Y.shape, dtype=torch.float32, device="cuda")
    dg.dg_standardize(Yd, mz, sz, out, ref=refs)
    assert np.allclose(out.cpu().numpy(), ((Z - mz) / sz).astype(np.float32), rtol=1e-6, atol=1e-6)
    # deterministic: the same call twice gives the same bits
    assert np.array_equal(dg.dg_column_stats(Yd, ref=refs)[1], sz)


def test_abs_quantile_and_gather(env):
    dg, torch = env
    rng = np.random.default_rng(32)
    Y = rng.normal(size=(20_001, 10)) * 10.0 ** rng.uniform(-5, 5, size=(20_001, 10))
    Yd = torch.from_numpy(Y).cuda()
    for c0, nc, q in ((0, 5, 0.99), (5, 5, 0.99), (0, 10, 0.5), (3, 1, 0.0), (2, 3, 1.0)):
        got = dg.dg_abs_quantile(Yd, c0, nc, q)
        want = np.quantile(np.abs(Y[:, c0:c0 + nc]).ravel(), q)  # linear interpolation
        assert abs(got - want) <= 1e-15 * abs(want), (c0, nc, q, got, want)
    X = torch.from_numpy(rng.normal(size=(1000, 7)).astype(np.float32)).cuda()
    idx_h = rng.integers(0, 1000, size=333).astype(np.int64)
    out = torch.empty((333, 7), dtype=torch.float32, device="cuda")
    dg.dg_gather_rows(X, torch.from_numpy(idx_h).cuda(), out)
    assert np.array_equal(out.cpu().numpy(), X.cpu().numpy()[idx_h])


def test_mlp_loss_against_oracle(env):
    dg, torch = env
    import oracle
    rng = np.random.default_rng(33)
    for no in (1, 10):
        p = (0.3 * rng.normal(size=oracle.mlp_nparams(no))).astype(np.float32)
        X = rng.normal(size=(5000, 7)).astype(np.float32)
        t = rng.normal(size=(5000, no)).astype(np.float32)
        loss_o, _ = oracle.mlp_loss_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64), no)
        tt = torch.from_numpy(t).cuda()
        got = dg.dg_mlp_loss(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(), tt if no > 1 else tt.reshape(-1))
        assert abs(got / loss_o - 1) < 1e-5, (no, got, loss_o)
