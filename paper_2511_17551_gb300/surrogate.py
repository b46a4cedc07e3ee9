"""Training drivers for the learned surrogates (temperature solve; chemistry source).

Data come from the plain solver itself: a mixture context is stepped with the plain
computations and ``dg_thermo_sample`` / ``dg_chem_sample`` draw node states after every
``steps_between`` RK steps (raw features and the plain FP64 results).  The drivers
standardise the data (``dg_column_stats``, ``dg_standardize``, ``dg_abs_quantile``),
initialise the network (Xavier-uniform from a seed) and run Adam epochs with
``dg_mlp_train_step`` on minibatches gathered by ``dg_gather_rows``; statistics, the asinh
target map, the trust box, forward, back-propagation, the gradient reduction, the update
and the validation loss all run in libdg's kernels.  PyTorch only holds the device
buffers; numpy draws the seeded permutations.
"""
import math

import numpy as np

from . import (DG_SRC_NSTATS, dg_abs_quantile, dg_chem_sample, dg_column_stats, dg_gather_rows,
               dg_mlp_loss, dg_mlp_nparams, dg_mlp_train_step, dg_mlp_workspace_bytes,
               dg_standardize, dg_step_rk, dg_thermo_sample)

NI, NH = 7, 64


def collect(ctx, n_total, n_snapshots, steps_between, cfl=0.3, seed=1):
    """Temperature surrogate data: n_total states from n_snapshots states of a plain run."""
    import torch
    per = int(math.ceil(n_total / n_snapshots))
    X = torch.empty((per * n_snapshots, NI), dtype=torch.float32, device="cuda")
    T = torch.empty((per * n_snapshots,), dtype=torch.float32, device="cuda")
    for s in range(n_snapshots):
        if s:
            dg_step_rk(ctx, steps_between, cfl)
        dg_thermo_sample(ctx, X[s * per:(s + 1) * per], T[s * per:(s + 1) * per],
                         seed=seed * 1000003 + s)
    return X[:n_total], T[:n_total]


def collect_source(ctx, n_total, n_snapshots, steps_between, cfl=0.05, dt_fixed=0.0, seed=1):
    """Source surrogate data: raw features [n][7] (float32) and the plain (omega, jpi)
    [n][10] (float64) from n_snapshots states of a plain reacting run."""
    import torch
    per = int(math.ceil(n_total / n_snapshots))
    X = torch.empty((per * n_snapshots, NI), dtype=torch.float32, device="cuda")
    Y = torch.empty((per * n_snapshots, 10), dtype=torch.float64, device="cuda")
    for s in range(n_snapshots):
        if s:
            dg_step_rk(ctx, steps_between, cfl, dt_fixed)
        dg_chem_sample(ctx, X[s * per:(s + 1) * per], Y[s * per:(s + 1) * per], seed=seed * 1000003 + s)
    return X[:n_total], Y[:n_total]


def xavier_params(seed=0, n_out=1):
    rng = np.random.default_rng(seed)
    p = np.zeros(dg_mlp_nparams(n_out), dtype=np.float32)
    o = 0
    for fan_in, fan_out in ((NI, NH), (NH, NH), (NH, n_out)):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        p[o:o + fan_in * fan_out] = rng.uniform(-lim, lim, fan_in * fan_out)
        o += fan_in * fan_out + fan_out  # weights then zero biases
    return p


def _std(sd, floor):
    return np.maximum(sd, floor)


def standardise(X, T):
    """Temperature surrogate statistics: mean/std of each feature and of T (float64 [16]),
    and the standardised arrays (device FP32)."""
    import torch
    mx, sx, _, _ = dg_column_stats(X)
    sx = _std(sx, 1e-12)
    T2 = T.reshape(-1, 1)
    mt, st_, _, _ = dg_column_stats(T2)
    st_ = _std(st_, 1e-12)
    stats = np.concatenate([mx, sx, mt, st_])
    Xn = torch.empty(X.shape, dtype=torch.float32, device=X.device)
    Tn = torch.empty(T2.shape, dtype=torch.float32, device=X.device)
    dg_standardize(X, mx, sx, Xn)
    dg_standardize(T2, mt, st_, Tn)
    return Xn, Tn.reshape(-1), stats


def fit(Xn, Yn, epochs=20, batch=4096, lr=1e-3, seed=0, val_frac=0.1, log=None, lr_final=None):
    """Adam on the mean-squared error of standardised targets Yn ([n] or [n][n_out]); with
    lr_final the step size decays from lr to lr_final over the epochs (cosine).
    Returns (params float32 [P] device, history of (epoch, train, val))."""
    import torch
    n_out = 1 if Yn.dim() == 1 else Yn.shape[1]
    Y2 = Yn.reshape(-1, n_out)
    n = Xn.shape[0]
    rng = np.random.default_rng(seed)
    dev = Xn.device
    perm = torch.from_numpy(rng.permutation(n).astype(np.int64)).to(dev)
    nval = max(1, int(val_frac * n))
    ntr = n - nval

    def gather(A, idx):
        out = torch.empty((idx.shape[0], A.shape[1]), dtype=torch.float32, device=dev)
        dg_gather_rows(A, idx, out)
        return out

    Xv, Yv = gather(Xn, perm[:nval]), gather(Y2, perm[:nval])
    Xt, Yt = gather(Xn, perm[nval:]), gather(Y2, perm[nval:])
    batch = min(batch, ntr)
    params = torch.from_numpy(xavier_params(seed, n_out)).to(dev)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    ws = torch.empty(dg_mlp_workspace_bytes(batch, n_out) // 4 + 1, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    xb = torch.empty((batch, NI), dtype=torch.float32, device=dev)
    tb = torch.empty((batch, n_out), dtype=torch.float32, device=dev)
    hist = []
    step = 0
    for ep in range(epochs):
        lr_ep = lr if lr_final is None else \
            lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * ep / max(1, epochs - 1)))
        order = torch.from_numpy(rng.permutation(ntr).astype(np.int64)).to(dev)
        tot, nb = 0.0, 0
        for b0 in range(0, ntr - batch + 1, batch):
            idx = order[b0:b0 + batch]
            dg_gather_rows(Xt, idx, xb)
            dg_gather_rows(Yt, idx, tb)
            step += 1
            dg_mlp_train_step(params, m, v, xb, tb if n_out > 1 else tb.reshape(-1), step, lr_ep, loss, ws)
            tot += loss.item() if (nb % 50 == 0) else 0.0
            nb += 1
        vloss = validation_loss(params, Xv, Yv if n_out > 1 else Yv.reshape(-1))
        hist.append((ep, tot, vloss))
        if log:
            log("epoch %d  val mse %.3e" % (ep, vloss))
    return params, hist


def train(X, T, epochs=20, batch=4096, lr=1e-3, seed=0, val_frac=0.1, log=None, lr_final=None):
    """Temperature surrogate.  Returns (params float32 [P] host, stats float64 [16],
    history of (epoch, train, val))."""
    Xn, Tn, stats = standardise(X, T)
    params, hist = fit(Xn, Tn, epochs, batch, lr, seed, val_frac, log, lr_final)
    return params.cpu().numpy(), stats, hist


def source_stats(X, Y, ref_quantile=0.99, ref_fraction=1e-3, tol_check=0.05, tol_mass=0.05,
                 floor_fraction=0.1, box_margin=0.01):
    """Statistics of the source surrogate (float64 [DG_SRC_NSTATS]) and the standardised
    training arrays.  omega_ref (jpi_ref) = ref_fraction x the ref_quantile of |omega|
    (of jpi) over the samples, so the asinh map is logarithmic over the rates that matter
    and linear near zero; the trust box is the per-feature range of the samples widened
    by box_margin of its width on each side; both rate checks carry the absolute floor
    floor_fraction omega_ref (the sampled-node check accepts |S_learned - S_plain| <=
    tol_check sum|S_plain| + floor)."""
    import torch
    w_ref = max(dg_abs_quantile(Y, 0, 5, ref_quantile) * ref_fraction, 1e-30)
    j_ref = max(dg_abs_quantile(Y, 5, 5, ref_quantile) * ref_fraction, 1e-30)
    ref = np.array([w_ref] * 5 + [j_ref] * 5)
    mz, sz, _, _ = dg_column_stats(Y, ref=ref)
    sz = _std(sz, 1e-6)
    mx, sx, lo, hi = dg_column_stats(X)
    sx = _std(sx, 1e-12)
    st = np.zeros(DG_SRC_NSTATS)
    st[0:7], st[7:14] = mx, sx
    st[14:24], st[24:34] = mz, sz
    st[34], st[35] = w_ref, j_ref
    st[36:43] = lo - box_margin * (hi - lo)
    st[43:50] = hi + box_margin * (hi - lo)
    st[50], st[51], st[52] = tol_check, tol_mass, floor_fraction * w_ref
    Xn = torch.empty(X.shape, dtype=torch.float32, device=X.device)
    Zn = torch.empty(Y.shape, dtype=torch.float32, device=X.device)
    dg_standardize(X, mx, sx, Xn)
    dg_standardize(Y, mz, sz, Zn, ref=ref)
    return Xn, Zn, st


def train_source(X, Y, epochs=30, batch=4096, lr=2e-3, seed=0, val_frac=0.1, log=None, lr_final=None,
                 **stat_kw):
    """Source surrogate (ten outputs).  Returns (params float32 [P] host, stats float64
    [DG_SRC_NSTATS], history)."""
    Xn, Zn, st = source_stats(X, Y, **stat_kw)
    params, hist = fit(Xn, Zn, epochs, batch, lr, seed, val_frac, log, lr_final)
    return params.cpu().numpy(), st, hist


def validation_loss(params, Xv, Yv):
    return dg_mlp_loss(params, Xv, Yv)
