"""Training driver for the learned temperature surrogate.

Data come from the plain solver itself: a mixture context is stepped with the plain
Newton temperature solve and ``dg_thermo_sample`` draws node states (raw features
Y_1..Y_5, ln rho, e and the converged T) after every ``steps_between`` RK steps.  The
driver standardises the data, initialises the network (Xavier-uniform from a seed) and
runs Adam epochs with ``dg_mlp_train_step``; forward, back-propagation, the gradient
reduction and the update all run in libdg's kernels.  PyTorch only holds the device
buffers and draws the epoch permutations.
"""
import math

import numpy as np

from . import (dg_mlp_nparams, dg_mlp_train_step, dg_mlp_workspace_bytes, dg_step_rk,
               dg_thermo_sample)

NI, NH = 7, 64


def collect(ctx, n_total, n_snapshots, steps_between, cfl=0.3, seed=1):
    """Sample n_total states from n_snapshots states of a plain-solver run."""
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


def xavier_params(seed=0):
    rng = np.random.default_rng(seed)
    p = np.zeros(dg_mlp_nparams(), dtype=np.float32)
    o = 0
    for fan_in, fan_out in ((NI, NH), (NH, NH), (NH, 1)):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        p[o:o + fan_in * fan_out] = rng.uniform(-lim, lim, fan_in * fan_out)
        o += fan_in * fan_out + fan_out  # weights then zero biases
    return p


def standardise(X, T):
    """Dataset statistics: mean/std of each feature and of T (float64 [16])."""
    mx = X.double().mean(0)
    sx = X.double().std(0).clamp_min(1e-12)
    mt = T.double().mean()
    st = T.double().std().clamp_min(1e-12)
    stats = np.concatenate([mx.cpu().numpy(), sx.cpu().numpy(), [mt.item(), st.item()]])
    Xn = ((X.double() - mx) / sx).float().contiguous()
    Tn = ((T.double() - mt) / st).float().contiguous()
    return Xn, Tn, stats


def train(X, T, epochs=20, batch=4096, lr=1e-3, seed=0, val_frac=0.1, log=None):
    """Adam on mean-squared error of the standardised temperature.

    Returns (params float32 [P] host, stats float64 [16], history of (epoch, train, val)).
    """
    import torch
    Xn, Tn, stats = standardise(X, T)
    n = Xn.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(n, generator=g).cuda()
    nval = max(1, int(val_frac * n))
    Xv, Tv = Xn[perm[:nval]], Tn[perm[:nval]]
    Xt, Tt = Xn[perm[nval:]], Tn[perm[nval:]]
    params = torch.from_numpy(xavier_params(seed)).cuda()
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    ws = torch.empty(dg_mlp_workspace_bytes(batch) // 4 + 1, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    hist = []
    step = 0
    for ep in range(epochs):
        order = torch.randperm(Xt.shape[0], generator=g).cuda()
        tot, nb = 0.0, 0
        for b0 in range(0, Xt.shape[0] - batch + 1, batch):
            idx = order[b0:b0 + batch]
            xb, tb = Xt[idx].contiguous(), Tt[idx].contiguous()
            step += 1
            dg_mlp_train_step(params, m, v, xb, tb, step, lr, loss, ws)
            tot += loss.item() if (nb % 50 == 0) else 0.0
            nb += 1
        vloss = validation_loss(params, Xv, Tv)
        hist.append((ep, tot, vloss))
        if log:
            log("epoch %d  val mse %.3e" % (ep, vloss))
    return params.cpu().numpy(), stats, hist


def validation_loss(params, Xv, Tv):
    import torch
    from . import dg_mlp_forward
    y = torch.empty_like(Tv)
    dg_mlp_forward(params, Xv, y, tensor_cores=0)
    return float(((y - Tv) ** 2).mean().item())
