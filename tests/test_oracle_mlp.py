"""Pins of the oracle's learned-temperature perceptron (forward, back-propagation, Adam)."""
import math

import numpy as np


def _params(orc, seed=0, scale=0.5):
    rng = np.random.default_rng(seed)
    return scale * rng.normal(size=orc.mlp_nparams())


def test_layout_size(orc):
    assert orc.mlp_nparams() == 64 * 7 + 64 + 64 * 64 + 64 + 64 + 1


def test_gelu_identities(orc):
    # gelu(x) - gelu(-x) = x for the tanh form; gelu(0) = 0; tanh form within 1e-3 of x Phi(x)
    for x in np.linspace(-6, 6, 49):
        assert abs(orc.gelu(x) - orc.gelu(-x) - x) < 1e-14 * max(1, abs(x))
        exact = 0.5 * x * (1 + math.erf(x / math.sqrt(2)))
        assert abs(orc.gelu(x) - exact) < 1e-3
        h = 1e-6
        fd = (orc.gelu(x + h) - orc.gelu(x - h)) / (2 * h)
        assert abs(orc.gelu_d(x) - fd) < 1e-8
    assert orc.gelu(0.0) == 0.0


def test_forward_single_path_by_hand(orc):
    """Only one path through the network carries weight: y = b3 + w3 gelu(W2 gelu(W1 x))."""
    p = np.zeros(orc.mlp_nparams())
    off_b1 = 64 * 7
    off_w2 = off_b1 + 64
    off_b2 = off_w2 + 64 * 64
    off_w3 = off_b2 + 64
    p[0 * 7 + 3] = 0.7          # W1[0][3]
    p[off_b1 + 0] = -0.2
    p[off_w2 + 5 * 64 + 0] = 1.3  # W2[5][0]
    p[off_b2 + 5] = 0.1
    p[off_w3 + 5] = -2.0
    p[-1] = 0.25
    x = np.array([[0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7]])
    h1 = orc.gelu(0.7 * 0.4 - 0.2)
    h2 = orc.gelu(1.3 * h1 + 0.1)
    # every other hidden unit sees gelu(0) = 0 except through the biases (zero here)
    assert abs(orc.mlp_forward(p, x)[0] - (0.25 - 2.0 * h2)) < 1e-15


def test_gradient_matches_finite_differences(orc):
    rng = np.random.default_rng(1)
    p = _params(orc, 1, 0.3)
    X = rng.normal(size=(5, 7))
    t = rng.normal(size=5)
    loss, g = orc.mlp_loss_grad(p, X, t)
    idx = rng.choice(len(p), size=60, replace=False)
    idx = np.concatenate([idx, [len(p) - 1, 64 * 7, 64 * 7 + 64 + 3]])
    for i in idx:
        h = 1e-5 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (orc.mlp_loss_grad(pp, X, t)[0] - orc.mlp_loss_grad(pm, X, t)[0]) / (2 * h)
        # central differences: truncation ~h^2, rounding ~eps*loss/h (~1e-10 absolute)
        assert abs(fd - g[i]) < 1e-6 * abs(g[i]) + 2e-9, (i, fd, g[i])
    y = orc.mlp_forward(p, X)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-14 * max(1, loss)


def test_adam_first_step_closed_form(orc):
    """At step 1 the bias-corrected moments are g and g^2: dp = -lr g / (|g| + eps)."""
    g = np.array([3.0, -1e-3, 0.0, 1e-9, -7.5])
    p = np.zeros(5)
    m = np.zeros(5)
    v = np.zeros(5)
    orc.adam_step(p, m, v, g, 1, lr=1e-3)
    assert np.allclose(p, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=0)
    # two steps with a constant gradient: still -lr g/(|g|+eps) per step
    orc.adam_step(p, m, v, g, 2, lr=1e-3)
    assert np.allclose(p, -2e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-20)


def test_training_reduces_loss_on_a_smooth_map(orc):
    """Full-batch Adam on a smooth 7-input target must reduce the loss tenfold."""
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, size=(256, 7))
    t = np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 0.3 * X[:, 6]
    p = _params(orc, 3, 0.2)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = orc.mlp_loss_grad(p, X, t)[0]
    for s in range(1, 301):
        _, g = orc.mlp_loss_grad(p, X, t)
        orc.adam_step(p, m, v, g, s, lr=3e-3)
    assert orc.mlp_loss_grad(p, X, t)[0] < 0.1 * l0


# ---- several outputs (the chemistry-source surrogate has ten)

def _slice(p, no, o):
    """Parameters of the one-output network made of output row o of an no-output one."""
    head = 64 * 7 + 64 + 64 * 64 + 64
    w3 = p[head:head + no * 64].reshape(no, 64)
    b3 = p[head + no * 64:]
    return np.concatenate([p[:head], w3[o], [b3[o]]])


def test_multi_output_layout(orc):
    for no in (1, 2, 10, 16):
        assert orc.mlp_nparams(no) == 64 * 7 + 64 + 64 * 64 + 64 + no * 64 + no
    assert orc.mlp_nparams(1) == orc.mlp_nparams()


def test_multi_output_rows_are_independent_heads(orc):
    """Output o of an n_out network equals the one-output network of row o (forward), and
    loss / gradients are the averages over outputs of the single-output ones: the shared
    hidden layers receive the mean of the heads' back-propagated signals."""
    rng = np.random.default_rng(5)
    no = 10
    p = 0.3 * rng.normal(size=orc.mlp_nparams(no))
    X = rng.normal(size=(6, 7))
    T = rng.normal(size=(6, no))
    Y = orc.mlp_forward(p, X, no)
    assert Y.shape == (6, no)
    loss, g = orc.mlp_loss_grad(p, X, T, no)
    head = 64 * 7 + 64 + 64 * 64 + 64
    g_shared = np.zeros(head)
    l_sum = 0.0
    for o in range(no):
        q = _slice(p, no, o)
        assert np.allclose(orc.mlp_forward(q, X), Y[:, o], rtol=0, atol=1e-14)
        lo, go = orc.mlp_loss_grad(q, X, T[:, o])
        l_sum += lo
        g_shared += go[:head]
        # the head's own weights: gradient of the mean loss = gradient of its loss / no
        assert np.allclose(g[head + o * 64:head + (o + 1) * 64], go[head:head + 64] / no, rtol=1e-12, atol=1e-16)
        assert abs(g[head + no * 64 + o] - go[-1] / no) < 1e-14
    assert abs(loss - l_sum / no) < 1e-13 * max(1.0, loss)
    assert np.allclose(g[:head], g_shared / no, rtol=1e-11, atol=1e-15)


def test_multi_output_gradient_matches_finite_differences(orc):
    rng = np.random.default_rng(7)
    no = 10
    p = 0.3 * rng.normal(size=orc.mlp_nparams(no))
    X = rng.normal(size=(4, 7))
    T = rng.normal(size=(4, no))
    loss, g = orc.mlp_loss_grad(p, X, T, no)
    idx = np.concatenate([rng.choice(len(p), size=40, replace=False), [len(p) - 1, len(p) - no - 1]])
    for i in idx:
        h = 1e-5 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (orc.mlp_loss_grad(pp, X, T, no)[0] - orc.mlp_loss_grad(pm, X, T, no)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * abs(g[i]) + 2e-9, (i, fd, g[i])
    Y = orc.mlp_forward(p, X, no)
    assert abs(loss - np.mean((Y - T) ** 2)) < 1e-14 * max(1, loss)


# ---- the oracle's learned-source evaluation (decode, acceptance flags, projection)

def _const_net(orc, c):
    """Ten-output network whose outputs are the constants c (W3 = 0, b3 = c)."""
    p = np.zeros(orc.mlp_nparams(10))
    p[-10:] = c
    return p


def _stats(mu, sd, w_ref=2.0, j_ref=3.0, lo=-1e30, hi=1e30, tol_mass=0.05):
    st = np.zeros(53)
    st[0:7] = [0.2, 0.2, 0.2, 0.2, 0.2, math.log(0.05), 2500.0]
    st[7:14] = [0.1, 0.1, 0.1, 0.1, 0.1, 1.0, 1500.0]
    st[14:24] = mu
    st[24:34] = sd
    st[34], st[35] = w_ref, j_ref
    st[36:43], st[43:50] = lo, hi
    st[50], st[51], st[52] = 0.05, tol_mass, 0.0
    return st


def test_source_surrogate_decode_closed_form(orc):
    """Constant network outputs y: omega_s = w_ref sinh(mu + sd y), jpi = max(0, j_ref
    sinh(...)), the projection sum-free, S = omega / (1 + dt jpi)."""
    c = np.array([0.3, -0.2, 0.1, 0.5, -0.4, 0.2, -1.0, 0.7, 0.0, 1.3])
    mu = np.linspace(-0.5, 0.5, 10)
    sd = np.linspace(0.5, 2.0, 10)
    st = _stats(mu, sd, tol_mass=10.0)
    rhos = np.array([[0.01, 0.02, 0.03, 0.005, 0.0015], [1.0, 0.1, 0.2, 0.3, 0.4]])
    T = np.array([3000.0, 800.0])
    dt = 1e-6
    S, ok, om, jpi = orc.chem_surrogate_source(_const_net(orc, c), st, rhos, T, dt)
    z = mu + sd * c
    om_ref = 2.0 * np.sinh(z[:5])
    jpi_ref = np.maximum(0.0, 3.0 * np.sinh(z[5:]))
    for r in range(2):
        assert np.allclose(om[r], om_ref, rtol=1e-14, atol=0)
        assert np.allclose(jpi[r], jpi_ref, rtol=1e-14, atol=0)
        proj = om_ref - np.abs(om_ref) * om_ref.sum() / np.abs(om_ref).sum()
        assert np.allclose(S[r], proj / (1.0 + dt * jpi_ref), rtol=1e-13, atol=1e-15)
        assert abs(S[r].sum() * 0 + (proj).sum()) < 1e-14 * np.abs(om_ref).sum()
    assert ok.all()


def test_source_surrogate_projection_is_mass_conserving(orc):
    rng = np.random.default_rng(11)
    p = 0.4 * rng.normal(size=orc.mlp_nparams(10))
    st = _stats(np.zeros(10), np.ones(10), w_ref=1e3, j_ref=1e2, tol_mass=1e9)
    rhos = rng.uniform(1e-3, 0.1, size=(64, 5))
    T = rng.uniform(300, 5000, size=64)
    S, ok, om, jpi = orc.chem_surrogate_source(p, st, rhos, T, dt=0.0)
    assert np.all(np.abs(S.sum(axis=1)) <= 1e-13 * np.abs(om).sum(axis=1))
    # a species whose raw rate is zero stays zero (the correction is proportional to |omega|)
    p2 = p.copy()
    head = 64 * 7 + 64 + 64 * 64 + 64
    p2[head + 2 * 64:head + 3 * 64] = 0.0   # head of output 2 (omega_3)
    p2[head + 10 * 64 + 2] = 0.0            # its bias
    S2, _, om2, _ = orc.chem_surrogate_source(p2, st, rhos, T)
    assert np.all(om2[:, 2] == 0.0) and np.all(S2[:, 2] == 0.0)


def test_source_surrogate_acceptance_flags(orc):
    c = np.array([0.3, -0.2, 0.1, 0.5, -0.4, 0, 0, 0, 0, 0])
    rhos = np.array([[0.01, 0.02, 0.03, 0.005, 0.0015]])
    T = np.array([3000.0])
    om = 2.0 * np.sinh(c[:5])
    imbalance = abs(om.sum()) / np.abs(om).sum()
    p = _const_net(orc, c)
    # mass balance just above / below the raw imbalance
    _, ok, _, _ = orc.chem_surrogate_source(p, _stats(np.zeros(10), np.ones(10), tol_mass=imbalance * 1.001), rhos, T)
    assert ok.all()
    _, ok, _, _ = orc.chem_surrogate_source(p, _stats(np.zeros(10), np.ones(10), tol_mass=imbalance * 0.999), rhos, T)
    assert not ok.any()
    # box: T outside [lo, hi] rejects
    lo = np.full(7, -1e30)
    hi = np.full(7, 1e30)
    hi[6] = 2999.0
    _, ok, _, _ = orc.chem_surrogate_source(p, _stats(np.zeros(10), np.ones(10), lo=lo, hi=hi, tol_mass=1.0), rhos, T)
    assert not ok.any()
