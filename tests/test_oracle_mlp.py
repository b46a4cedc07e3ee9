"""Pins of the oracle's learned-temperature perceptron (forward, back-propagation, Adam)."""
import math

import pytest

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


# ---- the oracle's learned-source evaluation (reading R18s: decode, trust box, mass
# balance, projection, sampled check, per-tile decision; rounding bound of the BF16 network)

def _const_net(orc, c):
    """Ten-output network whose outputs are the constants c (W3 = 0, b3 = c)."""
    p = np.zeros(orc.mlp_nparams(10))
    p[-10:] = c
    return p


def _stats(mu, sd, w_ref=2.0, j_ref=3.0, lo=-1e30, hi=1e30, tol_mass=0.05, tol_check=0.05, floor=0.0):
    st = np.zeros(53)
    st[0:7] = [0.2, 0.2, 0.2, 0.2, 0.2, math.log(0.05), 2500.0]
    st[7:14] = [0.1, 0.1, 0.1, 0.1, 0.1, 1.0, 1500.0]
    st[14:24] = mu
    st[24:34] = sd
    st[34], st[35] = w_ref, j_ref
    st[36:43], st[43:50] = lo, hi
    st[50], st[51], st[52] = tol_check, tol_mass, floor
    return st


def _net_for_rates(orc, omega, w_ref=1.0):
    """Constant network whose decoded rates are omega (mu 0, sd 1: b3 = asinh(omega/w_ref)),
    jpi = 0."""
    c = np.zeros(10)
    c[:5] = np.arcsinh(np.asarray(omega) / w_ref)
    return _const_net(orc, c)


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
    r = orc.chem_surrogate_source(_const_net(orc, c), st, rhos, T, dt)
    z = mu + sd * c
    om_ref = 2.0 * np.sinh(z[:5])
    jpi_ref = np.maximum(0.0, 3.0 * np.sinh(z[5:]))
    for k in range(2):
        assert np.allclose(r["omega"][k], om_ref, rtol=1e-14, atol=0)
        assert np.allclose(r["jpi"][k], jpi_ref, rtol=1e-14, atol=0)
        proj = om_ref - np.abs(om_ref) * om_ref.sum() / np.abs(om_ref).sum()
        assert np.allclose(r["S_learned"][k], proj / (1.0 + dt * jpi_ref), rtol=1e-13, atol=1e-15)
        assert abs(proj.sum()) < 1e-14 * np.abs(om_ref).sum()
    assert (r["inside"] & r["mass_ok"]).all()


def test_source_surrogate_projection_is_mass_conserving(orc):
    rng = np.random.default_rng(11)
    p = 0.4 * rng.normal(size=orc.mlp_nparams(10))
    st = _stats(np.zeros(10), np.ones(10), w_ref=1e3, j_ref=1e2, tol_mass=1e9)
    rhos = rng.uniform(1e-3, 0.1, size=(64, 5))
    T = rng.uniform(300, 5000, size=64)
    r = orc.chem_surrogate_source(p, st, rhos, T, dt=0.0)
    assert np.all(np.abs(r["S_learned"].sum(axis=1)) <= 1e-13 * np.abs(r["omega"]).sum(axis=1))
    # a species whose raw rate is zero stays zero (the correction is proportional to |omega|)
    p2 = p.copy()
    head = 64 * 7 + 64 + 64 * 64 + 64
    p2[head + 2 * 64:head + 3 * 64] = 0.0   # head of output 2 (omega_3)
    p2[head + 10 * 64 + 2] = 0.0            # its bias
    r2 = orc.chem_surrogate_source(p2, st, rhos, T)
    assert np.all(r2["omega"][:, 2] == 0.0) and np.all(r2["S_learned"][:, 2] == 0.0)


def test_mass_balance_threshold_both_sides(orc):
    """sum omega / sum |omega| = 0.11 / 3.11 = 0.0354 passes tau_m = 0.05; 0.17 / 3.17 =
    0.0536 fails; exactly at the threshold passes (<=)."""
    rhos = np.array([[0.01, 0.02, 0.03, 0.005, 0.0015]])
    T = np.array([3000.0])
    st = _stats(np.zeros(10), np.ones(10), w_ref=1.0)
    for last, ok in ((0.11, True), (0.17, False)):
        r = orc.chem_surrogate_source(_net_for_rates(orc, [1.0, -1.0, 0.5, -0.5, last]), st, rhos, T)
        assert bool(r["mass_ok"][0]) is ok


def test_floor_both_sides(orc):
    """One rate of 0.2: |sum| = sum|.| = 0.2 passes tau_m = 0.05 only through the floor:
    0.2 <= 0.01 + floor holds for floor 0.195, not for 0.185."""
    rhos = np.array([[0.01, 0.02, 0.03, 0.005, 0.0015]])
    T = np.array([3000.0])
    net = _net_for_rates(orc, [0.2, 0.0, 0.0, 0.0, 0.0])
    for floor, ok in ((0.195, True), (0.185, False)):
        r = orc.chem_surrogate_source(net, _stats(np.zeros(10), np.ones(10), w_ref=1.0, floor=floor), rhos, T)
        assert bool(r["mass_ok"][0]) is ok


def test_trust_box_both_sides(orc):
    rhos = np.array([[0.01, 0.02, 0.03, 0.005, 0.0015]])
    T = np.array([3000.0])
    net = _net_for_rates(orc, [0.3, -0.3, 0.0, 0.0, 0.0])
    lo, hi = np.full(7, -1e30), np.full(7, 1e30)
    for h, ok in ((3000.0, True), (2999.99, False)):
        hi[6] = h
        r = orc.chem_surrogate_source(net, _stats(np.zeros(10), np.ones(10), lo=lo, hi=hi), rhos, T)
        assert bool(r["inside"][0]) is ok
    hi[6] = 1e30
    for lval, ok in ((np.log(0.0665), True), (np.log(0.0666), False)):  # ln rho = ln 0.0665
        lo[5] = lval
        r = orc.chem_surrogate_source(net, _stats(np.zeros(10), np.ones(10), lo=lo, hi=hi), rhos, T)
        assert bool(r["inside"][0]) is ok


def _hot_state(n):
    rhos = np.tile(np.array([[0.012, 0.021, 0.030, 0.006, 0.0019]]), (n, 1))
    return rhos, np.full(n, 3500.0)


def test_sampled_check_both_sides_and_tiles(orc):
    """Learned rates = the plain source + d (e_1 - e_2): the sampled check passes at
    d = 0.9 (tau_c sum|S| + floor) and fails at 1.1 times it; 40 nodes make two tiles
    (32 + 8); a node of the second tile outside the box rejects that tile only, whose
    nodes then take the plain source."""
    import workloads as W
    sp, R = W.species_table(), W.reaction_table()
    n = 40
    rhos, T = _hot_state(n)
    _, _, S_p = orc.chem_eval(sp, R, rhos, T, 0.0)
    thr = 0.05 * np.abs(S_p[0]).sum()
    assert thr > 0
    w_ref = np.abs(S_p[0]).max()
    for kappa, flag in ((0.9, 0), (1.1, 2)):
        om = S_p[0].copy()
        om[0] += kappa * thr
        om[1] -= kappa * thr
        net = _net_for_rates(orc, om, w_ref)
        st = _stats(np.zeros(10), np.ones(10), w_ref=w_ref, tol_mass=0.05)
        r = orc.chem_surrogate_source(net, st, rhos, T, species=sp, reactions=R, call=3)
        assert list(r["tile_flag"]) == [flag, flag]
        assert not r["tile_ambiguous"].any()
    # tile granularity: node 35 outside the box (T above hi)
    T2 = T.copy()
    T2[35] = 3600.0
    hi = np.full(7, 1e30)
    hi[6] = 3550.0
    om = S_p[0].copy()
    om[0] += 0.5 * thr
    om[1] -= 0.5 * thr
    st = _stats(np.zeros(10), np.ones(10), w_ref=w_ref, hi=hi)
    r = orc.chem_surrogate_source(_net_for_rates(orc, om, w_ref), st, rhos, T2, species=sp, reactions=R, call=0)
    assert list(r["tile_flag"]) == [0, 1]
    assert np.allclose(r["S"][:32], om[None, :], rtol=1e-12, atol=1e-12 * w_ref)
    _, _, S_p2 = orc.chem_eval(sp, R, rhos, T2, 0.0)
    assert np.array_equal(r["S"][32:], S_p2[32:])
    # the sampled node of each tile lies inside it
    assert 0 <= r["sampled_node"][0] < 32 and 32 <= r["sampled_node"][1] < 40


def test_splitmix64_published_output(orc):
    """SplitMix64 (Steele, Lea & Flood 2014): the reference generator's first output from
    state 0 is 0xE220A8397B1DCDAF; the sampled-node hash is a single step of it."""
    assert orc.splitmix64([0])[0] == 0xE220A8397B1DCDAF
    # one step from state x: the output depends on x only through x + the golden increment
    g = 0x9E3779B97F4A7C15
    assert orc.splitmix64([g])[0] != orc.splitmix64([0])[0]


def _bf16(x):
    """Round float32 values to BF16 (round to nearest, ties to even), returned as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _gelu32(z, rng=None, eps=0.0):
    k = np.float32(math.sqrt(2.0 / math.pi))
    arg = (k * (z + np.float32(0.044715) * z * z * z)).astype(np.float32)
    t = np.tanh(arg.astype(np.float64))
    if rng is not None:
        t = t + rng.uniform(-eps, eps, size=t.shape)
    return (np.float32(0.5) * z * (np.float32(1.0) + t.astype(np.float32))).astype(np.float32)


def _emulated_forward(p, X, no, rng=None, eps=0.0):
    """The GPU's BF16 forward emulated bit for bit in its roundings: inputs, W1, W2 and the
    first hidden layer's activations rounded to BF16, sums in FP32 (products of BF16 values
    are exact in FP64), GELU in FP32 (tanh optionally perturbed by up to eps), output layer
    in FP32 with FP32 weights."""
    NI_, NH_ = 7, 64
    p32 = p.astype(np.float32)
    W1 = _bf16(p32[:NH_ * NI_].reshape(NH_, NI_))
    b1 = p32[NH_ * NI_:NH_ * NI_ + NH_]
    o = NH_ * NI_ + NH_
    W2 = _bf16(p32[o:o + NH_ * NH_].reshape(NH_, NH_))
    b2 = p32[o + NH_ * NH_:o + NH_ * NH_ + NH_]
    o3 = o + NH_ * NH_ + NH_
    W3 = p32[o3:o3 + no * NH_].reshape(no, NH_)
    b3 = p32[o3 + no * NH_:]
    xb = _bf16(X.astype(np.float32))
    z1 = ((xb.astype(np.float64) @ W1.T.astype(np.float64)).astype(np.float32) + b1).astype(np.float32)
    a1 = _bf16(_gelu32(z1, rng, eps))
    z2 = ((a1.astype(np.float64) @ W2.T.astype(np.float64)).astype(np.float32) + b2).astype(np.float32)
    a2 = _gelu32(z2, rng, eps)
    return (a2.astype(np.float64) @ W3.T.astype(np.float64)).astype(np.float32) + b3


@pytest.mark.parametrize("eps", [0.0, 2.0 ** -10.5])
def test_bf16_error_model_against_emulation(orc, eps):
    """The first-order model's standard deviation against the actual error of a BF16
    evaluation emulated bit for bit: every output error within 8 sd, and the RMS of
    error / sd between 0.3 and 1.3 (a model that drops a layer's rounding or misweights
    one is off by more)."""
    rng = np.random.default_rng(17)
    no = 10
    P = orc.mlp_nparams(no)
    p = np.zeros(P)
    lim1, lim2, lim3 = math.sqrt(6 / 71), math.sqrt(6 / 128), math.sqrt(6 / 74)
    p[:448] = rng.uniform(-lim1, lim1, 448) * 2.0
    p[448:512] = 0.1 * rng.normal(size=64)
    p[512:512 + 4096] = rng.uniform(-lim2, lim2, 4096) * 1.5
    p[4608:4672] = 0.1 * rng.normal(size=64)
    p[4672:4672 + 640] = rng.uniform(-lim3, lim3, 640)
    p[-10:] = 0.1 * rng.normal(size=10)
    p = p.astype(np.float32).astype(np.float64)
    X = rng.normal(size=(3000, 7))
    y, sd = orc.mlp_forward_sd(p, X, no, eps_t=eps)
    ye = _emulated_forward(p, X, no, rng if eps > 0 else None, eps).astype(np.float64)
    ratio = (ye - y) / sd
    assert np.abs(ratio).max() <= 8.0, np.abs(ratio).max()
    rms = math.sqrt(np.mean(ratio ** 2))
    assert 0.3 <= rms <= 1.3, rms


def test_bf16_rounding_ties_to_even(orc):
    """BF16 keeps 8 significand bits: near 1 the spacing is 2^-7.  1 + 2^-8 lies halfway
    between 1 and 1 + 2^-7 and goes to the even neighbour 1; 1 + 3 2^-8 lies halfway between
    1 + 2^-7 (odd) and 1 + 2^-6 (even); just above a halfway point rounds up."""
    x = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -20, -(1 + 2.0 ** -8 + 2.0 ** -20),
                  3.0, 2.0 ** -130], dtype=np.float32)
    want = np.array([1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -(1 + 2.0 ** -7), 3.0, 2.0 ** -130], dtype=np.float32)
    assert np.array_equal(orc.bf16(x), want)


def test_bf16_emulation_and_its_difference_model(orc):
    """The oracle's BF16 emulation equals this file's independent one bit for bit; a
    'GPU' that differs from it only where the GPU's arithmetic is not reproduced (FP32 sums
    in another order, tanh off by up to 2^-16) stays within 8 standard deviations of the
    difference model (u = 0) plus the effect of every hidden unit close enough to a BF16
    rounding boundary to round the other way."""
    rng = np.random.default_rng(23)
    no = 10
    p = (0.25 * rng.normal(size=orc.mlp_nparams(no))).astype(np.float32).astype(np.float64)
    X32 = rng.normal(size=(2000, 7)).astype(np.float32)
    y_o = orc.mlp_forward_bf16(p, X32, no)
    y_t = _emulated_forward(p, X32.astype(np.float64), no).astype(np.float64)
    assert np.array_equal(y_o, y_t)
    # a perturbed emulation: sequential FP32 sums and a perturbed tanh
    NI_, NH_ = 7, 64
    p32 = p.astype(np.float32)
    W1 = _bf16(p32[:448].reshape(NH_, NI_))
    b1 = p32[448:512]
    W2 = _bf16(p32[512:4608].reshape(NH_, NH_))
    b2 = p32[4608:4672]
    W3 = p32[4672:4672 + 640].reshape(no, NH_)
    b3 = p32[-no:]

    def seq(a, W, b):
        acc = np.tile(b.astype(np.float32), (a.shape[0], 1))
        for i in range(a.shape[1]):
            acc = (acc + a[:, i:i + 1] * W[:, i][None, :]).astype(np.float32)
        return acc

    xb = _bf16(X32)
    a1 = _bf16(_gelu32(seq(xb, W1, b1), rng, 2.0 ** -16))
    a2 = _gelu32(seq(a1, W2, b2), rng, 2.0 ** -16)
    y_g = seq(a2, W3, b3).astype(np.float64)
    _, sd = orc.mlp_forward_sd(p, X32.astype(np.float64), no, u=0.0)
    _, fl = orc.mlp_forward_bf16(p, X32, no, want_flip=True)
    r = np.abs(y_g - y_o) / (8.0 * sd + fl)
    assert r.max() <= 1.0, r.max()
    # without the flip allowance the largest differences are not covered: it is needed, and
    # it is added only at samples with a hidden unit near a rounding boundary
    assert (np.abs(y_g - y_o) / (8.0 * sd)).max() > 1.0
    assert 0.0 < np.mean(fl.max(axis=1) > 0) < 0.8


def test_positivity_rule_both_sides(orc):
    """Rule 5b: a learned consumption of species 1 at rate c (balanced by production of
    species 2) passes when rho_1 + dt S_1 >= 0 and fails when the step would take more than
    the species holds; with dt = 0 (a right-hand side) it always passes."""
    rhos = np.array([[0.01, 0.02, 0.03, 0.005, 0.0015]])
    T = np.array([3000.0])
    st = _stats(np.zeros(10), np.ones(10), w_ref=1.0)
    net = _net_for_rates(orc, [-100.0, 100.0, 0.0, 0.0, 0.0])
    for dt, ok in ((0.9e-4, True), (1.1e-4, False), (0.0, True)):  # rho_1 / 100 = 1e-4
        r = orc.chem_surrogate_source(net, st, rhos, T, dt)
        assert bool(r["positive"][0]) is ok and bool(r["mass_ok"][0]) is ok, (dt, r["positive"])


def _refresh_case(orc, n=96, seed=21):
    import workloads as W
    rng = np.random.default_rng(seed)
    sp, R = W.species_table(), W.reaction_table()
    rhos = np.array([[0.012, 0.021, 0.030, 0.006, 0.0019]]) * rng.uniform(0.5, 1.5, size=(n, 5))
    T = rng.uniform(2000.0, 4000.0, size=n)
    p = 0.4 * rng.normal(size=orc.mlp_nparams(10))
    om, jd, _ = orc.chem_eval(sp, R, rhos, T, 0.0)
    st = _stats(np.zeros(10), np.ones(10), w_ref=np.abs(om).mean(), j_ref=np.abs(jd).mean(), tol_mass=1e9)
    return sp, R, rhos, T, p, st


def test_plain_correction_is_exact_at_the_refresh_state(orc):
    """Step 9 of R18s: with the corrections taken at a state, the corrected network gives
    the plain rates there (omega, and jpi = max(0, -d omega / d rho) through the decoded
    value before its clamp), hence the plain point-implicit source and mass balance; nodes
    whose decoded jpi is negative while the plain one is positive are present, so a
    correction taken after the clamp would fail."""
    sp, R, rhos, T, p, st = _refresh_case(orc)
    dt = 3e-7
    om_p, jd, S_p = orc.chem_eval(sp, R, rhos, T, dt)
    c = orc.chem_surrogate_correction(p, st, rhos, T, species=sp, reactions=R)
    r = orc.chem_surrogate_source(p, st, rhos, T, dt, correction=c)
    raw = orc.chem_surrogate_source(p, st, rhos, T, dt)
    assert ((raw["jpi_raw"] < 0) & (-jd > 0)).sum() >= 10
    scale = np.abs(om_p).sum(axis=1, keepdims=True)
    # up to the rounding of (omega - omega^) + omega^ (FP64, relative to the larger part)
    eps = 2.0 ** -52
    tol_om = 4 * eps * (np.abs(om_p) + np.abs(raw["omega_net"]))
    assert np.all(np.abs(r["omega"] - om_p) <= tol_om)
    tol_j = 4 * eps * (np.abs(jd) + np.abs(raw["jpi_raw"]))
    assert np.all(np.abs(r["jpi"] - np.maximum(0.0, -jd)) <= tol_j)
    assert np.all(np.abs(r["S_learned"] - S_p) <= 1e-13 * scale + 2 * tol_om.sum(axis=1, keepdims=True))
    # the uncorrected network is far from the plain source on the same nodes
    assert np.median(np.abs(raw["S_learned"] - S_p).sum(axis=1) / scale[:, 0]) > 0.1


def test_plain_correction_error_is_first_order_in_the_state_change(orc):
    """A state u0 + h d away from the refresh state u0: the corrected error
    [net(u) - net(u0)] - [plain(u) - plain(u0)] halves with h (first order), while the
    uncorrected network's error stays of its own size."""
    sp, R, rhos, T, p, st = _refresh_case(orc, n=64, seed=22)
    rng = np.random.default_rng(23)
    d_rho = rhos * rng.uniform(-1.0, 1.0, size=rhos.shape)
    d_T = T * rng.uniform(-1.0, 1.0, size=T.shape)
    c = orc.chem_surrogate_correction(p, st, rhos, T, species=sp, reactions=R)
    errs, raw_errs = [], []
    for h in (2e-3, 1e-3, 5e-4):
        r1, T1 = rhos + h * d_rho, T + h * d_T
        _, _, S_p = orc.chem_eval(sp, R, r1, T1, 0.0)
        errs.append(np.linalg.norm(orc.chem_surrogate_source(p, st, r1, T1, correction=c)["S_learned"] - S_p))
        raw_errs.append(np.linalg.norm(orc.chem_surrogate_source(p, st, r1, T1)["S_learned"] - S_p))
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2, errs
    assert 0.9 < raw_errs[0] / raw_errs[-1] < 1.1, raw_errs
    assert errs[0] < 0.05 * raw_errs[0], (errs, raw_errs)


def test_refresh_full_check_both_sides_and_tiles(orc):
    """Step 9's full check at a refresh: learned rates = the plain source + d (e_1 - e_2)
    at every node trust both 32-node tiles of 40 nodes at d = 0.9 (tau_c sum|S| + floor)
    and neither at 1.1; a node of the second tile whose plain source moved (T 2500 K
    instead of 3500 K) leaves only that tile untrusted: flag 4 and the plain source there,
    the corrected (exact) source in the first tile."""
    import workloads as W
    sp, R = W.species_table(), W.reaction_table()
    n = 40
    rhos, T = _hot_state(n)
    _, _, S_p = orc.chem_eval(sp, R, rhos, T, 0.0)
    thr = 0.05 * np.abs(S_p[0]).sum()
    w_ref = np.abs(S_p[0]).max()
    st = _stats(np.zeros(10), np.ones(10), w_ref=w_ref, tol_mass=0.05)
    for kappa, trust in ((0.9, [True, True]), (1.1, [False, False])):
        om = S_p[0].copy()
        om[0] += kappa * thr
        om[1] -= kappa * thr
        c = orc.chem_surrogate_correction(_net_for_rates(orc, om, w_ref), st, rhos, T, species=sp, reactions=R)
        assert list(c["trust"]) == trust and not c["trust_ambiguous"].any()
    T2 = T.copy()
    T2[35] = 2500.0
    _, _, S_p2 = orc.chem_eval(sp, R, rhos, T2, 0.0)
    assert np.abs(S_p2[35] - S_p[0]).max() > 2 * thr
    om = S_p[0].copy()
    om[0] += 0.5 * thr
    om[1] -= 0.5 * thr
    net = _net_for_rates(orc, om, w_ref)
    c = orc.chem_surrogate_correction(net, st, rhos, T2, species=sp, reactions=R)
    assert list(c["trust"]) == [True, False]
    r = orc.chem_surrogate_source(net, st, rhos, T2, species=sp, reactions=R, call=0, correction=c)
    assert list(r["tile_flag"]) == [0, 4]
    assert np.array_equal(r["S"][32:], S_p2[32:])
    assert np.allclose(r["S"][:32], S_p2[:32], rtol=1e-12, atol=1e-12 * w_ref)
