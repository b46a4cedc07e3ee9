"""Pins of the oracle's finite-rate chemistry (appendix, Chemical Kinetics: Eqs. nrp,
forward_rate, backward, kedef, calc_prod) on the seeded five-species mechanism."""
import numpy as np
import pytest

import workloads as W

RU = 8.314462618
# atoms per species A, B, A2, B2, AB
ATOMS = np.array([[1, 0], [0, 1], [2, 0], [0, 2], [1, 1]], dtype=float)


def _states(rng, n, T_lo=1500, T_hi=6000):
    rho = 0.1 * rng.dirichlet(np.ones(5), size=n) * rng.uniform(0.5, 2.0, size=(n, 1))
    T = rng.uniform(T_lo, T_hi, size=n)
    return rho, T


def test_mechanism_is_element_balanced():
    R = W.reaction_table()
    assert R.shape == (17, 19)
    for row in R:
        dnu = row[5:10] - row[0:5]
        assert np.allclose(dnu @ ATOMS, 0)
    assert 3 <= int(R[:, 10].sum()) <= 5


def test_mass_and_element_conservation(orc):
    sp, R = W.species_table(), W.reaction_table()
    rng = np.random.default_rng(0)
    rho, T = _states(rng, 200)
    om, jd, S = orc.chem_eval(sp, R, rho, T)
    scale = np.abs(om).sum(1)
    assert np.all(np.abs(om.sum(1)) <= 1e-12 * scale + 1e-300)
    moles = om / sp[:, 0][None, :]
    elem = moles @ ATOMS
    assert np.all(np.abs(elem) <= 1e-12 * (np.abs(moles) @ ATOMS) + 1e-300)
    assert np.all(np.isfinite(om)) and scale.min() > 0


def test_jacobian_diagonal_matches_finite_differences(orc):
    sp, R = W.species_table(), W.reaction_table()
    rng = np.random.default_rng(1)
    rho, T = _states(rng, 20, 2500, 5000)
    om, jd, _ = orc.chem_eval(sp, R, rho, T)
    for s in range(5):
        # the rates are polynomials of degree <= 3 in rho_s: central differences with
        # h = 1e-3 rho_s have truncation error ~1e-7 and stay above the cancellation noise
        h = 1e-3 * rho[:, s]
        rp, rm = rho.copy(), rho.copy()
        rp[:, s] += h
        rm[:, s] -= h
        op, _, _ = orc.chem_eval(sp, R, rp, T)
        omn, _, _ = orc.chem_eval(sp, R, rm, T)
        fd = (op[:, s] - omn[:, s]) / (2 * h)
        assert np.allclose(jd[:, s], fd, rtol=1e-5, atol=1e-9 * np.abs(fd).max())


def test_point_implicit_scaling(orc):
    sp, R = W.species_table(), W.reaction_table()
    rng = np.random.default_rng(2)
    rho, T = _states(rng, 50)
    dt = 1e-7
    om, jd, S = orc.chem_eval(sp, R, rho, T, dt=dt)
    ref = om / (1.0 + dt * np.maximum(0.0, -jd))
    assert np.allclose(S, ref, rtol=1e-14, atol=0)
    _, _, S0 = orc.chem_eval(sp, R, rho, T, dt=0.0)
    assert np.array_equal(S0, om)


def _equilibrium_lnKc(orc, sp, row, T):
    """ln K_c of one reaction from the rate itself: bisect the free product concentration
    until the net rate vanishes (A2 + M <-> 2A + M type rows)."""
    nf, nb = row[0:5], row[5:10]
    dnu = nb - nf
    prod = int(np.argmax(dnu))  # species produced twice (2A or 2B) or once
    c = np.full(5, 1e-6)
    lo, hi = np.log(1e-30), np.log(1e-1)
    one = row[None, :]
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        c[prod] = np.exp(mid)
        rho = c * sp[:, 0] * 1e6
        om, _, _ = orc.chem_eval(sp, one, rho[None], np.array([T]))
        if om[0, prod] > 0:
            lo = mid
        else:
            hi = mid
    c[prod] = np.exp(0.5 * (lo + hi))
    return np.sum(dnu * np.log(c))


def test_equilibrium_constant_obeys_van_t_hoff(orc):
    """d ln K_c / dT = dH / (R T^2) - dnu / T with dH from the species enthalpies
    h/R = a1 T + a2 T^2/2 + a3 T^3/3 + a4 T^4/4 + a5 T^5/5 + a6."""
    sp, R = W.species_table(), W.reaction_table()
    rows = [r for r in R if r[10] == 0 and (r[5:10] - r[0:5]).max() == 2][:2]
    assert rows
    for row in rows:
        dnu = row[5:10] - row[0:5]
        T = 4000.0
        d = 1e-3 * T
        slope = (_equilibrium_lnKc(orc, sp, row, T + d) - _equilibrium_lnKc(orc, sp, row, T - d)) / (2 * d)
        a = sp[:, 1:8]
        h = a[:, 0] * T + a[:, 1] * T ** 2 / 2 + a[:, 2] * T ** 3 / 3 + a[:, 3] * T ** 4 / 4 + \
            a[:, 4] * T ** 5 / 5 + a[:, 5]
        expect = (dnu @ h) / T ** 2 - dnu.sum() / T
        assert abs(slope - expect) < 1e-5 * abs(expect)


def test_arrhenius_forward_rate(orc):
    """A single irreversible-in-practice step (products absent): the net rate is the forward
    rate k_f prod c^nu' (times M), so omega scales with A T^beta exp(-theta/T)."""
    sp = W.species_table()
    row = W.reaction_table()[0].copy()
    rho = np.zeros((1, 5))
    nf = row[0:5]
    rho[0] = np.where(nf > 0, 0.05, 0.0) + 1e-300
    T1, T2 = 3000.0, 4500.0
    o1, _, _ = orc.chem_eval(sp, row[None], rho, np.array([T1]))
    o2, _, _ = orc.chem_eval(sp, row[None], rho, np.array([T2]))
    beta, theta = row[17], row[18]
    ratio = (T2 / T1) ** beta * np.exp(-theta / T2 + theta / T1)
    s = int(np.argmax(nf))
    assert abs(o2[0, s] / o1[0, s] / ratio - 1) < 1e-10
