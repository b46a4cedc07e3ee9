"""Pins of the oracle's mixture thermodynamics (Eqs. total_energy, internal_energies, eos;
thermally perfect stand-in for the RRHO model of Eq. Internal_energy) and of the
multi-species Euler operator with the Ducros split-form flux."""
import numpy as np
import pytest

import cases
import workloads as W

RU = 8.314462618


def _Y(rng, n, ns=5):
    return rng.dirichlet(np.ones(ns), size=n)


def test_species_table_is_monotone_and_element_balanced():
    sp = W.species_table()
    T = np.linspace(200, 1e4, 2000)
    for s in range(5):
        a = sp[s, 1:6]
        cp = a[0] + a[1] * T + a[2] * T ** 2 + a[3] * T ** 3 + a[4] * T ** 4
        assert np.all(cp > 0) and np.all(np.diff(cp) >= 0)
    W_ = sp[:, 0]
    assert abs(W_[2] - 2 * W_[0]) < 1e-15 and abs(W_[4] - W_[0] - W_[1]) < 1e-15
    assert np.all((W_ >= 0.014) & (W_ <= 0.032))


def test_energy_matches_integral_of_cv(orc):
    """e(T2) - e(T1) = int cv dT (Gauss-Legendre, exact for the polynomial)."""
    sp = W.species_table()
    rng = np.random.default_rng(1)
    Y = _Y(rng, 50)
    T1 = rng.uniform(200, 3000, 50)
    T2 = T1 + rng.uniform(10, 5000, 50)
    e1, _ = orc.mixture_eval(sp, Y, T1)
    e2, _ = orc.mixture_eval(sp, Y, T2)
    x, w = np.polynomial.legendre.leggauss(8)
    integ = np.zeros(50)
    for xi, wi in zip(x, w):
        Tq = 0.5 * (T2 - T1) * xi + 0.5 * (T2 + T1)
        _, cv = orc.mixture_eval(sp, Y, Tq)
        integ += wi * cv * 0.5 * (T2 - T1)
    assert np.allclose(e2 - e1, integ, rtol=1e-12)


def test_cv_of_monatomic_constant_cp(orc):
    """cp/R = 5/2 constant (a monatomic gas): cv = 3/2 R_s, e = 3/2 R_s T + R_s a6."""
    sp = np.zeros((1, 8))
    sp[0, 0] = 0.004
    sp[0, 1] = 2.5
    sp[0, 6] = 0.0
    e, cv = orc.mixture_eval(sp, np.ones((3, 1)), np.array([300.0, 1000.0, 5000.0]))
    R = RU / 0.004
    assert np.allclose(cv, 1.5 * R, rtol=1e-15)
    assert np.allclose(e, 1.5 * R * np.array([300.0, 1000.0, 5000.0]), rtol=1e-15)


def test_newton_round_trip(orc):
    sp = W.species_table()
    rng = np.random.default_rng(2)
    n = 400
    Y = _Y(rng, n)
    T = np.exp(rng.uniform(np.log(220), np.log(9500), n))
    e, _ = orc.mixture_eval(sp, Y, T)
    Tr, it, bad = orc.mixture_temperature(sp, Y, e)
    assert not bad
    assert np.abs(Tr / T - 1).max() < 1e-12
    assert it.max() <= 12
    # warm start from a nearby temperature converges in very few steps
    Tw, itw, _ = orc.mixture_temperature(sp, Y, e, T0=T * (1 + 1e-3))
    assert np.abs(Tw / T - 1).max() < 1e-12 and itw.max() <= 4


def _mix_box(orc, N=3, shape=(3, 2, 2), warp=0.1, seed=7):
    x, _ = orc.lgl(N)
    xyz, nbr, face = W.box_mesh(shape, x, (-np.pi,) * 3, (np.pi,) * 3, periodic=True, warp=warp)
    sp = W.species_table()
    w = W.mixture_primitive(xyz, rho=0.1, vel=(300.0, -50.0, 20.0), T=1500.0, seed=seed)
    rng = np.random.default_rng(seed)
    w[:, 5:8] += 40.0 * rng.normal(size=w[:, 5:8].shape)
    w[:, 8] *= 1 + 0.05 * rng.uniform(-1, 1, size=w[:, 8].shape)
    o = orc.Oracle(3, N, xyz, nbr, face, n_species=5, volume_flux=orc.VF_DUCROS,
                   surface_flux=orc.SF_LLF, species=sp)
    return o, w


def _flux_scale(o, u, w):
    """Size of the contravariant flux differences per field: (|u| |v| + p) |Ja| / J * N^2."""
    sp = W.species_table()
    p = np.sum(w[:, :5] * (RU / sp[:, 0])[None, :, None], axis=1) * w[:, 8]
    vmax = np.abs(w[:, 5:8]).max()
    fs = np.abs(u).max(axis=(0, 2)) * vmax
    fs[5:] += p.max()
    return fs * np.abs(o.Ja).max() / o.J.min() * o.N ** 2


def test_mixture_free_stream_and_conservation(orc):
    o, w = _mix_box(orc)
    wc = w.copy()
    wc[:] = w[:1, :, :1]  # uniform state
    r = o.rhs(o.prim_to_cons(wc))
    u = o.prim_to_cons(wc)
    assert np.all(np.abs(r).max(axis=(0, 2)) < 1e-13 * _flux_scale(o, u, wc))
    u = o.prim_to_cons(w)
    r = o.rhs(u)
    _, wq = orc.lgl(o.N)
    idx = np.indices((o.N + 1,) * 3).reshape(3, -1)
    M = np.prod(wq[idx], axis=0)[None] * o.J
    for v in range(9):
        assert abs(np.sum(M * r[:, v])) < 1e-13 * np.sum(M * np.abs(r[:, v]))


def test_identical_species_reduce_to_ideal_gas(orc):
    """Five identical species with cp/R = 7/2 form a calorically perfect gas with gamma=1.4:
    the mixture operator (Ducros) must equal the one-gas operator (Ducros) on (rho, rho v, rho E)."""
    N = 3
    x, _ = orc.lgl(N)
    xyz, nbr, face = W.box_mesh((2, 3, 2), x, (-np.pi,) * 3, (np.pi,) * 3, periodic=True, warp=0.1)
    sp = np.zeros((5, 8))
    sp[:, 0] = 0.029
    sp[:, 1] = 3.5
    om = orc.Oracle(3, N, xyz, nbr, face, n_species=5, volume_flux=1, species=sp)
    og = orc.Oracle(3, N, xyz, nbr, face, n_species=0, volume_flux=1, gamma=1.4)
    rng = np.random.default_rng(4)
    K, npn = xyz.shape[0], 64
    Y = rng.dirichlet(np.ones(5), size=(K, npn)).transpose(0, 2, 1)
    rho = 1.0 + 0.1 * rng.uniform(size=(K, npn))
    T = 400 + 50 * rng.uniform(size=(K, npn))
    vel = 30 * rng.normal(size=(K, 3, npn))
    wm = np.concatenate([rho[:, None] * Y, vel, T[:, None]], axis=1)
    um = om.prim_to_cons(wm)
    R = RU / 0.029
    wg = np.concatenate([rho[:, None], vel, (rho * R * T)[:, None]], axis=1)
    ug = og.prim_to_cons(wg)
    assert np.allclose(um[:, 8], ug[:, 4], rtol=1e-13)
    rm, rg = om.rhs(um), og.rhs(ug)
    assert np.allclose(rm[:, :5].sum(axis=1), rg[:, 0], rtol=1e-11, atol=1e-11 * np.abs(rg[:, 0]).max())
    for k in range(4):
        assert np.allclose(rm[:, 5 + k], rg[:, 1 + k], rtol=1e-11, atol=1e-11 * np.abs(rg[:, 1 + k]).max())


def test_ducros_mixture_consistency_symmetry(orc):
    o, w = _mix_box(orc)
    u = o.prim_to_cons(w)
    rng = np.random.default_rng(3)
    for _ in range(10):
        a, b = u[rng.integers(o.K), :, rng.integers(64)], u[rng.integers(o.K), :, rng.integers(64)]
        n = rng.normal(size=3)
        assert np.allclose(o.flux_pair(a, a, n, 0), o.flux_pair(a, a, n, 2), rtol=1e-14)
        assert np.allclose(o.flux_pair(a, b, n, 0), o.flux_pair(b, a, n, 0), rtol=1e-14)
        assert np.allclose(o.flux_pair(a, a, n, 1), o.flux_pair(a, a, n, 2), rtol=1e-13)


def test_ogrid_mixture_wall_has_no_mass_flux(orc):
    """On the cylinder O-grid, uniform flow: the slip-wall faces carry no species mass flux,
    so d/dt of the total mass equals the inflow minus the outflow only (checked via a flow
    aligned with the wall: zero normal velocity everywhere on the wall)."""
    N = 3
    x, _ = orc.lgl(N)
    xyz, nbr, face = W.ogrid_mesh(x, 3, 4, 2)
    sp = W.species_table()
    w = W.mixture_primitive(xyz, rho=0.1, vel=(0.0, 0.0, 100.0), T=300.0)
    kinds = [orc.BC_INFLOW, orc.BC_OUTFLOW, orc.BC_SLIP_WALL]
    bcp = np.stack([w[0, :, 0]] * 3)
    o = orc.Oracle(3, N, xyz, nbr, face, n_species=5, volume_flux=1, species=sp,
                   bc_kind=kinds, bc_prim=bcp)
    wu = w.copy()
    wu[:] = w[:1, :, :1]  # uniform, flow along the cylinder axis (periodic z)
    r = o.rhs(o.prim_to_cons(wu))
    u = o.prim_to_cons(wu)
    # uniform axial flow past a slip wall, with inflow/outflow of the same state: steady
    assert np.all(np.abs(r).max(axis=(0, 2)) < 1e-13 * _flux_scale(o, u, wu))
