"""Pins of the oracle's Hennemann-Gassner shock indicator over its whole range (reading of
the shock-capturing paragraph: modal energy of rho p, threshold T(N) = 0.5 10^(-1.8 (N+1)^(1/4)),
sigmoid alpha = 1 / (1 + exp(-(s / T)(E - T))) with s = ln((1 - 1e-4) / 1e-4), alpha < 1e-3
dropped, clip to alpha_max, alpha <- max(alpha, 1/2 max over face neighbours)).

Each element carries rho p = A phi_0 + B phi_m, phi the orthonormal Legendre tensor modes
(built here with numpy, not with the oracle's Vandermonde matrix), so that its modal
energy fraction is E = B^2 / (A^2 + B^2) in closed form: phi_m of the highest degree N
enters the first criterion, of degree N - 1 the second.  The sigmoid's own meaning fixes
the expected values: alpha = 1/2 at E = T (the threshold is the midpoint), 1e-4 at E = 0
and 1 - 1e-4 at E = 2T (what s is defined by), so a wrong threshold exponent or constant,
a wrong sharpness, a dropped cut-off or smoothing rule fails here.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as L

import workloads as W

S = np.log((1.0 - 1e-4) / 1e-4)


def _thr(N):
    return 0.5 * 10.0 ** (-1.8 * (N + 1.0) ** 0.25)


def _phi(j, t):
    """Orthonormal Legendre polynomial of degree j on [-1, 1]."""
    c = np.zeros(j + 1)
    c[j] = 1.0
    return np.sqrt((2 * j + 1) / 2.0) * L.legval(t, c)


def _setup(orc, dim, N, n_el=3, alpha_max=1.0):
    x, _ = orc.lgl(N)
    shape = (n_el,) + (1,) * (dim - 1)
    xyz, nbr, face = W.box_mesh(shape, x, (0.0,) * dim, (float(n_el),) + (1.0,) * (dim - 1),
                                periodic=True)
    o = orc.Oracle(dim, N, xyz, nbr, face, alpha_max=alpha_max)
    # reference coordinates of every node (unit elements: xi = 2 (x - x_left) - 1)
    ref = np.empty_like(xyz)
    for d in range(dim):
        lo = np.floor(xyz[:, d].min(axis=1) + 1e-9)
        ref[:, d] = 2.0 * (xyz[:, d] - lo[:, None]) - 1.0
    return o, ref


def _state(o, ref, dim, rp):
    """Conserved state with rho p = rp [K][np], rho = 1 + 0.3 xi (so that p alone has a
    different spectrum), velocity 0."""
    K, npn = rp.shape
    rho = 1.0 + 0.3 * ref[:, 0]
    w = np.zeros((K, dim + 2, npn))
    w[:, 0] = rho
    w[:, dim + 1] = rp / rho
    return o.prim_to_cons(w)


def _field(ref, dim, E, mode):
    """A phi_0 + B phi_mode with B^2 / (A^2 + B^2) = E (A = 1) at every node of an element."""
    A = 1.0
    B = np.sqrt(E / (1.0 - E)) * A
    c0 = np.ones(ref.shape[0:1] + ref.shape[2:])
    cm = np.ones_like(c0)
    for d in range(dim):
        c0 = c0 * _phi(0, ref[:, d])
        cm = cm * _phi(mode[d], ref[:, d])
    return A * c0 + B * cm


def _alpha(E, N):
    a = 1.0 / (1.0 + np.exp(-(S / _thr(N)) * (E - _thr(N))))
    return 0.0 if a < 1e-3 else a


@pytest.mark.parametrize("N", [2, 3, 4, 7])
def test_alpha_is_one_half_at_the_threshold(orc, N):
    """E = T(N) through the highest-degree criterion (mode (N, 0)) and through the
    second-highest one (mode (N-1, 1)): alpha = 1/2 in the middle element."""
    dim = 2
    o, ref = _setup(orc, dim, N)
    T = _thr(N)
    for mode in ((N, 0), (N - 1, 1), (0, N)):
        rp = np.empty(ref.shape[0:1] + ref.shape[2:])
        rp[:] = _field(ref, dim, 1e-30, (0, 0))
        rp[1] = _field(ref[1:2], dim, T, mode)[0]
        a = o.indicator(_state(o, ref, dim, rp))
        assert abs(a[1] - 0.5) < 1e-10, (N, mode, a)
        # neighbours: half of it by smoothing
        assert abs(a[0] - 0.25) < 1e-10 and abs(a[2] - 0.25) < 1e-10, a


@pytest.mark.parametrize("N", [3, 4])
def test_sigmoid_values_and_cut_off(orc, N):
    """alpha at E = 2T is 1 - 1e-4, at E = T/2 it is 1 / (1 + sqrt(9999)), at E = 0.3T it
    is 1 / (1 + 9999^0.7) = 1.58e-3 (kept); at E = T/4 the raw value 1 / (1 + 9999^(3/4))
    = 9.99e-4 lies below the 1e-3 cut-off: 0."""
    dim = 2
    o, ref = _setup(orc, dim, N, n_el=1)
    T = _thr(N)
    expected = {2.0: 1.0 - 1e-4, 0.5: 1.0 / (1.0 + np.sqrt(9999.0)),
                0.3: 1.0 / (1.0 + 9999.0 ** 0.7), 0.25: 0.0}
    for f, want in expected.items():
        assert abs(_alpha(f * T, N) - want) < 1e-15 * max(1.0, want) + 1e-16
        rp = _field(ref, dim, f * T, (N, 0))
        a = o.indicator(_state(o, ref, dim, rp))
        # one element, periodic: its own neighbour (1/2 alpha < alpha, no change)
        assert abs(a[0] - want) < 1e-10 * max(want, 1e-3), (f, a[0], want)
    assert 1e-3 < 1.0 / (1.0 + 9999.0 ** 0.7) and 1.0 / (1.0 + 9999.0 ** 0.75) < 1e-3


def test_alpha_max_clip_and_smoothing_at_unsaturated_alpha(orc):
    """Three elements in a periodic row: raw alphas 0 (E = 0), 1/2 (E = T) and
    1 / (1 + 9999^0.05) = 0.387 (E = 0.95 T).  Smoothing max(alpha, 1/2 max neighbour):
    (0.25, 0.5, 0.387).  With alpha_max = 0.45 the middle clips first: (0.225, 0.45, 0.387)."""
    N, dim = 3, 2
    T = _thr(N)
    a_hi = 1.0 / (1.0 + 9999.0 ** 0.05)
    for amax, want in ((1.0, (0.25, 0.5, a_hi)), (0.45, (0.225, 0.45, a_hi))):
        o, ref = _setup(orc, dim, N, alpha_max=amax)
        rp = np.empty(ref.shape[0:1] + ref.shape[2:])
        rp[0] = _field(ref[0:1], dim, 1e-30, (0, 0))[0]
        rp[1] = _field(ref[1:2], dim, T, (N, 2))[0]
        rp[2] = _field(ref[2:3], dim, 0.95 * T, (1, N))[0]
        a = o.indicator(_state(o, ref, dim, rp))
        assert np.allclose(a, want, rtol=1e-10, atol=1e-14), (amax, a, want)


def test_three_dimensional_modes(orc):
    """3D, N = 3: a mixed mode (0, 3, 1) is of the highest degree, (2, 1, 2) of the second
    highest; both give alpha = 1/2 at E = T."""
    N, dim = 3, 3
    o, ref = _setup(orc, dim, N, n_el=1)
    T = _thr(N)
    for mode in ((0, 3, 1), (2, 1, 2)):
        a = o.indicator(_state(o, ref, dim, _field(ref, dim, T, mode)))
        assert abs(a[0] - 0.5) < 1e-10, (mode, a)
