"""Pins of the oracle's LGL basis (Eqs. lagrange_3d, lag, sbp, boundary_matrix)."""
import numpy as np
import numpy.polynomial.legendre as L
import pytest


def test_lgl_closed_forms(orc):
    x, w = orc.lgl(1)
    assert np.allclose(x, [-1, 1], atol=0) and np.allclose(w, [1, 1], atol=0)
    x, w = orc.lgl(2)
    assert np.allclose(x, [-1, 0, 1], atol=1e-16)
    assert np.allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    x, w = orc.lgl(3)
    s = 1 / np.sqrt(5)
    assert np.allclose(x, [-1, -s, s, 1], atol=1e-15)
    assert np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    x, w = orc.lgl(4)
    s = np.sqrt(3 / 7)
    assert np.allclose(x, [-1, -s, 0, s, 1], atol=1e-15)
    assert np.allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


@pytest.mark.parametrize("N", range(1, 16))
def test_lgl_against_legendre_library(orc, N):
    x, w = orc.lgl(N)
    # interior nodes are the roots of P_N' (numpy's Legendre series as the independent routine)
    c = np.zeros(N + 1)
    c[N] = 1
    roots = np.sort(np.real(L.legroots(L.legder(c)))) if N > 1 else np.array([])
    assert np.allclose(x[1:-1], roots, atol=1e-13)
    assert abs(w.sum() - 2) < 1e-14
    # quadrature exact to degree 2N-1
    for k in range(2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13


@pytest.mark.parametrize("N", range(1, 16))
def test_derivative_matrix(orc, N):
    x, w = orc.lgl(N)
    D = orc.dmat(N)
    for k in range(N + 1):
        d = k * x ** (k - 1) if k else 0 * x
        assert np.allclose(D @ x ** k, d, atol=1e-11 * max(1, N ** 2))
    # summation by parts: W D + (W D)^T = B  (Eq. sbp, Eq. boundary_matrix)
    Q = np.diag(w) @ D
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1, 1
    assert np.allclose(Q + Q.T, B, atol=1e-13)
    # the identities the diagonal-free split form relies on
    assert abs(2 * D[0, 0] + 1 / w[0]) < 1e-12 * N ** 2
    assert abs(2 * D[N, N] - 1 / w[N]) < 1e-12 * N ** 2


def test_N1_brute_force(orc):
    D = orc.dmat(1)
    assert np.array_equal(D, np.array([[-0.5, 0.5], [-0.5, 0.5]]))


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_vandermonde_orthonormal_modes(orc, N):
    x, w = orc.lgl(N)
    V = orc.vandermonde(N)
    for j in range(N + 1):
        c = np.zeros(N + 1)
        c[j] = np.sqrt((2 * j + 1) / 2)
        assert np.allclose(V[:, j], L.legval(x, c), atol=1e-14)
    # modal round trip
    f = np.random.default_rng(0).normal(size=N + 1)
    m = np.linalg.solve(V, f)
    assert np.allclose(V @ m, f, atol=1e-13)
