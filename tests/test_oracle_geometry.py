"""Pins of the oracle's metric terms (Eqs. mapp, mapped_equation, jacobian)."""
import numpy as np
import pytest

import workloads as W


def _affine_mesh(orc, N, A, b):
    x, _ = orc.lgl(N)
    idx = np.indices((N + 1,) * 3).reshape(3, -1)[::-1]  # idx[0] = x index, fastest
    r = x[idx]
    return (A @ r + b[:, None])[None]


def test_cartesian_metrics(orc):
    N = 3
    x, _ = orc.lgl(N)
    xyz, nbr, face = W.box_mesh((2, 3, 2), x, (0, 0, 0), (2.0, 6.0, 1.0))
    Ja, J = orc.geometry(3, N, xyz)
    h = np.array([1.0, 2.0, 0.5]) / 2
    assert np.allclose(J, np.prod(h), rtol=1e-14)
    for i in range(3):
        for n in range(3):
            ref = np.prod(h) / h[i] if i == n else 0.0
            assert np.allclose(Ja[:, i, n], ref, atol=1e-13)  # curl form: x_l * dx_m rounding


@pytest.mark.parametrize("N", [1, 2, 4])
def test_affine_metrics_match_inverse_jacobian(orc, N):
    rng = np.random.default_rng(1)
    A = np.eye(3) + 0.3 * rng.normal(size=(3, 3))
    if np.linalg.det(A) < 0:
        A[:, 0] *= -1
    xyz = _affine_mesh(orc, N, A, rng.normal(size=3))
    Ja, J = orc.geometry(3, N, xyz)
    detA = np.linalg.det(A)
    # Ja^i_n = J d(xi_i)/d(x_n) = det(A) * inv(A)[i, n]
    Ainv = np.linalg.inv(A)
    assert np.allclose(J, detA, rtol=1e-13)
    for i in range(3):
        for n in range(3):
            assert np.allclose(Ja[0, i, n], detA * Ainv[i, n], atol=1e-13)


@pytest.mark.parametrize("N", [2, 3, 5])
def test_warped_metric_identities(orc, N):
    x, _ = orc.lgl(N)
    xyz, nbr, face = W.tgv_config(x, 3, warp=0.1)
    Ja, J = orc.geometry(3, N, xyz)
    D = orc.dmat(N)
    n1 = N + 1
    for k in range(Ja.shape[0]):
        for n in range(3):
            div = np.zeros((n1, n1, n1))
            for i in range(3):
                a = Ja[k, i, n].reshape(n1, n1, n1)  # [z][y][x]
                axis = 2 - i
                div += np.moveaxis(np.tensordot(D, np.moveaxis(a, axis, 0), axes=(1, 0)), 0, axis)
            scale = np.abs(Ja[k]).max() * np.abs(D).max()
            assert np.abs(div).max() < 1e-13 * scale


def test_2d_polar_jacobian(orc):
    N = 4
    x, _ = orc.lgl(N)
    xyz, nbr, face = W.box_mesh((3, 4), x, (1.0, 0.2), (2.0, 1.4), periodic=False,
                                bc_ids=[0, 0, 0, 0])
    r, th = xyz[:, 0].copy(), xyz[:, 1].copy()
    xyz[:, 0] = r * np.cos(th)
    xyz[:, 1] = r * np.sin(th)
    Ja, J = orc.geometry(2, N, xyz)
    # the polar map restricted to an element is degree 1 in r and transcendental in theta;
    # J converges to r * (dr/dxi)(dth/deta) spectrally
    hr, ht = (1.0 / 3) / 2, (1.2 / 4) / 2
    assert np.allclose(J, r * hr * ht, rtol=2e-4)


def test_metric_identities_do_not_degrade_away_from_the_origin(orc):
    """The curl form is evaluated with x_l relative to each element's first node (a constant
    shift adds c curl grad x_m = 0): on the full 16^3 warped Taylor-Green mesh at N = 7,
    whose elements sit up to |x| / h = 8 element sizes from the origin, the discrete metric
    identities hold to the rounding of Ja's own size (measured 2.5e-14 of the scale); the
    products x_l grad x_m of size |x| h would leave about 1.7e-13."""
    N = 7
    x, _ = orc.lgl(N)
    xyz, nbr, face = W.box_mesh((16,) * 3, x, (-np.pi,) * 3, (np.pi,) * 3, warp=0.1)
    Ja, J = orc.geometry(3, N, xyz)
    D = orc.dmat(N)
    n1 = N + 1
    a = Ja.reshape(Ja.shape[0], 3, 3, n1, n1, n1)  # [k][i][n][z][y][x]
    div = (np.einsum("ab,kncdb->kncda", D, a[:, 0]) + np.einsum("ab,kncbd->kncad", D, a[:, 1]) +
           np.einsum("ab,knbcd->knacd", D, a[:, 2]))
    scale = np.abs(Ja).max() * np.abs(D).max()
    assert np.abs(div).max() < 6e-14 * scale
