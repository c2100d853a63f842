"""Pins of the oracle's Jacobian terms (the NOJAC kernels' input, Section 4:
det J and J^{-1} per element and quadrature point) against closed forms,
finite differences of the element map written out here, and an exact
symbolic volume."""
import numpy as np
import pytest

from paper_1310_1191_gb300 import inputs
from test_oracle_pins import _sympy_volume

TET, PRISM = 0, 1


def _prism_map(X, pts):
    """x(xi, eta, zeta) of a straight-edged prism from its six vertices."""
    xi, eta, ze = pts[..., 0], pts[..., 1], pts[..., 2]
    lam = [1 - xi - eta, xi, eta]
    out = 0.0
    for a in range(3):
        out = out + (lam[a] * (1 - ze) / 2)[..., None] * X[a] + (lam[a] * (1 + ze) / 2)[..., None] * X[a + 3]
    return out


def _fd_jacobian(X, pts, h=1e-2):
    """J[q][i][k] = d x_i / d xi_k by central differences; exact up to rounding
    because the map is linear in each reference coordinate separately."""
    J = np.zeros((pts.shape[0], 3, 3))
    for k in range(3):
        d = np.zeros(3)
        d[k] = h
        J[:, :, k] = (_prism_map(X, pts + d) - _prism_map(X, pts - d)) / (2 * h)
    return J


@pytest.mark.parametrize("p", [1, 2, 5])
def test_affine_prism_closed_form(orc, p):
    """Affine prism (parallel translate of a triangle): J = [e1, e2, v/2]
    everywhere, so det and J^{-1} are those of one fixed matrix."""
    x0, e1, e2, v = np.array([0.3, -0.2, 0.1]), np.array([0.7, 0.1, -0.2]), \
        np.array([-0.1, 0.6, 0.05]), np.array([0.1, -0.05, 0.9])
    bot = [x0, x0 + e1, x0 + e2]
    X = np.array(bot + [q + v for q in bot])[None]
    J = np.stack([e1, e2, v / 2], axis=1)
    T, st = orc.jacobian_terms(PRISM, p, X)
    assert st[0] == 0 and T.shape == (1, (p + 1) ** 3, 10)
    assert np.allclose(T[0, :, 0], np.linalg.det(J), rtol=1e-14, atol=0)
    Ji = np.linalg.inv(J)
    assert np.max(np.abs(T[0, :, 1:] - Ji.reshape(9)[None])) < 1e-14 * np.abs(Ji).max()


def test_tet_closed_form(orc):
    X = inputs.tet_mesh(2)[:5]
    T, st = orc.jacobian_terms(TET, 1, X)
    assert np.all(st == 0) and T.shape == (5, 4, 10)
    for e in range(5):
        J = np.stack([X[e, 1] - X[e, 0], X[e, 2] - X[e, 0], X[e, 3] - X[e, 0]], axis=1)
        assert np.allclose(T[e, :, 0], np.linalg.det(J), rtol=1e-13, atol=0)
        Ji = np.linalg.inv(J)
        assert np.max(np.abs(T[e, :, 1:] - Ji.reshape(9)[None])) < 1e-13 * np.abs(Ji).max()


@pytest.mark.parametrize("p", [1, 3, 7])
def test_jittered_prisms_against_finite_differences(orc, p):
    """Non-affine prisms: det = det(J_fd) and J^{-1} J_fd = I at every point."""
    E = 6
    X = inputs.prism_mesh(E)
    T, st = orc.jacobian_terms(PRISM, p, X)
    xi, _ = orc.rule(PRISM, p)
    assert np.all(st == 0)
    for e in range(E):
        Jfd = _fd_jacobian(X[e], xi)
        assert np.allclose(T[e, :, 0], np.linalg.det(Jfd), rtol=1e-11, atol=0)
        Ji = T[e, :, 1:].reshape(-1, 3, 3)
        assert np.max(np.abs(Ji @ Jfd - np.eye(3)[None])) < 1e-11


@pytest.mark.parametrize("p", [1, 4])
def test_weighted_det_sum_is_exact_volume(orc, p):
    """sum_q w_q det J_q = element volume (det J is a polynomial the rule
    integrates exactly), checked against a symbolic integral."""
    X = inputs.prism_mesh(4)
    T, _ = orc.jacobian_terms(PRISM, p, X)
    _, w = orc.rule(PRISM, p)
    for e in (0, 3):
        assert abs(np.dot(w, T[e, :, 0]) - _sympy_volume(X[e])) < 1e-15


def test_status_flags(orc):
    X = inputs.prism_mesh(4)
    X[1] = X[1][[1, 0, 2, 4, 3, 5]]  # mirrored: det J < 0
    X[2, 3, 1] = np.nan
    _, st = orc.jacobian_terms(PRISM, 2, X)
    assert st[0] == 0 and st[3] == 0
    assert st[1] == 1
    assert st[2] & 2
