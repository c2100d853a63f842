"""Pins of the elasticity oracle (the paper's model problem, Section 5.1):
block symmetry, rigid-body modes in the kernel, the trace identity with the
scalar Laplace stiffness, the load vector, and exact rational integrals on an
affine prism."""
from fractions import Fraction

import numpy as np
import pytest

from paper_1310_1191_gb300 import inputs
from test_oracle_pins import _exact_reference_moments

PRISM = 1


def _lame(Ey, nu):
    return Ey * nu / ((1 + nu) * (1 - 2 * nu)), Ey / (2 * (1 + nu))


def _relF(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("elem", [PRISM, 2])
@pytest.mark.parametrize("p", [1, 2, 4])
def test_block_symmetry_translations_load(orc, p, elem):
    """(elem 2: the paper's prism rule, Table 1 point counts)"""
    E = 6
    X = inputs.prism_mesh(E, dims=(2, 2, 1))[:E]
    C = inputs.elastic_coefficients(E)
    A, b, st = orc.integrate_elastic(p, X, C, elem=elem)
    assert np.all(st == 0)
    s = np.abs(A).max()
    for i in range(3):
        for k in range(3):
            assert np.max(np.abs(A[:, i, k] - A[:, k, i].transpose(0, 2, 1))) < 1e-13 * s
            # a translation (constant displacement, DOF 0 of component k) has no strain
            assert np.max(np.abs(A[:, i, k, :, 0])) < 1e-13 * s
    # load vector: b[i][0] = f_i V_e (phi_0 = 1); volumes from the scalar oracle
    Cs = np.zeros((11, E))
    Cs[9] = 1.0
    M, _, _ = orc.integrate(elem, p, X, Cs)
    V = M[:, 0, 0]
    assert np.allclose(b[:, :, 0], C[2:5].T * V[:, None], rtol=1e-13, atol=0)


def _map(Xe, pts):
    """Prism map x(xi) written out from the vertex shape functions."""
    xi, eta, ze = pts[:, 0], pts[:, 1], pts[:, 2]
    lam = [1 - xi - eta, xi, eta]
    out = np.zeros((pts.shape[0], 3))
    for a in range(3):
        out += np.outer(lam[a] * (1 - ze) / 2, Xe[a]) + np.outer(lam[a] * (1 + ze) / 2, Xe[a + 3])
    return out


@pytest.mark.parametrize("elem", [PRISM, 2])
@pytest.mark.parametrize("p", [1, 3])
def test_rigid_rotations_in_kernel(orc, p, elem):
    """u = w x x has zero strain: its coefficient vectors (fitted exactly in the
    basis, which contains the map) are annihilated by A^e, with either rule."""
    E = 4
    X = inputs.prism_mesh(E, dims=(2, 1, 1))[:E]
    C = inputs.elastic_coefficients(E)
    A, _, _ = orc.integrate_elastic(p, X, C, elem=elem)
    rng = np.random.default_rng(1)
    pts = []
    while len(pts) < 400:
        x, y = rng.uniform(0, 1, 2)
        if x + y <= 1:
            pts.append([x, y, rng.uniform(-1, 1)])
    pts = np.array(pts)
    phi = orc.basis(PRISM, p, pts)[:, 0, :]  # [npts][NS]
    NS = phi.shape[1]
    for e in range(E):
        x = _map(X[e], pts)
        coef, res, *_ = np.linalg.lstsq(phi, x, rcond=None)  # x_m = sum_r coef[r][m] phi_r
        assert np.max(np.abs(phi @ coef - x)) < 1e-12
        for w in np.eye(3):
            u = np.cross(w, coef)  # coefficients of w x x, [NS][3]
            U = u.T.reshape(3 * NS)
            Ae = A[e].transpose(0, 2, 1, 3).reshape(3 * NS, 3 * NS)
            r = Ae @ U
            assert np.linalg.norm(r) < 1e-11 * np.linalg.norm(Ae) * np.linalg.norm(U)


@pytest.mark.parametrize("elem", [PRISM, 2])
@pytest.mark.parametrize("p", [2, 5])
def test_trace_is_scaled_laplacian(orc, p, elem):
    """sum_i A^{ii} = (lam + 4 mu) times the scalar stiffness with D = I."""
    E = 3
    X = inputs.prism_mesh(E, dims=(2, 1, 1))[:E]
    C = inputs.elastic_coefficients(E)
    A, _, _ = orc.integrate_elastic(p, X, C, elem=elem)
    lam, mu = _lame(C[0], C[1])
    Cs = np.zeros((11, E))
    Cs[0:3] = (lam + 4 * mu)[None, :]
    K, _, _ = orc.integrate(elem, p, X, Cs)
    assert _relF(A[:, 0, 0] + A[:, 1, 1] + A[:, 2, 2], K) < 1e-13


@pytest.mark.slow
def test_affine_prism_exact_rational(orc):
    """Affine prism: every block equals its exact integral, computed with
    rationals from the symbolic basis moments."""
    p = 1
    x0 = [Fraction(1, 3), Fraction(-1, 5), Fraction(2, 7)]
    e1 = [Fraction(3, 4), Fraction(1, 8), Fraction(-1, 6)]
    e2 = [Fraction(-1, 9), Fraction(2, 3), Fraction(1, 10)]
    v = [Fraction(1, 7), Fraction(-1, 11), Fraction(4, 5)]
    bot = [x0, [x0[i] + e1[i] for i in range(3)], [x0[i] + e2[i] for i in range(3)]]
    verts = bot + [[q[i] + v[i] for i in range(3)] for q in bot]
    J = [[e1[i], e2[i], v[i] / 2] for i in range(3)]
    det = (J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
           - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
           + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]))
    Ji = [[None] * 3 for _ in range(3)]
    for k in range(3):
        for m in range(3):
            r0, r1, c0, c1 = (m + 1) % 3, (m + 2) % 3, (k + 1) % 3, (k + 2) % 3
            Ji[k][m] = (J[r0][c0] * J[r1][c1] - J[r0][c1] * J[r1][c0]) / det
    Ey, nu = Fraction(7, 2), Fraction(3, 10)
    lam, mu = Ey * nu / ((1 + nu) * (1 - 2 * nu)), Ey / (2 * (1 + nu))

    def c(i, j, k, l):
        return lam * (i == j) * (k == l) + mu * ((i == k) * (j == l) + (i == l) * (j == k))

    M = _exact_reference_moments(p)
    NS = len(M[0][0])
    Aex = np.zeros((3, 3, NS, NS))
    for i in range(3):
        for k in range(3):
            G = [[det * sum(Ji[a][j] * c(i, j, k, l) * Ji[b][l] for j in range(3) for l in range(3))
                  for b in range(3)] for a in range(3)]
            for s in range(NS):
                for r in range(NS):
                    Aex[i, k, s, r] = float(sum(G[a][b] * M[1 + a][1 + b][s][r]
                                                for a in range(3) for b in range(3)))
    X = np.array([[float(q) for q in row] for row in verts])[None]
    C = np.array([[float(Ey)], [float(nu)], [0.0], [0.0], [0.0]])
    A, _, st = orc.integrate_elastic(p, X, C)
    assert st[0] == 0
    assert _relF(A[0], Aex) < 1e-14
