"""Pins of the oracle's element-operator apply y_e = A_e x_e against closed
forms that do not go through the oracle: textbook P1 integrals on tets, and on
the reference prism (x = xi, y = eta, z = zeta) the integrals of the
Dubiner x Legendre basis that orthogonality and the fundamental theorem of
calculus fix (int_T T_t = |T| delta_t0, int L_k' = L_k(1) - L_k(-1))."""
import numpy as np
import pytest

from paper_1310_1191_gb300 import inputs

TET, PRISM = 0, 1
REF_PRISM = np.array([[0, 0, -1], [1, 0, -1], [0, 1, -1], [0, 0, 1], [1, 0, 1], [0, 1, 1]], float)


def _coef(E, D=None, b=(0, 0, 0), c=0.0):
    out = np.zeros((11, E))
    if D is not None:
        D = np.asarray(D, float)
        out[0], out[1], out[2] = D[0, 0], D[1, 1], D[2, 2]
        out[3], out[4], out[5] = D[0, 1], D[0, 2], D[1, 2]
    out[6:9] = np.asarray(b, float)[:, None]
    out[9] = c
    return out


def test_apply_tet_closed_form(orc):
    """General D, b, c on P1 tets: y = (V G D G^T + V/4 1 (G b)^T + c V (1 + I)/20) x."""
    X = inputs.tet_mesh(2)
    E = X.shape[0]
    C = inputs.coefficients(E)
    x = np.random.default_rng(3).standard_normal((E, 4))
    y, st = orc.apply(TET, 1, X, C, x)
    assert np.all(st == 0)
    for e in range(E):
        Mx = np.hstack([np.ones((4, 1)), X[e]])
        G = np.linalg.inv(Mx)[1:, :].T
        V = abs(np.linalg.det(Mx)) / 6.0
        D = np.array([[C[0, e], C[3, e], C[4, e]], [C[3, e], C[1, e], C[5, e]],
                      [C[4, e], C[5, e], C[2, e]]])
        op = V * G @ D @ G.T + (V / 4.0) * np.outer(np.ones(4), G @ C[6:9, e]) + \
            C[9, e] * V * (np.ones((4, 4)) + np.eye(4)) / 20.0
        ref = op @ x[e]
        assert np.linalg.norm(y[e] - ref) <= 1e-13 * np.linalg.norm(op) * np.linalg.norm(x[e])


@pytest.mark.parametrize("p", [1, 2, 3, 5, 7])
def test_apply_reference_prism_diffusion(orc, p):
    """D = I on the reference prism, x = the DOF of zeta (t = 0, k = 1):
    y_i = int dphi_i/dzeta = |T| (L_k(1) - L_k(-1)) delta_t0 = 1 for t = 0 and
    odd k, 0 otherwise."""
    NT = (p + 1) * (p + 2) // 2
    n = orc.ns(PRISM, p)
    x = np.zeros((1, n))
    x[0, NT] = 1.0
    y, st = orc.apply(PRISM, p, REF_PRISM[None], _coef(1, D=np.eye(3)), x)
    ref = np.zeros(n)
    ref[[NT * k for k in range(1, p + 1, 2)]] = 1.0
    assert st[0] == 0
    assert np.max(np.abs(y[0] - ref)) < 1e-13


@pytest.mark.parametrize("p", [2, 4, 6])
def test_apply_reference_prism_convection(orc, p):
    """b = e_z on the reference prism, x = the DOF of zeta: y_i = int phi_i
    (b . grad zeta) = |K| delta_i0 = 1 for i = 0 only.  The transposed product
    would pick up int L_k' zeta != 0 for even k >= 2, so this fixes the
    orientation of the product (A x, not A^T x)."""
    NT = (p + 1) * (p + 2) // 2
    n = orc.ns(PRISM, p)
    x = np.zeros((1, n))
    x[0, NT] = 1.0
    y, _ = orc.apply(PRISM, p, REF_PRISM[None], _coef(1, b=(0.0, 0.0, 1.0)), x)
    ref = np.zeros(n)
    ref[0] = 1.0
    assert np.max(np.abs(y[0] - ref)) < 1e-13


@pytest.mark.parametrize("p", [1, 3, 7])
def test_apply_extruded_prism_reaction_and_constant_mode(orc, p):
    """Straight (un-jittered) prisms, det J constant: reaction only gives
    y = c V e_0 for x = e_0 (the basis is orthogonal to the constant); with
    c = 0 any D and b annihilate the constant (y = 0)."""
    dims = (2, 2, 1)
    E = 2 * 2 * 2
    X = inputs.prism_mesh(E, jitter=0.0, dims=dims)
    n = orc.ns(PRISM, p)
    x = np.zeros((E, n))
    x[:, 0] = 1.0
    c = 0.7
    y, st = orc.apply(PRISM, p, X, _coef(E, c=c), x)
    assert np.all(st == 0)
    V = np.abs(np.linalg.det(np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], 2))) / 2.0
    ref = np.zeros((E, n))
    ref[:, 0] = c * V
    assert np.max(np.abs(y - ref)) < 1e-13 * c * V.max()
    C = inputs.coefficients(E)
    C[9] = 0.0
    y, _ = orc.apply(PRISM, p, inputs.prism_mesh(E, dims=dims), C, x)
    assert np.max(np.abs(y)) < 1e-12 * np.abs(C[:9]).max()


@pytest.mark.parametrize("p", [2, 5])
def test_apply_symmetry_and_energy(orc, p):
    """b = 0: z . (A x) = x . (A z) (symmetric form) and x . (A x) > 0 (D SPD, c > 0)."""
    E = 4
    X = inputs.prism_mesh(E, dims=(2, 1, 1))
    C = inputs.coefficients(E)
    C[6:9] = 0.0
    n = orc.ns(PRISM, p)
    rng = np.random.default_rng(5)
    x, z = rng.standard_normal((2, E, n))
    yx, _ = orc.apply(PRISM, p, X, C, x)
    yz, _ = orc.apply(PRISM, p, X, C, z)
    a, b = np.einsum("ei,ei->e", z, yx), np.einsum("ei,ei->e", x, yz)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))
    assert np.all(np.einsum("ei,ei->e", x, yx) > 0)
