"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: printed
table values, closed-form integrals, library routines for special cases,
invariants of the weak form and exact rational brute force on affine elements.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1310_1191_gb300 import inputs

TET, PRISM = 0, 1
HERE = os.path.dirname(os.path.abspath(__file__))

REF_PRISM = np.array([[0, 0, -1], [1, 0, -1], [0, 1, -1], [0, 0, 1], [1, 0, 1], [0, 1, 1]], float)


def _coef(E, D=None, b=(0, 0, 0), c=0.0, f=0.0):
    out = np.zeros((11, E))
    if D is not None:
        D = np.asarray(D, float)
        out[0], out[1], out[2] = D[0, 0], D[1, 1], D[2, 2]
        out[3], out[4], out[5] = D[0, 1], D[0, 2], D[1, 2]
    out[6:9] = np.asarray(b, float)[:, None]
    out[9] = c
    out[10] = f
    return out


def _relF(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------- tables


def test_paper_table1_table2_sizes(orc):
    """N_sh and Table 2 array sizes printed in the paper (Tables 1, 2)."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "paper_tables_1_2.txt"))
            if l.strip() and not l.startswith("#")][1:]
    for p, nsh, per_pt, blocks, nq in (map(int, r) for r in rows):
        assert orc.ns(PRISM, p) == nsh
        assert 4 * orc.ns(PRISM, p) == per_pt
        assert orc.ns(PRISM, p) ** 2 == blocks
        assert orc.nq(PRISM, p) == (p + 1) ** 3
        assert orc.nq(orc.PRISM_T1, p) == nq
        assert orc.rule(orc.PRISM_T1, p)[0].shape == (nq, 3)


def test_jacobi_vs_scipy(orc):
    from scipy.special import eval_jacobi
    rng = np.random.default_rng(0)
    for n in range(0, 9):
        for a in (0, 1, 3, 7, 15):
            for x in rng.uniform(-1, 1, 5):
                ref = eval_jacobi(n, a, 0, x)
                assert abs(orc.jacobi(n, a, 0, x) - ref) <= 1e-12 * max(1, abs(ref))
                h = 1e-6
                fd = (eval_jacobi(n, a, 0, x + h) - eval_jacobi(n, a, 0, x - h)) / (2 * h)
                assert abs(orc.djacobi(n, a, 0, x) - fd) <= 1e-6 * max(1, abs(fd))


def test_gauss_rules_vs_library(orc):
    """Gauss-Legendre = numpy.leggauss; Gauss-Jacobi(1,0) = scipy.roots_jacobi."""
    from scipy.special import roots_jacobi
    for n in range(1, 9):
        x, w = orc.gauss_jacobi(n, 0, 0)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.allclose(x, xr, atol=1e-15, rtol=0) and np.allclose(w, wr, atol=1e-15, rtol=0)
        x, w = orc.gauss_jacobi(n, 1, 0)
        xr, wr = roots_jacobi(n, 1, 0)
        assert np.allclose(x, xr, atol=1e-14, rtol=0) and np.allclose(w, wr, atol=1e-14, rtol=0)


@pytest.mark.parametrize("p", range(1, 8))
def test_prism_rule_exactness(orc, p):
    """Exact on random polynomials of degree <= 2p:
    int_T xi^a eta^b = a! b! / (a+b+2)!, int_{-1}^{1} zeta^c = 2/(c+1) (c even)."""
    xi, w = orc.rule(PRISM, p)
    assert abs(w.sum() - 1.0) < 1e-14
    rng = np.random.default_rng(p)
    for trial in range(20):
        a = int(rng.integers(0, 2 * p + 1))
        b = int(rng.integers(0, 2 * p + 1 - a))
        c = int(rng.integers(0, 2 * p + 1))
        exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2) * (
            2.0 / (c + 1) if c % 2 == 0 else 0.0)
        got = np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c)
        assert abs(got - exact) <= 1e-14 * max(1.0, abs(exact)), (a, b, c)
    # random polynomial of total degree <= 2p (combination of monomials)
    terms = [(a, b, c) for a in range(2 * p + 1) for b in range(2 * p + 1 - a)
             for c in range(2 * p + 1)]
    coef = rng.standard_normal(len(terms))
    got = sum(k * np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c)
              for k, (a, b, c) in zip(coef, terms))
    exact = sum(k * math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
                * (2.0 / (c + 1) if c % 2 == 0 else 0.0) for k, (a, b, c) in zip(coef, terms))
    assert abs(got - exact) < 1e-12


def test_tet_rule_textbook(orc):
    """4-point rule exact to degree 2: int_tet x^a y^b z^c = a!b!c!/(a+b+c+3)!."""
    xi, w = orc.rule(TET, 1)
    for a in range(3):
        for b in range(3 - a):
            for c in range(3 - a - b):
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(
                    a + b + c + 3)
                got = np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c)
                assert abs(got - exact) < 1e-16


# ---------------------------------------------------------------- basis


@pytest.mark.parametrize("p", range(1, 8))
def test_basis_orthogonality_identity_prism(orc, p):
    """Mass matrix on the reference prism is diagonal with entries
    1/((2i+1)(i+j+1)(2k+1)) for the unnormalised Dubiner x Legendre basis."""
    NS = orc.ns(PRISM, p)
    X = REF_PRISM[None]
    A, b, st = orc.integrate(PRISM, p, X, _coef(1, c=1.0, f=1.0))
    M = A[0]
    NT = (p + 1) * (p + 2) // 2
    expect = np.zeros(NS)
    t = 0
    for n in range(p + 1):
        for i in range(n, -1, -1):
            j = n - i
            for k in range(p + 1):
                expect[t + NT * k] = 1.0 / ((2 * i + 1) * (i + j + 1) * (2 * k + 1))
            t += 1
    assert np.max(np.abs(np.diag(M) - expect)) < 1e-14
    assert np.max(np.abs(M - np.diag(np.diag(M)))) < 1e-14
    assert abs(b[0, 0] - 1.0) < 1e-14 and np.max(np.abs(b[0, 1:])) < 1e-14
    assert st[0] == 0


@pytest.mark.parametrize("p", [1, 3, 7])
def test_basis_derivatives_finite_difference(orc, p):
    rng = np.random.default_rng(10 + p)
    pts = []
    while len(pts) < 6:
        x, y = rng.uniform(0.05, 0.9, 2)
        if x + y < 0.95:
            pts.append([x, y, rng.uniform(-0.9, 0.9)])
    pts = np.array(pts)
    phi = orc.basis(PRISM, p, pts)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (orc.basis(PRISM, p, pts + e)[:, 0] - orc.basis(PRISM, p, pts - e)[:, 0]) / (2 * h)
        scale = np.max(np.abs(phi[:, 1 + k])) + 1
        assert np.max(np.abs(phi[:, 1 + k] - fd)) < 2e-6 * scale


# ---------------------------------------------------------------- P1 tetrahedra


def test_p1_tet_closed_form(orc):
    """A = V G G^T, b = f V / 4 (G = barycentric gradients); row/column sums
    vanish; sum of volumes = 1 on the unit cube mesh."""
    X = inputs.tet_mesh(4)
    E = X.shape[0]
    A, b, st = orc.integrate(TET, 1, X, inputs.coefficients(E, kind="laplace"))
    assert np.all(st == 0)
    for e in range(E):
        Mx = np.hstack([np.ones((4, 1)), X[e]])
        Ginv = np.linalg.inv(Mx)  # columns: barycentric coordinate coefficients
        G = Ginv[1:, :].T  # [4][3] gradients
        V = abs(np.linalg.det(Mx)) / 6.0
        assert np.max(np.abs(A[e] - V * G @ G.T)) < 1e-13 * np.max(np.abs(A[e]))
        assert np.allclose(b[e], V / 4.0, rtol=1e-14, atol=0)
    assert np.max(np.abs(A.sum(axis=1))) < 1e-14 and np.max(np.abs(A.sum(axis=2))) < 1e-14
    assert abs(b.sum() - 1.0) < 1e-13


def test_p1_tet_general_form(orc):
    """General D, b, c on P1: closed form with exact integrals of barycentric
    products (int lam_i = V/4, int lam_i lam_j = V (1+delta_ij)/20)."""
    X = inputs.tet_mesh(2)
    E = X.shape[0]
    C = inputs.coefficients(E)
    A, b, st = orc.integrate(TET, 1, X, C)
    for e in range(E):
        Mx = np.hstack([np.ones((4, 1)), X[e]])
        G = np.linalg.inv(Mx)[1:, :].T
        V = abs(np.linalg.det(Mx)) / 6.0
        D = np.array([[C[0, e], C[3, e], C[4, e]], [C[3, e], C[1, e], C[5, e]],
                      [C[4, e], C[5, e], C[2, e]]])
        bb, c, f = C[6:9, e], C[9, e], C[10, e]
        M = V * (np.ones((4, 4)) + np.eye(4)) / 20.0
        ref = V * G @ D @ G.T + (V / 4.0) * np.outer(np.ones(4), G @ bb) + c * M
        assert _relF(A[e], ref) < 1e-14
        assert np.allclose(b[e], f * V / 4.0, rtol=1e-13, atol=1e-18)


# ---------------------------------------------------------------- prisms


def _sympy_volume(X):
    """Exact volume of a straight-edged prism: integral of det J over the
    reference prism, done symbolically with the vertices as rationals."""
    import sympy as sp
    xi, eta, ze = sp.symbols("xi eta zeta")
    lam = [1 - xi - eta, xi, eta]
    N = [lam[a] * (1 - ze) / 2 for a in range(3)] + [lam[a] * (1 + ze) / 2 for a in range(3)]
    Xr = [[sp.Rational(float(v)) for v in row] for row in X]
    x = [sum(N[v] * Xr[v][i] for v in range(6)) for i in range(3)]
    J = sp.Matrix(3, 3, lambda i, k: sp.diff(x[i], [xi, eta, ze][k]))
    d = sp.expand(J.det())
    return float(sp.integrate(sp.integrate(sp.integrate(d, (eta, 0, 1 - xi)), (xi, 0, 1)),
                              (ze, -1, 1)))


@pytest.mark.parametrize("p", [1, 2, 4, 7])
def test_prism_volume_and_load(orc, p):
    """D = 0, b = 0, c = 1: A[0][0] = V_e (phi_0 = 1); b_e[0] = f V_e; the
    volumes of a full grid add up to the box; two elements checked against an
    exact symbolic integral of det J."""
    dims = (3, 3, 2)
    E = 2 * 3 * 3 * 2
    X = inputs.prism_mesh(E, dims=dims)
    f = 0.37
    A, b, st = orc.integrate(PRISM, p, X, _coef(E, c=1.0, f=f))
    assert np.all(st == 0)
    V = A[:, 0, 0]
    assert abs(V.sum() - inputs.prism_box_volume(E, dims)) < 1e-14
    assert np.allclose(b[:, 0], f * V, rtol=1e-14, atol=0)
    if p == 1:
        for e in (0, 7):
            assert abs(V[e] - _sympy_volume(X[e])) < 1e-15


@pytest.mark.parametrize("p", [1, 3, 5])
def test_prism_constant_mode(orc, p):
    """Pure diffusion annihilates the constant (DOF 0) on both sides;
    diffusion + convection still annihilates it as trial function (column 0)."""
    E = 6
    X = inputs.prism_mesh(E, dims=(2, 2, 2))
    C = inputs.coefficients(E)
    Cd = C.copy()
    Cd[6:10] = 0.0
    A, _, _ = orc.integrate(PRISM, p, X, Cd)
    s = np.abs(A).max()
    assert np.max(np.abs(A[:, :, 0])) < 1e-13 * s and np.max(np.abs(A[:, 0, :])) < 1e-13 * s
    Cc = C.copy()
    Cc[9] = 0.0
    A, _, _ = orc.integrate(PRISM, p, X, Cc)
    assert np.max(np.abs(A[:, :, 0])) < 1e-13 * s
    assert np.max(np.abs(A[:, 0, :])) > 1e-3 * s  # convection does act on the test side


@pytest.mark.parametrize("p", [2, 6])
def test_prism_symmetry(orc, p):
    E = 4
    X = inputs.prism_mesh(E, dims=(2, 2, 1))
    A, _, _ = orc.integrate(PRISM, p, X, inputs.coefficients(E, kind="symmetric"))
    assert np.max(np.abs(A - A.transpose(0, 2, 1))) < 1e-13 * np.abs(A).max()


def _rot(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("p", [1, 3])
def test_prism_invariances(orc, p):
    """Rotation with D' = R D R^T, b' = R b and translation leave A unchanged;
    scaling x -> s x scales diffusion by s, convection by s^2, reaction by s^3."""
    rng = np.random.default_rng(5)
    X = inputs.prism_mesh(4, dims=(2, 2, 1))[:1]
    C = inputs.coefficients(1)
    A0, _, _ = orc.integrate(PRISM, p, X, C)
    R = _rot(rng)
    D = np.array([[C[0, 0], C[3, 0], C[4, 0]], [C[3, 0], C[1, 0], C[5, 0]],
                  [C[4, 0], C[5, 0], C[2, 0]]])
    D2 = R @ D @ R.T
    C2 = C.copy()
    C2[0:6, 0] = [D2[0, 0], D2[1, 1], D2[2, 2], D2[0, 1], D2[0, 2], D2[1, 2]]
    C2[6:9, 0] = R @ C[6:9, 0]
    X2 = (X[0] @ R.T + np.array([0.3, -1.2, 2.0]))[None]
    A1, _, _ = orc.integrate(PRISM, p, X2, C2)
    assert _relF(A1, A0) < 1e-13
    s = 1.7
    parts = []
    for sel in ("diff", "conv", "reac"):
        Cs = C.copy()
        if sel != "diff":
            Cs[0:6] = 0
        if sel != "conv":
            Cs[6:9] = 0
        if sel != "reac":
            Cs[9] = 0
        parts.append((orc.integrate(PRISM, p, X, Cs)[0], orc.integrate(PRISM, p, X * s, Cs)[0]))
    for (a, as_), k in zip(parts, (1, 2, 3)):
        assert _relF(as_, a * s ** k) < 1e-13


def _exact_reference_moments(p):
    """Exact rational moments M[d][d'][i][j] = int_ref dphi_i/dxi_d dphi_j/dxi_d'
    (d = 0 value, 1..3 reference derivatives) of the Dubiner x Legendre basis,
    built symbolically from sympy's Jacobi polynomials."""
    import sympy as sp
    x, y, z = sp.symbols("x y z")
    r, s = 2 * x - 1, 2 * y - 1
    a = 2 * (1 + r) / (1 - s) - 1
    tri = []
    for n in range(p + 1):
        for i in range(n, -1, -1):
            j = n - i
            e = sp.jacobi(i, 0, 0, a) * ((1 - s) / 2) ** i * sp.jacobi(j, 2 * i + 1, 0, s)
            tri.append(sp.Poly(sp.cancel(sp.expand(e)), x, y))
    basis = []
    for k in range(p + 1):
        L = sp.Poly(sp.expand(sp.jacobi(k, 0, 0, z)), z)
        for t in tri:
            basis.append(sp.Poly(t.as_expr() * L.as_expr(), x, y, z, domain="QQ"))
    fun = [[b, b.diff(x), b.diff(y), b.diff(z)] for b in basis]

    def integ(poly):
        tot = Fraction(0)
        for (ea, eb, ec), cf in poly.terms():
            if ec % 2:
                continue
            v = Fraction(math.factorial(ea) * math.factorial(eb), math.factorial(ea + eb + 2))
            tot += Fraction(int(cf.p), int(cf.q)) * v * Fraction(2, ec + 1)
        return tot

    NS = len(basis)
    M = [[[[integ(fun[i][d] * fun[j][dd]) for j in range(NS)] for i in range(NS)]
          for dd in range(4)] for d in range(4)]
    return M


@pytest.mark.slow
@pytest.mark.parametrize("elem", [PRISM, 2])
@pytest.mark.parametrize("p", [1, 2])
def test_affine_prism_exact_rational(orc, p, elem):
    """Affine prism, constant coefficients: the integrand is a polynomial of
    degree <= 2p, so the oracle's quadrature sum equals the exact integral,
    computed here with rationals from a symbolic basis; with the collapsed
    rule and with the paper's rule (elem 2, Table 1 point counts)."""
    x0 = [Fraction(1, 3), Fraction(-1, 5), Fraction(2, 7)]
    e1 = [Fraction(3, 4), Fraction(1, 8), Fraction(-1, 6)]
    e2 = [Fraction(-1, 9), Fraction(2, 3), Fraction(1, 10)]
    v = [Fraction(1, 7), Fraction(-1, 11), Fraction(4, 5)]  # top = bottom + v
    bot = [x0, [x0[i] + e1[i] for i in range(3)], [x0[i] + e2[i] for i in range(3)]]
    verts = bot + [[q[i] + v[i] for i in range(3)] for q in bot]
    # J columns: dx/dxi = e1, dx/deta = e2, dx/dzeta = v/2
    J = [[e1[i], e2[i], v[i] / 2] for i in range(3)]

    def det3(m):
        return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
                - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
                + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))

    det = det3(J)
    Ji = [[None] * 3 for _ in range(3)]
    for k in range(3):
        for m in range(3):
            r0, r1, c0, c1 = (m + 1) % 3, (m + 2) % 3, (k + 1) % 3, (k + 2) % 3
            Ji[k][m] = (J[r0][c0] * J[r1][c1] - J[r0][c1] * J[r1][c0]) / det
    D = [[Fraction(2), Fraction(1, 2), Fraction(-1, 3)], [Fraction(1, 2), Fraction(3), Fraction(1, 4)],
         [Fraction(-1, 3), Fraction(1, 4), Fraction(5, 2)]]
    bb = [Fraction(1, 2), Fraction(-3, 4), Fraction(1, 3)]
    c = Fraction(2, 3)
    # G[d][d'] on reference derivatives
    G = [[Fraction(0)] * 4 for _ in range(4)]
    G[0][0] = det * c
    for k in range(3):
        G[0][1 + k] = det * sum(Ji[k][m] * bb[m] for m in range(3))
        for l in range(3):
            G[1 + k][1 + l] = det * sum(Ji[k][m] * D[m][n] * Ji[l][n] for m in range(3)
                                        for n in range(3))
    M = _exact_reference_moments(p)
    NS = len(M[0][0])
    Aex = np.array([[float(sum(G[d][dd] * M[d][dd][i][j] for d in range(4) for dd in range(4)))
                     for j in range(NS)] for i in range(NS)])
    X = np.array([[float(q) for q in row] for row in verts])[None]
    C = _coef(1, D=np.array(D, dtype=float), b=np.array(bb, dtype=float), c=float(c))
    A, _, st = orc.integrate(elem, p, X, C)
    assert st[0] == 0
    assert _relF(A[0], Aex) < 1e-14


def test_status_flags(orc):
    X = inputs.prism_mesh(4, dims=(2, 1, 1))
    X[1] = X[1][[1, 0, 2, 4, 3, 5]]  # mirrored -> det J < 0
    C = inputs.coefficients(4)
    C[9, 2] = np.nan
    _, _, st = orc.integrate(PRISM, 2, X, C)
    assert st[0] == 0 and st[1] & 1 and st[2] & 2 and st[3] == 0


# ---------------------------------------------------------------- nonlinear law


def test_law_newton(orc):
    """k = 1 + 0.5 exp(-u^2) + 0.2 log(1 + k g): 8 Newton steps leave a
    residual <= 1e-12; g = 0 gives the closed form; matches a bracketing
    root finder."""
    from scipy.optimize import brentq
    rng = np.random.default_rng(3)
    for u, g in zip(rng.uniform(-3, 3, 50), rng.uniform(0, 400, 50)):
        k = orc.law_k(u, g)
        assert abs(orc.law_residual(u, g, k)) <= 1e-12
        kr = brentq(lambda kk: kk - 1 - 0.5 * math.exp(-u * u) - 0.2 * math.log(1 + kk * g), 1.0,
                    100.0, xtol=1e-15)
        assert abs(k - kr) < 1e-12 * kr
    for u in (-1.5, 0.0, 0.7):
        assert abs(orc.law_k(u, 0.0) - (1 + 0.5 * math.exp(-u * u))) < 1e-15


def test_integrate_nonlinear_law_reduces_to_constant(orc):
    """With u = const (only DOF 0 set) the gradient vanishes, so k = 1 +
    0.5 exp(-u^2) at every point: same as constant D = k I."""
    p = 2
    E = 3
    X = inputs.prism_mesh(E, dims=(2, 1, 1))
    C = inputs.coefficients(E)
    NS = orc.ns(PRISM, p)
    U = np.zeros((E, NS))
    U[:, 0] = [0.3, -0.8, 1.1]
    A, b, _ = orc.integrate(PRISM, p, X, C, law=1, ucoef=U)
    C2 = C.copy()
    k = 1 + 0.5 * np.exp(-U[:, 0] ** 2)
    C2[0] = C2[1] = C2[2] = k
    C2[3:6] = 0
    A2, b2, _ = orc.integrate(PRISM, p, X, C2)
    assert _relF(A, A2) < 1e-14 and _relF(b, b2) < 1e-15


# ---------------------------------------------------------------- MLP


def test_mlp_against_torch_and_fd(orc):
    """FP64 forward/backprop of the 2->H->H->1 tanh network vs torch.nn with
    the same parameters (inputs u and s = |grad u|, u mapped linearly and
    log s linearly onto [-1, 1]), and vs central finite differences."""
    import torch
    H = 8
    rng = np.random.default_rng(11)
    P = orc.mlp_nparams(H)
    assert P == 2 * H + H + H * H + H + H + 1
    th = rng.standard_normal(P) * 0.5
    box = np.array([-2.0, 2.0, 1.0, 50.0])
    u = rng.uniform(-2, 2, 32)
    g = rng.uniform(1, 50, 32)  # s = |grad u|
    t = rng.uniform(1, 2, 32)
    L, grad = orc.mlp_loss_grad(H, th, box, u, g, t)
    # torch reference
    net = torch.nn.Sequential(torch.nn.Linear(2, H), torch.nn.Tanh(), torch.nn.Linear(H, H),
                              torch.nn.Tanh(), torch.nn.Linear(H, 1)).double()
    o = 0
    for layer, (r, c) in zip([net[0], net[2], net[4]], [(H, 2), (H, H), (1, H)]):
        layer.weight.data = torch.tensor(th[o:o + r * c].reshape(r, c))
        o += r * c
        layer.bias.data = torch.tensor(th[o:o + r])
        o += r
    xin = torch.tensor(np.stack([2 * (u + 2) / 4 - 1, 2 * np.log(g) / np.log(50.0) - 1], 1))
    y = net(xin)[:, 0]
    Lt = ((y - torch.tensor(t)) ** 2).mean()
    Lt.backward()
    gt = np.concatenate([np.concatenate([l.weight.grad.numpy().ravel(), l.bias.grad.numpy()])
                         for l in (net[0], net[2], net[4])])
    assert abs(L - Lt.item()) < 1e-13
    assert np.max(np.abs(grad - gt)) < 1e-13
    assert np.allclose(orc.mlp_forward(H, th, box, u, g), y.detach().numpy(), rtol=0, atol=1e-14)
    # central finite differences
    h = 1e-6
    for k in rng.choice(P, 12, replace=False):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (orc.mlp_loss_grad(H, tp, box, u, g, t)[0] - orc.mlp_loss_grad(H, tm, box, u, g, t)[0]) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(grad[k]))


def test_integrate_mlp_law_inside_and_outside_box(orc):
    """law=2 equals law=1 when the network reproduces the law exactly outside
    of its box (fallback flagged), and uses the network inside: a network whose
    output is a constant k0 (all weights zero, b3 = k0) gives D = k0 I."""
    p = 2
    E = 4
    X = inputs.prism_mesh(E, dims=(2, 1, 1))
    C = inputs.coefficients(E)
    NS = orc.ns(PRISM, p)
    U = np.stack([2.0 * inputs.draw_uniform(5, np.arange(E, dtype=np.uint64), k) - 1.0
                  for k in range(NS)], 1)
    H = 8
    th = np.zeros(orc.mlp_nparams(H))
    th[-1] = 2.5
    big = np.array([-1e9, 1e9, 1e-12, 1e12])
    A2, b2, st2 = orc.integrate(PRISM, p, X, C, law=2, ucoef=U, mlp=(H, th, big))
    C2 = C.copy()
    C2[0] = C2[1] = C2[2] = 2.5
    C2[3:6] = 0
    A0, b0, _ = orc.integrate(PRISM, p, X, C2)
    assert _relF(A2, A0) < 1e-14 and np.all(st2 == 0)
    tiny = np.array([1e8, 2e8, 1e8, 2e8])  # nothing inside: exact law everywhere
    A3, _, st3 = orc.integrate(PRISM, p, X, C, law=2, ucoef=U, mlp=(H, th, tiny))
    A1, _, _ = orc.integrate(PRISM, p, X, C, law=1, ucoef=U)
    assert _relF(A3, A1) < 1e-15 and np.all(st3 == 8)


# ------------------------------------------- law with a non-zero field gradient


def _sheared_affine_prism():
    """An affine image x = M xi + t of the reference prism with a shear (M is
    not symmetric, so J^{-1} and J^{-T} differ), det M > 0."""
    M = np.array([[1.2, 0.35, -0.2], [-0.15, 0.9, 0.25], [0.3, -0.1, 0.6]])
    t = np.array([0.4, -0.3, 1.1])
    assert np.linalg.det(M) > 0
    return M, t, REF_PRISM @ M.T + t


def _linear_field_coefficients(orc, elem, p, X, M, t, a, c0):
    """Dubiner coefficients of u(x) = a.x + c0 on the affine element, by
    least squares over the oracle's quadrature points (u is linear in the
    reference coordinates, so the fit is exact)."""
    xi, _ = orc.rule(elem, p)
    phi0 = orc.basis(elem, p, xi)[:, 0, :]
    x = xi @ M.T + t
    U, *_ = np.linalg.lstsq(phi0, x @ a + c0, rcond=None)
    assert np.max(np.abs(phi0 @ U - (x @ a + c0))) < 1e-13
    return U, x


def _law_root(u, g):
    from scipy.optimize import brentq
    return brentq(lambda kk: kk - 1 - 0.5 * math.exp(-u * u) - 0.2 * math.log(1 + kk * g), 1.0,
                  100.0, xtol=1e-15)


@pytest.mark.parametrize("elem,p", [(PRISM, 1), (PRISM, 2), (PRISM, 3), (TET, 1)])
def test_point_law_linear_field_closed_form(orc, elem, p):
    """A linear physical field u = a.x + c0 on a sheared affine element: at
    every quadrature point u = a.x(xi_Q) + c0, |grad u| = |a| exactly, and k
    solves the law with g = |a|^2 (checked by a bracketing root finder).
    |a| != 1 separates g from |grad u|; the shear separates J^{-T} from J^{-1}."""
    M, t, X = _sheared_affine_prism()
    if elem == TET:
        X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) @ M.T + t
    a = np.array([1.3, -0.7, 2.1])
    c0 = 0.25
    U, x = _linear_field_coefficients(orc, elem, p, X, M, t, a, c0)
    u, s, k, st = orc.point_law(elem, p, X[None], U[None], law=1)
    assert st[0] == 0
    assert np.max(np.abs(u[0] - (x @ a + c0))) < 1e-12
    assert np.max(np.abs(s[0] - np.linalg.norm(a))) < 1e-12
    g = float(a @ a)
    kr = np.array([_law_root(uq, g) for uq in u[0]])
    assert np.max(np.abs(k[0] - kr) / kr) < 1e-12


def test_integrate_network_law_gradient_only_network(orc):
    """law=2 on a linear field: a network whose first layer ignores u (zero
    u-column) sees only |grad u| = |a|, constant over the element, so its
    output k0 is constant and integrate(law=2) equals integrate(law=0) with
    D = k0 I (b, c, f unchanged).  k0 comes from the network forward pass,
    which is pinned against torch.nn."""
    M, t, X = _sheared_affine_prism()
    p = 3
    a = np.array([1.3, -0.7, 2.1])
    U, _ = _linear_field_coefficients(orc, PRISM, p, X, M, t, a, 0.25)
    H = 8
    rng = np.random.default_rng(21)
    th = rng.standard_normal(orc.mlp_nparams(H)) * 0.4
    th[0:2 * H:2] = 0.0  # W1[:, 0] = 0: the network ignores u
    s0 = float(np.linalg.norm(a))
    box = np.array([-1e3, 1e3, 0.5 * s0, 2.0 * s0])
    k0 = float(orc.mlp_forward(H, th, box, np.array([0.0]), np.array([s0]))[0])
    C = inputs.coefficients(1)
    A2, b2, st2 = orc.integrate(PRISM, p, X[None], C, law=2, ucoef=U[None], mlp=(H, th, box))
    assert st2[0] == 0
    C0 = C.copy()
    C0[0] = C0[1] = C0[2] = k0
    C0[3:6] = 0
    A0, b0, _ = orc.integrate(PRISM, p, X[None], C0)
    # |grad u| at the points is |a| up to rounding (about 1e-13), hence 1e-12
    assert _relF(A2, A0) < 1e-12 and _relF(b2, b0) < 1e-15
    # the exact law at the same points (law=1) is not constant: it differs
    A1, _, _ = orc.integrate(PRISM, p, X[None], C, law=1, ucoef=U[None])
    assert _relF(A1, A0) > 1e-3
