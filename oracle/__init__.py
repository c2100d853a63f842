"""FP64 CPU oracle for per-element numerical integration (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never calls it.  The arithmetic lives in ``fem_oracle.c``, plain
C with OpenMP over elements, which writes out the quadrature sum of the weak
form (Section 2, eq. sum_int); this module compiles it with gcc on first use
and wraps it with ctypes.

Prism rules: elem PRISM uses the collapsed (p+1)^3-point rule; elem PRISM_T1
the paper's point counts (Table 1), a fully symmetric triangle rule found by
this oracle's own search (tri_search; stored in prism_rules_table1.txt by
make_prism_rules.py) times Gauss-Legendre in zeta.

Parity status of each function (what pins it is in tests/test_oracle_*.py):
  rule, basis, integrate (constant coefficients), law_k, mlp_loss_grad,
  apply (the element operator applied to a coefficient vector): pinned;
  point_law (u, |grad u| and k at the points): pinned by a linear physical
  field on a sheared affine prism (u, |grad u| and k in closed form);
  integrate with law=1/2: pinned by the constant-field reduction (law 1) and
  by a network that sees only |grad u|, constant for a linear field (law 2),
  both against law=0 with D = k I.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "fem_oracle.c")
_SO = os.path.join(_BUILD, "libfem_oracle.so")

TET, PRISM = 0, 1
PRISM_T1 = 2  # prism with the paper's rule (Table 1 point counts)
ST_DET, ST_NONFINITE, ST_FALLBACK = 1, 2, 8
_RULES = os.path.join(_HERE, "prism_rules_table1.txt")

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile fem_oracle.c into a shared library (gcc -O2 -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
            P = ctypes.c_void_p
            lib.orc_ns.argtypes = [i, i]
            lib.orc_nq.argtypes = [i, i]
            lib.orc_jacobi.argtypes = [i, i, i, d]
            lib.orc_jacobi.restype = d
            lib.orc_djacobi.argtypes = [i, i, i, d]
            lib.orc_djacobi.restype = d
            lib.orc_gauss_jacobi.argtypes = [i, i, i, P, P]
            lib.orc_rule.argtypes = [i, i, P, P]
            lib.orc_basis.argtypes = [i, i, i, P, P]
            lib.orc_law_k.argtypes = [d, d]
            lib.orc_law_k.restype = d
            lib.orc_law_residual.argtypes = [d, d, d]
            lib.orc_law_residual.restype = d
            lib.orc_mlp_nparams.argtypes = [i]
            lib.orc_mlp_forward.argtypes = [i, P, P, i64, P, P, P]
            lib.orc_mlp_loss_grad.argtypes = [i, P, P, i64, P, P, P, P]
            lib.orc_mlp_loss_grad.restype = d
            lib.orc_integrate_ex.argtypes = [i, i, i64, P, P, i64, i, P, i, P, P, P, P, P, i]
            lib.orc_point_law.argtypes = [i, i, i64, P, P, i, i, P, P, P, P, P, P]
            lib.orc_integrate_elastic.argtypes = [i, i64, P, P, i64, P, P, P, i]
            lib.orc_integrate_elastic_ex.argtypes = [i, i, i64, P, P, i64, P, P, P, i]
            lib.orc_jacobian_terms.argtypes = [i, i, i64, P, P, P]
            lib.orc_max_threads.argtypes = []
            lib.orc_tri_search.argtypes = [i, i64, ctypes.c_uint64, i, P, P]
            lib.orc_tri_unknowns.argtypes = [i]
            lib.orc_tri_points.argtypes = [i]
            lib.orc_set_tri_rule.argtypes = [i, P]
            lib.orc_tri_rule.argtypes = [i, P, P, P]
            for p, params in read_tri_rules().items():
                lib.orc_set_tri_rule(p, _f64(params).ctypes.data_as(ctypes.c_void_p))
            _lib = lib
    return _lib


def read_tri_rules(path: str = _RULES) -> dict:
    """{p: orbit parameters} of the stored symmetric triangle rules (the
    oracle's own search, written by make_prism_rules.py); {} if absent."""
    out = {}
    if not os.path.exists(path):
        return out
    for line in open(path):
        f = line.split()
        if f and f[0] == "rule":
            out[int(f[1])] = np.array([float(v) for v in f[7:]])
    return out


def tri_search(p: int, trials: int, seed: int = 1310, max_sol: int = 64):
    """Distinct positive-interior symmetric triangle rules of degree 2p found
    by `trials` continuation paths: (params [n][unknowns], smallest
    barycentric coordinate [n]), the largest coordinate first."""
    lib = _load()
    nu = lib.orc_tri_unknowns(p)
    sol = np.zeros((max_sol, nu))
    mb = np.zeros(max_sol)
    n = lib.orc_tri_search(p, trials, seed, max_sol, _ptr(sol), _ptr(mb))
    if n < 0:
        raise ValueError("bad degree")
    return sol[:n], mb[:n]


def tri_rule(p: int):
    """(xi [n], eta [n], w [n]) of the stored symmetric triangle rule of degree 2p."""
    x, y, w = np.zeros(64), np.zeros(64), np.zeros(64)
    n = _load().orc_tri_rule(p, _ptr(x), _ptr(y), _ptr(w))
    if n < 0:
        raise ValueError("no stored triangle rule for p = %d" % p)
    return x[:n], y[:n], w[:n]


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def ns(elem: int, p: int) -> int:
    return _load().orc_ns(elem, p)


def nq(elem: int, p: int) -> int:
    return _load().orc_nq(elem, p)


def max_threads() -> int:
    return _load().orc_max_threads()


def jacobi(n, a, b, x):
    return _load().orc_jacobi(n, a, b, float(x))


def djacobi(n, a, b, x):
    return _load().orc_djacobi(n, a, b, float(x))


def gauss_jacobi(n: int, a: int, b: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _load().orc_gauss_jacobi(n, a, b, _ptr(x), _ptr(w))
    return x, w


def rule(elem: int, p: int):
    """Quadrature points [NQ][3] and weights [NQ] on the reference element."""
    n = nq(elem, p)
    if n < 0:
        raise ValueError("unsupported element/degree")
    xi = np.zeros((n, 3))
    w = np.zeros(n)
    _load().orc_rule(elem, p, _ptr(xi), _ptr(w))
    return xi, w


def basis(elem: int, p: int, pts) -> np.ndarray:
    """Shape function values and reference derivatives [npts][4][NS]."""
    pts = _f64(pts).reshape(-1, 3)
    n = ns(elem, p)
    out = np.zeros((pts.shape[0], 4, n))
    _load().orc_basis(elem, p, pts.shape[0], _ptr(pts), _ptr(out))
    return out


def law_k(u: float, g: float) -> float:
    return _load().orc_law_k(float(u), float(g))


def law_residual(u: float, g: float, k: float) -> float:
    return _load().orc_law_residual(float(u), float(g), float(k))


def mlp_nparams(H: int) -> int:
    return _load().orc_mlp_nparams(H)


def mlp_forward(H, theta, box, u, s):
    """MLP(u, s) with s = |grad u|; box = (u0, u1, s0, s1)."""
    theta, box, u, s = _f64(theta), _f64(box), _f64(u), _f64(s)
    y = np.zeros(u.shape[0])
    _load().orc_mlp_forward(H, _ptr(theta), _ptr(box), u.shape[0], _ptr(u), _ptr(s), _ptr(y))
    return y


def mlp_loss_grad(H, theta, box, u, s, t):
    """Mean squared error of MLP(u, s) against t and its gradient (backprop)."""
    theta, box, u, s, t = _f64(theta), _f64(box), _f64(u), _f64(s), _f64(t)
    grad = np.zeros(mlp_nparams(H))
    L = _load().orc_mlp_loss_grad(H, _ptr(theta), _ptr(box), u.shape[0], _ptr(u), _ptr(s),
                                  _ptr(t), _ptr(grad))
    return L, grad


def integrate(elem: int, p: int, coords, coeffs, law: int = 0, ucoef=None, mlp=None,
              nthreads: int = 0):
    """Element matrices A [E][NS][NS], load vectors b [E][NS], status [E] (FP64).

    coords [E][nv][3]; coeffs SoA [11][E]; law 0 constant, 1 exact nonlinear
    law (ucoef [E][NS]), 2 MLP inside its box else the exact law
    (mlp = (H, theta, box)).
    """
    coords = _f64(coords)
    coeffs = _f64(coeffs)
    E = coords.shape[0]
    n = ns(elem, p)
    if n < 0:
        raise ValueError("unsupported element/degree")
    A = np.zeros((E, n, n))
    b = np.zeros((E, n))
    st = np.zeros(E, dtype=np.int32)
    uc = _f64(ucoef) if ucoef is not None else None
    H, th, box = (0, None, None) if mlp is None else (mlp[0], _f64(mlp[1]), _f64(mlp[2]))
    if law and uc is None:
        raise ValueError("law needs ucoef")
    if law == 2 and mlp is None:
        raise ValueError("law 2 needs mlp")
    rc = _load().orc_integrate_ex(elem, p, E, _ptr(coords), _ptr(coeffs), coeffs.shape[1], law,
                                  _ptr(uc), H, _ptr(th), _ptr(box), _ptr(A), _ptr(b), _ptr(st),
                                  nthreads)
    if rc != 0:
        raise RuntimeError("oracle integrate failed")
    return A, b, st


def point_law(elem: int, p: int, coords, ucoef, law: int = 1, mlp=None):
    """The coefficient stage of ``integrate`` with law 1 or 2 at every
    quadrature point: u [E][NQ], s = |grad u| [E][NQ], k [E][NQ], status [E]."""
    coords = _f64(coords)
    uc = _f64(ucoef)
    E = coords.shape[0]
    n = nq(elem, p)
    if n < 0:
        raise ValueError("unsupported element/degree")
    H, th, box = (0, None, None) if mlp is None else (mlp[0], _f64(mlp[1]), _f64(mlp[2]))
    if law == 2 and mlp is None:
        raise ValueError("law 2 needs mlp")
    u = np.zeros((E, n))
    s = np.zeros((E, n))
    k = np.zeros((E, n))
    st = np.zeros(E, dtype=np.int32)
    rc = _load().orc_point_law(elem, p, E, _ptr(coords), _ptr(uc), law, H, _ptr(th), _ptr(box),
                               _ptr(u), _ptr(s), _ptr(k), _ptr(st))
    if rc != 0:
        raise RuntimeError("oracle point_law failed")
    return u, s, k, st


def apply(elem: int, p: int, coords, coeffs, x, nthreads: int = 0):
    """Element operator applied to per-element coefficient vectors (FP64).

    y[e] = A_e x[e] with A_e the element matrix of ``integrate`` (constant
    coefficients): the element-level matrix-vector product that a Krylov
    solver of the assembled system performs with the element matrices left
    in device memory (Section 4), here by its definition, the formed matrix
    times the vector.  Returns (y [E][NS], status [E]).
    """
    A, _, st = integrate(elem, p, coords, coeffs, nthreads=nthreads)
    x = _f64(x)
    if x.shape != A.shape[:2]:
        raise ValueError("x must be [E][NS]")
    return np.einsum("eij,ej->ei", A, x), st


def jacobian_terms(elem: int, p: int, coords):
    """Per element and quadrature point: det J and J^{-1} (the NOJAC kernels'
    input, Section 4).  Returns terms [E][NQ][10] (det, then (J^{-1})[k][m] at
    1 + 3k + m) and status [E]."""
    coords = _f64(coords)
    E = coords.shape[0]
    n = nq(elem, p)
    if n < 0:
        raise ValueError("unsupported element/degree")
    terms = np.zeros((E, n, 10))
    st = np.zeros(E, dtype=np.int32)
    if _load().orc_jacobian_terms(elem, p, E, _ptr(coords), _ptr(terms), _ptr(st)) != 0:
        raise RuntimeError("oracle jacobian_terms failed")
    return terms, st


def integrate_elastic(p: int, coords, coeffs, nthreads: int = 0, elem: int = PRISM):
    """Linear elastostatics on prisms: A [E][3][3][NS][NS], b [E][3][NS], status.

    coeffs SoA [5][E]: Young modulus, Poisson ratio, body force fx, fy, fz;
    elem PRISM (collapsed rule) or PRISM_T1 (the paper's rule)."""
    coords = _f64(coords)
    coeffs = _f64(coeffs)
    E = coords.shape[0]
    n = ns(PRISM, p)
    A = np.zeros((E, 3, 3, n, n))
    b = np.zeros((E, 3, n))
    st = np.zeros(E, dtype=np.int32)
    rc = _load().orc_integrate_elastic_ex(elem, p, E, _ptr(coords), _ptr(coeffs), coeffs.shape[1], _ptr(A),
                                          _ptr(b), _ptr(st), nthreads)
    if rc != 0:
        raise RuntimeError("oracle integrate_elastic failed")
    return A, b, st
