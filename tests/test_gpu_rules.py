"""The paper's prism rules (Section 2, Table 1: N_Q = 6 ... 336 points,
a fully symmetric degree-2p triangle rule x (p+1)-point Gauss-Legendre in
zeta) on the GPU: tables built with FEM_RULE_TABLE1, every precision of
fem_integrate, against the oracle with the same rule (elem PRISM_T1), element
by element."""
import numpy as np
import pytest

from _util import TOL, SWEEP_E, ns, rel_frob, unpack_upper
from paper_1310_1191_gb300 import inputs

pytestmark = pytest.mark.gpu

T1 = 2  # oracle element code of the prism with the paper's rule
TOL_ALL = {0: TOL[0], 1: TOL[1], 2: 3e-5, 3: 3e-5}
# element counts spanning several CTAs / tensor-core M tiles and a ragged tail
E_OF = {1: 301, 2: 301, 3: 203, 4: 101, 5: 41, 6: 21, 7: 11}


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1310_1191_gb300 import _lib, build
    assert torch.cuda.is_available()
    build.build()
    _lib.load()
    return _lib


@pytest.fixture(scope="module")
def t1(lib):
    t = lib.fem_tables_build_ex(lib.FEM_PRISM6, lib.FEM_RULE_TABLE1, 1, 7)
    yield t
    t.close()


def _run(lib, t, p, X, C, prec, layout=0, stride=None):
    import torch
    E = X.shape[0]
    n = ns(1, p)
    dt = torch.float64 if prec == 0 else torch.float32
    m = lib.fem_matrix_size(lib.FEM_PRISM6, p, layout)
    A = torch.full((E, m), float("nan"), dtype=dt, device="cuda")
    b = torch.full((E, n), float("nan"), dtype=dt, device="cuda")
    st = torch.full((E,), -1, dtype=torch.int32, device="cuda")
    lib.fem_integrate(t, E, torch.from_numpy(X).cuda(), None, p, torch.from_numpy(C).cuda(), stride or C.shape[1],
                      None, prec, layout, A, b, st)
    torch.cuda.synchronize()
    return A.double().cpu().numpy(), b.double().cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("p", range(1, 8))
def test_table1_rule_parity(orc, lib, t1, p, prec):
    E = E_OF[p]
    X, C = inputs.prism_mesh(E), inputs.coefficients(E)
    n = ns(1, p)
    A, b, st = _run(lib, t1, p, X, C, prec)
    RA, Rb, Rst = orc.integrate(T1, p, X, C)
    err = rel_frob(A.reshape(E, n, n), RA)
    assert err.max() <= TOL_ALL[prec], (p, prec, err.max())
    assert rel_frob(b, Rb).max() <= TOL_ALL[prec]
    assert np.array_equal(st, Rst)


def test_table1_rule_differs_from_collapsed(orc, lib, t1):
    """The tables really carry the other rule: on the jittered mesh the
    result differs from the collapsed rule's by its quadrature error, far
    above the FP64 tolerance, and matches the oracle's collapsed result only
    through that rule."""
    p, E = 4, 64
    X, C = inputs.prism_mesh(E), inputs.coefficients(E)
    A, _, _ = _run(lib, t1, p, X, C, 0)
    R0, _, _ = orc.integrate(1, p, X, C)
    n = ns(1, p)
    d = rel_frob(A.reshape(E, n, n), R0)
    assert d.max() > 1e-8


def test_table1_rule_sympacked_and_flags(orc, lib, t1):
    p, E = 3, 40
    X, C = inputs.prism_mesh(E), inputs.coefficients(E, kind="symmetric")
    n = ns(1, p)
    A, b, st = _run(lib, t1, p, X, C, 0, layout=1)
    RA, Rb, _ = orc.integrate(T1, p, X, C)
    assert rel_frob(unpack_upper(A, n), np.triu(RA)).max() <= TOL[0]
    assert np.all(st == 0)
    Xb, Cb = X.copy(), inputs.coefficients(E)
    Xb[3] = Xb[3][[1, 0, 2, 4, 3, 5]]  # mirrored: det J < 0
    Cb[10, 7] = np.inf
    for prec in (0, 1, 2):
        _, _, st = _run(lib, t1, p, Xb, Cb, prec)
        _, _, Rst = orc.integrate(T1, p, Xb, Cb)
        assert np.array_equal(st, Rst), prec
        assert st[3] & lib.FEM_ST_DET and st[7] & lib.FEM_ST_NONFINITE


def test_table1_rule_other_entry_points_refuse(lib, t1):
    """The paper's rule has kernels for the constant-coefficient scalar form
    and for elasticity only: the law, split-geometry, apply and mixed-degree
    entry points give FEM_EUNSUPPORTED with these tables, before any launch."""
    import torch
    E, p = 4, 2
    X = torch.from_numpy(inputs.prism_mesh(E)).cuda()
    C = torch.from_numpy(inputs.coefficients(E)).cuda()
    A = torch.zeros(E * 400, dtype=torch.float64, device="cuda")
    U = torch.zeros((E, 18), dtype=torch.float32, device="cuda")
    calls = [
        lambda: lib.fem_integrate_law(t1, p, E, X, C, E, U, lib.FEM_LAW_EXACT, None, 0, 0, A),
        lambda: lib.fem_jacobian_terms(t1, p, E, X, A),
        lambda: lib.fem_apply(t1, p, E, X, C, E, 0, A, A[E * 18:]),
        lambda: lib.fem_plan_create(t1, np.full(E, p, dtype=np.int8), 0),
        lambda: lib.fem_integrate(t1, E, X, np.full(E, p, dtype=np.int8), 0, C, E, None, 0, 0, A),
    ]
    for k, call in enumerate(calls):
        with pytest.raises(lib.FemError) as ei:
            call()
        assert ei.value.code == lib.FEM_EUNSUPPORTED, k
        assert "TABLE1" in lib.last_error(), k


@pytest.mark.slow
@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("p", [1, 4, 7])
def test_table1_rule_full_size_sampled(orc, lib, t1, p, prec):
    """The degree sweep's element counts in one launch, as the benchmark runs
    them; a seeded sample of elements (first, last and 14 others) vs the oracle."""
    import torch
    E = SWEEP_E[p]
    X, C = inputs.prism_mesh(E), inputs.coefficients(E)
    n = ns(1, p)
    dt = torch.float64 if prec == 0 else torch.float32
    A = torch.empty((E, n * n), dtype=dt, device="cuda")
    b = torch.empty((E, n), dtype=dt, device="cuda")
    st = torch.empty((E,), dtype=torch.int32, device="cuda")
    lib.fem_integrate(t1, E, torch.from_numpy(X).cuda(), None, p, torch.from_numpy(C).cuda(), E, None, prec, 0,
                      A, b, st)
    torch.cuda.synchronize()
    rng = np.random.default_rng(p)
    idx = np.unique(np.concatenate([[0, E - 1], rng.choice(E, 14, replace=False)]))
    RA, Rb, _ = orc.integrate(T1, p, X[idx], C[:, idx])
    Ah = A[torch.from_numpy(idx).cuda()].double().cpu().numpy().reshape(len(idx), n, n)
    assert rel_frob(Ah, RA).max() <= TOL_ALL[prec]
    assert int((st != 0).sum().item()) == 0


E_EL = {1: 64, 2: 40, 3: 24, 4: 12, 5: 6, 6: 4, 7: 3}


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("p", range(1, 8))
def test_table1_rule_elasticity_parity(orc, lib, t1, p, prec):
    """Linear elastostatics (the paper's model problem, Section 5.1) with the
    paper's own rule: every element and block against the oracle's
    elasticity with the same rule."""
    import torch
    E = E_EL[p]
    X, C = inputs.prism_mesh(E), inputs.elastic_coefficients(E)
    n = ns(1, p)
    dt = torch.float64 if prec == 0 else torch.float32
    A = torch.full((E, 9 * n * n), float("nan"), dtype=dt, device="cuda")
    b = torch.full((E, 3 * n), float("nan"), dtype=dt, device="cuda")
    st = torch.full((E,), -1, dtype=torch.int32, device="cuda")
    lib.fem_integrate_elastic(t1, p, E, torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(), E, prec, A, b, st)
    torch.cuda.synchronize()
    RA, Rb, Rst = orc.integrate_elastic(p, X, C, elem=T1)
    err = rel_frob(A.double().cpu().numpy().reshape(E, 9 * n * n), RA.reshape(E, -1))
    assert err.max() <= TOL_ALL[prec], (p, prec, err.max())
    assert rel_frob(b.double().cpu().numpy(), Rb.reshape(E, -1)).max() <= TOL_ALL[prec]
    assert np.array_equal(st.cpu().numpy(), Rst)
