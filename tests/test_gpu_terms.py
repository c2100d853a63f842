"""Split geometry (NOJAC): the device Jacobian-terms pass against the oracle's
terms, and integration from stored terms against the oracle's element
matrices, through the C ABI."""
import numpy as np
import pytest

from _util import PRISM, SWEEP_E, TET, TOL, ns, rel_frob, unpack_upper, workload
from paper_1310_1191_gb300 import inputs

pytestmark = pytest.mark.gpu

# several CTAs of the terms pass (512 points per CTA) and of the FMA kernels, plus a ragged tail
SMALL_E = {1: 42 * 3 + 5, 2: 14 * 3 + 5, 3: 2 * 5 + 1, 4: 5, 5: 3, 6: 3, 7: 3}


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1310_1191_gb300 import _lib, build
    assert torch.cuda.is_available()
    build.build()
    _lib.load()
    return _lib


@pytest.fixture(scope="module")
def prism_tables(lib):
    t = lib.fem_tables_build(lib.FEM_PRISM6, 1, 7)
    yield t
    t.close()


@pytest.fixture(scope="module")
def tet_tables(lib):
    t = lib.fem_tables_build(lib.FEM_TET4, 1, 1)
    yield t
    t.close()


def _nq(elem, p):
    return 4 if elem == TET else (p + 1) ** 3


def _terms(lib, tables, elem, p, X):
    import torch
    E = X.shape[0]
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    T = torch.full((max(E, 1), _nq(elem, p), 10), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.full((max(E, 1),), -1, dtype=torch.int32, device="cuda")
    lib.fem_jacobian_terms(tables, p, E, Xd, T, st)
    torch.cuda.synchronize()
    return T, st


def _integrate_terms(lib, tables, elem, p, Td, C, prec, layout=0):
    import torch
    E = C.shape[1]
    dt = torch.float64 if prec == 0 else torch.float32
    Cd = torch.from_numpy(np.ascontiguousarray(C)).cuda()
    m = lib.fem_matrix_size(elem, p, layout)
    A = torch.full((E, m), float("nan"), dtype=dt, device="cuda")
    b = torch.full((E, ns(elem, p)), float("nan"), dtype=dt, device="cuda")
    st = torch.full((E,), -1, dtype=torch.int32, device="cuda")
    lib.fem_integrate_terms(tables, p, E, Td, Cd, E, prec, layout, A, b, st)
    torch.cuda.synchronize()
    return A.double().cpu().numpy(), b.double().cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("p", range(1, 8))
def test_terms_match_oracle(orc, lib, prism_tables, p):
    E = SMALL_E[p]
    X, _ = workload(PRISM, p, E)
    T, st = _terms(lib, prism_tables, PRISM, p, X)
    R, Rst = orc.jacobian_terms(PRISM, p, X)
    assert np.array_equal(st.cpu().numpy(), Rst)
    assert rel_frob(T.cpu().numpy(), R).max() <= 1e-13


def test_terms_tets(orc, lib, tet_tables):
    X = inputs.tet_mesh(4)
    T, st = _terms(lib, tet_tables, TET, 1, X)
    R, Rst = orc.jacobian_terms(TET, 1, X)
    assert np.array_equal(st.cpu().numpy(), Rst) and np.all(Rst == 0)
    assert rel_frob(T.cpu().numpy(), R).max() <= 1e-13


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", range(1, 8))
def test_integrate_terms_match_oracle(orc, lib, prism_tables, p, prec):
    """Device terms -> NOJAC integration vs the oracle's fused computation."""
    E = SMALL_E[p]
    X, C = workload(PRISM, p, E)
    T, _ = _terms(lib, prism_tables, PRISM, p, X)
    A, b, st = _integrate_terms(lib, prism_tables, PRISM, p, T, C, prec)
    RA, Rb, Rst = orc.integrate(PRISM, p, X, C)
    n = ns(PRISM, p)
    assert np.array_equal(st, Rst) and np.all(st == 0)
    assert rel_frob(A.reshape(E, n, n), RA).max() <= TOL[prec]
    assert rel_frob(b, Rb).max() <= TOL[prec]


@pytest.mark.parametrize("p", [2, 5])
def test_integrate_oracle_terms(orc, lib, prism_tables, p):
    """The oracle's own terms as input: checks the terms layout contract
    independently of the device terms pass."""
    import torch
    E = SMALL_E[p]
    X, C = workload(PRISM, p, E)
    R, _ = orc.jacobian_terms(PRISM, p, X)
    A, b, st = _integrate_terms(lib, prism_tables, PRISM, p, torch.from_numpy(R).cuda(), C, 0)
    RA, Rb, _ = orc.integrate(PRISM, p, X, C)
    n = ns(PRISM, p)
    assert rel_frob(A.reshape(E, n, n), RA).max() <= TOL[0]
    assert rel_frob(b, Rb).max() <= TOL[0]


@pytest.mark.parametrize("prec", [0, 1])
def test_integrate_terms_tets_and_packed(orc, lib, tet_tables, prism_tables, prec):
    X = inputs.tet_mesh(3)
    E = X.shape[0]
    C = inputs.coefficients(E)
    T, _ = _terms(lib, tet_tables, TET, 1, X)
    A, b, st = _integrate_terms(lib, tet_tables, TET, 1, T, C, prec)
    RA, Rb, _ = orc.integrate(TET, 1, X, C)
    assert rel_frob(A.reshape(E, 4, 4), RA).max() <= TOL[prec]
    p = 3
    Xp, Cp = workload(PRISM, p, SMALL_E[p], kind="symmetric")
    Tp, _ = _terms(lib, prism_tables, PRISM, p, Xp)
    Ap, _, stp = _integrate_terms(lib, prism_tables, PRISM, p, Tp, Cp, prec, layout=1)
    RA, _, _ = orc.integrate(PRISM, p, Xp, Cp)
    assert rel_frob(unpack_upper(Ap, ns(PRISM, p)), np.triu(RA)).max() <= TOL[prec]
    assert np.all(stp == 0)


def test_status_flags_and_errors(orc, lib, prism_tables):
    import torch
    p = 2
    X, C = workload(PRISM, p, 6)
    X[1] = X[1][[1, 0, 2, 4, 3, 5]]  # mirrored: det J < 0
    X[4, 2, 0] = np.nan               # non-finite coordinate
    C[9, 3] = np.nan                  # non-finite coefficient
    T, st = _terms(lib, prism_tables, PRISM, p, X)
    _, Rst_t = orc.jacobian_terms(PRISM, p, X)
    assert np.array_equal(st.cpu().numpy(), Rst_t)
    _, _, sti = _integrate_terms(lib, prism_tables, PRISM, p, T, C, 0)
    _, _, Rst = orc.integrate(PRISM, p, X, C)
    assert list(sti) == list(Rst)
    assert sti[1] & 1 and sti[3] & 2 and sti[4] & 2 and sti[0] == 0
    # empty input, bad alignment, tensor-core precision
    Xd = torch.from_numpy(X).cuda()
    Tb = torch.zeros(6 * 27 * 10 + 2, dtype=torch.float64, device="cuda")
    lib.fem_jacobian_terms(prism_tables, p, 0, Xd, Tb)
    with pytest.raises(lib.FemError) as ei:
        lib.fem_jacobian_terms(prism_tables, p, 6, Xd, Tb.data_ptr() + 8)
    assert ei.value.code == lib.FEM_EINVAL
    Cd = torch.from_numpy(C).cuda()
    A = torch.zeros(6 * 324, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.FemError) as ei:
        lib.fem_integrate_terms(prism_tables, p, 6, T, Cd, 6, lib.FEM_BF16X3, 0, A)
    assert ei.value.code == lib.FEM_EUNSUPPORTED


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", [1, 3])
def test_elastic_from_terms(orc, lib, prism_tables, p, prec):
    import torch
    E = 7
    X = inputs.prism_mesh(E)
    C = inputs.elastic_coefficients(E)
    T, _ = _terms(lib, prism_tables, PRISM, p, X)
    n = ns(PRISM, p)
    dt = torch.float64 if prec == 0 else torch.float32
    A = torch.full((E, 3, 3, n, n), float("nan"), dtype=dt, device="cuda")
    b = torch.full((E, 3, n), float("nan"), dtype=dt, device="cuda")
    st = torch.full((E,), -1, dtype=torch.int32, device="cuda")
    lib.fem_integrate_elastic_terms(prism_tables, p, E, T, torch.from_numpy(C).cuda(), E, prec, A, b, st)
    torch.cuda.synchronize()
    RA, Rb, Rst = orc.integrate_elastic(p, X, C)
    assert np.array_equal(st.cpu().numpy(), Rst)
    assert rel_frob(A.double().cpu().numpy(), RA).max() <= TOL[prec]
    assert rel_frob(b.double().cpu().numpy(), Rb).max() <= TOL[prec]


@pytest.mark.slow
@pytest.mark.parametrize("p", [1, 4, 7])
def test_full_size_sampled(orc, lib, prism_tables, p):
    """Sweep element counts (about 2 GB of FP64 output): terms pass + NOJAC
    integration in one stream; a seeded sample vs the oracle."""
    import torch
    E = SWEEP_E[p]
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    n = ns(PRISM, p)
    Xd = torch.from_numpy(X).cuda()
    Cd = torch.from_numpy(C).cuda()
    T = torch.empty((E, _nq(PRISM, p), 10), dtype=torch.float64, device="cuda")
    A = torch.full((E, n * n), float("nan"), dtype=torch.float64, device="cuda")
    b = torch.full((E, n), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.full((E,), -1, dtype=torch.int32, device="cuda")
    lib.fem_jacobian_terms(prism_tables, p, E, Xd, T, st)
    lib.fem_integrate_terms(prism_tables, p, E, T, Cd, E, 0, 0, A, b, st)
    torch.cuda.synchronize()
    assert int((st != 0).sum().item()) == 0
    assert not bool(torch.isnan(A).any().item())
    rng = np.random.default_rng(300 + p)
    idx = np.array(sorted(set([0, E - 1]) | set(rng.choice(E, 12, replace=False).tolist())))
    Ai = A[torch.from_numpy(idx).cuda()].cpu().numpy().reshape(-1, n, n)
    RA, Rb, _ = orc.integrate(PRISM, p, X[idx], C[:, idx])
    assert rel_frob(Ai, RA).max() <= TOL[0]
    assert rel_frob(b[torch.from_numpy(idx).cuda()].cpu().numpy(), Rb).max() <= TOL[0]
