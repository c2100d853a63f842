"""The single integration entry point of include/fem.h, fem_integrate, through
the C ABI: per-element degrees (the host classifies the elements by degree,
Section 4.2) and a coefficient law (the coefficients depend on the old
solution, Section 2) on the same call, and the synchronous status query
fem_sync_status that turns per-element flags into FEM_EELEMENT."""
import numpy as np
import pytest

from _util import PRISM, TOL, ns, rel_frob
from paper_1310_1191_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_TC = 3e-5  # tensor-core forms (FP32 accumulation over K = 4 NQ)


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1310_1191_gb300 import _lib, build
    assert torch.cuda.is_available()
    build.build()
    _lib.load()
    return _lib


@pytest.fixture(scope="module")
def tables(lib):
    t = lib.fem_tables_build(lib.FEM_PRISM6, 1, 7)
    yield t
    t.close()


def _oracle_mixed(orc, X, C, P):
    ref = {}
    for p in range(1, 8):
        sel = np.flatnonzero(P == p)
        if sel.size:
            A, b, st = orc.integrate(PRISM, p, X[sel], C[:, sel])
            for k, e in enumerate(sel):
                ref[int(e)] = (A[k], b[k], st[k])
    return ref


def _mixed_call(lib, tables, X, C, P, prec, layout=0):
    import torch
    offA, offb, totA, totb = lib.fem_output_offsets(lib.FEM_PRISM6, P, layout)
    dt = torch.float64 if prec == 0 else torch.float32
    E = X.shape[0]
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    A = torch.full((totA,), float("nan"), dtype=dt, device="cuda")
    b = torch.full((totb,), float("nan"), dtype=dt, device="cuda")
    st = torch.full((E,), -1, dtype=torch.int32, device="cuda")
    lib.fem_integrate(tables, E, Xd, P, 0, Cd, C.shape[1], None, prec, layout, A, b, st)
    torch.cuda.synchronize()
    return A.double().cpu().numpy(), b.double().cpu().numpy(), st.cpu().numpy(), offA, offb


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_per_element_degree_matches_oracle(orc, lib, tables, prec):
    """700 prisms with degrees 1..7 through fem_integrate(p_per_elem): every
    element vs the oracle (FP64 1e-12, FP32 1e-5, BF16x3 3e-5), twice (the
    second call replays the plan the tables keep)."""
    E = 700
    X, C, P = inputs.prism_mesh(E), inputs.coefficients(E), inputs.mixed_degrees(E)
    assert set(np.unique(P)) == set(range(1, 8))
    ref = _oracle_mixed(orc, X, C, P)
    tol = {0: TOL[0], 1: TOL[1], 2: TOL_TC}[prec]
    for call in range(2):
        A, b, st, offA, offb = _mixed_call(lib, tables, X, C, P, prec)
        errs = []
        for e in range(E):
            n = ns(PRISM, int(P[e]))
            RA, Rb, Rst = ref[e]
            errs.append(rel_frob(A[offA[e]:offA[e] + n * n].reshape(1, n, n), RA[None])[0])
            assert rel_frob(b[offb[e]:offb[e] + n][None], Rb[None])[0] <= tol, (call, e)
            assert st[e] == Rst
        assert max(errs) <= tol, (call, max(errs))


def test_per_element_degree_changes_rebuild_the_plan(orc, lib, tables):
    """A call with other degrees (and then the first ones again) after a plan
    was kept: each result matches the oracle (the kept plan is replaced)."""
    E = 300
    X, C = inputs.prism_mesh(E), inputs.coefficients(E)
    P1 = inputs.mixed_degrees(E)
    P2 = np.ascontiguousarray(P1[::-1])
    for P in (P1, P2, P1):
        ref = _oracle_mixed(orc, X, C, P)
        A, b, st, offA, offb = _mixed_call(lib, tables, X, C, P, 1)
        for e in range(0, E, 7):
            n = ns(PRISM, int(P[e]))
            assert rel_frob(A[offA[e]:offA[e] + n * n].reshape(1, n, n), ref[e][0][None])[0] <= TOL[1]


def test_uniform_degree_is_the_direct_launch(lib, tables):
    """p_per_elem = NULL with a constant law is fem_integrate_uniform: the
    same bits."""
    import torch
    E, p = 64, 4
    X, C = inputs.prism_mesh(E), inputs.coefficients(E)
    n = ns(PRISM, p)
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    A1 = torch.empty((E, n * n), dtype=torch.float64, device="cuda")
    A2 = torch.empty_like(A1)
    lib.fem_integrate(tables, E, Xd, None, p, Cd, E, None, 0, 0, A1)
    lib.fem_integrate_uniform(tables, p, E, Xd, Cd, E, 0, 0, A2)
    torch.cuda.synchronize()
    assert torch.equal(A1, A2)


@pytest.mark.parametrize("prec", [0, 1])
def test_law_through_fem_integrate_matches_oracle(orc, lib, tables, prec):
    """The exact nonlinear law through fem_integrate's law argument vs the
    oracle (law = 1)."""
    import torch
    E, p = 30, 3
    NS = ns(PRISM, p)
    X, C = inputs.prism_mesh(E), inputs.coefficients(E)
    U = inputs.field_coefficients(E, NS).astype(np.float32)
    dt = torch.float64 if prec == 0 else torch.float32
    A = torch.empty((E, NS * NS), dtype=dt, device="cuda")
    b = torch.empty((E, NS), dtype=dt, device="cuda")
    st = torch.empty(E, dtype=torch.int32, device="cuda")
    Ud = torch.from_numpy(U).cuda()
    law = lib.coef_law(lib.FEM_LAW_EXACT, Ud)
    lib.fem_integrate(tables, E, torch.from_numpy(X).cuda(), None, p, torch.from_numpy(C).cuda(), E, law,
                      prec, 0, A, b, st)
    torch.cuda.synchronize()
    RA, Rb, Rst = orc.integrate(PRISM, p, X, C, law=1, ucoef=U.astype(np.float64))
    assert rel_frob(A.cpu().numpy().reshape(E, NS, NS), RA).max() <= TOL[prec]
    assert rel_frob(b.cpu().numpy(), Rb).max() <= TOL[prec]
    assert np.array_equal(st.cpu().numpy(), Rst)
    # a law with per-element degrees is refused before any launch
    P = np.full(E, p, dtype=np.int8)
    with pytest.raises(lib.FemError) as ei:
        lib.fem_integrate(tables, E, torch.from_numpy(X).cuda(), P, 0, torch.from_numpy(C).cuda(), E, law,
                          prec, 0, A, b, st)
    assert ei.value.code == lib.FEM_EUNSUPPORTED


def test_sync_status_reports_flagged_elements(lib, tables):
    """fem_sync_status: FEM_OK on a clean mesh; FEM_EELEMENT with the number
    of flagged elements for det J < 0 and a NaN coefficient; FEM_EELEMENT with
    FEM_ST_NONSYM for packed output of a form with convection; the
    informational FEM_ST_FALLBACK alone stays FEM_OK."""
    import torch
    E, p = 40, 2
    n = ns(PRISM, p)
    X, C = inputs.prism_mesh(E), inputs.coefficients(E)
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    A = torch.empty((E, n * n), dtype=torch.float64, device="cuda")
    st = torch.full((E,), -1, dtype=torch.int32, device="cuda")
    lib.fem_integrate(tables, E, Xd, None, p, Cd, E, None, 0, 0, A, None, st)
    assert lib.fem_sync_status(tables, st, E) == (lib.FEM_OK, 0, 0)
    Xb, Cb = X.copy(), C.copy()
    Xb[5] = Xb[5][[1, 0, 2, 4, 3, 5]]  # mirrored: det J < 0
    Cb[9, 17] = np.nan
    lib.fem_integrate(tables, E, torch.from_numpy(Xb).cuda(), None, p, torch.from_numpy(Cb).cuda(), E, None,
                      0, 0, A, None, st)
    code, bits, nflag = lib.fem_sync_status(tables, st, E)
    assert code == lib.FEM_EELEMENT and nflag == 2
    assert bits == lib.FEM_ST_DET | lib.FEM_ST_NONFINITE
    Ap = torch.empty((E, n * (n + 1) // 2), dtype=torch.float64, device="cuda")
    lib.fem_integrate(tables, E, Xd, None, p, Cd, E, None, 0, lib.FEM_OUT_SYMPACKED, Ap, None, st)
    code, bits, nflag = lib.fem_sync_status(tables, st, E)
    assert code == lib.FEM_EELEMENT and nflag == E and bits == lib.FEM_ST_NONSYM
    info = torch.full((E,), lib.FEM_ST_FALLBACK, dtype=torch.int32, device="cuda")
    assert lib.fem_sync_status(tables, info, E) == (lib.FEM_OK, lib.FEM_ST_FALLBACK, 0)
    assert lib.fem_sync_status(tables, None, 0) == (lib.FEM_OK, 0, 0)
