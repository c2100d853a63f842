"""The allocation-free mixed-degree entry point (fem_integrate_mixed_noalloc).

It exists for callers that cannot allocate device memory (fixed pools or
budgets, paths where an allocation's implicit synchronisation is not
allowed): its scratch lives in a fixed static device array of the library.
This file is collected last so that a failure here cannot hide another test's
result.  It checks, through the C ABI, that two calls in a row give the same
element matrices and load vectors as the plan entry point (fem_plan_execute)
within the tolerance of the parity tests (full and upper-packed output), and
that calls beyond the fixed scratch size, on tetrahedron tables or in a
tensor-core precision are refused."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1310_1191_gb300 import _lib, build
    assert torch.cuda.is_available()
    build.build()
    _lib.load()
    return _lib


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_plan_two_calls(lib, prec, layout):
    """Full output of the random form, and upper-packed output of the
    symmetric form (no convection)."""
    import torch
    from paper_1310_1191_gb300 import inputs
    E = 3000
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E, kind="random" if layout == 0 else "symmetric")
    P = inputs.mixed_degrees(E)
    t = lib.fem_tables_build(lib.FEM_PRISM6, 1, 7)
    offA, offb, totA, totb = lib.fem_output_offsets(lib.FEM_PRISM6, P, layout)
    dt = torch.float64 if prec == 0 else torch.float32
    Xd = torch.from_numpy(X).cuda()
    Cd = torch.from_numpy(C).cuda()
    # reference: the plan entry point
    A0 = torch.zeros(totA, dtype=dt, device="cuda")
    b0 = torch.zeros(totb, dtype=dt, device="cuda")
    plan = lib.fem_plan_create(t, P, prec, layout, 0, None)
    lib.fem_plan_execute(plan, Xd, Cd, E, A0, b0)
    torch.cuda.synchronize()
    plan.close()
    # the allocation-free entry point, twice in a row into fresh outputs
    for call in range(2):
        A1 = torch.full((totA,), float("nan"), dtype=dt, device="cuda")
        b1 = torch.full((totb,), float("nan"), dtype=dt, device="cuda")
        st = torch.full((E,), -1, dtype=torch.int32, device="cuda")
        lib.fem_integrate_mixed_noalloc(t, P, Xd, Cd, E, prec, layout, A1, b1, st)
        torch.cuda.synchronize()
        assert int((st != 0).sum().item()) == 0, call
        Ah, Rh = A1.double().cpu().numpy(), A0.double().cpu().numpy()
        bh, Rb = b1.double().cpu().numpy(), b0.double().cpu().numpy()
        assert not np.isnan(Ah).any() and not np.isnan(bh).any(), call
        for e in range(0, E, 37):
            p = int(P[e])
            n = (p + 1) ** 2 * (p + 2) // 2
            m = n * n if layout == 0 else n * (n + 1) // 2
            sa = slice(int(offA[e]), int(offA[e]) + m)
            sb = slice(int(offb[e]), int(offb[e]) + n)
            assert _rel(Ah[sa], Rh[sa]) <= TOL[prec], (call, e)
            assert _rel(bh[sb], Rb[sb]) <= TOL[prec], (call, e)
        assert _rel(Ah, Rh) <= TOL[prec] and _rel(bh, Rb) <= TOL[prec], call
    t.close()


def test_noalloc_rejects_too_many_elements(lib):
    import torch
    t = lib.fem_tables_build(lib.FEM_PRISM6, 1, 2)
    P = np.ones(16385, dtype=np.int8)
    X = torch.zeros((16385, 6, 3), dtype=torch.float64, device="cuda")
    C = torch.zeros((11, 16385), dtype=torch.float64, device="cuda")
    A = torch.zeros(16385 * 36, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.FemError) as ei:
        lib.fem_integrate_mixed_noalloc(t, P, X, C, 16385, lib.FEM_F32, lib.FEM_OUT_FULL, A)
    assert ei.value.code == lib.FEM_EINVAL and "16384" in lib.last_error()
    t.close()


def test_noalloc_rejects_other_element_and_precision(lib):
    """Tetrahedron tables and the tensor-core precisions are refused on the
    host, with the code and message of include/fem.h."""
    import torch
    P = np.ones(8, dtype=np.int8)
    X = torch.zeros((8, 6, 3), dtype=torch.float64, device="cuda")
    C = torch.zeros((11, 8), dtype=torch.float64, device="cuda")
    A = torch.zeros(8 * 36, dtype=torch.float32, device="cuda")
    tt = lib.fem_tables_build(lib.FEM_TET4, 1, 1)
    with pytest.raises(lib.FemError) as ei:
        lib.fem_integrate_mixed_noalloc(tt, P, X, C, 8, lib.FEM_F32, lib.FEM_OUT_FULL, A)
    assert ei.value.code == lib.FEM_EINVAL and "prism" in lib.last_error()
    tt.close()
    t = lib.fem_tables_build(lib.FEM_PRISM6, 1, 2)
    for prec in (lib.FEM_BF16X3, lib.FEM_F16X3):
        with pytest.raises(lib.FemError) as ei:
            lib.fem_integrate_mixed_noalloc(t, P, X, C, 8, prec, lib.FEM_OUT_FULL, A)
        assert ei.value.code == lib.FEM_EUNSUPPORTED and "FP64 / FP32" in lib.last_error()
    t.close()
