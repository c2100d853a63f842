"""Matrix-free element-operator apply (fem_apply) through the C ABI against the
FP64 oracle's y_e = A_e x_e: every degree and both precisions on several
element groups with a ragged tail, many groups per CTA, P1 tets, status
flags, argument errors, and the full-size apply workload sampled."""
import numpy as np
import pytest

from _util import PRISM, TET, TOL, ns
from paper_1310_1191_gb300 import inputs

pytestmark = pytest.mark.gpu

# elements per group of the prism kernel (about one quadrature point per thread)
EB = {p: max(1, 256 // (p + 1) ** 2) for p in range(1, 8)}
# about 1 GB of algorithmic FP64 traffic per degree: x, y, coordinates, coefficients
APPLY_E = {p: round(1e9 / (8 * (2 * ns(PRISM, p) + 29))) for p in range(1, 8)}


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


def _x(E, n, seed):
    return np.random.default_rng(seed).standard_normal((E, n))


def _run(lib, t, p, X, C, x, prec, tensors=False):
    import torch
    E = X.shape[0]
    dt = torch.float64 if prec == 0 else torch.float32
    xd = torch.from_numpy(x).to("cuda", dt)
    y = torch.full_like(xd, float("nan"))
    st = torch.full((E,), -1, dtype=torch.int32, device="cuda")
    lib.fem_apply(t, p, E, torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(), E, prec, xd, y, st)
    torch.cuda.synchronize()
    if tensors:
        return y, st
    return y.double().cpu().numpy(), st.cpu().numpy()


def _rel(y, r):
    return np.linalg.norm(y - r, axis=1) / np.linalg.norm(r, axis=1)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", range(1, 8))
def test_apply_parity_small(orc, lib, tables, p, prec):
    """Three element groups and a ragged tail, every element vs the oracle."""
    E = 3 * EB[p] + 1
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    x = _x(E, ns(PRISM, p), p)
    if prec == 1:
        x = x.astype(np.float32).astype(np.float64)  # the oracle applies A to the same x
    y, st = _run(lib, tables, p, X, C, x, prec)
    R, Rst = orc.apply(PRISM, p, X, C, x)
    err = _rel(y, R)
    print("apply p=%d prec=%d: max %.3e" % (p, prec, err.max()))
    assert np.array_equal(st, Rst) and np.all(st == 0)
    assert err.max() <= TOL[prec]


@pytest.mark.parametrize("p,E", [(1, 70000), (3, 20000), (5, 2500)])
def test_apply_many_groups_per_cta(orc, lib, tables, p, E):
    """More groups than resident CTAs, so every CTA pipelines several groups
    through its two buffers; every element vs the oracle."""
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    x = _x(E, ns(PRISM, p), 10 + p)
    y, st = _run(lib, tables, p, X, C, x, 0)
    R, Rst = orc.apply(PRISM, p, X, C, x)
    assert np.array_equal(st, Rst)
    assert _rel(y, R).max() <= TOL[0]


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_tets(orc, lib, prec):
    from _util import workload
    t = lib.fem_tables_build(lib.FEM_TET4, 1, 1)
    try:
        X, _ = workload(TET, 1, 3000)
        E = X.shape[0]
        C = inputs.coefficients(E)
        x = _x(E, 4, 7)
        if prec == 1:
            x = x.astype(np.float32).astype(np.float64)
        y, st = _run(lib, t, 1, X, C, x, prec)
        R, Rst = orc.apply(TET, 1, X, C, x)
        assert np.array_equal(st, Rst)
        assert _rel(y, R).max() <= TOL[prec]
    finally:
        t.close()


def test_apply_flags(orc, lib, tables):
    p, E = 3, 2 * EB[3] + 3
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    X[1] = X[1][[1, 0, 2, 4, 3, 5]]  # mirrored: det J < 0
    C[2, 5] = np.nan
    X[EB[3] + 2, 4, 1] = np.inf       # second group
    x = _x(E, ns(PRISM, p), 3)
    for prec in (0, 1):
        y, st = _run(lib, tables, p, X, C, x, prec)
        R, Rst = orc.apply(PRISM, p, X, C, x)
        assert list(st) == list(Rst)
        assert st[1] & 1 and st[5] & 2 and st[EB[3] + 2] & 2 and st[0] == 0
        ok = Rst == 0
        assert _rel(y[ok], R[ok]).max() <= TOL[prec]


def test_apply_errors(lib, tables):
    import torch
    X = torch.from_numpy(inputs.prism_mesh(4)).cuda()
    C = torch.from_numpy(inputs.coefficients(4)).cuda()
    x = torch.zeros(4 * 40 + 1, dtype=torch.float64, device="cuda")
    y = torch.zeros(4 * 40, dtype=torch.float64, device="cuda")
    lib.fem_apply(tables, 3, 0, None, None, 0, 0, None, None)  # n = 0: no-op
    with pytest.raises(lib.FemError):
        lib.fem_apply(tables, 3, 4, X, C, 4, lib.FEM_BF16X3, x, y)
    with pytest.raises(lib.FemError):
        lib.fem_apply(tables, 3, 4, X, C, 3, 0, x, y)  # coeff_stride < n
    with pytest.raises(lib.FemError):
        lib.fem_apply(tables, 3, 4, X, C, 4, 0, x.data_ptr() + 4, y)  # x not 8-byte aligned
    with pytest.raises(lib.FemError):
        lib.fem_apply(tables, 3, 4, X, C, 4, 0, x, x[8:])  # x and y overlap


@pytest.mark.slow
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", range(1, 8))
def test_apply_full_size_sampled(orc, lib, tables, p, prec):
    """The bench's apply workload (about 1 GB of FP64 traffic per degree):
    no flags, no NaN, sampled elements vs the oracle."""
    import torch
    E = APPLY_E[p]
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    x = inputs.dof_vectors(E, ns(PRISM, p))
    y, st = _run(lib, tables, p, X, C, x, prec, tensors=True)
    assert int((st != 0).sum().item()) == 0
    assert not bool(torch.isnan(y).any().item())
    rng = np.random.default_rng(900 + p)
    idx = np.array(sorted(set([0, E - 1]) | set(rng.choice(E, 16, replace=False).tolist())))
    xs = x[idx].astype(np.float32).astype(np.float64) if prec == 1 else x[idx]
    R, _ = orc.apply(PRISM, p, X[idx], C[:, idx], xs)
    ys = y[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    assert _rel(ys, R).max() <= TOL[prec]
