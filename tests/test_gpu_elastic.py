"""Linear elastostatics (the paper's model problem) through the C ABI vs the
FP64 oracle: all degrees, both precisions, a ragged tail of virtual elements
(9 blocks per element), status flags, and the full-size sweep sampled."""
import numpy as np
import pytest

from _util import PRISM, TOL, ns, rel_frob
from paper_1310_1191_gb300 import inputs

pytestmark = pytest.mark.gpu

# elements per degree: a few CTAs of virtual elements and a ragged tail
SMALL_E = {1: 23, 2: 11, 3: 5, 4: 3, 5: 2, 6: 2, 7: 1}
# about 2 GB of FP64 output per degree: round(2e9 / (8 (9 NS^2 + 3 NS)))
ELASTIC_SWEEP_E = {p: round(2e9 / (8 * (9 * ns(PRISM, p) ** 2 + 3 * ns(PRISM, p)))) for p in range(1, 8)}


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


def _run(lib, tables, p, X, C, prec, tensors=False):
    import torch
    E = X.shape[0]
    n = ns(PRISM, p)
    dt = torch.float64 if prec == 0 else torch.float32
    A = torch.full((E, 3, 3, n, n), float("nan"), dtype=dt, device="cuda")
    b = torch.full((E, 3, n), float("nan"), dtype=dt, device="cuda")
    st = torch.full((E,), -1, dtype=torch.int32, device="cuda")
    lib.fem_integrate_elastic(tables, p, E, torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(), E,
                              prec, A, b, st)
    torch.cuda.synchronize()
    if tensors:
        return A, b, st
    return A.cpu().numpy(), b.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", range(1, 8))
def test_elastic_parity_small(orc, lib, tables, p, prec):
    E = SMALL_E[p]
    X = inputs.prism_mesh(E)
    C = inputs.elastic_coefficients(E)
    A, b, st = _run(lib, tables, p, X, C, prec)
    RA, Rb, Rst = orc.integrate_elastic(p, X, C)
    n = ns(PRISM, p)
    eA = rel_frob(A.reshape(E, 9 * n * n), RA.reshape(E, 9 * n * n))
    eb = rel_frob(b.reshape(E, 3 * n), Rb.reshape(E, 3 * n))
    assert np.array_equal(st, Rst) and np.all(st == 0)
    assert eA.max() <= TOL[prec] and eb.max() <= TOL[prec], (eA.max(), eb.max())


def test_elastic_flags(orc, lib, tables):
    p = 2
    X = inputs.prism_mesh(4)
    C = inputs.elastic_coefficients(4)
    X[1] = X[1][[1, 0, 2, 4, 3, 5]]  # mirrored: det J < 0
    C[1, 2] = np.nan
    A, b, st = _run(lib, tables, p, X, C, 0)
    _, _, Rst = orc.integrate_elastic(p, X, C)
    assert list(st) == list(Rst) and st[1] & 1 and st[2] & 2 and st[0] == 0


@pytest.mark.slow
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", range(1, 8))
def test_elastic_full_size_sampled(orc, lib, tables, p, prec):
    import torch
    E = ELASTIC_SWEEP_E[p]
    X = inputs.prism_mesh(E)
    C = inputs.elastic_coefficients(E)
    A, b, st = _run(lib, tables, p, X, C, prec, tensors=True)
    assert int((st != 0).sum().item()) == 0
    assert not bool(torch.isnan(A).any().item())
    rng = np.random.default_rng(700 + p)
    idx = np.array(sorted(set([0, E - 1]) | set(rng.choice(E, 4 if p >= 6 else 12, replace=False).tolist())))
    n = ns(PRISM, p)
    ti = torch.from_numpy(idx).cuda()
    Ai = A[ti].double().cpu().numpy().reshape(len(idx), -1)
    RA, Rb, _ = orc.integrate_elastic(p, X[idx], C[:, idx])
    assert rel_frob(Ai, RA.reshape(len(idx), -1)).max() <= TOL[prec]
    assert rel_frob(b[ti].double().cpu().numpy().reshape(len(idx), -1), Rb.reshape(len(idx), -1)).max() <= TOL[prec]


# ---- tensor-core forms (BF16x3, FP16x3): the bound of the scalar
# tensor-core form, which the FP32 accumulator sets (it grows with K = 4 NQ,
# not with the form)
TOL_TC = 3e-5


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("p", range(1, 8))
def test_elastic_tc_parity_small(orc, lib, tables, p, prec):
    E = SMALL_E[p]
    X = inputs.prism_mesh(E)
    C = inputs.elastic_coefficients(E)
    A, b, st = _run(lib, tables, p, X, C, prec)
    assert lib.fem_error_flag(tables) == lib.FEM_OK
    RA, Rb, Rst = orc.integrate_elastic(p, X, C)
    n = ns(PRISM, p)
    eA = rel_frob(A.reshape(E, 9 * n * n), RA.reshape(E, 9 * n * n))
    eb = rel_frob(b.reshape(E, 3 * n), Rb.reshape(E, 3 * n))
    print("elastic tc p=%d prec=%d: A max %.3e b max %.3e" % (p, prec, eA.max(), eb.max()))
    assert np.array_equal(st, Rst) and np.all(st == 0)
    assert eA.max() <= TOL_TC and eb.max() <= TOL_TC


def test_elastic_tc_many_tiles_vs_oracle(orc, lib, tables):
    """About ten M tiles per CTA (consecutive tiles share elements), every element."""
    p, E = 3, 600
    X = inputs.prism_mesh(E)
    C = inputs.elastic_coefficients(E)
    A, b, st = _run(lib, tables, p, X, C, lib.FEM_BF16X3)
    RA, Rb, Rst = orc.integrate_elastic(p, X, C)
    n = ns(PRISM, p)
    assert np.array_equal(st, Rst)
    assert rel_frob(A.reshape(E, -1), RA.reshape(E, -1)).max() <= TOL_TC
    assert rel_frob(b.reshape(E, -1), Rb.reshape(E, -1)).max() <= TOL_TC


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("p,E", [(5, 150), (7, 80)])
def test_elastic_tc_many_tiles_vs_fp64_kernel(orc, lib, tables, p, E, prec):
    """Eight or more M tiles per CTA, every element against the FP64 kernel
    (itself within 1e-12 of the oracle, checked on one element)."""
    X = inputs.prism_mesh(E)
    C = inputs.elastic_coefficients(E)
    A, b, st = _run(lib, tables, p, X, C, prec)
    A64, b64, st64 = _run(lib, tables, p, X, C, lib.FEM_F64)
    RA, _, _ = orc.integrate_elastic(p, X[:1], C[:, :1])
    assert rel_frob(A64[:1].reshape(1, -1), RA.reshape(1, -1)).max() <= 1e-12
    assert np.array_equal(st, st64) and np.all(st == 0)
    eA = rel_frob(A.reshape(E, -1), A64.reshape(E, -1))
    print("elastic tc many tiles p=%d prec=%d: A max %.3e" % (p, prec, eA.max()))
    assert eA.max() <= TOL_TC and rel_frob(b.reshape(E, -1), b64.reshape(E, -1)).max() <= TOL_TC


def test_elastic_tc_flags(orc, lib, tables):
    p = 2
    X = inputs.prism_mesh(4)
    C = inputs.elastic_coefficients(4)
    X[1] = X[1][[1, 0, 2, 4, 3, 5]]  # mirrored: det J < 0
    C[1, 2] = np.nan
    _, _, Rst = orc.integrate_elastic(p, X, C)
    for prec in (lib.FEM_BF16X3, lib.FEM_F16X3):
        _, _, st = _run(lib, tables, p, X, C, prec)
        assert list(st) == list(Rst)


def test_elastic_f16_small_load(orc, lib, tables):
    """FP16x3 with a body force 1e-6 of the stiffness scale: the load-vector
    row has its own power-of-two scale, so b stays accurate."""
    p, E = 3, 6
    X = inputs.prism_mesh(E)
    C = inputs.elastic_coefficients(E)
    C[2:5] *= 1e-6
    A, b, st = _run(lib, tables, p, X, C, lib.FEM_F16X3)
    RA, Rb, _ = orc.integrate_elastic(p, X, C)
    assert rel_frob(A.reshape(E, -1), RA.reshape(E, -1)).max() <= TOL_TC
    assert rel_frob(b.reshape(E, -1), Rb.reshape(E, -1)).max() <= TOL_TC
