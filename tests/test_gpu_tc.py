"""Tensor-core path (tcgen05, BF16/FP16 hi+lo split, FP32 accumulation) vs
the FP64 oracle, through the C ABI.

Tolerances (per-element relative Frobenius error of A_e and b_e), derived
from the arithmetic: a 16-bit hi + lo pair keeps 16 (BF16) or 22 (FP16)
significant bits of each operand (error about 2^-16 resp. 2^-21 per product
after dropping lo*lo), and the tensor core's FP32 accumulator adds up to about
one FP32 ulp (2^-24) of the running sum per accumulation step, 3 K/16 steps
for K = 4 NQ (384 at p = 7: about 2.3e-5).  Measured, the accumulator term
dominates for both types (the error grows linearly with K: ~2.5e-6 at p = 4,
~9e-6 at p = 7).  Bound: 3e-5 for both.  The measured max / median are
printed for the record."""
import numpy as np
import pytest

from _util import PRISM, gpu_integrate, ns, rel_frob, unpack_upper, workload
from paper_1310_1191_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_TC = {2: 3e-5, 3: 3e-5}
# several M tiles of 128 rows (NS+1 rows per element) and a ragged last tile
SMALL_E = {1: 300, 2: 70, 3: 37, 4: 23, 5: 9, 6: 5, 7: 4}


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


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("p", range(1, 8))
def test_tc_parity_small(orc, lib, tables, p, prec):
    E = SMALL_E[p]
    X, C = workload(PRISM, p, E)
    A, b, st = gpu_integrate(tables, PRISM, p, X, C, prec)
    assert lib.fem_error_flag(tables) == lib.FEM_OK
    RA, Rb, Rst = orc.integrate(PRISM, p, X, C)
    n = ns(PRISM, p)
    eA = rel_frob(A.reshape(E, n, n), RA)
    eb = rel_frob(b, Rb)
    print("p=%d prec=%d A max %.3e median %.3e  b max %.3e" % (p, prec, eA.max(), np.median(eA), eb.max()))
    assert np.all(st == Rst)
    assert eA.max() <= TOL_TC[prec] and eb.max() <= TOL_TC[prec]


# about 10 or more M tiles per persistent CTA (152 CTAs), so consecutive tiles
# of one CTA share elements (the ring of element slots) and the ranges of
# neighbouring CTAs split elements between them
MANY_E_ORACLE = {1: 40000, 2: 12000, 3: 5000, 4: 2000}
MANY_E_FP64 = {5: 1600, 6: 1100, 7: 800}


@pytest.mark.parametrize("p", sorted(MANY_E_ORACLE))
def test_tc_many_tiles_per_cta_vs_oracle(orc, lib, tables, p):
    """Every element of a mesh with about ten tiles per CTA vs the oracle (BF16x3)."""
    E = MANY_E_ORACLE[p]
    X, C = workload(PRISM, p, E)
    A, b, st = gpu_integrate(tables, PRISM, p, X, C, 2)
    assert lib.fem_error_flag(tables) == lib.FEM_OK
    RA, Rb, Rst = orc.integrate(PRISM, p, X, C)
    n = ns(PRISM, p)
    eA = rel_frob(A.reshape(E, n, n), RA)
    print("many tiles p=%d: A max %.3e" % (p, eA.max()))
    assert np.all(st == Rst)
    assert eA.max() <= TOL_TC[2] and rel_frob(b, Rb).max() <= TOL_TC[2]


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("p", sorted(MANY_E_FP64))
def test_tc_many_tiles_per_cta_vs_fp64_kernel(orc, lib, tables, p, prec):
    """Every element of a mesh with ten or more tiles per CTA vs the FP64 kernel
    (itself within 1e-12 of the oracle, checked here on a sample)."""
    E = MANY_E_FP64[p]
    X, C = workload(PRISM, p, E)
    A, b, st = gpu_integrate(tables, PRISM, p, X, C, prec)
    A64, b64, st64 = gpu_integrate(tables, PRISM, p, X, C, 0)
    assert lib.fem_error_flag(tables) == lib.FEM_OK
    idx = np.array([0, E // 2, E - 1])
    RA, _, _ = orc.integrate(PRISM, p, X[idx], C[:, idx])
    n = ns(PRISM, p)
    assert rel_frob(A64[idx].reshape(-1, n, n), RA).max() <= 1e-12
    eA = rel_frob(A.reshape(E, n, n), A64.reshape(E, n, n))
    print("many tiles p=%d prec=%d: A max %.3e" % (p, prec, eA.max()))
    assert np.all(st == st64) and np.all(st == 0)
    assert eA.max() <= TOL_TC[prec] and rel_frob(b, b64).max() <= TOL_TC[prec]


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("p", [3, 7])
def test_tc_sympacked_and_flags(orc, lib, tables, p, prec):
    E = SMALL_E[p]
    X, C = workload(PRISM, p, E, kind="symmetric")
    X[1] = X[1][[1, 0, 2, 4, 3, 5]]  # mirrored element: det J < 0 (flagged, still integrated)
    A, b, st = gpu_integrate(tables, PRISM, p, X, C, prec, layout=1)
    RA, Rb, Rst = orc.integrate(PRISM, p, X, C)
    n = ns(PRISM, p)
    assert list(st) == list(Rst) and st[1] & 1
    assert rel_frob(unpack_upper(A, n), np.triu(RA)).max() <= TOL_TC[prec]
    assert rel_frob(b, Rb).max() <= TOL_TC[prec]


def test_tc_bounded_wait_expires_and_recovers(orc, lib, tables):
    """Failure detection without a fault: the next launch withholds its
    operand copies, its waits run out (about 1 s), the device error word and
    the elements' status say so, and the next launch is correct again."""
    import torch
    p, E = 4, 20
    X, C = workload(PRISM, p, E)
    lib.fem_error_flag(tables)  # clear
    lib.fem_debug_stall_next(tables)
    A, b, st = gpu_integrate(tables, PRISM, p, X, C, lib.FEM_BF16X3)
    assert lib.fem_error_flag(tables) == lib.FEM_ETIMEOUT
    assert np.all(st & lib.FEM_ST_TIMEOUT)
    assert lib.fem_error_flag(tables) == lib.FEM_OK  # cleared by the previous call
    A, b, st = gpu_integrate(tables, PRISM, p, X, C, lib.FEM_BF16X3)
    assert lib.fem_error_flag(tables) == lib.FEM_OK and np.all(st == 0)
    RA, _, _ = orc.integrate(PRISM, p, X, C)
    n = ns(PRISM, p)
    assert rel_frob(A.reshape(E, n, n), RA).max() <= TOL_TC[2]


def test_tc_tet_unsupported(lib):
    import torch
    t = lib.fem_tables_build(lib.FEM_TET4, 1, 1)
    X = torch.zeros((2, 4, 3), dtype=torch.float64, device="cuda")
    C = torch.zeros((11, 2), dtype=torch.float64, device="cuda")
    A = torch.zeros((2, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(lib.FemError) as ei:
        lib.fem_integrate_uniform(t, 1, 2, X, C, 2, lib.FEM_BF16X3, 0, A)
    assert ei.value.code == lib.FEM_EUNSUPPORTED
    t.close()


@pytest.mark.slow
@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("p", [4, 5, 6, 7])
def test_tc_parity_full_size_sampled(orc, lib, tables, p, prec):
    """200,000 prisms per degree (the mixed-precision workload), full launch;
    a seeded sample vs the oracle, all statuses clean, no NaN."""
    import torch
    E = 200000
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    A, b, st = gpu_integrate(tables, PRISM, p, X, C, prec, return_tensors=True)
    assert lib.fem_error_flag(tables) == lib.FEM_OK
    rng = np.random.default_rng(200 + p)
    idx = np.array(sorted(set([0, E - 1]) | set(rng.choice(E, 6, replace=False).tolist())))
    n = ns(PRISM, p)
    ti = torch.from_numpy(idx).cuda()
    Ai = A[ti].double().cpu().numpy().reshape(-1, n, n)
    bi = b[ti].double().cpu().numpy()
    assert int((st != 0).sum().item()) == 0
    assert not bool(torch.isnan(A).any().item())
    RA, Rb, _ = orc.integrate(PRISM, p, X[idx], C[:, idx])
    eA = rel_frob(Ai, RA)
    print("full p=%d prec=%d A max %.3e median %.3e" % (p, prec, eA.max(), np.median(eA)))
    assert eA.max() <= TOL_TC[prec] and rel_frob(bi, Rb).max() <= TOL_TC[prec]
    del A, b, st
    torch.cuda.empty_cache()
