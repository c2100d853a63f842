"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Small cases span several CTAs and a ragged tail of elements; full-size cases
run the degree sweep's element counts in the benchmark's launch configuration
and check a seeded sample of elements against the oracle.  Tolerances are the
per-element relative Frobenius bounds 1e-12 (FP64) and 1e-5 (FP32)."""
import numpy as np
import pytest

from _util import PRISM, SWEEP_E, TET, TOL, gpu_integrate, ns, rel_frob, unpack_upper, workload
from paper_1310_1191_gb300 import inputs

pytestmark = pytest.mark.gpu

# element groups per CTA of the FMA kernels: small cases cover a few CTAs + a ragged tail
SMALL_E = {1: 42 * 3 + 5, 2: 14 * 3 + 5, 3: 2 * 5 + 1, 4: 5, 5: 3, 6: 3, 7: 2}


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


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", range(1, 8))
def test_prism_parity_small(orc, prism_tables, p, prec):
    E = SMALL_E[p]
    X, C = workload(PRISM, p, E)
    A, b, st = gpu_integrate(prism_tables, PRISM, p, X, C, prec)
    RA, Rb, Rst = orc.integrate(PRISM, p, X, C)
    n = ns(PRISM, p)
    eA = rel_frob(A.reshape(E, n, n), RA)
    eb = rel_frob(b, Rb)
    assert np.all(st == Rst) and np.all(st == 0)
    assert eA.max() <= TOL[prec], (eA.max(), np.median(eA))
    assert eb.max() <= TOL[prec], (eb.max(), np.median(eb))


@pytest.mark.parametrize("prec", [0, 1])
def test_tet_parity_full_mesh(orc, tet_tables, prec):
    """All 24576 jittered P1 tetrahedra of the unit cube (16^3 cells x 6)."""
    X = inputs.tet_mesh(16)
    E = X.shape[0]
    assert E == 24576
    C = inputs.coefficients(E, kind="laplace")
    A, b, st = gpu_integrate(tet_tables, TET, 1, X, C, prec)
    RA, Rb, _ = orc.integrate(TET, 1, X, C)
    assert rel_frob(A.reshape(E, 4, 4), RA).max() <= TOL[prec]
    assert rel_frob(b, Rb).max() <= TOL[prec]
    assert np.all(st == 0)
    assert abs(b.sum() - 1.0) < (1e-12 if prec == 0 else 1e-4)  # volumes add up to the cube


@pytest.mark.parametrize("prec", [0, 1])
def test_tet_general_coefficients(orc, tet_tables, prec):
    X = inputs.tet_mesh(3)
    E = X.shape[0]
    C = inputs.coefficients(E)
    A, b, _ = gpu_integrate(tet_tables, TET, 1, X, C, prec)
    RA, Rb, _ = orc.integrate(TET, 1, X, C)
    assert rel_frob(A.reshape(E, 4, 4), RA).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 3, 5, 7])
def test_prism_sympacked(orc, prism_tables, p, prec):
    """Symmetric form (b = 0): upper-packed rows equal the oracle's upper triangle."""
    E = SMALL_E[p]
    X, C = workload(PRISM, p, E, kind="symmetric")
    A, b, st = gpu_integrate(prism_tables, PRISM, p, X, C, prec, layout=1)
    RA, _, _ = orc.integrate(PRISM, p, X, C)
    n = ns(PRISM, p)
    U = unpack_upper(A, n)
    R = np.triu(RA)
    assert rel_frob(U, R).max() <= TOL[prec]
    assert np.all(st == 0)


def test_status_flags_and_nonsym(orc, prism_tables):
    p = 2
    X, C = workload(PRISM, p, 6)
    X[1] = X[1][[1, 0, 2, 4, 3, 5]]  # mirrored: det J < 0
    C[9, 3] = np.nan
    A, b, st = gpu_integrate(prism_tables, PRISM, p, X, C, 0)
    _, _, Rst = orc.integrate(PRISM, p, X, C)
    assert list(st) == list(Rst)
    assert st[1] & 1 and st[3] & 2 and st[0] == 0
    # packed output of a non-symmetric form is flagged per element
    _, _, st2 = gpu_integrate(prism_tables, PRISM, p, X, C, 0, layout=1)
    assert np.all(st2 & 4)


def test_empty_and_no_load_vector(orc, prism_tables):
    X, C = workload(PRISM, 3, 3)
    A, b, st = gpu_integrate(prism_tables, PRISM, 3, X[:0], C[:, :0], 0)
    assert A.shape[0] == 0
    A, b, st = gpu_integrate(prism_tables, PRISM, 3, X, C, 0, want_b=False)
    RA, _, _ = orc.integrate(PRISM, 3, X, C)
    assert rel_frob(A.reshape(3, 40, 40), RA).max() <= TOL[0]


def test_coefficient_stride(orc, prism_tables):
    """SoA coefficients with a row stride larger than n_elem."""
    X, C = workload(PRISM, 2, 20)
    Cw = np.zeros((11, 33))
    Cw[:, :20] = C
    A, b, st = gpu_integrate(prism_tables, PRISM, 2, X, Cw, 0, coeff_stride=33)
    RA, Rb, _ = orc.integrate(PRISM, 2, X, C)
    assert rel_frob(A.reshape(20, 18, 18), RA).max() <= TOL[0]


def test_device_errors_are_reported(lib, prism_tables):
    import torch
    X, C = workload(PRISM, 2, 4)
    Xd = torch.from_numpy(X).cuda()
    Cd = torch.from_numpy(C).cuda()
    A = torch.zeros(4 * 324 + 2, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.FemError) as ei:  # misaligned output
        lib.fem_integrate_uniform(prism_tables, 2, 4, Xd, Cd, 4, 0, 0, A.data_ptr() + 8)
    assert ei.value.code == lib.FEM_EINVAL
    with pytest.raises(lib.FemError) as ei:  # degree outside the tables
        t = lib.fem_tables_build(lib.FEM_PRISM6, 1, 2)
        lib.fem_integrate_uniform(t, 3, 4, Xd, Cd, 4, 0, 0, A)
    assert ei.value.code == lib.FEM_EINVAL
    with pytest.raises(lib.FemError) as ei:
        lib.fem_integrate_uniform(prism_tables, 2, 4, Xd, Cd, 3, 0, 0, A)  # stride < n
    assert ei.value.code == lib.FEM_EINVAL


def _sample(E, k, seed):
    rng = np.random.default_rng(seed)
    idx = set([0, E - 1]) | set(rng.choice(E, size=min(k, E), replace=False).tolist())
    return np.array(sorted(idx))


@pytest.mark.slow
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("p", range(1, 8))
def test_prism_parity_full_size_sampled(orc, prism_tables, p, prec):
    """Degree sweep element counts (~2 GB of FP64 output per degree), whole
    launch as in the benchmark; a seeded sample of elements vs the oracle."""
    import torch
    E = SWEEP_E[p]
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    A, b, st = gpu_integrate(prism_tables, PRISM, p, X, C, prec, return_tensors=True)
    idx = _sample(E, 24 if p <= 5 else 6, 100 + p)
    n = ns(PRISM, p)
    Ai = A[torch.from_numpy(idx).cuda()].double().cpu().numpy().reshape(-1, n, n)
    bi = b[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    assert int((st != 0).sum().item()) == 0
    assert not bool(torch.isnan(A).any().item())
    RA, Rb, _ = orc.integrate(PRISM, p, X[idx], C[:, idx])
    assert rel_frob(Ai, RA).max() <= TOL[prec]
    assert rel_frob(bi, Rb).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_integrate_host_buffers(orc, lib, prism_tables, prec):
    """fem_integrate_host (host buffers, chunked copy/compute pipeline with a
    ragged last chunk) gives the device path's results."""
    import torch
    p, E = 3, 301
    X, C = workload(PRISM, p, E)
    n = ns(PRISM, p)
    dt = torch.float64 if prec == 0 else torch.float32
    Ah = torch.empty((E, n * n), dtype=dt).pin_memory()
    bh = torch.empty((E, n), dtype=dt).pin_memory()
    sh = torch.empty((E,), dtype=torch.int32).pin_memory()
    Xh = torch.from_numpy(X).pin_memory()
    Ch = torch.from_numpy(C).pin_memory()
    lib.fem_integrate_host(prism_tables, p, E, Xh, Ch, E, prec, 0, Ah, bh, sh, chunk=37)
    A, b, st = gpu_integrate(prism_tables, PRISM, p, X, C, prec)
    assert np.array_equal(Ah.numpy(), A) and np.array_equal(bh.numpy(), b)
    assert np.array_equal(sh.numpy(), st)
    RA, Rb, _ = orc.integrate(PRISM, p, X, C)
    assert rel_frob(Ah.numpy().reshape(E, n, n), RA).max() <= TOL[prec]
