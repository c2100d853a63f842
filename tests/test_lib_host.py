"""Host-side checks of the CUDA library that need no GPU: it loads, exports
every symbol of include/fem.h, its reference tables agree with the oracle's
independent construction, and argument validation rejects bad calls before
anything is enqueued."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    from paper_1310_1191_gb300 import build, _lib
    build.build()
    return _lib


def _header_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(fem_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib):
    declared = _header_functions()
    assert declared, "no declarations found"
    assert declared == set(lib.EXPORTS), declared ^ set(lib.EXPORTS)
    so = lib.load()
    for name in declared:
        assert hasattr(so, name), name


@pytest.mark.parametrize("p", range(1, 8))
def test_prism_tables_match_oracle(lib, orc, p):
    xi, w, phi = lib.fem_reference_rule(lib.FEM_PRISM6, p)
    oxi, ow = orc.rule(1, p)
    assert np.max(np.abs(xi - oxi)) < 1e-15
    assert np.max(np.abs(w - ow) / ow) < 1e-14
    ophi = orc.basis(1, p, oxi)
    scale = np.abs(ophi).max(axis=(0, 2), keepdims=True)
    assert np.max(np.abs(phi - ophi) / scale) < 1e-14


@pytest.mark.parametrize("p", range(1, 8))
def test_table1_prism_rule_matches_oracle(lib, orc, p):
    """The paper's prism rule (Table 1 point counts): the library's triangle
    rules (tri_rules_gen.cpp: continuation on the symmetric invariants e2, e3
    in its own parameters) and the oracle's (its own search on the monomial
    moments) are the same point set with the same weights, in the same order;
    the tables' shape functions at those points agree.  The orbit parameters
    of the degree-14 rule are determined by its moments only to about 1e-13
    (the system's condition number times the rounding of the moments), hence
    the tolerances."""
    xi, w, phi = lib.fem_reference_rule_ex(lib.FEM_PRISM6, lib.FEM_RULE_TABLE1, p)
    oxi, ow = orc.rule(orc.PRISM_T1, p)
    assert xi.shape == oxi.shape
    assert np.max(np.abs(xi - oxi)) < 1e-12
    assert np.max(np.abs(w - ow) / ow) < 1e-11
    ophi = orc.basis(1, p, oxi)
    scale = np.abs(ophi).max(axis=(0, 2), keepdims=True)
    assert np.max(np.abs(phi - ophi) / scale) < 1e-11


def test_tet_tables_match_oracle(lib, orc):
    xi, w, phi = lib.fem_reference_rule(lib.FEM_TET4, 1)
    oxi, ow = orc.rule(0, 1)
    assert np.max(np.abs(xi - oxi)) < 1e-15 and np.max(np.abs(w - ow)) < 1e-17
    assert np.max(np.abs(phi - orc.basis(0, 1, oxi))) < 1e-15


@pytest.mark.parametrize("p", [1, 4, 7])
def test_prism_table_factors(lib, p):
    """The structure fem_apply's sum factorisation relies on, read off the
    library's own table: DOF t + NT k at point iz NAB + iab is the triangle
    factor of (iab, t) times the zeta factor of (iz, k), for the value and all
    three reference derivatives (d/dzeta from the Legendre derivative)."""
    _, _, phi = lib.fem_reference_rule(lib.FEM_PRISM6, p)
    N = p + 1
    NT, NAB = N * (N + 1) // 2, N * N
    T = phi[:NAB, :3, :NT]                 # zeta level 0, k = 0 (L_0 = 1)
    L = phi[::NAB, 0, ::NT][:N, :N]        # first triangle point, t = 0 (T_0 = 1)
    dL = phi[::NAB, 3, ::NT][:N, :N]
    q = np.arange(N * NAB)
    iz, iab = q // NAB, q % NAB
    dof = np.arange(NT * N)
    k, t = dof // NT, dof % NT
    for d in range(3):
        ref = T[iab][:, d][:, t] * L[iz][:, k]
        assert np.max(np.abs(phi[:, d, :] - ref)) <= 1e-13 * np.abs(phi[:, d, :]).max()
    ref = T[iab][:, 0][:, t] * dL[iz][:, k]
    assert np.max(np.abs(phi[:, 3, :] - ref)) <= 1e-13 * np.abs(phi[:, 3, :]).max()


def test_sizes_and_strings(lib):
    assert lib.fem_matrix_size(lib.FEM_PRISM6, 7, lib.FEM_OUT_FULL) == 288 * 288
    assert lib.fem_matrix_size(lib.FEM_PRISM6, 3, lib.FEM_OUT_SYMPACKED) == 40 * 41 // 2
    assert lib.fem_matrix_size(lib.FEM_TET4, 1, lib.FEM_OUT_FULL) == 16
    assert lib.fem_matrix_size(lib.FEM_TET4, 2, lib.FEM_OUT_FULL) == -1
    assert lib.fem_matrix_size(lib.FEM_PRISM6, 8, lib.FEM_OUT_FULL) == -1
    assert lib.status_str(lib.FEM_EINVAL) == "invalid argument"


def test_invalid_arguments_rejected_on_host(lib):
    so = lib.load()
    with pytest.raises(lib.FemError) as ei:
        lib.fem_reference_rule(lib.FEM_PRISM6, 9)
    assert ei.value.code == lib.FEM_EINVAL
    # NULL tables handle
    rc = so.fem_integrate(None, 10, 8, None, 2, 8, 10, None, lib.FEM_F64, lib.FEM_OUT_FULL, 16, None,
                          None, None)
    assert rc == lib.FEM_EINVAL and "tables" in lib.last_error()
    rc = so.fem_integrate_uniform(None, 2, 10, 8, 8, 10, lib.FEM_F64, lib.FEM_OUT_FULL, 16, None, None,
                                  None)
    assert rc == lib.FEM_EINVAL and "tables" in lib.last_error()
    rc = so.fem_sync_status(None, 8, 10, None, None, None)
    assert rc == lib.FEM_EINVAL and "tables" in lib.last_error()
    rc = so.fem_apply(None, 2, 10, 8, 8, 10, lib.FEM_F64, 8, 16, None, None)
    assert rc == lib.FEM_EINVAL and "tables" in lib.last_error()
    # unknown rule, or the paper's rule on tetrahedra
    with pytest.raises(lib.FemError) as ei:
        lib.fem_reference_rule_ex(lib.FEM_PRISM6, 5, 2)
    assert ei.value.code == lib.FEM_EINVAL
    with pytest.raises(lib.FemError) as ei:
        lib.fem_reference_rule_ex(lib.FEM_TET4, lib.FEM_RULE_TABLE1, 1)
    assert ei.value.code == lib.FEM_EINVAL
    # bad degree range for the builder
    h = ctypes.c_void_p()
    assert so.fem_tables_build(lib.FEM_PRISM6, 3, 2, ctypes.byref(h)) == lib.FEM_EINVAL
    assert so.fem_tables_build(lib.FEM_TET4, 1, 2, ctypes.byref(h)) == lib.FEM_EINVAL
    assert so.fem_tables_build(lib.FEM_PRISM6, 1, 1, None) == lib.FEM_EINVAL
