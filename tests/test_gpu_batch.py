"""Mixed-degree meshes through fem_plan_* (p-binned persistent launch, CUDA
graph replay, autotuned tile shapes, per-degree launch loop) vs the oracle."""
import os

import numpy as np
import pytest

from _util import PRISM, TOL, ns, rel_frob
from paper_1310_1191_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def _mesh(E, seed_first=0):
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    P = inputs.mixed_degrees(E)
    return X, C, P


def _oracle_by_degree(orc, X, C, P, idx=None):
    """Oracle A_e, b_e for the elements idx (all if None), grouped by degree."""
    idx = np.arange(X.shape[0]) if idx is None else np.asarray(idx)
    out = {}
    for p in range(1, 8):
        sel = idx[P[idx] == p]
        if sel.size == 0:
            continue
        A, b, st = orc.integrate(PRISM, p, X[sel], C[:, sel])
        for k, e in enumerate(sel):
            out[int(e)] = (A[k], b[k], st[k])
    return out


def _run(lib, tables, X, C, P, prec, layout=0, flags=0, cache=None, plan=None, reps=1):
    import torch
    offA, offb, totA, totb = lib.fem_output_offsets(lib.FEM_PRISM6, P, layout)
    dt = torch.float64 if prec == 0 else torch.float32
    Xd = torch.from_numpy(X).cuda()
    Cd = torch.from_numpy(C).cuda()
    A = torch.full((totA,), float("nan"), dtype=dt, device="cuda")
    b = torch.full((totb,), float("nan"), dtype=dt, device="cuda")
    st = torch.full((X.shape[0],), -1, dtype=torch.int32, device="cuda")
    own = plan is None
    if own:
        plan = lib.fem_plan_create(tables, P, prec, layout, flags, cache)
    for _ in range(reps):
        lib.fem_plan_execute(plan, Xd, Cd, C.shape[1], A, b, st)
    torch.cuda.synchronize()
    res = (A.cpu().numpy(), b.cpu().numpy(), st.cpu().numpy(), offA, offb)
    if own:
        plan.close()
    return res


def _check(ref, P, res, prec, layout=0, idx=None):
    A, b, st, offA, offb = res
    idx = sorted(ref) if idx is None else idx
    errs = []
    for e in idx:
        p = int(P[e])
        n = ns(PRISM, p)
        RA, Rb, Rst = ref[e]
        if layout == 0:
            Ae = A[offA[e]:offA[e] + n * n].reshape(n, n)
            R = RA
        else:
            Ae = np.zeros((n, n))
            Ae[np.triu_indices(n)] = A[offA[e]:offA[e] + n * (n + 1) // 2]
            R = np.triu(RA)
        errs.append(rel_frob(Ae[None], R[None])[0])
        assert rel_frob(b[offb[e]:offb[e] + n][None], Rb[None])[0] <= TOL[prec]
        assert st[e] == Rst
    errs = np.array(errs)
    assert errs.max() <= TOL[prec], errs.max()
    return errs


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("mode", ["graph", "nograph", "loop", "concurrent", "concurrent_nograph"])
def test_plan_modes_match_oracle(orc, lib, tables, prec, mode):
    E = 700
    X, C, P = _mesh(E)
    assert set(np.unique(P)) == set(range(1, 8))
    ref = _oracle_by_degree(orc, X, C, P)
    flags = {"graph": 0, "nograph": lib.FEM_PLAN_NOGRAPH, "loop": lib.FEM_PLAN_LOOP,
             "concurrent": lib.FEM_PLAN_CONCURRENT,
             "concurrent_nograph": lib.FEM_PLAN_CONCURRENT | lib.FEM_PLAN_NOGRAPH}[mode]
    _check(ref, P, _run(lib, tables, X, C, P, prec, flags=flags, reps=2), prec)


@pytest.mark.parametrize("mode", ["loop", "concurrent"])
def test_per_degree_plans_tune_three_candidates(orc, lib, tables, tmp_path, mode):
    """Per-degree plans default to the uniform-degree kernels (variant 2) and,
    with autotuning, keep the fastest of the three candidates per degree,
    each timed as one launch over the bin; results stay exact."""
    E = 1500
    X, C, P = _mesh(E)
    idx = np.arange(0, E, 11)
    ref = _oracle_by_degree(orc, X, C, P, idx)
    base = {"loop": lib.FEM_PLAN_LOOP, "concurrent": lib.FEM_PLAN_CONCURRENT}[mode]
    plan = lib.fem_plan_create(tables, P, 1, 0, base, None)
    assert all(plan.variant(p)[0] == 2 for p in range(1, 8))
    _check(ref, P, _run(lib, tables, X, C, P, 1, plan=plan), 1, idx=list(idx))
    plan.close()
    cache = str(tmp_path / "tune.txt")
    plan = lib.fem_plan_create(tables, P, 1, 0, base | lib.FEM_PLAN_AUTOTUNE, cache)
    _check(ref, P, _run(lib, tables, X, C, P, 1, plan=plan, reps=2), 1, idx=list(idx))
    for p in range(1, 8):
        v, ms = plan.variant(p)
        assert v in (0, 1, 2) and ms[:3].min() > 0 and ms[v] == ms[:3].min() and ms[3] == 0
    chosen = [plan.variant(p)[0] for p in range(1, 8)]
    plan.close()
    # the cache is keyed by execution mode: a persistent plan ignores these entries
    plan = lib.fem_plan_create(tables, P, 1, 0, lib.FEM_PLAN_AUTOTUNE, cache)
    _check(ref, P, _run(lib, tables, X, C, P, 1, plan=plan), 1, idx=list(idx))
    assert all(plan.variant(p)[0] in (0, 1) for p in range(1, 8))
    plan.close()
    plan = lib.fem_plan_create(tables, P, 1, 0, base | lib.FEM_PLAN_AUTOTUNE, cache)
    _run(lib, tables, X, C, P, 1, plan=plan)
    assert [plan.variant(p)[0] for p in range(1, 8)] == chosen
    plan.close()


TOL_TC = 3e-5  # the tensor-core forms' bound (FP32 accumulation over K = 4 NQ)


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("mode", ["loop", "concurrent"])
def test_tensor_core_plans_match_oracle(orc, lib, tables, prec, mode):
    """Per-degree plans with a tensor-core precision: the p >= 3 bins run the
    tensor-core kernel on the plan's permutation and output offsets, the
    p <= 2 bins an FP32 kernel; every element vs the oracle."""
    E = 700
    X, C, P = _mesh(E)
    ref = _oracle_by_degree(orc, X, C, P)
    flags = {"loop": lib.FEM_PLAN_LOOP, "concurrent": lib.FEM_PLAN_CONCURRENT}[mode]
    plan = lib.fem_plan_create(tables, P, prec, 0, flags, None)
    assert [plan.variant(p)[0] for p in range(1, 8)] == [2, 2, 3, 3, 3, 3, 3]
    A, b, st, offA, offb = _run(lib, tables, X, C, P, prec, plan=plan, reps=2)
    plan.close()
    assert lib.fem_error_flag(tables) == lib.FEM_OK
    errs = []
    for e in range(E):
        p = int(P[e])
        n = ns(PRISM, p)
        RA, Rb, Rst = ref[e]
        errs.append(rel_frob(A[offA[e]:offA[e] + n * n].reshape(1, n, n), RA[None])[0])
        assert rel_frob(b[offb[e]:offb[e] + n][None], Rb[None])[0] <= TOL_TC
        assert st[e] == Rst
    print("tensor-core plan prec=%d %s: max %.2e" % (prec, mode, max(errs)))
    assert max(errs) <= TOL_TC


def test_tensor_core_plan_autotune_and_persistent_refused(orc, lib, tables):
    E = 1500
    X, C, P = _mesh(E)
    idx = np.arange(0, E, 13)
    ref = _oracle_by_degree(orc, X, C, P, idx)
    plan = lib.fem_plan_create(tables, P, lib.FEM_BF16X3, 0, lib.FEM_PLAN_CONCURRENT | lib.FEM_PLAN_AUTOTUNE, None)
    A, b, st, offA, offb = _run(lib, tables, X, C, P, 2, plan=plan, reps=2)
    for p in range(1, 8):
        v, ms = plan.variant(p)
        assert v in (0, 1, 2, 3) and ms.min() > 0 and ms[v] == ms.min()
    plan.close()
    for e in idx:
        p = int(P[e])
        n = ns(PRISM, p)
        assert rel_frob(A[offA[e]:offA[e] + n * n].reshape(1, n, n), ref[int(e)][0][None])[0] <= TOL_TC
    with pytest.raises(lib.FemError) as ei:
        lib.fem_plan_create(tables, P, lib.FEM_BF16X3, 0, 0, None)
    assert ei.value.code == lib.FEM_EUNSUPPORTED


@pytest.mark.parametrize("prec", [0, 1])
def test_plan_sympacked(orc, lib, tables, prec):
    E = 300
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E, kind="symmetric")
    P = inputs.mixed_degrees(E)
    ref = _oracle_by_degree(orc, X, C, P)
    _check(ref, P, _run(lib, tables, X, C, P, prec, layout=1), prec, layout=1)


def test_plan_autotune_and_cache(orc, lib, tables, tmp_path):
    E = 2000
    X, C, P = _mesh(E)
    idx = np.arange(0, E, 7)
    ref = _oracle_by_degree(orc, X, C, P, idx)
    cache = str(tmp_path / "tune.txt")
    plan = lib.fem_plan_create(tables, P, 1, 0, lib.FEM_PLAN_AUTOTUNE, cache)
    res = _run(lib, tables, X, C, P, 1, plan=plan, reps=2)
    _check(ref, P, res, 1, idx=list(idx))
    chosen = {}
    for p in range(1, 8):
        v, ms = plan.variant(p)
        assert v in (0, 1) and ms[v] > 0 and ms[v] <= ms[1 - v]
        chosen[p] = v
    plan.close()
    lines = open(cache).read().split("\n")
    assert len([l for l in lines if l.strip()]) == 7
    plan2 = lib.fem_plan_create(tables, P, 1, 0, lib.FEM_PLAN_AUTOTUNE, cache)
    res2 = _run(lib, tables, X, C, P, 1, plan=plan2)
    assert all(plan2.variant(p)[0] == chosen[p] for p in range(1, 8))
    _check(ref, P, res2, 1, idx=list(idx))
    plan2.close()


def test_plan_replay_and_rebind(orc, lib, tables):
    """Graph replays with the same buffers and re-captures with new ones."""
    import torch
    E = 400
    X, C, P = _mesh(E)
    ref = _oracle_by_degree(orc, X, C, P)
    plan = lib.fem_plan_create(tables, P, 0, 0, 0, None)
    r1 = _run(lib, tables, X, C, P, 0, plan=plan, reps=3)
    r2 = _run(lib, tables, X, C, P, 0, plan=plan, reps=1)  # new buffers
    _check(ref, P, r1, 0)
    _check(ref, P, r2, 0)
    plan.close()


def test_plan_errors(lib, tables):
    P = np.array([1, 2, 8], dtype=np.int8)
    with pytest.raises(lib.FemError) as ei:
        lib.fem_plan_create(tables, P, 1)
    assert ei.value.code == lib.FEM_EINVAL
    with pytest.raises(lib.FemError) as ei:
        lib.fem_plan_create(tables, np.array([3], dtype=np.int8), lib.FEM_BF16X3)
    assert ei.value.code == lib.FEM_EUNSUPPORTED


@pytest.mark.slow
@pytest.mark.parametrize("prec", [1, 0])
def test_plan_full_size_sampled(orc, lib, tables, prec):
    """500,000 prisms with seeded mixed degrees, one graph launch; a seeded
    sample of elements vs the oracle, statuses clean, no NaN."""
    import torch
    E = 500000
    X, C, P = _mesh(E)
    offA, offb, totA, totb = lib.fem_output_offsets(lib.FEM_PRISM6, P, 0)
    dt = torch.float64 if prec == 0 else torch.float32
    Xd = torch.from_numpy(X).cuda()
    Cd = torch.from_numpy(C).cuda()
    A = torch.full((totA,), float("nan"), dtype=dt, device="cuda")
    b = torch.full((totb,), float("nan"), dtype=dt, device="cuda")
    st = torch.full((E,), -1, dtype=torch.int32, device="cuda")
    plan = lib.fem_plan_create(tables, P, prec, 0, lib.FEM_PLAN_AUTOTUNE, None)
    lib.fem_plan_execute(plan, Xd, Cd, E, A, b, st)
    lib.fem_plan_execute(plan, Xd, Cd, E, A, b, st)
    torch.cuda.synchronize()
    assert int((st != 0).sum().item()) == 0
    assert not bool(torch.isnan(A).any().item()) and not bool(torch.isnan(b).any().item())
    rng = np.random.default_rng(400)
    idx = [0, E - 1] + sorted(rng.choice(E, 40, replace=False).tolist())
    idx = [e for e in idx if P[e] <= 6 or e in (0, E - 1)][:30]
    ref = _oracle_by_degree(orc, X, C, P, np.array(idx))
    Ah = {}
    for e in idx:
        n = ns(PRISM, int(P[e]))
        Ah[e] = A[int(offA[e]):int(offA[e]) + n * n].double().cpu().numpy().reshape(n, n)
    errs = [rel_frob(Ah[e][None], ref[e][0][None])[0] for e in idx]
    assert max(errs) <= TOL[prec]
    plan.close()
