"""Child process of test_gpu_checked.py: loads the checked library variant
(FEM_GB300_CHECKED=1 set by the parent) and runs mixed-degree integrations
through it.  Prints one line "OK <cases>" when every check passed."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from _util import PRISM, ns, rel_frob  # noqa: E402
from paper_1310_1191_gb300 import _lib, inputs  # noqa: E402

TOL = {0: 1e-12, 2: 3e-5}


def _oracle(X, C, P):
    out = {}
    for p in range(1, 8):
        sel = np.nonzero(P == p)[0]
        if sel.size == 0:
            continue
        A, b, _ = oracle.integrate(PRISM, p, X[sel], C[:, sel])
        for k, e in enumerate(sel):
            out[int(e)] = (A[k], b[k])
    return out


def _errors(ref, P, A, b, offA, offb, skip=()):
    worst = 0.0
    for e, (RA, Rb) in ref.items():
        n = ns(PRISM, int(P[e]))
        be = b[offb[e]:offb[e] + n]
        worst = max(worst, float(rel_frob(be[None], Rb[None])[0]))
        Ae = A[offA[e]:offA[e] + n * n]
        if e in skip:
            assert np.all(np.isnan(Ae)), "skipped block was written"
            continue
        worst = max(worst, float(rel_frob(Ae.reshape(1, n, n), RA[None])[0]))
    return worst


def main():
    lib = _lib
    lib.load()
    assert os.path.basename(lib._lib._name) == "libfem_gb300_checked.so", lib._lib._name
    oracle.build()
    t = lib.fem_tables_build(lib.FEM_PRISM6, 1, 7)
    E = 97
    X, C = inputs.prism_mesh(E), inputs.coefficients(E)
    P = inputs.mixed_degrees(E)
    P[E - 1] = 3  # the last block (the one the hook cuts) of a known degree
    ref = _oracle(X, C, P)
    offA, offb, totA, totb = lib.fem_output_offsets(lib.FEM_PRISM6, P, 0)
    assert offA[E - 1] + ns(PRISM, 3) ** 2 == totA
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    cases = 0
    for prec in (lib.FEM_F64, lib.FEM_BF16X3):
        dt = torch.float64 if prec == lib.FEM_F64 else torch.float32
        A = torch.full((totA,), float("nan"), dtype=dt, device="cuda")
        b = torch.full((totb,), float("nan"), dtype=dt, device="cuda")
        st = torch.full((E,), -1, dtype=torch.int32, device="cuda")
        # tensor-core plans run per degree (graph branches)
        flag_modes = [0, lib.FEM_PLAN_LOOP] if prec == lib.FEM_F64 else [lib.FEM_PLAN_CONCURRENT]
        for flags in flag_modes:
            plan = lib.fem_plan_create(t, P, prec, 0, flags)
            # every check holds on a well-formed plan
            lib.fem_plan_execute(plan, Xd, Cd, E, A, b, st)
            assert lib.fem_error_flag(t) == lib.FEM_OK, lib.last_error()
            err = _errors(ref, P, A.double().cpu().numpy(), b.double().cpu().numpy(), offA, offb)
            assert err <= TOL[prec], (prec, flags, err)
            assert int((st != 0).sum().item()) == 0
            # the hook shortens A_out by one value: the last block is refused
            A.fill_(float("nan"))
            b.fill_(float("nan"))
            lib.fem_debug_shrink_bound(plan)
            lib.fem_plan_execute(plan, Xd, Cd, E, A, b, st)
            code = lib.fem_error_flag(t)
            assert code == lib.FEM_ECHECKED, (prec, flags, code)
            err = _errors(ref, P, A.double().cpu().numpy(), b.double().cpu().numpy(), offA, offb,
                          skip=(E - 1,))
            assert err <= TOL[prec], (prec, flags, err)
            # the next execution is normal again and the word was cleared
            lib.fem_plan_execute(plan, Xd, Cd, E, A, b, st)
            assert lib.fem_error_flag(t) == lib.FEM_OK
            plan.close()
            cases += 1
    # the allocation-free entry point under the same checks
    A = torch.full((totA,), float("nan"), dtype=torch.float64, device="cuda")
    b = torch.full((totb,), float("nan"), dtype=torch.float64, device="cuda")
    lib.fem_integrate_mixed_noalloc(t, P, Xd, Cd, E, lib.FEM_F64, 0, A, b)
    assert lib.fem_error_flag(t) == lib.FEM_OK
    err = _errors(ref, P, A.cpu().numpy(), b.cpu().numpy(), offA, offb)
    assert err <= TOL[0], err
    cases += 1
    t.close()
    print("OK %d" % cases)


if __name__ == "__main__":
    main()
