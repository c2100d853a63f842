"""Helpers shared by the GPU tests: seeded workloads, device calls through the
C ABI, and per-element error measures."""
import numpy as np

from paper_1310_1191_gb300 import inputs

TET, PRISM = 0, 1
# tolerance on the per-element relative Frobenius error, by precision
TOL = {0: 1e-12, 1: 1e-5}

# element counts of the ~2 GB-per-degree prism sweep (FP64 full output):
# E_p = round(2e9 / (8 (NS^2 + NS)))
SWEEP_E = {1: 5952381, 2: 730994, 3: 152439, 4: 43860, 5: 15623, 6: 6475, 7: 3004}


def ns(elem, p):
    return 4 if elem == TET else (p + 1) ** 2 * (p + 2) // 2


def workload(elem, p, E, kind="random", first=0):
    """(coords [E][nv][3], coeffs [11][E]) of the seeded synthetic workload."""
    if elem == TET:
        X = inputs.tet_mesh(16)[first:first + E]
        C = inputs.coefficients(X.shape[0], kind="laplace" if kind == "random" else kind)
    else:
        X = inputs.prism_mesh(E)
        C = inputs.coefficients(E, kind=kind)
    return np.ascontiguousarray(X), np.ascontiguousarray(C)


def rel_frob(A, R):
    """Per-element ||A - R||_F / ||R||_F over the trailing axes."""
    ax = tuple(range(1, A.ndim))
    num = np.sqrt(np.sum((A.astype(np.float64) - R) ** 2, axis=ax))
    den = np.sqrt(np.sum(R ** 2, axis=ax))
    return num / np.where(den > 0, den, 1.0)


def unpack_upper(P, n):
    """[E][n(n+1)/2] upper-packed rows -> [E][n][n] upper triangles (lower = 0)."""
    E = P.shape[0]
    out = np.zeros((E, n, n), dtype=np.float64)
    iu = np.triu_indices(n)
    out[:, iu[0], iu[1]] = P
    return out


def gpu_integrate(tables, elem, p, X, C, prec, layout=0, want_b=True, stream=None,
                  coeff_stride=None, return_tensors=False):
    """Run fem_integrate on device copies of X, C; returns numpy (A, b, status)."""
    import torch
    from paper_1310_1191_gb300 import _lib
    E = X.shape[0]
    dt = torch.float64 if prec == 0 else torch.float32
    dev = torch.device("cuda")
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    Cd = torch.from_numpy(np.ascontiguousarray(C)).to(dev)
    m = _lib.fem_matrix_size(elem, p, layout)
    A = torch.full((max(E, 1), m), float("nan"), dtype=dt, device=dev)
    b = torch.full((max(E, 1), ns(elem, p)), float("nan"), dtype=dt, device=dev) if want_b else None
    st = torch.full((max(E, 1),), -1, dtype=torch.int32, device=dev)
    _lib.fem_integrate_uniform(tables, p, E, Xd, Cd, coeff_stride or C.shape[1], prec, layout, A,
                               b, st, stream)
    torch.cuda.synchronize()
    if return_tensors:
        return A, b, st
    return (A.cpu().numpy()[:E], None if b is None else b.cpu().numpy()[:E],
            st.cpu().numpy()[:E])
