"""Host checks of the mirrored pairs that the FMA kernels use (no GPU).

The kernels compute a tile (or micro-tile) of A_e below the diagonal from
the one above it:  A[j][i] = A[i][j] + sum_Q (phi_0[Q][j] V[Q][i] -
phi_0[Q][i] V[Q][j]),  V[Q][j] = sum_{d=1..3} G_Q[0][d] phi_d[Q][j].  This
holds because the per-point coefficient matrix G_Q of the weak form has a
symmetric diffusion block G[1..3][1..3], a reaction entry G[0][0] and a
convection row G[0][1..3], with G[1..3][0] = 0.  The first test checks that
identity on the dense quadrature sum with random tables; the second the
work ratios that bench.py reports beside the algorithmic roofline."""
import numpy as np
import pytest


def _dense(phi, G):
    # A[i][j] = sum_Q sum_{d,d'} phi[Q][d][i] G_Q[d][d'] phi[Q][d'][j]
    return np.einsum("qdi,qde,qej->ij", phi, G, phi)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lower_triangle_from_upper_plus_convection(seed):
    rng = np.random.default_rng(seed)
    nq, ns = 17, 11
    phi = rng.standard_normal((nq, 4, ns))
    G = np.zeros((nq, 4, 4))
    for q in range(nq):
        m = rng.standard_normal((3, 3))
        G[q, 1:, 1:] = m @ m.T              # SPD diffusion block (w det J^-1 D J^-T)
        G[q, 0, 0] = rng.uniform(0.0, 1.0)  # reaction
        G[q, 0, 1:] = rng.uniform(-1.0, 1.0, 3)  # convection: test value x trial derivative
    A = _dense(phi, G)
    V = np.einsum("qd,qdj->qj", G[:, 0, 1:], phi[:, 1:, :])
    phi0 = phi[:, 0, :]
    corr = np.einsum("qj,qi->ij", phi0, V) - np.einsum("qi,qj->ij", phi0, V)  # [i][j]
    # A[j][i] = A[i][j] + corr[i][j] for every pair, hence A^T = A + corr
    assert np.allclose(A.T, A + corr, rtol=0, atol=1e-11 * np.abs(A).max())
    # without convection the matrix is symmetric and the correction vanishes
    G[:, 0, 1:] = 0.0
    A0 = _dense(phi, G)
    assert np.allclose(A0, A0.T, rtol=0, atol=1e-11 * np.abs(A0).max())


def test_executed_work_ratios():
    import bench
    # (T (T + 1) / 2 full + T (T - 1) / 2 half tiles) / T^2 of the contraction
    expect = {(8, 4): 1900 / 2500, (8, 5): 1344 / 1764, (8, 6): 14 / 16, (8, 7): 30 / 36, (4, 7): 30 / 36}
    for (osz, p), ratio in expect.items():
        n, q = bench.ns_of(p), bench.nq_of(p)
        full = bench.flops_per_elem(p)
        assert bench.executed_flops_per_elem(p, osz) == pytest.approx(full - 8 * q * n * n * (1 - ratio), rel=1e-12)
    for osz, p in ((8, 1), (8, 2), (8, 3), (4, 5), (4, 6)):
        assert bench.executed_flops_per_elem(p, osz) == bench.flops_per_elem(p)
