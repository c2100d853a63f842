"""Nonlinear coefficient law and learned surrogate on the GPU vs the oracle:
training samples, network forward and gradients, training, field samples,
integration with the exact law and with the network, checkpointing, and the
measured gain of the network over the exact law."""
import os
import time

import numpy as np
import pytest

from _util import PRISM, rel_frob
from paper_1310_1191_gb300 import inputs

pytestmark = pytest.mark.gpu

P3, NS3, NQ3 = 3, 40, 64


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


def _field(E, ns, first=0):
    return inputs.field_coefficients(E, ns, first=first).astype(np.float32)


BOX = np.array([-5.4, 5.5, 58.0, 4900.0])  # about the 0.1/99.9 percentiles of the p=3 workload


def test_law_samples_match_generator_and_oracle_law(orc, lib):
    import torch
    n = 4096
    us = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    k = torch.empty(n, dtype=torch.float32, device="cuda")
    lib.fem_law_samples(n, BOX, 42, us, k)
    torch.cuda.synchronize()
    us, k = us.cpu().numpy(), k.cpu().numpy()
    idx = np.arange(n, dtype=np.uint64)
    u_ref = BOX[0] + (BOX[1] - BOX[0]) * inputs.draw_uniform(42, idx, 0)
    s_ref = np.exp(np.log(BOX[2]) + (np.log(BOX[3]) - np.log(BOX[2])) * inputs.draw_uniform(42, idx, 1))
    assert np.allclose(us[:, 0], u_ref.astype(np.float32), rtol=2e-7, atol=1e-6)
    assert np.allclose(us[:, 1], s_ref.astype(np.float32), rtol=2e-7)
    kr = np.array([orc.law_k(u, s * s) for u, s in zip(u_ref, s_ref)])
    assert np.max(np.abs(k - kr) / kr) <= 2e-7


def test_mlp_forward_and_gradient_vs_oracle(orc, lib):
    import torch
    m = lib.fem_mlp_create(BOX, 7)
    master, wc, box = m.params()
    assert np.array_equal(box, BOX)
    # compute weights are the master weights rounded to BF16
    bf = (master.view(np.uint32).astype(np.uint64) + 0x7FFF + ((master.view(np.uint32) >> 16) & 1))
    assert np.array_equal(wc, ((bf >> 16) << 16).astype(np.uint32).view(np.float32))
    n = 2048
    rng = np.random.default_rng(3)
    u = rng.uniform(BOX[0], BOX[1], n)
    s = np.exp(rng.uniform(np.log(BOX[2]), np.log(BOX[3]), n))
    tgt = np.array([orc.law_k(a, b * b) for a, b in zip(u, s)])
    us_d = torch.from_numpy(np.stack([u, s], 1).astype(np.float32)).cuda()
    t_d = torch.from_numpy(tgt.astype(np.float32)).cuda()
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    lib.fem_mlp_forward(m, n, us_d, y)
    grad = torch.empty(lib.fem_mlp_nparams(), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    lib.fem_mlp_loss_grad(m, n, us_d, t_d, grad, loss)
    torch.cuda.synchronize()
    u32 = us_d.cpu().numpy().astype(np.float64)
    t32 = t_d.cpu().numpy().astype(np.float64)
    yr = orc.mlp_forward(64, wc.astype(np.float64), BOX, u32[:, 0], u32[:, 1])
    assert np.max(np.abs(y.cpu().numpy() - yr)) <= 1e-5 * np.max(np.abs(yr))
    Lr, gr = orc.mlp_loss_grad(64, wc.astype(np.float64), BOX, u32[:, 0], u32[:, 1], t32)
    g = grad.cpu().numpy()
    assert abs(loss.item() - Lr) <= 1e-4 * Lr
    assert np.max(np.abs(g - gr)) <= 1e-4 * np.max(np.abs(gr))
    m.close()


def test_mlp_training_fits_law_and_checkpoint(orc, lib, tmp_path):
    import torch
    N = 1_000_000
    us = torch.empty((N, 2), dtype=torch.float32, device="cuda")
    k = torch.empty(N, dtype=torch.float32, device="cuda")
    lib.fem_law_samples(N, BOX, 42, us, k)
    m = lib.fem_mlp_create(BOX, 42)
    L1 = lib.fem_mlp_train(m, N, us, k, 3000, 8192, 1e-3, 1)
    L2 = lib.fem_mlp_train(m, N, us, k, 1000, 8192, 3e-4, 2)
    assert L2[-100:].mean() < 1e-3 * L1[:10].mean()
    M = 200_000
    hus = torch.empty((M, 2), dtype=torch.float32, device="cuda")
    hk = torch.empty(M, dtype=torch.float32, device="cuda")
    lib.fem_law_samples(M, BOX, 4242, hus, hk)
    y = torch.empty(M, dtype=torch.float32, device="cuda")
    lib.fem_mlp_forward(m, M, hus, y)
    torch.cuda.synchronize()
    rel = ((y - hk).abs() / hk).cpu().numpy()
    print("surrogate held-out relative error: median %.2e p99 %.2e max %.2e"
          % (np.median(rel), np.percentile(rel, 99), rel.max()))
    assert np.median(rel) < 2e-3 and rel.max() < 2e-2
    # checkpoint round trip: identical outputs
    path = str(tmp_path / "net.bin")
    lib.fem_mlp_save(m, path)
    m2 = lib.fem_mlp_load(path)
    y2 = torch.empty(M, dtype=torch.float32, device="cuda")
    lib.fem_mlp_forward(m2, M, hus, y2)
    torch.cuda.synchronize()
    assert torch.equal(y, y2)
    m.close()
    m2.close()


def test_field_samples_vs_host_reference(orc, lib, tables):
    import torch
    E = 50
    X = inputs.prism_mesh(E)
    U = _field(E, NS3)
    out = torch.empty((E, NQ3, 2), dtype=torch.float32, device="cuda")
    lib.fem_field_samples(tables, P3, E, torch.from_numpy(X).cuda(), torch.from_numpy(U).cuda(), out)
    torch.cuda.synchronize()
    out = out.cpu().numpy()
    xi, w = orc.rule(PRISM, P3)
    phi = orc.basis(PRISM, P3, xi)
    for e in range(0, E, 7):
        for q in range(0, NQ3, 5):
            x, y, z = xi[q]
            lo, hi = (1 - z) / 2, (1 + z) / 2
            Xe = X[e]
            J = np.stack([lo * (Xe[1] - Xe[0]) + hi * (Xe[4] - Xe[3]),
                          lo * (Xe[2] - Xe[0]) + hi * (Xe[5] - Xe[3]),
                          0.5 * ((1 - x - y) * (Xe[3] - Xe[0]) + x * (Xe[4] - Xe[1]) + y * (Xe[5] - Xe[2]))], 1)
            u = U[e] @ phi[q, 0]
            gr = np.linalg.solve(J.T, phi[q, 1:] @ U[e])
            assert abs(out[e, q, 0] - u) <= 1e-5 * max(1.0, abs(u))
            assert abs(out[e, q, 1] - np.linalg.norm(gr)) <= 1e-5 * np.linalg.norm(gr)


@pytest.mark.parametrize("p", [1, 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_integrate_exact_law_vs_oracle(orc, lib, tables, p, prec):
    import torch
    E = 30
    NS = (p + 1) ** 2 * (p + 2) // 2
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    U = _field(E, NS)
    dt = torch.float64 if prec == 0 else torch.float32
    A = torch.empty((E, NS * NS), dtype=dt, device="cuda")
    b = torch.empty((E, NS), dtype=dt, device="cuda")
    st = torch.empty(E, dtype=torch.int32, device="cuda")
    lib.fem_integrate_law(tables, p, E, torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(), E,
                          torch.from_numpy(U).cuda(), lib.FEM_LAW_EXACT, None, prec, 0, A, b, st)
    torch.cuda.synchronize()
    RA, Rb, Rst = orc.integrate(PRISM, p, X, C, law=1, ucoef=U.astype(np.float64))
    tol = 1e-12 if prec == 0 else 1e-5
    assert rel_frob(A.cpu().numpy().reshape(E, NS, NS), RA).max() <= tol
    assert rel_frob(b.cpu().numpy(), Rb).max() <= tol
    assert np.array_equal(st.cpu().numpy(), Rst)


@pytest.mark.parametrize("prec", [0, 1])
def test_integrate_network_vs_oracle(orc, lib, tables, prec):
    """Network coefficient inside a box that holds every point (no fallback),
    and a box that holds none (exact law everywhere, every element flagged)."""
    import torch
    E = 24
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    U = _field(E, NS3)
    dt = torch.float64 if prec == 0 else torch.float32
    Xd, Cd, Ud = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(), torch.from_numpy(U).cuda()
    for box, flag in ((np.array([-1e3, 1e3, 1e-3, 1e6]), 0), (np.array([1e3, 2e3, 1e8, 2e8]), 8)):
        m = lib.fem_mlp_create(box, 11)
        _, wc, _ = m.params()
        A = torch.empty((E, NS3 * NS3), dtype=dt, device="cuda")
        st = torch.empty(E, dtype=torch.int32, device="cuda")
        lib.fem_integrate_law(tables, P3, E, Xd, Cd, E, Ud, lib.FEM_LAW_MLP, m, prec, 0, A, None, st)
        torch.cuda.synchronize()
        RA, _, Rst = orc.integrate(PRISM, P3, X, C, law=2, ucoef=U.astype(np.float64),
                                   mlp=(64, wc.astype(np.float64), box))
        # the network runs in FP32 in both kernels
        assert rel_frob(A.cpu().numpy().reshape(E, NS3, NS3), RA).max() <= 1e-5
        assert np.all(st.cpu().numpy() == flag) and np.all(Rst == flag)
        m.close()


TOL_TC = 3e-5  # the tensor-core forms' bound (FP32 accumulation over K = 4 NQ)


@pytest.mark.parametrize("p,E", [(1, 400), (3, 30), (3, 5000), (5, 12)])
def test_tensor_core_exact_law_vs_oracle(orc, lib, tables, p, E):
    """The law on the tensor-core kernel (BF16x3): every element vs the
    oracle; p = 3 with 5,000 elements puts about ten M tiles on each CTA."""
    import torch
    NS = (p + 1) ** 2 * (p + 2) // 2
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    U = _field(E, NS)
    A = torch.empty((E, NS * NS), dtype=torch.float32, device="cuda")
    b = torch.empty((E, NS), dtype=torch.float32, device="cuda")
    st = torch.empty(E, dtype=torch.int32, device="cuda")
    lib.fem_integrate_law(tables, p, E, torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(), E,
                          torch.from_numpy(U).cuda(), lib.FEM_LAW_EXACT, None, lib.FEM_BF16X3, 0, A, b, st)
    torch.cuda.synchronize()
    assert lib.fem_error_flag(tables) == lib.FEM_OK
    RA, Rb, Rst = orc.integrate(PRISM, p, X, C, law=1, ucoef=U.astype(np.float64))
    eA = rel_frob(A.cpu().numpy().reshape(E, NS, NS), RA)
    print("tensor-core exact law p=%d E=%d: max %.2e" % (p, E, eA.max()))
    assert eA.max() <= TOL_TC and rel_frob(b.cpu().numpy(), Rb).max() <= TOL_TC
    assert np.array_equal(st.cpu().numpy(), Rst)


def test_tensor_core_network_vs_oracle(orc, lib, tables):
    """Network on the tensor-core kernel: a box that holds every point (no
    fallback) and one that holds none (exact law everywhere, every element
    flagged).  Boxes that cut through the points are left out: the GPU takes
    the in-box decision in FP32 and the oracle in FP64, so a point on the
    edge could go either way."""
    import torch
    E = 40
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    U = _field(E, NS3)
    Xd, Cd, Ud = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(), torch.from_numpy(U).cuda()
    for box, flag in ((np.array([-1e3, 1e3, 1e-3, 1e6]), 0), (np.array([1e3, 2e3, 1e8, 2e8]), 8)):
        m = lib.fem_mlp_create(box, 11)
        _, wc, _ = m.params()
        A = torch.empty((E, NS3 * NS3), dtype=torch.float32, device="cuda")
        st = torch.empty(E, dtype=torch.int32, device="cuda")
        lib.fem_integrate_law(tables, P3, E, Xd, Cd, E, Ud, lib.FEM_LAW_MLP, m, lib.FEM_BF16X3, 0, A, None, st)
        torch.cuda.synchronize()
        RA, _, Rst = orc.integrate(PRISM, P3, X, C, law=2, ucoef=U.astype(np.float64),
                                   mlp=(64, wc.astype(np.float64), box))
        eA = rel_frob(A.cpu().numpy().reshape(E, NS3, NS3), RA)
        print("tensor-core network flag=%s: max %.2e" % (flag, eA.max()))
        assert eA.max() <= TOL_TC
        assert np.array_equal(st.cpu().numpy(), Rst) and np.all(Rst == flag)
        m.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_law_more_newton_steps_converged(orc, lib, tables, prec):
    """The exact law with 16 and 32 Newton steps through fem_integrate's law
    descriptor: 8 steps have converged (residual <= 1e-12, pinned on the CPU),
    so the element matrices match the oracle's 8-step law within the
    precision's tolerance."""
    import torch
    E = 30
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    U = _field(E, NS3)
    dt = torch.float64 if prec == 0 else torch.float32
    RA, _, Rst = orc.integrate(PRISM, P3, X, C, law=1, ucoef=U.astype(np.float64))
    tol = {0: 1e-12, 1: 1e-5, 2: TOL_TC}[prec]
    for steps in (16, 32):
        A = torch.empty((E, NS3 * NS3), dtype=dt, device="cuda")
        st = torch.empty(E, dtype=torch.int32, device="cuda")
        law = lib.coef_law(lib.FEM_LAW_EXACT, torch.from_numpy(U).cuda(), newton_steps=steps)
        lib.fem_integrate(tables, E, torch.from_numpy(X).cuda(), None, P3, torch.from_numpy(C).cuda(), E, law, prec,
                          0, A, None, st)
        torch.cuda.synchronize()
        assert rel_frob(A.double().cpu().numpy().reshape(E, NS3, NS3), RA).max() <= tol, steps
        assert np.array_equal(st.cpu().numpy(), Rst)


@pytest.mark.parametrize("prec", [1, 2])
def test_network_hardware_tanh_within_its_bound(orc, lib, tables, prec):
    """The network with tanh.approx.f32 activations against the oracle's
    network (FP64, exact tanh).  With an activation error of at most eps
    the output moves by at most sum_n |W3_n| (1 + sum_m |W2_nm|) eps, so the
    element matrices (linear in k in their diffusion part) move by at most
    that over the smallest k, plus the kernel's own tolerance; eps = 2^-10.5
    is taken as the approximation's bound."""
    import torch
    E = 40
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    U = _field(E, NS3)
    box = np.array([-1e3, 1e3, 1e-3, 1e6])
    m = lib.fem_mlp_create(box, 11)
    # an output layer that keeps k in [1.5, 2.5] (sum |W3| <= 0.5, b3 = 2), as a
    # trained surrogate of the law does, so that the bound relative to k is tight
    H = 64
    master, _, _ = m.params()
    o3 = 3 * H + H * H + H
    master[o3:o3 + H] *= 0.5 / np.abs(master[o3:o3 + H]).sum()
    master[o3 + H] = 2.0
    m.set_params(master)
    _, wc, _ = m.params()
    W2 = wc[3 * H:3 * H + H * H].reshape(H, H)
    W3 = wc[o3:o3 + H]
    eps = 2.0 ** -10.5
    dk = float(np.sum(np.abs(W3) * (1.0 + np.abs(W2).sum(1)))) * eps
    dt = torch.float32
    A = torch.empty((E, NS3 * NS3), dtype=dt, device="cuda")
    st = torch.empty(E, dtype=torch.int32, device="cuda")
    law = lib.coef_law(lib.FEM_LAW_MLP, torch.from_numpy(U).cuda(), m, hw_tanh=True)
    lib.fem_integrate(tables, E, torch.from_numpy(X).cuda(), None, P3, torch.from_numpy(C).cuda(), E, law, prec, 0,
                      A, None, st)
    torch.cuda.synchronize()
    RA, _, Rst = orc.integrate(PRISM, P3, X, C, law=2, ucoef=U.astype(np.float64),
                               mlp=(64, wc.astype(np.float64), box))
    _, _, kref, _ = orc.point_law(PRISM, P3, X, U.astype(np.float64), law=2, mlp=(64, wc.astype(np.float64), box))
    bound = dk / np.abs(kref).min() + (1e-5 if prec == 1 else TOL_TC)
    err = rel_frob(A.cpu().numpy().reshape(E, NS3, NS3), RA)
    print("hardware tanh, prec %d: max %.2e (bound %.2e)" % (prec, err.max(), bound))
    assert err.max() <= bound
    assert np.array_equal(st.cpu().numpy(), Rst)
    m.close()


@pytest.mark.slow
def test_surrogate_gain_measured(orc, lib, tables):
    """What the trained network gains over the exact law on the nonlinear
    workload (p = 3, FP32): element-matrix error vs the FP64 oracle (exact
    law) and device time of the whole integration, both reported.  The
    network must stay within 5e-3 of the oracle; the time ratio is measured,
    not assumed (the 8-step Newton law is cheap, so the network can lose)."""
    import torch
    E = 200_000
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    U = _field(E, NS3)
    Xd, Cd, Ud = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(), torch.from_numpy(U).cuda()
    pil = torch.empty((20000, NQ3, 2), dtype=torch.float32, device="cuda")
    lib.fem_field_samples(tables, P3, 20000, Xd, Ud, pil)
    box = lib.fem_box_from_samples(pil.cpu().numpy())
    N = 2_000_000
    us = torch.empty((N, 2), dtype=torch.float32, device="cuda")
    k = torch.empty(N, dtype=torch.float32, device="cuda")
    lib.fem_law_samples(N, box, 42, us, k)
    m = lib.fem_mlp_create(box, 42)
    lib.fem_mlp_train(m, N, us, k, 4000, 8192, 1e-3, 1)
    lib.fem_mlp_train(m, N, us, k, 2000, 8192, 3e-4, 2)
    A = torch.empty((E, NS3 * NS3), dtype=torch.float32, device="cuda")
    st = torch.empty(E, dtype=torch.int32, device="cuda")
    times, errs = {}, {}
    idx = np.arange(0, E, E // 48)[:48]
    RA, _, _ = orc.integrate(PRISM, P3, X[idx], C[:, idx], law=1, ucoef=U[idx].astype(np.float64))
    for name, law, mm, steps, hw in (("exact", lib.FEM_LAW_EXACT, None, 8, False),
                                     ("exact32", lib.FEM_LAW_EXACT, None, 32, False),
                                     ("network", lib.FEM_LAW_MLP, m, 0, False),
                                     ("network_hw", lib.FEM_LAW_MLP, m, 0, True)):
        cl = lib.coef_law(law, Ud, mm, newton_steps=steps, hw_tanh=hw)
        run = lambda: lib.fem_integrate(tables, E, Xd, None, P3, Cd, E, cl, 1, 0, A, None, st)
        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            run()
        e1.record()
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1) / 3
        Ai = A[torch.from_numpy(idx).cuda()].double().cpu().numpy().reshape(-1, NS3, NS3)
        errs[name] = rel_frob(Ai, RA)
    fb = int(((st & 8) != 0).sum().item())
    print("exact law: %.2f ms, err max %.2e | network: %.2f ms, err max %.2e median %.2e | "
          "time ratio network/exact %.2f | fallback elements %.1f%%"
          % (times["exact"], errs["exact"].max(), times["network"], errs["network"].max(),
             np.median(errs["network"]), times["network"] / times["exact"], 100.0 * fb / E))
    slope = (times["exact32"] - times["exact"]) / 24.0
    for net in ("network", "network_hw"):
        cross = 8 + (times[net] - times["exact"]) / slope if slope > 0 else float("inf")
        print("%s: %.2f ms, err max %.2e; the exact law costs as much at about %.0f Newton steps"
              % (net, times[net], errs[net].max(), cross))
    assert errs["exact"].max() <= 1e-5 and errs["exact32"].max() <= 1e-5
    assert errs["network"].max() <= 5e-3 and errs["network_hw"].max() <= 5e-3
    m.close()
