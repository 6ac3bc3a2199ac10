"""Richardson(m)-FNS (Sec. 3.1, eqs. 19-20 with T = I): the unrolled chain's symbol and
weight gradients against central differences of the FP64 oracle, and the symbol's
training step (Algorithm 2, Meta-Lambda stage with the symbol held directly)."""
import numpy as np
import pytest

import richm_synth as synth
from gpu_util import make_op, to_dev
from oracle.fourier import fourier_correction
from oracle.iterations import inner_steps, jacobi_binv
from oracle.operators import assemble_q1
from paper_2412_08076_gb300 import fns, richm

pytestmark = pytest.mark.gpu


def _r32(a):
    return np.asarray(a).astype(np.float32).astype(np.float64)


def test_fns_chain_gradients_match_oracle_differences():
    import torch
    n, m, M, C = 7, 2, 4, 2
    insts = [synth.AnisoInstance(1e-2, 0.4, n), synth.AnisoInstance(0.5, 2.0, n)]
    B = len(insts)
    op = make_op(insts)
    As = [assemble_q1(n, t.eps, t.theta) for t in insts]
    fs = [_r32(synth.rhs_normal(3, i, n)) for i in range(B)]
    S = synth.fourier_symbol(n, seed=5) * 0.3
    S = S.astype(np.complex64).astype(np.complex128)
    w = _r32(np.array([[0.5, 0.7], [0.6, 0.4]]))

    def oracle_loss(SS, ww):
        tot = 0.0
        for b in range(B):
            u = np.zeros(n * n)
            for _ in range(C):
                u, _ = inner_steps(As[b], fs[b].ravel(), u, None, ww[b], K=M, Binv=jacobi_binv(As[b]))
                u = fourier_correction(As[b], fs[b].ravel(), u, SS)
            tot += np.log(np.linalg.norm(fs[b].ravel() - As[b] @ u) / np.linalg.norm(fs[b]))
        return tot / B

    h = 1e-6
    ref_dS = np.zeros((n, n), dtype=np.complex128)
    for k1 in range(n):
        for k2 in range(n):
            E = np.zeros((n, n))
            E[k1, k2] = 1.0
            re = (oracle_loss(S + h * E, w) - oracle_loss(S - h * E, w)) / (2 * h)
            im = (oracle_loss(S + 1j * h * E, w) - oracle_loss(S - 1j * h * E, w)) / (2 * h)
            ref_dS[k1, k2] = re + 1j * im
    ref_gw = np.zeros_like(w)
    for b in range(B):
        for i in range(m):
            E = np.zeros_like(w)
            E[b, i] = h
            ref_gw[b, i] = (oracle_loss(S, w + E) - oracle_loss(S, w - E)) / (2 * h)
    b_dev = to_dev(op, fs, richm.F32)
    f = fns.FNS(op, torch.tensor(w, dtype=torch.float32, device="cuda"), m, M,
                torch.tensor(S.astype(np.complex64), device="cuda"), precond=1)
    loss, dS, gw = f.loss_and_grads(b_dev, C)
    assert abs(float(loss.item()) - oracle_loss(S, w)) <= 1e-5 * abs(oracle_loss(S, w)) + 1e-6
    got = dS.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref_dS) <= 1e-3 * np.linalg.norm(ref_dS)
    np.testing.assert_allclose(gw.cpu().numpy(), ref_gw, atol=1e-3 * np.abs(ref_gw).max())


def test_fns_symbol_training_lowers_the_loss():
    import torch
    n, m, M, C, B = 31, 1, 10, 2, 4
    insts = [synth.AnisoInstance(1e-2, 0.0, n)] * B
    op = make_op(insts)
    b_dev = to_dev(op, [_r32(synth.rhs_normal(1, i, n)) for i in range(B)], richm.F32)
    coef = op.stencil(0)
    S0 = fns.periodic_inverse_symbol(coef, n, delta=1e-2 * 4 * coef[0])
    S = torch.tensor(S0.astype(np.complex64), device="cuda")
    w = torch.full((B, m), 0.5, dtype=torch.float32, device="cuda")
    f0 = fns.FNS(op, w.clone(), m, M, S.clone(), precond=1)
    f = fns.FNS(op, w, m, M, S, precond=1)
    hist = fns.train_alternating(f, [b_dev], C=C, rounds=1, steps=20, lr_symbol=2e-2, lr_w=1e-3)
    assert len(hist) == 60 and np.all(np.isfinite(hist))
    assert hist[-1] < hist[0] - 0.03  # FP64 run of the same schedule: -1.949 -> -2.081
    # Outer iterations to a relative residual of 1e-2 (an FP32 state cannot reach the
    # paper's 1e-6 on this problem without refinement); the same schedule in FP64 gives
    # 40-57 with the initial parameters and 32-48 trained.
    its0 = f0.iterations(b_dev, tol=1e-2, max_outer=300)
    its = f.iterations(b_dev, tol=1e-2, max_outer=300)
    assert all(c is not None for c in its0 + its)
    assert max(its) < max(its0)


def test_fns_parameter_maps_match_oracle():
    import torch
    from oracle.fourier import symbol_from_stencil, transition_band
    for n in (1, 16, 33):
        q = [1.3, -0.4, 0.08, -0.38, 0.05, 0.02]
        o = np.array([0.1, -0.2, 0.05, 0.3, -0.1, 0.4], dtype=np.float32)
        S = richm.symbol_from_stencil(n, q, torch.tensor(o, device="cuda"))
        ref = symbol_from_stencil(q, o.astype(np.float64), n)
        assert np.abs(S.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()
        tau = np.array([1.0, 0.1, -0.2, 0.05, 0.3, -0.15, 0.02, 0.07, -0.01], dtype=np.float32)
        t = richm.transition_from_band(n, torch.tensor(tau, device="cuda"))
        tref = transition_band(tau.astype(np.float64), n)
        assert np.abs(t.cpu().numpy() - tref).max() <= 1e-5 * np.abs(tref).max()
        # reverse modes: against the oracle's maps by central differences of <G, map>
        rng = np.random.default_rng(n)
        G = rng.standard_normal((n, n))
        dS = torch.tensor((G + 1j * rng.standard_normal((n, n))).astype(np.complex64), device="cuda")
        d_o = richm.symbol_from_stencil_vjp(n, q, torch.tensor(o, device="cuda"), dS).cpu().numpy()
        dtau = richm.transition_from_band_vjp(n, torch.tensor(G.astype(np.float32), device="cuda")).cpu().numpy()
        h = 1e-5
        Gf = G.astype(np.float32).astype(np.float64)
        for m in range(6):
            e = np.zeros(6)
            e[m] = h
            fd = (np.sum(Gf * symbol_from_stencil(q, o + e, n).real) -
                  np.sum(Gf * symbol_from_stencil(q, o - e, n).real)) / (2 * h)
            assert abs(d_o[m] - fd) <= 1e-3 * max(1.0, abs(fd)), (n, m, d_o[m], fd)
        for k in range(9):
            e = np.zeros(9)
            e[k] = h
            fd = (np.sum(Gf * transition_band(tau + e, n)) - np.sum(Gf * transition_band(tau - e, n))) / (2 * h)
            assert abs(dtau[k] - fd) <= 1e-3 * max(1.0, abs(fd)), (n, k, dtau[k], fd)


def test_fns_chain_with_transition_and_maps_matches_oracle_differences():
    # the FNS chain (C outer iterations of M Jacobi-Richardson(m) sweeps and the correction
    # with the symbol and transition maps) against central differences of the FP64 oracle
    import torch
    from oracle.fourier import fourier_correction_t, symbol_from_stencil, transition_band
    n, m, M, C = 7, 2, 4, 2
    insts = [synth.AnisoInstance(1e-2, 0.4, n)] * 2
    B = len(insts)
    op = make_op(insts)
    A = assemble_q1(n, 1e-2, 0.4)
    fs = [_r32(synth.rhs_normal(3, i, n)) for i in range(B)]
    c = op.stencil(0)
    q = [c[0], c[1], c[2], c[3], c[4], 0.05 * c[0]]
    o = np.array([0.05, -0.1, 0.2, 0.0, 0.1, -0.3], dtype=np.float32).astype(np.float64)
    tau = np.array([1.0, 0.1, -0.05, 0.02, 0.08, -0.04, 0.01, 0.03, -0.02], dtype=np.float32).astype(np.float64)
    w = _r32(np.array([[0.5, 0.7], [0.5, 0.7]]))

    def oracle_loss(o_, tau_):
        S = symbol_from_stencil(q, o_, n).astype(np.complex64).astype(np.complex128)
        t = transition_band(tau_, n).astype(np.float32).astype(np.float64)
        tot = 0.0
        for bi in range(B):
            u = np.zeros(n * n)
            for _ in range(C):
                u, _ = inner_steps(A, fs[bi].ravel(), u, None, w[bi], K=M, Binv=jacobi_binv(A))
                u = fourier_correction_t(A, fs[bi].ravel(), u, S, t)
            tot += np.log(np.linalg.norm(fs[bi].ravel() - A @ u) / np.linalg.norm(fs[bi]))
        return tot / B

    o_t = torch.tensor(o.astype(np.float32), device="cuda")
    tau_t = torch.tensor(tau.astype(np.float32), device="cuda")
    S = richm.symbol_from_stencil(n, q, o_t)
    t = richm.transition_from_band(n, tau_t)
    f = fns.FNS(op, torch.tensor(w, dtype=torch.float32, device="cuda"), m, M, S, precond=1, transition=t)
    loss, dS, gw, dt = f.loss_and_grads(to_dev(op, fs, richm.F32), C, want_dt=True)
    assert abs(float(loss.item()) - oracle_loss(o, tau)) <= 1e-4 * abs(oracle_loss(o, tau))
    d_o = richm.symbol_from_stencil_vjp(n, q, o_t, dS).cpu().numpy()
    d_tau = richm.transition_from_band_vjp(n, dt).cpu().numpy()
    h = 1e-4
    scale = max(np.abs(d_o).max(), np.abs(d_tau).max())
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        fd = (oracle_loss(o + e, tau) - oracle_loss(o - e, tau)) / (2 * h)
        assert abs(d_o[k] - fd) <= 2e-3 * scale, (k, d_o[k], fd)
    for k in range(9):
        e = np.zeros(9)
        e[k] = h
        fd = (oracle_loss(o, tau + e) - oracle_loss(o, tau - e)) / (2 * h)
        assert abs(d_tau[k] - fd) <= 2e-3 * scale, (k, d_tau[k], fd)


def test_algorithm2_with_meta_networks_lowers_the_loss():
    # Algorithm 2 over two (eps, theta): Meta-Lambda and Meta-T with Meta-omega frozen at
    # 0.5, then Meta-omega, then Meta-Lambda and Meta-T again
    import torch
    n, B = 31, 4
    batches = []
    for k, (eps, th) in enumerate([(1e-2, 0.0), (1e-1, 0.7)]):
        insts = [synth.AnisoInstance(eps, th, n)] * B
        op = make_op(insts)
        b = to_dev(op, [_r32(synth.rhs_normal(20 + k, i, n)) for i in range(B)], richm.F32)
        X = torch.tensor(synth.meta_inputs(insts), dtype=torch.float32, device="cuda")
        batches.append((op, b, X[:1].contiguous(), X))
    net = fns.MetaFNS(m=4, M=8)
    its0 = [net.iterations(op, b, X1, XB, tol=1e-2, max_outer=300) for op, b, X1, XB in batches]
    hist = fns.train_algorithm2(net, batches, C=2, cycles=1, steps=16, lr=2e-3)
    assert len(hist) == 48 and np.all(np.isfinite(hist))
    assert np.mean(hist[-4:]) < np.mean(hist[:4]) - 0.02
    its = [net.iterations(op, b, X1, XB, tol=1e-2, max_outer=300) for op, b, X1, XB in batches]
    print(f"\nAlgorithm 2 (Meta-omega, Meta-Lambda, Meta-T): loss {hist[0]:.3f} -> {hist[-1]:.3f}; "
          f"outer iterations to 1e-2 {its0} -> {its}")
    # (the initial networks may not reach the tolerance within 300 iterations: None)
    for a, c in zip(its0, its):
        assert all(v is not None for v in c)
        assert max(c) <= max(301 if v is None else v for v in a)
