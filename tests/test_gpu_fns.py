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
