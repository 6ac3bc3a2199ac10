"""GPU Fourier-domain correction (eqs. 19-20 with T = I) against the oracle."""
import numpy as np
import pytest

import richm_synth as synth
from gpu_util import from_dev, make_op, to_dev
from oracle.fourier import fourier_correction, fourier_correction_vjp
from oracle.operators import assemble_q1
from paper_2412_08076_gb300 import richm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,batch", [(33, 3), (63, 2), (1, 1)])
def test_fourier_correction_matches_oracle(n, batch):
    import torch
    insts = [synth.AnisoInstance(1e-4, np.pi / 3, n)] * batch
    op = make_op(insts)
    A = assemble_q1(n, 1e-4, np.pi / 3)
    S = synth.fourier_symbol(n, seed=3)
    us = [(0.3 * synth.rhs_uniform(8, i, n)).astype(np.float32).astype(np.float64) for i in range(batch)]
    fs = [synth.rhs_uniform(9, i, n).astype(np.float32).astype(np.float64) for i in range(batch)]
    U, F = to_dev(op, us, richm.F32), to_dev(op, fs, richm.F32)
    St = torch.tensor(S.astype(np.complex64), device="cuda")
    op.fourier_correction(U, F, St)
    got = from_dev(op, U, richm.F32)
    S32 = S.astype(np.complex64).astype(np.complex128)
    for i in range(batch):
        ref = fourier_correction(A, fs[i].ravel(), us[i].ravel(), S32)
        assert np.linalg.norm(got[i].ravel() - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,batch,inplace", [(32, 3, False), (31, 2, True), (1, 1, False)])
def test_fourier_vjp_matches_oracle(n, batch, inplace):
    # instances of one size with different coefficients; dS is the batch sum
    import torch
    insts = [synth.AnisoInstance([1e-4, 1e-1, 1.0][i % 3], [np.pi / 3, 0.4, 2.5][i % 3], n) for i in range(batch)]
    op = make_op(insts)
    As = [assemble_q1(n, t.eps, t.theta) for t in insts]
    S = synth.fourier_symbol(n, seed=5)
    r32 = lambda a: a.astype(np.float32).astype(np.float64)
    us = [r32(0.3 * synth.rhs_uniform(8, i, n)) for i in range(batch)]
    fs = [r32(synth.rhs_uniform(9, i, n)) for i in range(batch)]
    gs = [r32(synth.rhs_uniform(7, i, n)) for i in range(batch)]
    U, F, G = to_dev(op, us, richm.F32), to_dev(op, fs, richm.F32), to_dev(op, gs, richm.F32)
    St = torch.tensor(S.astype(np.complex64), device="cuda")
    dS = torch.full((n, n), float("nan"), dtype=torch.complex64, device="cuda")
    GX = G if inplace else torch.full_like(G, float("nan"))
    op.fourier_correction_vjp(U, F, G, St, dsymbol=dS, g_x=GX)
    S32 = S.astype(np.complex64).astype(np.complex128)
    ref_dS = np.zeros((n, n), dtype=np.complex128)
    got_gx = from_dev(op, GX, richm.F32)
    for i in range(batch):
        d, du = fourier_correction_vjp(As[i], fs[i].ravel(), us[i].ravel(), S32, gs[i].ravel())
        ref_dS += d
        assert np.linalg.norm(got_gx[i].ravel() - du) <= 1e-5 * np.linalg.norm(du)
    got_dS = dS.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got_dS - ref_dS) <= 1e-5 * np.linalg.norm(ref_dS)


def test_fourier_vjp_optional_outputs_and_errors():
    import torch
    n, batch = 16, 2
    insts = [synth.AnisoInstance(1e-2, 0.3, n)] * batch
    op = make_op(insts)
    S = torch.tensor(synth.fourier_symbol(n, seed=5).astype(np.complex64), device="cuda")
    G = to_dev(op, [synth.rhs_uniform(7, i, n) for i in range(batch)], richm.F32)
    GX = torch.zeros_like(G)
    op.fourier_correction_vjp(None, None, G, S, dsymbol=None, g_x=GX)  # no symbol gradient: x, b unused
    A = assemble_q1(n, 1e-2, 0.3)
    S32 = S.cpu().numpy().astype(np.complex128)
    for i, gx in enumerate(from_dev(op, GX, richm.F32)):
        g = synth.rhs_uniform(7, i, n).astype(np.float32).astype(np.float64).ravel()
        _, du = fourier_correction_vjp(A, np.zeros(n * n), np.zeros(n * n), S32, g)
        assert np.linalg.norm(gx.ravel() - du) <= 1e-5 * np.linalg.norm(du)
    dS = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    with pytest.raises(richm.RichmError):
        op.fourier_correction_vjp(None, None, G, S, dsymbol=dS)  # the symbol gradient needs x and b
    with pytest.raises(richm.RichmError):
        op.fourier_correction_vjp(G, G, G, S, dsymbol=dS, work=torch.empty(256, dtype=torch.uint8, device="cuda"))


def _transition(n, w=1, seed=4):
    from oracle.fourier import transition_field
    rng = np.random.default_rng(seed)
    k = 2 * w + 1
    tau = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
    tau = 0.5 * (tau + np.conj(tau[::-1, ::-1]))
    tau[w, w] = 1.0
    return transition_field(0.3 * tau, n)


@pytest.mark.parametrize("n,batch", [(33, 3), (32, 2), (1, 1)])
def test_transition_correction_and_vjp_match_oracle(n, batch):
    # the FNS correction with a banded transition T (eq. 20), forward and reverse mode
    import torch
    from oracle.fourier import fourier_correction_t, fourier_correction_t_vjp
    insts = [synth.AnisoInstance([1e-4, 1e-1, 1.0][i % 3], [np.pi / 3, 0.4, 2.5][i % 3], n) for i in range(batch)]
    op = make_op(insts)
    As = [assemble_q1(n, t.eps, t.theta) for t in insts]
    S = synth.fourier_symbol(n, seed=5)
    t = _transition(n).astype(np.float32)
    r32 = lambda a: a.astype(np.float32).astype(np.float64)
    us = [r32(0.3 * synth.rhs_uniform(8, i, n)) for i in range(batch)]
    fs = [r32(synth.rhs_uniform(9, i, n)) for i in range(batch)]
    gs = [r32(synth.rhs_uniform(7, i, n)) for i in range(batch)]
    St = torch.tensor(S.astype(np.complex64), device="cuda")
    Tt = torch.tensor(t, device="cuda")
    S32 = S.astype(np.complex64).astype(np.complex128)
    t64 = t.astype(np.float64)
    U, F = to_dev(op, us, richm.F32), to_dev(op, fs, richm.F32)
    op.fourier_correction(U, F, St, transition=Tt)
    got = from_dev(op, U, richm.F32)
    for i in range(batch):
        ref = fourier_correction_t(As[i], fs[i].ravel(), us[i].ravel(), S32, t64)
        assert np.linalg.norm(got[i].ravel() - ref) <= 1e-5 * np.linalg.norm(ref)
    U, G = to_dev(op, us, richm.F32), to_dev(op, gs, richm.F32)
    dS = torch.full((n, n), float("nan"), dtype=torch.complex64, device="cuda")
    dT = torch.full((n, n), float("nan"), dtype=torch.float32, device="cuda")
    GX = torch.full_like(G, float("nan"))
    op.fourier_correction_t_vjp(U, F, G, St, Tt, dsymbol=dS, dtransition=dT, g_x=GX)
    ref_dS = np.zeros((n, n), complex)
    ref_dT = np.zeros((n, n))
    got_gx = from_dev(op, GX, richm.F32)
    for i in range(batch):
        d, dt, du = fourier_correction_t_vjp(As[i], fs[i].ravel(), us[i].ravel(), S32, t64, gs[i].ravel())
        ref_dS += d
        ref_dT += dt
        assert np.linalg.norm(got_gx[i].ravel() - du) <= 1e-5 * np.linalg.norm(du)
    assert np.linalg.norm(dS.cpu().numpy().astype(np.complex128) - ref_dS) <= 1e-5 * np.linalg.norm(ref_dS)
    assert np.linalg.norm(dT.cpu().numpy().astype(np.float64) - ref_dT) <= 1e-5 * np.linalg.norm(ref_dT)
    # t = 1 through the transition entry points equals the plain correction's reverse mode
    ones = torch.ones((n, n), device="cuda")
    GX1, GX2 = torch.zeros_like(G), torch.zeros_like(G)
    dS1, dS2 = torch.zeros_like(dS), torch.zeros_like(dS)
    op.fourier_correction_t_vjp(U, F, G, St, ones, dsymbol=dS1, g_x=GX1)
    op.fourier_correction_vjp(U, F, G, St, dsymbol=dS2, g_x=GX2)
    assert torch.equal(GX1, GX2) and torch.equal(dS1, dS2)
