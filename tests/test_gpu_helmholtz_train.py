"""Differentiation of complex (Helmholtz) sweeps: the log-residual loss with its A^H
gradient and the complex adjoint against the FP64 oracle and central differences,
and the log-omega training of the NAG-Richardson(m) smoother used as the FGMRES
preconditioner (Sec. 3.2)."""
import math

import numpy as np
import pytest
import torch

import richm_synth as synth
from gpu_util import coef, from_dev, to_dev
from oracle.operators import assemble_helmholtz, assemble_helmholtz_sponge
from oracle.training import loss_and_grads_general
from paper_2412_08076_gb300 import richm

pytestmark = pytest.mark.gpu


def _omega(N):
    return 2 * math.pi * 10 * N / 128


SPECS = [(richm.HELMHOLTZ_FD5_SPONGE, 31, _omega(32)), (richm.HELMHOLTZ_FD5_ABC, 20, 15.0),
         (richm.HELMHOLTZ_FD5_SPONGE, 70, _omega(71)), (richm.HELMHOLTZ_FD5_DIRICHLET, 9, 7.0),
         (richm.HELMHOLTZ_FD5_SPONGE, 1, 20.0)]


def _setup(specs=SPECS, m=4, seed=5, single=False):
    op = richm.Operator([(kind, n, 1.0, 0.0, k) for kind, n, k in specs])
    mats = []
    for kind, n, k in specs:
        if kind == richm.HELMHOLTZ_FD5_SPONGE:
            mats.append(assemble_helmholtz_sponge(n, k).tocsr())
        else:
            mats.append(assemble_helmholtz(n, k, absorbing=kind == richm.HELMHOLTZ_FD5_ABC).tocsr())
    G = np.array(op.gershgorin())
    rng = np.random.default_rng(seed)
    B = len(specs)
    w = rng.uniform(0.3, 1.2, (B, m)) / G[:, None]
    a = rng.uniform(0.1, 0.4, (B, m))
    at = rng.uniform(0.0, 0.5, (B, m))
    fs = [synth.rhs_uniform(seed, i, n) + 1j * synth.rhs_uniform(seed + 1, i, n) for i, (_, n, _) in enumerate(specs)]
    x0 = [0.1 * (synth.rhs_uniform(seed + 2, i, n) - 0.5j * synth.rhs_uniform(seed + 3, i, n))
          for i, (_, n, _) in enumerate(specs)]
    if single:
        fs = [v.astype(np.complex64).astype(np.complex128) for v in fs]
        x0 = [v.astype(np.complex64).astype(np.complex128) for v in x0]
        w, a, at = (v.astype(np.float32).astype(np.float64) for v in (w, a, at))
    return op, mats, w, a, at, fs, x0


def _gpu_grads(op, dtype, x0, fs, w, a, at, m, K, every):
    X0 = to_dev(op, x0, dtype)
    B = to_dev(op, fs, dtype)
    W = coef(w, dtype)
    A_ = None if a is None else coef(a, dtype)
    AT = None if at is None else coef(at, dtype)
    ck = torch.zeros(op.checkpoint_elems(K, every), dtype=richm.TORCH_DTYPE[dtype], device="cuda")
    XK = op.zeros(dtype)
    op.forward_checkpointed(dtype, X0, B, W, A_, AT, m, K, every, 0, ck, XK)
    gK = op.zeros(dtype)
    loss = op.loss_log_residual(dtype, XK, B, gK)
    gw = torch.zeros_like(W)
    ga = None if a is None else torch.zeros_like(W)
    gat = None if at is None else torch.zeros_like(W)
    gx0 = op.zeros(dtype)
    op.sweeps_adjoint(dtype, ck, every, B, gK, W, A_, AT, m, K, 0, gw, ga, gat, gx0)
    return (loss.item(), gw.cpu().numpy(), None if ga is None else ga.cpu().numpy(),
            None if gat is None else gat.cpu().numpy(), from_dev(op, gx0, dtype))


def _close(got, ref, rtol):
    ref = np.asarray(ref)
    np.testing.assert_allclose(got, ref, rtol=rtol, atol=rtol * np.abs(ref).max())


@pytest.mark.parametrize("method", ["nagex", "nag", "richardson"])
@pytest.mark.parametrize("every", [1, 4, 12])
def test_complex128_adjoint_matches_oracle(method, every):
    op, mats, w, a, at, fs, x0 = _setup()
    m, K = 4, 12
    a_ = None if method == "richardson" else a
    at_ = at if method == "nagex" else None
    L, gw, ga, gat, gx0 = _gpu_grads(op, richm.C128, x0, fs, w, a_, at_, m, K, every)
    Lo, gwo, gao, gato, gxo = loss_and_grads_general(mats, [f.ravel() for f in fs], [x.ravel() for x in x0], w, a_,
                                                     at_, K)
    assert abs(L - Lo) <= 1e-12 * abs(Lo)
    _close(gw, gwo, 1e-9)
    if method == "nag":
        _close(ga, gao, 1e-9)  # the at-gradient is folded into alpha's (at = a)
    if method == "nagex":
        _close(ga, gao, 1e-9)
        _close(gat, gato, 1e-9)
    for i in range(len(mats)):
        _close(gx0[i].ravel(), gxo[i], 1e-8)


def test_complex64_adjoint_close_to_oracle():
    op, mats, w, a, at, fs, x0 = _setup(single=True)
    m, K = 4, 12
    L, gw, ga, gat, gx0 = _gpu_grads(op, richm.C64, x0, fs, w, a, at, m, K, 4)
    Lo, gwo, gao, gato, gxo = loss_and_grads_general(mats, [f.ravel() for f in fs], [x.ravel() for x in x0], w, a,
                                                     at, K)
    assert abs(L - Lo) <= 1e-5 * abs(Lo)
    _close(gw, gwo, 2e-3)
    _close(ga, gao, 2e-3)
    _close(gat, gato, 2e-3)


def test_complex_adjoint_matches_central_differences():
    # the FP64 complex adjoint within 1e-6 relative of central differences of the
    # library's own forward loss, for weights and the real and imaginary parts of x0
    specs = [(richm.HELMHOLTZ_FD5_SPONGE, 31, _omega(32)), (richm.HELMHOLTZ_FD5_ABC, 24, 12.0)]
    op, mats, w, a, at, fs, x0 = _setup(specs)
    m, K, every = 4, 16, 8
    L, gw, ga, gat, gx0 = _gpu_grads(op, richm.C128, x0, fs, w, a, at, m, K, every)

    def loss_of(w_, a_, at_, x0_):
        return _gpu_grads(op, richm.C128, x0_, fs, w_, a_, at_, m, K, every)[0]

    def fd(loss_at, g, h):
        d1 = (loss_at(h) - loss_at(-h)) / (2 * h)
        d2 = (loss_at(h / 2) - loss_at(-h / 2)) / h
        rx = (4 * d2 - d1) / 3
        scale = max(abs(rx), 1e-3)
        assert abs(g - rx) <= 1e-6 * scale, (g, rx, d1)

    for b in range(2):
        for i in (0, 3):
            for name, arr, g in (("w", w, gw), ("a", a, ga), ("at", at, gat)):
                h = 1e-4 * abs(arr[b, i])

                def loss_at(d, name=name, arr=arr, b=b, i=i):
                    p = arr.copy()
                    p[b, i] += d
                    kw = dict(w_=w, a_=a, at_=at, x0_=x0)
                    kw[name + "_"] = p
                    return loss_of(**kw)
                fd(loss_at, g[b, i], h)
        for (r, c) in ((3, 4), (10, 7)):
            for unit in (1.0, 1j):
                def loss_at(d, b=b, r=r, c=c, unit=unit):
                    xp = [x.copy() for x in x0]
                    xp[b][r, c] += d * unit
                    return loss_of(w, a, at, xp)
                comp = gx0[b][r, c].real if unit == 1.0 else gx0[b][r, c].imag
                fd(loss_at, comp, 1e-4)


def test_complex_dtype_refuses_preconditioners():
    op, mats, w, a, at, fs, x0 = _setup()
    X0 = to_dev(op, x0, richm.C128)
    ck = torch.zeros(op.checkpoint_elems(4, 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(richm.RichmError):
        op.forward_checkpointed(richm.C128, X0, X0, coef(w, richm.C128), None, None, 4, 4, 4, 1, ck, op.zeros(
            richm.C128))


def test_meta_omega_training_lowers_the_preconditioner_loss():
    # Algorithm 1 for the Helmholtz smoother: the meta network's log-weights and momentum
    # trained on the complex adjoint lower the log residual of the preconditioner
    # (5 NAG sweeps from zero) on fresh right-hand sides; FGMRES(20) preconditioned by the
    # initial and by the trained smoother is run on point sources at N = 128
    from paper_2412_08076_gb300 import helmholtz as hz
    specs = [(richm.HELMHOLTZ_FD5_SPONGE, N - 1, _omega(N)) for N in (64, 128) for _ in range(2)]
    net = hz.SmootherNet(m=5, K=5)
    N = 128
    ev = [(richm.HELMHOLTZ_FD5_SPONGE, N - 1, _omega(N))] * 4
    op = richm.Operator([(kind, n, 1.0, 0.0, k) for kind, n, k in ev])
    X = torch.tensor(hz.instance_inputs(ev), device="cuda")
    G = torch.tensor(np.array(op.gershgorin()), dtype=torch.float32, device="cuda")
    src = np.zeros((4, (N - 1) ** 2), np.complex128)
    for s_, (i, j) in enumerate(synth.point_sources(N - 1, 4, seed=6)):
        src[s_, i * (N - 1) + j] = 1.0
    Bp = op.pack(torch.tensor(src.ravel(), device="cuda"), richm.C128)

    def fgmres_its():
        w, a, _ = net.coefficients(X, G)
        Xs = op.zeros(richm.C128)
        st, info = op.fgmres(Bp, Xs, w, a, None, restart=20, tol=1e-6, max_iters=3000, m=5, sweeps=5,
                             inner=richm.C64)
        assert st == richm.OK
        return [i_ for i_, _, _ in info]

    Bv = hz.random_rhs(op, ev, 900)
    loss0 = float(net.loss_and_grads(op, X, G, Bv)[0].item())
    its0 = fgmres_its()
    hist = hz.train(net, specs, steps=100, lr=3e-3)
    assert np.all(np.isfinite(hist))
    loss1 = float(net.loss_and_grads(op, X, G, Bv)[0].item())
    its1 = fgmres_its()
    print(f"\nmeta-omega (NAG-Richardson(5), Helmholtz with sponge): training loss {hist[0]:.3f} -> "
          f"{hist[-1]:.3f}; held-out loss at N = 128 {loss0:.3f} -> {loss1:.3f}; FGMRES(20) iterations "
          f"{its0} -> {its1}")
    assert np.mean(hist[-10:]) < np.mean(hist[:10]) - 0.02
    assert loss1 < loss0
