"""The sponge-layer Helmholtz operator (eq. 21) and the batched FGMRES (Sec. 3.2,
Table 9) against the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

import richm_synth as synth
from gpu_util import coef, from_dev, to_dev
from oracle.iterations import chebyshev_weights, inner_steps
from oracle.krylov import fgmres, richardson_preconditioner
from oracle.operators import assemble_helmholtz, assemble_helmholtz_sponge, gershgorin_max
from paper_2412_08076_gb300 import richm

pytestmark = pytest.mark.gpu


def _omega(N):
    # Table 9's ratio: omega / 2 pi = 10 at N = 128 (about 12.8 grid spacings per wavelength)
    return 2 * math.pi * 10 * N / 128


def _batch(specs):
    """specs: (kind, n, k) -> operator and oracle matrices"""
    op = richm.Operator([(kind, n, 1.0, 0.0, k) for kind, n, k in specs])
    mats = []
    for kind, n, k in specs:
        if kind == richm.HELMHOLTZ_FD5_SPONGE:
            mats.append(assemble_helmholtz_sponge(n, k))
        else:
            mats.append(assemble_helmholtz(n, k, absorbing=kind == richm.HELMHOLTZ_FD5_ABC))
    return op, mats


def _rhs(specs, seed):
    out = []
    for i, (_, n, _) in enumerate(specs):
        out.append(synth.rhs_uniform(seed, i, n) + 1j * synth.rhs_uniform(seed + 1, i, n))
    return out


SPECS = [(richm.HELMHOLTZ_FD5_SPONGE, 31, _omega(32)), (richm.HELMHOLTZ_FD5_SPONGE, 63, _omega(64)),
         (richm.HELMHOLTZ_FD5_ABC, 40, 20.0), (richm.HELMHOLTZ_FD5_DIRICHLET, 17, 9.0),
         (richm.HELMHOLTZ_FD5_SPONGE, 1, 30.0), (richm.HELMHOLTZ_FD5_SPONGE, 100, _omega(101))]


@pytest.mark.parametrize("dtype", [richm.C128, richm.C64])
def test_sponge_residual_and_sweeps_match_oracle(dtype):
    op, mats = _batch(SPECS)
    xs, bs = _rhs(SPECS, 10), _rhs(SPECS, 12)
    X, B = to_dev(op, xs, dtype), to_dev(op, bs, dtype)
    R = op.zeros(dtype)
    rn, bn, rel = op.residual_norm(dtype, X, B, r_out=R)
    rs = from_dev(op, R, dtype)
    tol = 1e-12 if dtype == richm.C128 else 1e-5
    for i, A in enumerate(mats):
        xi = xs[i].ravel().astype(np.complex64 if dtype == richm.C64 else np.complex128).astype(np.complex128)
        bi = bs[i].ravel().astype(np.complex64 if dtype == richm.C64 else np.complex128).astype(np.complex128)
        r = bi - A @ xi
        assert np.abs(rs[i].ravel() - r).max() <= tol * np.abs(r).max()
        assert abs(rn[i].item() - np.linalg.norm(r)) <= 1e-12 * np.linalg.norm(r) + (0 if dtype == richm.C128 else
                                                                                     1e-6 * np.linalg.norm(r))
    # eight Jacobi-preconditioned NAG sweeps (one sweep per launch for the sponge layer)
    m = 4
    G = np.array(op.gershgorin())
    for i, A in enumerate(mats):
        assert abs(G[i] - gershgorin_max(A)) <= 1e-12 * G[i]
    w = np.stack([np.array([0.2, 0.5, 0.35, 0.6]) for _ in SPECS])
    a = np.full_like(w, 0.3)
    X = op.zeros(dtype)
    XP = op.zeros(dtype)
    op.apply_sweeps(dtype, X, XP, B, coef(w, dtype), coef(a, dtype), None, K=8, m=m, precond=1)
    got = from_dev(op, X, dtype)
    for i, A in enumerate(mats):
        bi = bs[i].ravel().astype(np.complex64 if dtype == richm.C64 else np.complex128).astype(np.complex128)
        d = A.diagonal()
        ref, _ = inner_steps(A, bi, np.zeros_like(bi), None, w[i], a[i], K=8, Binv=lambda r, d=d: r / d)
        assert np.abs(got[i].ravel() - ref).max() <= (1e-12 if dtype == richm.C128 else 1e-5) * np.abs(ref).max()


def _smoother(G, m=5, beta=0.3):
    # the upper part of the spectrum, [G/4, G], damped by Chebyshev weights (eqs. 8-9)
    w = np.stack([chebyshev_weights(g, g / 4.0, m) for g in G])
    return w, np.full_like(w, beta)


def test_fgmres_follows_the_oracle_iteration():
    # complex128 smoother: the same iteration as the oracle's (modified Gram-Schmidt
    # there, classical Gram-Schmidt twice here); 12 Arnoldi steps with restart 5
    op, mats = _batch(SPECS)
    bs = _rhs(SPECS, 20)
    x0 = [0.01 * v for v in _rhs(SPECS, 22)]
    G = np.array(op.gershgorin())
    w, a = _smoother(G)
    B, X = to_dev(op, bs, richm.C128), to_dev(op, x0, richm.C128)
    st, info = op.fgmres(B, X, coef(w, richm.C128), coef(a, richm.C128), None, restart=5, tol=0.0, max_iters=12,
                         sweeps=5, inner=richm.C128)
    assert st == richm.ERR_NOT_CONVERGED
    got = from_dev(op, X, richm.C128)
    for i, A in enumerate(mats):
        M = richardson_preconditioner(A, w[i], a[i], K=5)
        ref, its, est = fgmres(A, bs[i].ravel(), x0[i].ravel(), M, m=5, tol=0.0, max_iters=12)
        # the one-unknown instance breaks down (|w| = 0) after every first step: its
        # count depends on when its residual rounds to zero; every other takes 12 steps
        assert info[i][0] == 12 or SPECS[i][1] == 1
        err = np.abs(got[i].ravel() - ref).max() / np.abs(ref).max()
        assert err <= 1e-9, (i, err)
        rel = np.linalg.norm(bs[i].ravel() - A @ got[i].ravel()) / np.linalg.norm(bs[i])
        assert abs(info[i][1] - rel) <= 1e-10 * rel


def test_fgmres_mixed_precision_solves_to_tolerance():
    # complex64 smoother, complex128 basis and iterate: every instance to 1e-9, the
    # residual recomputed by the oracle
    op, mats = _batch(SPECS)
    bs = _rhs(SPECS, 30)
    G = np.array(op.gershgorin())
    w, a = _smoother(G)
    B, X = to_dev(op, bs, richm.C128), op.zeros(richm.C128)
    st, info = op.fgmres(B, X, coef(w, richm.C64), coef(a, richm.C64), None, restart=20, tol=1e-9, max_iters=5000,
                         sweeps=5, inner=richm.C64)
    assert st == richm.OK, info
    got = from_dev(op, X, richm.C128)
    for i, A in enumerate(mats):
        rel = np.linalg.norm(bs[i].ravel() - A @ got[i].ravel()) / np.linalg.norm(bs[i])
        assert rel <= 1e-9 * (1 + 1e-6), (i, rel)
        assert abs(info[i][1] - rel) <= 1e-6 * rel


def test_fgmres_without_preconditioner_is_gmres():
    op, mats = _batch(SPECS[:3])
    bs = _rhs(SPECS[:3], 40)
    B, X = to_dev(op, bs, richm.C128), op.zeros(richm.C128)
    st, info = op.fgmres(B, X, None, None, None, restart=7, tol=0.0, max_iters=14, sweeps=0, inner=richm.C128)
    got = from_dev(op, X, richm.C128)
    for i, A in enumerate(mats):
        ref, its, est = fgmres(A, bs[i].ravel(), None, None, m=7, tol=0.0, max_iters=14)
        assert np.abs(got[i].ravel() - ref).max() <= 1e-9 * np.abs(ref).max()


def test_fgmres_complex64_basis_solves_to_tolerance():
    # complex64 smoother and Arnoldi basis (the cycles on the FP32 pipe), complex128
    # iterate and restart residual: every instance to 1e-9 against the oracle's
    # recomputed residual, in about as many steps as with the complex128 basis
    op, mats = _batch(SPECS)
    bs = _rhs(SPECS, 30)
    G = np.array(op.gershgorin())
    w, a = _smoother(G)
    B = to_dev(op, bs, richm.C128)
    its = {}
    for basis in (richm.C128, richm.C64):
        X = op.zeros(richm.C128)
        st, info = op.fgmres(B, X, coef(w, richm.C64), coef(a, richm.C64), None, restart=20, tol=1e-9,
                             max_iters=5000, sweeps=5, inner=richm.C64, basis=basis)
        assert st == richm.OK, info
        got = from_dev(op, X, richm.C128)
        for i, A in enumerate(mats):
            rel = np.linalg.norm(bs[i].ravel() - A @ got[i].ravel()) / np.linalg.norm(bs[i])
            assert rel <= 1e-9 * (1 + 1e-6), (basis, i, rel)
            assert abs(info[i][1] - rel) <= 1e-6 * rel
        its[basis] = [i_ for i_, _, _ in info]
    print(f"\nFGMRES(20) to 1e-9, Arnoldi steps: complex128 basis {its[richm.C128]}, complex64 basis {its[richm.C64]}")
    for i128, i64 in zip(its[richm.C128], its[richm.C64]):
        assert i64 <= 1.15 * i128 + 20, (i128, i64)


def test_fgmres_basis_option_is_checked():
    op, mats = _batch(SPECS[:2])
    B, X = op.zeros(richm.C128), op.zeros(richm.C128)
    w = coef(np.full((2, 5), 1e-4), richm.C128)
    with pytest.raises(richm.RichmError):  # a complex64 basis needs the complex64 smoother
        op.fgmres(B, X, w, None, None, sweeps=5, m=5, inner=richm.C128, basis=richm.C64)
    with pytest.raises(richm.RichmError):
        op.fgmres(B, X, w, None, None, sweeps=5, m=5, inner=richm.C128, basis=richm.F32)


@pytest.mark.parametrize("K", [8, 6])
def test_sponge_fused_complex64_sweeps_match_oracle(K):
    # the fused complex64 kernel with the sponge layer's per-node diagonal: passes of four
    # sweeps (K = 6: one pass and two single sweeps), no preconditioner, against the
    # oracle's eq. 21 matrix; the one-sweep kernel agrees with it to FP32 rounding
    op, mats = _batch(SPECS)
    bs = _rhs(SPECS, 14)
    B = to_dev(op, bs, richm.C64)
    G = np.array(op.gershgorin())
    w = np.stack([np.array([0.3, 0.7, 0.5, 0.9]) / g for g in G])
    a = np.full_like(w, 0.3)
    out = {}
    for fuse in (4, 1):
        X, XP = op.zeros(richm.C64), op.zeros(richm.C64)
        op.apply_sweeps(richm.C64, X, XP, B, coef(w, richm.C64), coef(a, richm.C64), None, K=K, m=4, fuse=fuse)
        out[fuse] = from_dev(op, X, richm.C64)
    for i, A in enumerate(mats):
        bi = bs[i].ravel().astype(np.complex64).astype(np.complex128)
        ref, _ = inner_steps(A, bi, np.zeros_like(bi), None, w[i].astype(np.float32).astype(np.float64),
                             a[i].astype(np.float32).astype(np.float64), K=K)
        scale = np.abs(ref).max()
        assert np.abs(out[4][i].ravel() - ref).max() <= 1e-5 * scale, (i, np.abs(out[4][i].ravel() - ref).max())
        assert np.abs(out[4][i] - out[1][i]).max() <= 1e-5 * scale
