"""SSOR-preconditioned sweeps (eq. 17 with the SSOR preconditioner) against the FP64 oracle."""
import math

import numpy as np
import pytest

import richm_synth as synth
from gpu_util import coef, from_dev, make_op, to_dev
from oracle.iterations import inner_steps, ssor_binv
from oracle.operators import assemble_q1
from paper_2412_08076_gb300 import richm

pytestmark = pytest.mark.gpu

# one and several row chunks (512 columns per chunk in FP32, 256 in FP64), ragged sizes;
# a batch whose rows all fit one chunk runs the register-resident row kernels, any wider
# instance sends the whole batch through the chunked kernels
SIZES = [1, 2, 3, 5, 17, 31, 64, 130, 255, 300, 513]
SIZES_ONE_CHUNK = {"f32": [1, 2, 5, 31, 64, 130, 300, 511], "f64": [1, 2, 5, 31, 64, 130, 255]}


def _instances(seed, sizes):
    u = synth.uniform(synth.stream_key(seed), 2 * len(sizes))
    return [synth.AnisoInstance(10 ** (-6 * u[2 * i]), math.pi * u[2 * i + 1], n) for i, n in enumerate(sizes)]


def _case(dtype, variant, relax, K, k_start=2, sizes=SIZES, wscale=1.0):
    insts = _instances(21, sizes)
    op = make_op(insts)
    m = 3
    # B^{-1} A has its spectrum in (0, 1]: weights of order 1 (wscale > 1: larger steps)
    w = np.tile(wscale * np.array([0.9, 1.3, 0.7]), (len(insts), 1))
    a = np.tile(np.array([0.2, 0.35, 0.1]), (len(insts), 1))
    at = None
    if variant == "richardson":
        a = None
    elif variant == "nagex":
        at = np.tile(np.array([0.5, 0.0, 0.3]), (len(insts), 1))
    x0 = [0.5 * synth.rhs_uniform(41, i, t.n) for i, t in enumerate(insts)]
    xp0 = [x - 0.05 * synth.rhs_uniform(42, i, t.n) for i, (x, t) in enumerate(zip(x0, insts))]
    bs = [synth.rhs_uniform(43, i, t.n) for i, t in enumerate(insts)]
    if dtype == richm.F32:
        rnd = lambda v: None if v is None else np.asarray(v, dtype=np.float32).astype(np.float64)
        x0 = [rnd(v) for v in x0]
        xp0 = [rnd(v) for v in xp0]
        bs = [rnd(v) for v in bs]
        w, a, at = rnd(w), rnd(a), rnd(at)
        relax = float(np.float32(relax))
    X = to_dev(op, x0, dtype)
    XP = to_dev(op, xp0, dtype)
    B = to_dev(op, bs, dtype)
    op.apply_sweeps(dtype, X, XP if a is not None else None, B, coef(w, dtype),
                    None if a is None else coef(a, dtype), None if at is None else coef(at, dtype),
                    K=K, m=m, k_start=k_start, precond=2, relax=relax)
    got = from_dev(op, X, dtype)
    gotp = from_dev(op, XP, dtype) if a is not None else None
    out = []
    for i, t in enumerate(insts):
        A = assemble_q1(t.n, t.eps, t.theta)
        v0 = None if a is None else (x0[i] - xp0[i]).ravel()
        ref, refv = inner_steps(A, bs[i].ravel(), x0[i].ravel(), v0, w[i], None if a is None else a[i],
                                None if at is None else at[i], K=K, k_start=k_start, Binv=ssor_binv(A, relax))
        out.append((t, got[i].ravel(), ref, None if gotp is None else gotp[i].ravel(), ref - refv))
    return out


@pytest.mark.parametrize("variant", ["richardson", "nag", "nagex"])
@pytest.mark.parametrize("relax", [1.0, 1.6])
@pytest.mark.parametrize("chunks", ["one", "several"])
def test_fp64_ssor_sweeps_match_oracle(variant, relax, chunks):
    sizes = SIZES_ONE_CHUNK["f64"] if chunks == "one" else SIZES
    for t, g, ref, gp, refp in _case(richm.F64, variant, relax, K=3, sizes=sizes):
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(g - ref).max() <= 1e-12 * scale, (t, np.abs(g - ref).max() / scale)
        if gp is not None:
            assert np.abs(gp - refp).max() <= 1e-12 * max(np.abs(refp).max(), 1e-300)


@pytest.mark.parametrize("variant", ["richardson", "nag"])
@pytest.mark.parametrize("chunks", ["one", "several"])
def test_fp32_ssor_sweeps_within_1e5(variant, chunks):
    # damping weights (every mode of B^{-1} A contracts), two sweeps from the same
    # FP32-rounded state: FP32 rounding of the two triangular solves stays ~1e-6 relative
    sizes = SIZES_ONE_CHUNK["f32"] if chunks == "one" else SIZES
    for t, g, ref, gp, refp in _case(richm.F32, variant, 1.2, K=2, wscale=0.7, sizes=sizes):
        scale = max(np.abs(ref).max(), 1.0)
        assert np.abs(g - ref).max() <= 1e-5 * scale, (t, np.abs(g - ref).max() / scale)


def test_ssor_sweep_leaves_padding_zero_and_rejects_bad_arguments():
    insts = _instances(22, [31, 100])
    op = make_op(insts)
    X, XP, B = op.zeros(richm.F64), op.zeros(richm.F64), op.zeros(richm.F64)
    B.copy_(to_dev(op, [np.ones((t.n, t.n)) for t in insts], richm.F64))
    w = coef(np.ones((2, 3)), richm.F64)
    a = coef(np.full((2, 3), 0.2), richm.F64)
    op.apply_sweeps(richm.F64, X, XP, B, w, a, K=4, m=3, precond=2, relax=1.3)
    host = X.cpu().numpy()
    for b_, t in enumerate(insts):
        lay = op.layout(b_)
        blk = host[lay.offset:lay.offset + lay.rows * lay.pitch].reshape(lay.rows, lay.pitch)
        assert np.all(blk[0] == 0) and np.all(blk[-1] == 0) and np.all(blk[:, t.n:] == 0)
        assert np.abs(blk[1:-1, :t.n]).max() > 0
    for bad in (0.0, 2.0, -0.5):
        with pytest.raises(richm.RichmError):
            op.apply_sweeps(richm.F64, X, XP, B, w, a, K=1, m=3, precond=2, relax=bad)


def _paper_instances(sizes, theta=math.pi / 10, eps=1e-6):
    return [synth.AnisoInstance(eps, theta, n) for n in sizes]


@pytest.mark.parametrize("inner", [richm.F32, richm.F64])
def test_ssor_preconditioned_solve_to_1e10_checked_by_oracle(inner):
    # eps = 1e-6, theta = pi/10 (the setting of the paper's SSOR tables); B^{-1} A has its
    # spectrum in (0, 1], so the momentum-aware Chebyshev weights take the bound 1
    from gpu_util import nag_weights
    insts = _paper_instances([15, 31, 63])
    op = make_op(insts)
    w, a = nag_weights(np.ones(len(insts)), 16, beta=0.3)
    bs = [synth.rhs_uniform(44, i, t.n) for i, t in enumerate(insts)]
    B = to_dev(op, bs, richm.F64)
    X = op.zeros(richm.F64)
    opts = op.solve_opts(16, tol=1e-10, max_sweeps=200000, refine_every=64, inner=inner, precond=2, fuse=1,
                         relax=1.0)
    st, info = op.solve(B, X, coef(w, inner), coef(a, inner), None, opts)
    assert st == richm.OK, info
    xs = from_dev(op, X, richm.F64)
    for i, t in enumerate(insts):
        A = assemble_q1(t.n, t.eps, t.theta)
        r = np.linalg.norm(bs[i].ravel() - A @ xs[i].ravel()) / np.linalg.norm(bs[i])
        assert r <= 1e-10, (t, r)
        assert abs(info[i][1] - r) <= 1e-3 * r + 1e-14


def test_ssor_needs_fewer_sweeps_than_jacobi():
    # the same NAG(16) weight construction on each preconditioned spectrum: (0, 1] for
    # SSOR, (0, G / d] for Jacobi (d the diagonal, G the Gershgorin bound)
    from gpu_util import nag_weights
    insts = _paper_instances([31, 63])
    op = make_op(insts)
    G = np.array(op.gershgorin())
    d = np.array([op.stencil(i)[0] for i in range(len(insts))])
    bs = [synth.rhs_uniform(45, i, t.n) for i, t in enumerate(insts)]
    B = to_dev(op, bs, richm.F64)
    sweeps = {}
    for pc, bound in ((1, G / d), (2, np.ones(len(insts)))):
        w, a = nag_weights(bound, 16, beta=0.3)
        X = op.zeros(richm.F64)
        opts = op.solve_opts(16, tol=1e-8, max_sweeps=400000, refine_every=64, inner=richm.F64, precond=pc, fuse=1,
                             relax=1.0)
        st, info = op.solve(B, X, coef(w, richm.F64), coef(a, richm.F64), None, opts)
        assert st == richm.OK, (pc, info)
        sweeps[pc] = [s for s, _, _ in info]
    assert all(s2 < s1 for s1, s2 in zip(sweeps[1], sweeps[2])), sweeps
