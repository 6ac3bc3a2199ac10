"""GPU sweeps (Table 1 iterations, eq. 17) against the FP64 oracle, element by element."""
import math

import numpy as np
import pytest
import torch

import richm_synth as synth
from gpu_util import coef, fp32_bound, from_dev, make_op, nag_weights, period_amplification, to_dev
from oracle.iterations import inner_steps, jacobi_binv
from oracle.operators import assemble_helmholtz, assemble_q1, gershgorin_max, helmholtz_wavenumber
from paper_2412_08076_gb300 import richm

pytestmark = pytest.mark.gpu

# sizes spanning one / several warp tiles, ragged row blocks and column blocks
SIZES = [1, 2, 3, 5, 8, 17, 31, 63, 64, 70, 127, 130]


def _instances(seed=11, sizes=SIZES):
    u = synth.uniform(synth.stream_key(seed), 2 * len(sizes))
    return [synth.AnisoInstance(10 ** (-3 * u[2 * i]), math.pi * u[2 * i + 1], n) for i, n in enumerate(sizes)]


def _run_case(dtype, variant, K, k_start=0, precond=0, sizes=SIZES, fuse=0, rows=None):
    insts = _instances(sizes=sizes)
    op = make_op(insts)
    if rows is not None:
        op.set_tuning(fuse, rows)
    m = 6
    As = [assemble_q1(t.n, t.eps, t.theta) for t in insts]
    G = np.array([gershgorin_max(A) for A in As])
    w, a = nag_weights(G, m, beta=0.25)
    at = None
    if variant == "richardson":
        a = None
    elif variant == "mom":
        at = np.zeros_like(a)
    elif variant == "nagex":
        at = a * 0.5 + 0.1
    if precond:
        d = np.array([A.diagonal()[0] for A in As])
        w = w * d[:, None]  # B^{-1} = D^{-1}: the weights act on D^{-1} r
    x0 = [0.5 * synth.rhs_uniform(31, i, t.n) for i, t in enumerate(insts)]
    v0 = [0.05 * synth.rhs_uniform(32, i, t.n) for i, t in enumerate(insts)]
    bs = [synth.rhs_uniform(33, i, t.n) for i, t in enumerate(insts)]
    if dtype == richm.F32:  # both sides start from the same FP32-rounded state
        x0 = [v.astype(np.float32).astype(np.float64) for v in x0]
        v0 = [v.astype(np.float32).astype(np.float64) for v in v0]
        bs = [v.astype(np.float32).astype(np.float64) for v in bs]
        w = w.astype(np.float32).astype(np.float64)
        a = None if a is None else a.astype(np.float32).astype(np.float64)
        at = None if at is None else at.astype(np.float32).astype(np.float64)
    xprev0 = [x - v for x, v in zip(x0, v0)]
    if dtype == richm.F32:
        xprev0 = [v.astype(np.float32).astype(np.float64) for v in xprev0]
        v0 = [x - p for x, p in zip(x0, xprev0)]
    X = to_dev(op, x0, dtype)
    XP = to_dev(op, xprev0, dtype)
    B = to_dev(op, bs, dtype)
    op.apply_sweeps(dtype, X, XP if a is not None else None, B, coef(w, dtype),
                    None if a is None else coef(a, dtype), None if at is None else coef(at, dtype),
                    K=K, m=m, k_start=k_start, precond=precond, fuse=fuse)
    got = from_dev(op, X, dtype)
    gotp = from_dev(op, XP, dtype) if a is not None else None
    out = []
    for i, t in enumerate(insts):
        Binv = jacobi_binv(As[i]) if precond else None
        wi = w[i] / As[i].diagonal()[0] if precond else w[i]
        ref, refv = inner_steps(As[i], bs[i].ravel(), x0[i].ravel(), None if a is None else v0[i].ravel(), w[i],
                                None if a is None else a[i], None if at is None else at[i], K=K,
                                k_start=k_start, Binv=Binv)
        out.append((got[i].ravel(), ref, None if gotp is None else gotp[i].ravel(), ref - refv,
                    w[i] if not precond else wi, None if a is None else a[i], None if at is None else at[i], G[i]))
    return out


@pytest.mark.parametrize("variant", ["richardson", "nag", "mom", "nagex"])
@pytest.mark.parametrize("precond", [0, 1])
def test_fp64_sweeps_match_oracle(variant, precond):
    for g, ref, gp, refp, *_ in _run_case(richm.F64, variant, K=13, k_start=4, precond=precond):
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(g - ref).max() <= 1e-12 * scale
        if gp is not None:
            assert np.abs(gp - refp).max() <= 1e-12 * max(np.abs(refp).max(), 1e-300)


def test_fp64_zero_sweeps_is_noop():
    insts = _instances(sizes=[5, 40])
    op = make_op(insts)
    x0 = [synth.rhs_uniform(1, i, t.n) for i, t in enumerate(insts)]
    X = to_dev(op, x0, richm.F64)
    op.apply_sweeps(richm.F64, X, None, X.clone(), coef(np.ones((2, 3)), richm.F64), K=0, m=3)
    for g, r in zip(from_dev(op, X, richm.F64), x0):
        np.testing.assert_array_equal(g, r)


def _fp32_bound(w, a, at, G, k_start, K, xmax, bmax):
    return fp32_bound(w, a, at, G, k_start, K, xmax, bmax)


@pytest.mark.parametrize("variant", ["richardson", "nag", "nagex"])
def test_fp32_block_matches_oracle(variant):
    # one fused block of 8 sweeps from the same FP32-rounded state
    K, k_start = 8, 2
    worst = 0.0
    for g, ref, gp, refp, w, a, at, G in _run_case(richm.F32, variant, K=K, k_start=k_start):
        xmax = max(np.abs(ref).max(), 1.0)
        err = np.abs(g - ref).max()
        bound = _fp32_bound(w, a, at, G, k_start, K, xmax, 1.0)
        assert err <= bound, (err, bound)
        worst = max(worst, err / xmax)
    print(f"worst FP32 block error (rel. to max|x|): {worst:.2e}")


def test_fp32_block_mild_weights_within_1e5():
    # weights with |1 - w lambda| <= 1 on the spectrum: no mode is amplified, so the
    # FP32 block stays within 1e-5 of max|x| (the FP32 sweep tolerance)
    insts = _instances(sizes=[31, 63, 127, 130])
    op = make_op(insts)
    As = [assemble_q1(t.n, t.eps, t.theta) for t in insts]
    G = np.array([gershgorin_max(A) for A in As])
    m, K = 4, 16
    w = np.outer(1.0 / G, [0.4, 0.7, 1.0, 1.3]).astype(np.float32).astype(np.float64)
    a = np.full_like(w, 0.25).astype(np.float32).astype(np.float64)
    x0 = [synth.rhs_uniform(41, i, t.n).astype(np.float32).astype(np.float64) for i, t in enumerate(insts)]
    bs = [synth.rhs_uniform(42, i, t.n).astype(np.float32).astype(np.float64) for i, t in enumerate(insts)]
    X = to_dev(op, x0, richm.F32)
    XP = to_dev(op, x0, richm.F32)
    B = to_dev(op, bs, richm.F32)
    op.apply_sweeps(richm.F32, X, XP, B, coef(w, richm.F32), coef(a, richm.F32), None, K=K, m=m)
    for i, g in enumerate(from_dev(op, X, richm.F32)):
        ref, _ = inner_steps(As[i], bs[i].ravel(), x0[i].ravel(), None, w[i], a[i], K=K)
        rel = np.linalg.norm(g.ravel() - ref) / np.linalg.norm(ref)
        assert rel <= 1e-5, rel


@pytest.mark.parametrize("dtype", [richm.C128, richm.C64])
def test_helmholtz_sweeps_match_oracle(dtype):
    sizes = [1, 3, 9, 33, 64, 100]
    insts = [synth.AnisoInstance(1.0, 0.0, n) for n in sizes]
    ks = [helmholtz_wavenumber(n) for n in sizes]
    # one operator per k (k is per instance in the library; the oracle assembles each)
    op = richm.Operator([(richm.HELMHOLTZ_FD5_ABC, n, 1.0, 0.0, k) for n, k in zip(sizes, ks)])
    m, K = 8, 12
    ws = np.stack([synth.helmholtz_weights(m, 1.0 / (n + 1), seed=4) for n in sizes])
    a = np.full_like(ws, 0.3)
    x0 = [0.1 * (synth.rhs_uniform(51, i, n) + 1j * synth.rhs_uniform(52, i, n)) for i, n in enumerate(sizes)]
    bs = [synth.point_source_rhs(n, 1, seed=5 + i)[0] for i, n in enumerate(sizes)]
    if dtype == richm.C64:
        x0 = [v.astype(np.complex64).astype(np.complex128) for v in x0]
        ws = ws.astype(np.float32).astype(np.float64)
        a = a.astype(np.float32).astype(np.float64)
    X = to_dev(op, x0, dtype)
    XP = to_dev(op, x0, dtype)
    B = to_dev(op, bs, dtype)
    op.apply_sweeps(dtype, X, XP, B, coef(ws, dtype), coef(a, dtype), None, K=K, m=m)
    tol = 1e-12 if dtype == richm.C128 else 1e-5
    for i, g in enumerate(from_dev(op, X, dtype)):
        H = assemble_helmholtz(sizes[i], ks[i])
        ref, _ = inner_steps(H, bs[i].ravel(), x0[i].ravel(), None, ws[i], a[i], K=K)
        rel = np.linalg.norm(g.ravel() - ref) / np.linalg.norm(ref)
        assert rel <= tol, (sizes[i], rel)


@pytest.mark.parametrize("variant", ["nag", "nagex", "richardson"])
@pytest.mark.parametrize("kind", [richm.HELMHOLTZ_FD5_ABC, richm.HELMHOLTZ_FD5_DIRICHLET])
def test_helmholtz_fused_passes_match_oracle(variant, kind):
    # complex fused passes of 4 sweeps (64-column tiles, 32-column tails at 65..88
    # columns, several tiles from 89 on), 32-row bands (pairs of tail tiles and an odd
    # one), plus a one-sweep remainder
    sizes = [5, 64, 70, 88, 150, 130]
    ks = [helmholtz_wavenumber(n) for n in sizes]
    op = richm.Operator([(kind, n, 1.0, 0.0, k) for n, k in zip(sizes, ks)])
    op.set_tuning(4, 32)
    m, K = 8, 9
    ws = np.stack([synth.helmholtz_weights(m, 1.0 / (n + 1), seed=4) for n in sizes]).astype(np.float32)
    a = np.full_like(ws, 0.3)
    at = None
    if variant == "richardson":
        a = None
    elif variant == "nagex":
        at = np.full_like(ws, 0.1)
    x0 = [(0.1 * (synth.rhs_uniform(51, i, n) + 1j * synth.rhs_uniform(52, i, n))).astype(np.complex64)
          for i, n in enumerate(sizes)]
    v0 = [(0.01 * (synth.rhs_uniform(53, i, n) - 1j * synth.rhs_uniform(54, i, n))).astype(np.complex64)
          for i, n in enumerate(sizes)]
    xp0 = [(x - v).astype(np.complex64) for x, v in zip(x0, v0)]
    bs = [synth.point_source_rhs(n, 1, seed=5 + i)[0].astype(np.complex64) for i, n in enumerate(sizes)]
    X, XP, B = to_dev(op, x0, richm.C64), to_dev(op, xp0, richm.C64), to_dev(op, bs, richm.C64)
    op.apply_sweeps(richm.C64, X, XP if a is not None else None, B, coef(ws, richm.C64),
                    None if a is None else coef(a, richm.C64), None if at is None else coef(at, richm.C64),
                    K=K, m=m, fuse=4)
    for i, g in enumerate(from_dev(op, X, richm.C64)):
        H = assemble_helmholtz(sizes[i], ks[i], absorbing=kind == richm.HELMHOLTZ_FD5_ABC)
        v = None if a is None else (x0[i].astype(np.complex128) - xp0[i].astype(np.complex128)).ravel()
        ref, _ = inner_steps(H, bs[i].astype(np.complex128).ravel(), x0[i].astype(np.complex128).ravel(), v,
                             ws[i].astype(np.float64), None if a is None else a[i].astype(np.float64),
                             None if at is None else at[i].astype(np.float64), K=K)
        rel = np.linalg.norm(g.ravel() - ref) / np.linalg.norm(ref)
        assert rel <= 1e-5, (sizes[i], rel)


def test_helmholtz_fused_equals_one_sweep_passes_closely():
    sizes = [33, 88, 200]
    ks = [helmholtz_wavenumber(n) for n in sizes]
    res = []
    for fuse in (1, 4):
        op = richm.Operator([(richm.HELMHOLTZ_FD5_ABC, n, 1.0, 0.0, k) for n, k in zip(sizes, ks)])
        ws = np.stack([synth.helmholtz_weights(8, 1.0 / (n + 1), seed=4) for n in sizes])
        x0 = [0.1 * (synth.rhs_uniform(55, i, n) + 1j * synth.rhs_uniform(56, i, n)) for i, n in enumerate(sizes)]
        X, XP = to_dev(op, x0, richm.C64), to_dev(op, x0, richm.C64)
        B = to_dev(op, [synth.point_source_rhs(n, 1, seed=9 + i)[0] for i, n in enumerate(sizes)], richm.C64)
        op.apply_sweeps(richm.C64, X, XP, B, coef(ws, richm.C64), coef(np.full_like(ws, 0.3), richm.C64), None,
                        K=16, m=8, fuse=fuse)
        res.append(from_dev(op, X, richm.C64))
    for g1, g4 in zip(*res):
        assert np.abs(g1 - g4).max() <= 1e-5 * max(np.abs(g1).max(), 1e-30)


def test_helmholtz_jacobi_preconditioned():
    sizes = [4, 33]
    ks = [helmholtz_wavenumber(n) for n in sizes]
    op = richm.Operator([(richm.HELMHOLTZ_FD5_ABC, n, 1.0, 0.0, k) for n, k in zip(sizes, ks)])
    m, K = 3, 7
    ws = np.array([[0.3, 0.5, 0.4]] * 2)
    a = np.full_like(ws, 0.2)
    x0 = [0.1 * synth.rhs_uniform(61, i, n) + 0j for i, n in enumerate(sizes)]
    bs = [synth.point_source_rhs(n, 1, seed=9)[0] for n in sizes]
    X = to_dev(op, x0, richm.C128)
    XP = to_dev(op, x0, richm.C128)
    B = to_dev(op, bs, richm.C128)
    op.apply_sweeps(richm.C128, X, XP, B, coef(ws, richm.C128), coef(a, richm.C128), None, K=K, m=m, precond=1)
    for i, g in enumerate(from_dev(op, X, richm.C128)):
        H = assemble_helmholtz(sizes[i], ks[i])
        ref, _ = inner_steps(H, bs[i].ravel(), x0[i].ravel(), None, ws[i], a[i], K=K, Binv=jacobi_binv(H))
        assert np.linalg.norm(g.ravel() - ref) <= 1e-12 * np.linalg.norm(ref)


def test_pack_unpack_roundtrip_and_halo_zero():
    insts = _instances(sizes=[1, 7, 64, 129])
    op = make_op(insts)
    arrs = [synth.rhs_uniform(71, i, t.n) for i, t in enumerate(insts)]
    for dt in (richm.F64, richm.F32):
        buf = to_dev(op, arrs, dt)
        back = from_dev(op, buf, dt)
        for a_, b_ in zip(arrs, back):
            np.testing.assert_array_equal(b_, a_.astype(richm.TORCH_DTYPE[dt].__str__().split(".")[-1]))
        host = buf.cpu().numpy()
        for i, lay in enumerate(op.layouts):
            n = op.ns[i]
            blk = host[lay.offset:lay.offset + lay.rows * lay.pitch].reshape(lay.rows, lay.pitch)
            assert np.all(blk[0] == 0) and np.all(blk[-1] == 0) and np.all(blk[:, n:] == 0)


@pytest.mark.parametrize("fuse", [4, 8])
@pytest.mark.parametrize("variant", ["nag", "richardson", "nagex"])
def test_fp32_fused_sweeps_match_oracle(fuse, variant):
    # temporally blocked passes (+ a one-sweep remainder) against the oracle from the
    # same FP32 state, bounded by the derived rounding bound; sizes span one and
    # several 128-column tiles (n > 128 has interior tile edges) and ragged 64-row blocks
    sizes = [1, 5, 63, 127, 128, 129, 200, 255, 300]
    K, k_start = 2 * fuse + 1, 3
    for g, ref, gp, refp, w, a, at, G in _run_case(richm.F32, variant, K=K, k_start=k_start, sizes=sizes,
                                                   fuse=fuse):
        xmax = max(np.abs(ref).max(), 1.0)
        bound = _fp32_bound(w, a, at, G, k_start, K, xmax, 1.0)
        assert np.abs(g - ref).max() <= bound
        if gp is not None:
            assert np.abs(gp - refp).max() <= bound


@pytest.mark.parametrize("fuse", [4, 8])
@pytest.mark.parametrize("variant", ["nag", "nagex"])
def test_fp32_fused_jacobi_preconditioned_sweeps_match_oracle(fuse, variant):
    # the fused kernels' B^{-1} = D^{-1} variants (weights scaled by the constant 1/d)
    sizes = [5, 127, 129, 255, 300]
    K, k_start = 2 * fuse, 2
    for g, ref, gp, refp, w, a, at, G in _run_case(richm.F32, variant, K=K, k_start=k_start, sizes=sizes,
                                                   precond=1, fuse=fuse):
        xmax = max(np.abs(ref).max(), 1.0)
        bound = _fp32_bound(w, a, at, G, k_start, K, xmax, 1.0)
        assert np.abs(g - ref).max() <= bound
        assert np.abs(gp - refp).max() <= bound


@pytest.mark.parametrize("fuse", [4, 8])
@pytest.mark.parametrize("rows", [16, 48, 64])
def test_fused_tail_tiles_match_oracle(fuse, rows):
    # sizes whose last column block is a 64-column tail tile (129..176 and 241..288
    # columns at 8 sweeps per pass, 129..184 and 249..304 at 4), with an even and an
    # odd number of row bands: tail tiles of two bands share a warp, an odd one out
    # runs with idle lanes
    sizes = [129, 150, 176, 241, 255, 288, 300, 511]
    K, k_start = 2 * fuse, 1
    for g, ref, gp, refp, w, a, at, G in _run_case(richm.F32, "nag", K=K, k_start=k_start, sizes=sizes, fuse=fuse,
                                                   rows=rows):
        xmax = max(np.abs(ref).max(), 1.0)
        bound = _fp32_bound(w, a, at, G, k_start, K, xmax, 1.0)
        assert np.abs(g - ref).max() <= bound
        assert np.abs(gp - refp).max() <= bound


@pytest.mark.parametrize("fuse", [4, 8])
def test_fused_equals_single_sweeps_closely(fuse):
    # same arithmetic per point, different launch structure: agreement to a few ulps
    sizes = [31, 127, 129, 255, 511]
    a1 = _run_case(richm.F32, "nag", K=2 * fuse, k_start=1, sizes=sizes, fuse=1)
    a2 = _run_case(richm.F32, "nag", K=2 * fuse, k_start=1, sizes=sizes, fuse=fuse)
    for (g1, ref, *_), (g2, *_r) in zip(a1, a2):
        scale = max(np.abs(ref).max(), 1.0)
        assert np.abs(g1 - g2).max() <= 1e-5 * scale


def test_autotune_picks_a_supported_pass_length():
    insts = _instances(sizes=[127, 255, 511, 63])
    op = make_op(insts)
    fuse, ms = op.autotune(16, momentum=True)
    assert fuse in (1, 4, 8) and ms > 0


@pytest.mark.parametrize("fuse", [4, 8])
def test_bf16_state_fused_pass_matches_oracle(fuse):
    # bfloat16 iterate, FP32 arithmetic and right-hand side: one pass from the same
    # bf16-representable state is the FP32 result rounded once to bfloat16
    sizes = [5, 63, 130, 255]
    insts = _instances(sizes=sizes)
    op = make_op(insts)
    As = [assemble_q1(t.n, t.eps, t.theta) for t in insts]
    G = np.array([gershgorin_max(A) for A in As])
    m = 16
    w, a = nag_weights(G, m, beta=0.3)
    w = w.astype(np.float32).astype(np.float64)
    a = a.astype(np.float32).astype(np.float64)
    bf = lambda v: torch.tensor(v).to(torch.bfloat16).to(torch.float64).numpy()  # noqa: E731
    x0 = [bf(0.5 * synth.rhs_uniform(31, i, t.n)) for i, t in enumerate(insts)]
    xp0 = [bf(x - 0.02 * synth.rhs_uniform(32, i, t.n)) for i, (x, t) in enumerate(zip(x0, insts))]
    bs = [synth.rhs_uniform(33, i, t.n).astype(np.float32).astype(np.float64) for i, t in enumerate(insts)]
    X, XP = to_dev(op, x0, richm.BF16), to_dev(op, xp0, richm.BF16)
    B = to_dev(op, bs, richm.F32)
    op.apply_sweeps(richm.BF16, X, XP, B, coef(w, richm.F32), coef(a, richm.F32), None, K=fuse, m=m, k_start=3,
                    fuse=fuse)
    got = [g.astype(np.float64) for g in from_dev(op, X, richm.BF16)]
    for i, t in enumerate(insts):
        ref, _ = inner_steps(As[i], bs[i].ravel(), x0[i].ravel(), (x0[i] - xp0[i]).ravel(), w[i], a[i], K=fuse,
                             k_start=3)
        xmax = max(np.abs(ref).max(), 1.0)
        bound = fp32_bound(w[i], a[i], None, G[i], 3, fuse, xmax, 1.0) + 2.0 ** -8 * np.abs(ref).max()
        assert np.abs(got[i].ravel() - ref).max() <= bound


def test_bf16_state_requires_fused_passes():
    insts = _instances(sizes=[31])
    op = make_op(insts)
    X = op.zeros(richm.BF16)
    B = op.zeros(richm.F32)
    with pytest.raises(richm.RichmError) as ei:
        op.apply_sweeps(richm.BF16, X, None, B, coef(np.ones((1, 4)), richm.F32), K=6, m=4, fuse=4)
    assert ei.value.status == richm.ERR_UNSUPPORTED
