"""GPU residual norms, refinement and the batched solve against the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

import richm_synth as synth
from gpu_util import coef, fp32_bound, from_dev, make_op, nag_weights, to_dev
from oracle.iterations import inner_steps, refined_steps
from oracle.operators import assemble_helmholtz, assemble_q1, gershgorin_max, helmholtz_wavenumber
from paper_2412_08076_gb300 import richm

pytestmark = pytest.mark.gpu


def _insts(sizes, seed=5):
    u = synth.uniform(synth.stream_key(seed), 2 * len(sizes))
    return [synth.AnisoInstance(10 ** (-3 * u[2 * i]), math.pi * u[2 * i + 1], n) for i, n in enumerate(sizes)]


@pytest.mark.parametrize("dtype", [richm.F64, richm.F32])
def test_residual_norm_matches_oracle(dtype):
    insts = _insts([1, 4, 33, 64, 127, 200])
    op = make_op(insts)
    xs = [synth.rhs_uniform(3, i, t.n) for i, t in enumerate(insts)]
    bs = [synth.rhs_uniform(4, i, t.n) for i, t in enumerate(insts)]
    if dtype == richm.F32:
        xs = [v.astype(np.float32).astype(np.float64) for v in xs]
        bs = [v.astype(np.float32).astype(np.float64) for v in bs]
    X, B = to_dev(op, xs, dtype), to_dev(op, bs, dtype)
    R = op.zeros(dtype)
    rn, bn, rel = op.residual_norm(dtype, X, B, r_out=R)
    rs = from_dev(op, R, dtype)
    for i, t in enumerate(insts):
        A = assemble_q1(t.n, t.eps, t.theta)
        r = bs[i].ravel() - A @ xs[i].ravel()
        tol = 1e-13 if dtype == richm.F64 else 1e-6
        assert abs(rn[i].item() - np.linalg.norm(r)) <= 1e-13 * np.linalg.norm(r)
        assert abs(bn[i].item() - np.linalg.norm(bs[i])) <= 1e-13 * np.linalg.norm(bs[i])
        assert abs(rel[i].item() - np.linalg.norm(r) / np.linalg.norm(bs[i])) <= 1e-12
        assert np.abs(rs[i].ravel() - r).max() <= tol * np.abs(r).max()


def test_residual_norm_complex():
    sizes = [5, 40]
    op = richm.Operator([(richm.HELMHOLTZ_FD5_ABC, n, 1.0, 0.0, helmholtz_wavenumber(n)) for n in sizes])
    xs = [synth.rhs_uniform(3, i, n) + 1j * synth.rhs_uniform(6, i, n) for i, n in enumerate(sizes)]
    bs = [synth.rhs_uniform(4, i, n) + 0j for i, n in enumerate(sizes)]
    X, B = to_dev(op, xs, richm.C128), to_dev(op, bs, richm.C128)
    rn, bn, rel = op.residual_norm(richm.C128, X, B)
    for i, n in enumerate(sizes):
        H = assemble_helmholtz(n, helmholtz_wavenumber(n))
        r = bs[i].ravel() - H @ xs[i].ravel()
        assert abs(rn[i].item() - np.linalg.norm(r)) <= 1e-12 * np.linalg.norm(r)


def _solve_setup(sizes, m=16, beta=0.3, seed=5):
    insts = _insts(sizes, seed)
    op = make_op(insts)
    As = [assemble_q1(t.n, t.eps, t.theta) for t in insts]
    G = np.array([gershgorin_max(A) for A in As])
    w, a = nag_weights(G, m, beta=beta)
    bs = [synth.rhs_uniform(2, i, t.n) for i, t in enumerate(insts)]
    return insts, op, As, w, a, bs


@pytest.mark.parametrize("refine_every", [128, 256])
def test_solve_with_long_refinement_intervals_checked_by_oracle(refine_every):
    # the benchmark's interval: FP32 sweeps carry the momentum across refinements, so a
    # longer interval only moves where FP32 rounding is corrected
    insts, op, As, w, a, bs = _solve_setup([15, 63, 130, 255])
    B = to_dev(op, bs, richm.F64)
    X = op.zeros(richm.F64)
    opts = op.solve_opts(16, tol=1e-10, max_sweeps=400000, refine_every=refine_every, inner=richm.F32, fuse=8)
    st, info = op.solve(B, X, coef(w, richm.F32), coef(a, richm.F32), None, opts)
    assert st == richm.OK, info
    xs = from_dev(op, X, richm.F64)
    for i, t in enumerate(insts):
        r = np.linalg.norm(bs[i].ravel() - As[i] @ xs[i].ravel()) / np.linalg.norm(bs[i])
        assert r <= 1e-10, (t, r)
        assert info[i][0] % refine_every == 0


@pytest.mark.parametrize("use_graph,fuse", [(1, 1), (0, 1), (1, 4), (1, 8)])
def test_solve_to_1e10_checked_by_oracle(use_graph, fuse):
    insts, op, As, w, a, bs = _solve_setup([1, 2, 15, 31, 63, 64, 130])
    B = to_dev(op, bs, richm.F64)
    X = op.zeros(richm.F64)
    opts = op.solve_opts(16, tol=1e-10, max_sweeps=400000, refine_every=64, inner=richm.F32, use_graph=use_graph,
                         fuse=fuse)
    st, info = op.solve(B, X, coef(w, richm.F32), coef(a, richm.F32), None, opts)
    assert st == richm.OK, info
    xs = from_dev(op, X, richm.F64)
    for i, t in enumerate(insts):
        r = np.linalg.norm(bs[i].ravel() - As[i] @ xs[i].ravel()) / np.linalg.norm(bs[i])
        assert r <= 1e-10, (t, r)
        sweeps, rel, s = info[i]
        assert s == richm.OK and sweeps % 64 == 0
        assert abs(rel - r) <= 1e-3 * r + 1e-14


@pytest.mark.parametrize("inner", [richm.F32, richm.F64])
def test_refinement_residual_norm_matches_oracle(inner):
    # tol = 0 stops every instance after max_sweeps; the reported relative residual is
    # the solver's refinement residual (b folded into the FP64 stencil, |b| from the
    # first residual) of the x it returns
    insts, op, As, w, a, bs = _solve_setup([1, 5, 33, 64, 97, 130])
    B = to_dev(op, bs, richm.F64)
    X = op.zeros(richm.F64)
    opts = op.solve_opts(16, tol=0.0, max_sweeps=128, refine_every=64, inner=inner, fuse=1 if inner == richm.F64 else 8)
    st, info = op.solve(B, X, coef(w, inner), coef(a, inner), None, opts)
    assert st == richm.ERR_NOT_CONVERGED
    xs = from_dev(op, X, richm.F64)
    for i, t in enumerate(insts):
        r = np.linalg.norm(bs[i].ravel() - As[i] @ xs[i].ravel()) / np.linalg.norm(bs[i])
        assert info[i][0] == 128
        # both sides round b - A x in FP64 in different orders: an absolute difference of
        # a few ulp of |b| + |A||x|, relative to |b| (instances that converged far)
        assert abs(info[i][1] - r) <= 1e-12 * r + 1e-13, (t, info[i][1], r)


def test_fused_refinement_norm_over_a_wide_range():
    # the fused refinement sums |r|^2 as FP32 pairs from r's binary32 split; right-hand
    # sides whose entries span 1e-30 .. 1e6 (residual entries below 2^-74 take the
    # unsplit path) give the FP64 relative residual to 1e-12
    insts, op, As, w, a, bs = _solve_setup([33, 64, 130])
    rng = np.random.default_rng(17)
    bs = [v * 10.0 ** rng.uniform(-30, 6, v.shape) for v in bs]
    B = to_dev(op, bs, richm.F64)
    for sweeps in (64, 192):
        X = op.zeros(richm.F64)
        opts = op.solve_opts(16, tol=0.0, max_sweeps=sweeps, refine_every=64, inner=richm.F32, fuse=8)
        st, info = op.solve(B, X, coef(w, richm.F32), coef(a, richm.F32), None, opts)
        xs = from_dev(op, X, richm.F64)
        for i, t in enumerate(insts):
            r = np.linalg.norm(bs[i].ravel() - As[i] @ xs[i].ravel()) / np.linalg.norm(bs[i])
            assert info[i][0] == sweeps
            assert abs(info[i][1] - r) <= 1e-12 * r + 1e-15, (t, info[i][1], r)


@pytest.mark.parametrize("scale,fp64", [(1.0, 0), (1e-28, 0), (1e33, 0), (1.0, 1)])
def test_fused_refinement_right_hand_side_matches_the_oracle(scale, fp64):
    # the refinement after fused cycles forms r = b - A x in 64-bit fixed point per tile
    # (scale 1), or in FP64 where the tile's values fall outside that form's range
    # (1e-28, 1e33) or when the options ask for it (fp64_residual); either way its FP32
    # right-hand side is the oracle's FP64 residual of the x it wrote, rounded to FP32:
    # within one unit in the last place plus a few FP64 units of |b| + |A||x| (the
    # oracle's own rounding where the sum cancels)
    insts, op, As, w, a, bs = _solve_setup([33, 64, 130])
    bs = [v * scale for v in bs]
    B = to_dev(op, bs, richm.F64)
    X = op.zeros(richm.F64)
    opts = op.solve_opts(16, tol=0.0, max_sweeps=10 ** 6, refine_every=64, inner=richm.F32, fuse=8,
                         fp64_residual=fp64)
    S = richm.Solver(op, opts, coef(w, richm.F32), coef(a, richm.F32))
    S.start(B, X)
    for cycles in (1, 2):
        S.step(1)
        _, rhs, _ = S.views()
        rhs = from_dev(op, rhs.clone(), richm.F32)
        st, info = S.finish()
        xs = from_dev(op, X, richm.F64)
        for i, t in enumerate(insts):
            x = xs[i].ravel()
            r = bs[i].ravel() - As[i] @ x
            mag = np.abs(bs[i].ravel()) + abs(As[i]) @ np.abs(x)
            got = rhs[i].ravel().astype(np.float64)
            tol = np.spacing(np.abs(r).astype(np.float32)).astype(np.float64) + 2.0 ** -50 * mag
            bad = np.abs(got - r) > tol
            assert not bad.any(), (t, cycles, got[bad][:4], r[bad][:4])
            assert info[i][0] == 64 * cycles
            rel = np.linalg.norm(r) / np.linalg.norm(bs[i])
            assert abs(info[i][1] - rel) <= 1e-12 * rel, (t, info[i][1], rel)
    S.close()


def test_solve_with_either_refinement_residual_reaches_1e10():
    # the fixed-point and the FP64-arithmetic refinement residual both take every instance
    # to 1e-10 (oracle-recomputed), and the options check refuses other values
    insts, op, As, w, a, bs = _solve_setup([15, 63, 130, 255])
    B = to_dev(op, bs, richm.F64)
    res = []
    for fp64 in (0, 1):
        X = op.zeros(richm.F64)
        opts = op.solve_opts(16, tol=1e-10, max_sweeps=400000, refine_every=64, inner=richm.F32, fuse=8,
                             fp64_residual=fp64)
        st, info = op.solve(B, X, coef(w, richm.F32), coef(a, richm.F32), None, opts)
        assert st == richm.OK
        xs = from_dev(op, X, richm.F64)
        for i, t in enumerate(insts):
            r = np.linalg.norm(bs[i].ravel() - As[i] @ xs[i].ravel()) / np.linalg.norm(bs[i])
            # near 1e-10 the two FP64-level evaluations of |b - A x| / |b| differ by their
            # rounding, a few 1e-16 of |A||x| / |b|
            assert r <= 1e-10 and abs(info[i][1] - r) <= 1e-12 * r + 2e-14, (fp64, t, r, info[i])
        res.append([i_[0] for i_ in info])
    print(f"\nsweeps to 1e-10, fixed-point / FP64 refinement residual: {res[0]} / {res[1]}")
    with pytest.raises(richm.RichmError):
        op.solve(B, op.zeros(richm.F64), coef(w, richm.F32), coef(a, richm.F32), None,
                 op.solve_opts(16, fp64_residual=2))


def test_integer_field_conversions_match_hardware():
    assert richm.selftest_conversions() == (0, 0)


def test_solve_graph_and_plain_launches_agree_bitwise():
    res = []
    for g in (1, 0):
        insts, op, As, w, a, bs = _solve_setup([17, 40, 63])
        B = to_dev(op, bs, richm.F64)
        X = op.zeros(richm.F64)
        opts = op.solve_opts(16, tol=1e-9, max_sweeps=100000, refine_every=32, use_graph=g)
        st, info = op.solve(B, X, coef(w, richm.F32), coef(a, richm.F32), None, opts)
        res.append((X.cpu().numpy(), info))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]


def test_fp64_inner_solver_follows_the_oracle_iteration():
    # tol = 0: every instance runs exactly max_sweeps; FP64 inner sweeps with FP64
    # refinement are the same iteration as the oracle's plain sweeps.
    # (a) Steps that damp every mode (w lambda in (0, 1.5], momentum 0.3): FP64 rounding is
    # not amplified, and the solver matches the oracle to 1e-12 after 160 sweeps.
    # (b) The momentum-aware Chebyshev weights (w lambda up to ~24): the rounding made at a
    # sweep is carried by the long later steps of its period (per-mode factors up to ~1e4),
    # so two FP64 evaluation orders of the same iteration differ by more than 1e-12; the
    # oracle's own split and unsplit runs do too. There the state is held to the rounding
    # bound derived from the arithmetic with the FP64 unit roundoff.
    insts, op, As, w, a, bs = _solve_setup([9, 31, 70])
    G = np.array([gershgorin_max(A) for A in As])
    rng = np.random.default_rng(17)
    mild = rng.uniform(0.3, 1.5, w.shape) / G[:, None]
    B = to_dev(op, bs, richm.F64)
    for case, wc in (("mild", mild), ("chebyshev", w)):
        X = op.zeros(richm.F64)
        opts = op.solve_opts(16, tol=0.0, max_sweeps=160, refine_every=32, inner=richm.F64)
        st, info = op.solve(B, X, coef(wc, richm.F64), coef(a, richm.F64), None, opts)
        assert st == richm.ERR_NOT_CONVERGED
        xs = from_dev(op, X, richm.F64)
        for i, t in enumerate(insts):
            ref, _ = inner_steps(As[i], bs[i].ravel(), np.zeros(t.n * t.n), None, wc[i], a[i], K=160)
            assert info[i][0] == 160
            err = np.abs(xs[i].ravel() - ref).max() / np.abs(ref).max()
            if case == "mild":
                assert err <= 1e-12, (t.n, err)
            else:
                bound = fp32_bound(wc[i], a[i], None, G[i], 0, 160, np.abs(ref).max(), np.abs(bs[i]).max(),
                                   u=2.0 ** -53) / np.abs(ref).max()
                split = refined_steps(As[i], bs[i].ravel(), np.zeros(t.n * t.n), 160, wc[i], a[i], refine_every=32)
                assert err <= bound, (t.n, err, bound)
                assert np.abs(split - ref).max() / np.abs(ref).max() <= bound


@pytest.mark.parametrize("fuse", [1, 8])
def test_solver_finish_between_steps_leaves_the_iterate_in_x(fuse):
    # fused cycles alternate between x and a workspace buffer: finish (callable between
    # steps) must leave every instance's newest iterate in x, also for instances that
    # stopped on an odd cycle, and stepping on afterwards must not change the result
    insts, op, As, w, a, bs = _solve_setup([31, 63, 100])
    B = to_dev(op, bs, richm.F64)
    res = []
    for pause in (None, 3):
        X = op.zeros(richm.F64)
        S = richm.Solver(op, op.solve_opts(16, tol=1e-8, max_sweeps=10**6, fuse=fuse), coef(w, richm.F32),
                         coef(a, richm.F32))
        S.start(B, X)
        done = 0
        active = len(insts)
        while active:
            active = S.step(1)
            done += 1
            if pause is not None and done == pause:
                st, info = S.finish()
                xs = from_dev(op, X, richm.F64)
                for i, t in enumerate(insts):
                    r = np.linalg.norm(bs[i].ravel() - As[i] @ xs[i].ravel()) / np.linalg.norm(bs[i])
                    assert abs(info[i][1] - r) <= 1e-9 * r + 1e-14, (i, info[i][1], r)
        st, info = S.finish()
        assert st == richm.OK
        res.append((X.cpu().numpy(), info))
        S.close()
    np.testing.assert_array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]


def test_solver_session_steps_and_reports():
    insts, op, As, w, a, bs = _solve_setup([31, 63])
    B = to_dev(op, bs, richm.F64)
    X = op.zeros(richm.F64)
    wt, at = coef(w, richm.F32), coef(a, richm.F32)
    S = richm.Solver(op, op.solve_opts(16, tol=1e-10, max_sweeps=10**6), wt, at)
    S.start(B, X)
    assert S.step(0) == 2
    total = 0
    active = 2
    while active:
        active = S.step(4)
        total += 4
        assert total < 100000
    st, info = S.finish()
    assert st == richm.OK
    S.close()


def test_solve_reports_divergence_and_not_converged():
    insts, op, As, w, a, bs = _solve_setup([15, 31])
    B = to_dev(op, bs, richm.F64)
    X = op.zeros(richm.F64)
    G = np.array([gershgorin_max(A) for A in As])
    wbad = np.tile((3.0 / G)[:, None], (1, 4))  # |1 - w lam| up to 2: diverges
    st, info = op.solve(B, X, coef(wbad, richm.F32), None, None,
                        op.solve_opts(4, tol=1e-10, max_sweeps=100000, refine_every=16))
    assert st == richm.ERR_DIVERGED
    assert all(s == richm.ERR_DIVERGED for _, _, s in info)
    X.zero_()
    st, info = op.solve(B, X, coef(w, richm.F32), coef(a, richm.F32), None,
                        op.solve_opts(16, tol=1e-10, max_sweeps=64, refine_every=32))
    assert st == richm.ERR_NOT_CONVERGED
    assert all(s == richm.ERR_NOT_CONVERGED and sw == 64 for sw, _, s in info)


def test_refine_entry_matches_definition():
    insts, op, As, w, a, bs = _solve_setup([9, 33])
    xs = [synth.rhs_uniform(81, i, t.n) for i, t in enumerate(insts)]
    es = [1e-3 * synth.rhs_uniform(82, i, t.n) for i, t in enumerate(insts)]
    eps_ = [1e-3 * synth.rhs_uniform(83, i, t.n) for i, t in enumerate(insts)]
    X, B = to_dev(op, xs, richm.F64), to_dev(op, bs, richm.F64)
    E, EP = to_dev(op, es, richm.F64), to_dev(op, eps_, richm.F64)
    R = op.zeros(richm.F64)
    rel = op.refine(X, B, E, EP, richm.F64, R)
    for i, t in enumerate(insts):
        xn = xs[i] + es[i]
        r = bs[i].ravel() - As[i] @ xn.ravel()
        np.testing.assert_allclose(from_dev(op, X, richm.F64)[i], xn, rtol=0, atol=1e-15)
        np.testing.assert_allclose(from_dev(op, EP, richm.F64)[i], eps_[i] - es[i], rtol=0, atol=1e-18)
        assert np.all(from_dev(op, E, richm.F64)[i] == 0)
        np.testing.assert_allclose(from_dev(op, R, richm.F64)[i].ravel(), r, rtol=0, atol=1e-13)
        assert abs(rel[i].item() - np.linalg.norm(r) / np.linalg.norm(bs[i])) <= 1e-13


def test_solve_host_matches_device_solve():
    # host buffers in and out, zero initial guess: the same iteration as richm_solve
    insts, op, As, w, a, bs = _solve_setup([15, 40, 63, 100])
    wt, at = coef(w, richm.F32), coef(a, richm.F32)
    opts = op.solve_opts(16, tol=1e-10, max_sweeps=400000)
    B = to_dev(op, bs, richm.F64)
    X = op.zeros(richm.F64)
    st_d, info_d = op.solve(B, X, wt, at, None, opts)
    hb = torch.tensor(np.concatenate([v.ravel() for v in bs])).pin_memory()
    hx = torch.full((op.dense_elems(),), np.nan, dtype=torch.float64).pin_memory()
    st_h, info_h = op.solve_host(hb, hx, wt, at, None, opts)
    assert st_d == st_h == richm.OK
    assert info_d == info_h
    np.testing.assert_array_equal(hx.numpy(), op.unpack(X, richm.F64).cpu().numpy())
    off = 0
    for i, t in enumerate(insts):
        u = hx.numpy()[off:off + t.n * t.n]
        off += t.n * t.n
        assert np.linalg.norm(bs[i].ravel() - As[i] @ u) / np.linalg.norm(bs[i]) <= 1e-10


def test_kept_session_repeats_and_rebinds():
    # richm_solve keeps its session in the operator for the next call with the same
    # options, weights and workspace: repeated solves (graphs reused), new weight values
    # behind the same pointers, another x buffer, other options and an interleaved host
    # solve each give the bits of a solve on a fresh operator
    sizes = [15, 40, 63, 130]

    def fresh(bs_, w_, a_, opts_kw):
        insts, op, As, w, a, bs = _solve_setup(sizes)
        X = op.zeros(richm.F64)
        st, info = op.solve(to_dev(op, bs_, richm.F64), X, coef(w_, richm.F32), coef(a_, richm.F32), None,
                            op.solve_opts(16, **opts_kw))
        x = X.cpu().numpy()
        op.close()
        return st, info, x

    kw1 = dict(tol=1e-10, max_sweeps=400000, refine_every=64, use_graph=1, fuse=8)
    kw2 = dict(tol=1e-9, max_sweeps=400000, refine_every=32, use_graph=1, fuse=4)
    insts, op, As, w, a, bs = _solve_setup(sizes)
    wt, at = coef(w, richm.F32), coef(a, richm.F32)
    B = to_dev(op, bs, richm.F64)
    work = op.workspace(op._ws("richm_solve_workspace", richm.C.byref(op.solve_opts(16, **kw1))))
    ref1 = fresh(bs, w, a, kw1)
    X = op.zeros(richm.F64)
    for _ in range(3):
        X.zero_()
        st, info = op.solve(B, X, wt, at, None, op.solve_opts(16, **kw1), work=work)
        assert (st, info) == ref1[:2]
        np.testing.assert_array_equal(X.cpu().numpy(), ref1[2])
    # new weights written into the same device arrays
    w2 = w * 0.97
    wt.copy_(coef(w2, richm.F32))
    ref2 = fresh(bs, w2, a, kw1)
    X.zero_()
    st, info = op.solve(B, X, wt, at, None, op.solve_opts(16, **kw1), work=work)
    assert (st, info) == ref2[:2]
    np.testing.assert_array_equal(X.cpu().numpy(), ref2[2])
    # another x buffer (the kept graphs are captured again)
    X2 = op.zeros(richm.F64)
    st, info = op.solve(B, X2, wt, at, None, op.solve_opts(16, **kw1), work=work)
    np.testing.assert_array_equal(X2.cpu().numpy(), ref2[2])
    # other options
    ref3 = fresh(bs, w2, a, kw2)
    X2.zero_()
    st, info = op.solve(B, X2, wt, at, None, op.solve_opts(16, **kw2), work=work)
    assert (st, info) == ref3[:2]
    np.testing.assert_array_equal(X2.cpu().numpy(), ref3[2])
    # a host solve in between, then the device solve again
    hb = torch.tensor(np.concatenate([v.ravel() for v in bs])).pin_memory()
    hx = torch.empty(op.dense_elems(), dtype=torch.float64).pin_memory()
    for _ in range(2):
        st_h, info_h = op.solve_host(hb, hx, wt, at, None, op.solve_opts(16, **kw1))
        assert info_h == ref2[1]
        dense = op.unpack(torch.tensor(ref2[2], device="cuda"), richm.F64).cpu().numpy()
        np.testing.assert_array_equal(hx.numpy(), dense)
    X.zero_()
    st, info = op.solve(B, X, wt, at, None, op.solve_opts(16, **kw1), work=work)
    np.testing.assert_array_equal(X.cpu().numpy(), ref2[2])
    op.close()


def test_bf16_inner_state_converges_with_mild_steps_and_reports_divergence_otherwise():
    # bfloat16 inner iterate (FP32 arithmetic), FP64 refinement. With steps that damp
    # every mode (|1 - w lam| <= 1) the refinement removes the storage rounding and the
    # FP64 tolerance is reached; with the large steps of a Chebyshev-type schedule the
    # rounding made at each pass boundary is amplified by the following steps, and the
    # solver must report divergence instead of producing garbage.
    insts, op, As, w, a, bs = _solve_setup([15, 31])
    G = np.array([gershgorin_max(A) for A in As])
    mild = np.tile((1.0 / G)[:, None], (1, 16))
    B = to_dev(op, bs, richm.F64)
    X = op.zeros(richm.F64)
    opts = op.solve_opts(16, tol=1e-10, max_sweeps=2_000_000, inner=richm.BF16, fuse=8)
    st, info = op.solve(B, X, coef(mild, richm.F32), coef(np.full_like(mild, 0.2), richm.F32), None, opts)
    assert st == richm.OK, info
    xs = from_dev(op, X, richm.F64)
    for i, t in enumerate(insts):
        assert np.linalg.norm(bs[i].ravel() - As[i] @ xs[i].ravel()) / np.linalg.norm(bs[i]) <= 1e-10
    X.zero_()
    st, info = op.solve(B, X, coef(w, richm.F32), coef(a, richm.F32), None, opts)
    assert st in (richm.OK, richm.ERR_DIVERGED)
    for sweeps, rel, status in info:
        assert status in (richm.OK, richm.ERR_DIVERGED)
        if status == richm.OK:
            assert rel <= 1e-10
