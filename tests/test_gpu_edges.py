"""Edge cases of the sweep path against the oracle: the largest grid the tests run,
degenerate coefficients (isotropic, axis-aligned anisotropy), the shortest and longest
weight periods, zero weights and a batch of identical instances."""
import math

import numpy as np
import pytest

import richm_synth as synth
from gpu_util import coef, fp32_bound, from_dev, make_op, to_dev
from oracle.iterations import inner_steps
from oracle.operators import assemble_q1, gershgorin_max
from oracle.sampling import sampled_sweeps
from paper_2412_08076_gb300 import meta as meta_mod
from paper_2412_08076_gb300 import richm

pytestmark = pytest.mark.gpu


def test_largest_grid_fused_pass_sampled():
    # one 16383^2 instance (268 M unknowns, 1 GB per FP32 buffer): one fused pass of 8
    # NAG sweeps from x = 0, sampled at corners, edges, tile and band boundaries and
    # random points against the oracle's windowed evaluation
    n = 16383
    t = synth.AnisoInstance(1e-3, 2.0, n)
    op = make_op([t])
    G = op.gershgorin()[0]
    wn = (meta_mod.chebyshev_unit_weights(16) / G).astype(np.float32)[None, :]
    a = np.full_like(wn, 0.3)
    b = synth.rhs_uniform(7, 0, n).astype(np.float32)
    B = to_dev(op, [b], richm.F32)
    X, XP = op.zeros(richm.F32), op.zeros(richm.F32)
    K = 8
    op.apply_sweeps(richm.F32, X, XP, B, coef(wn, richm.F32), coef(a, richm.F32), None, K=K, m=16, fuse=8)
    got = from_dev(op, X, richm.F32)[0]
    rng = np.random.default_rng(17)
    pts = {(0, 0), (n - 1, n - 1), (0, n - 1), (n - 1, 0), (255, 111), (256, 112), (8191, 8192), (n - 1, 4000)}
    while len(pts) < 16:
        pts.add((int(rng.integers(0, n)), int(rng.integers(0, n))))
    pts = sorted(pts)
    ref = sampled_sweeps(("q1", t.eps, t.theta), n, np.zeros((n, n)), None, b.astype(np.float64),
                         wn[0].astype(np.float64), a[0].astype(np.float64), None, K, pts)
    bound = fp32_bound(wn[0].astype(np.float64), a[0].astype(np.float64), None, G, 0, K,
                       max(1.0, np.abs(ref).max()), 1.0)
    for (p, q), r in zip(pts, ref):
        assert abs(got[p, q] - r) <= bound, (p, q, got[p, q], r, bound)
    op.close()


@pytest.mark.parametrize("m", [1, 64])
def test_degenerate_coefficients_and_period_lengths(m):
    # isotropic (eps = 1), axis-aligned anisotropy (theta = 0, pi/2: the corner couplings
    # are equal), a near-diagonal direction, and a duplicated instance; FP64 to 1e-12
    insts = [synth.AnisoInstance(1.0, 0.7, 33), synth.AnisoInstance(1e-4, 0.0, 40),
             synth.AnisoInstance(1e-4, math.pi / 2, 40), synth.AnisoInstance(1e-2, math.pi / 4, 65),
             synth.AnisoInstance(1e-2, math.pi / 4, 65)]
    op = make_op(insts)
    As = [assemble_q1(t.n, t.eps, t.theta) for t in insts]
    G = np.array([gershgorin_max(A) for A in As])
    u = synth.uniform(synth.stream_key(88), m)
    w = (0.3 + 0.6 * u)[None, :] / G[:, None]
    a = np.full_like(w, 0.2)
    # instances 3 and 4 are the same problem with the same data
    x0 = [synth.rhs_uniform(60, min(i, 3), t.n) for i, t in enumerate(insts)]
    bs = [synth.rhs_uniform(61, min(i, 3), t.n) for i, t in enumerate(insts)]
    X, XP, B = to_dev(op, x0, richm.F64), to_dev(op, x0, richm.F64), to_dev(op, bs, richm.F64)
    K = 2 * m + 3
    op.apply_sweeps(richm.F64, X, XP, B, coef(w, richm.F64), coef(a, richm.F64), None, K=K, m=m, k_start=1)
    got = from_dev(op, X, richm.F64)
    for i, t in enumerate(insts):
        ref, _ = inner_steps(As[i], bs[i].ravel(), x0[i].ravel(), None, w[i], a[i], K=K, k_start=1)
        assert np.abs(got[i].ravel() - ref).max() <= 1e-12 * np.abs(ref).max(), t
    np.testing.assert_array_equal(got[3], got[4])


def test_zero_weights_and_zero_momentum_leave_the_state_unchanged():
    insts = [synth.AnisoInstance(1e-2, 1.0, n) for n in (7, 130)]
    op = make_op(insts)
    x0 = [synth.rhs_uniform(62, i, t.n) for i, t in enumerate(insts)]
    X, XP = to_dev(op, x0, richm.F64), to_dev(op, x0, richm.F64)
    B = to_dev(op, [synth.rhs_uniform(63, i, t.n) for i, t in enumerate(insts)], richm.F64)
    zeros = coef(np.zeros((2, 4)), richm.F64)
    op.apply_sweeps(richm.F64, X, XP, B, zeros, zeros, None, K=9, m=4)
    for g, x in zip(from_dev(op, X, richm.F64), x0):
        np.testing.assert_array_equal(g, x)
