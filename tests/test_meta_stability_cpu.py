"""Long-run stability of the weights the meta network supplies.

A symmetric A evolves each eigenvector independently under NAG-Richardson(m), so one
period is a 2x2 map per eigenvalue; the solve cannot diverge if its spectral radius
is <= 1 on the whole spectrum, which lies in (0, sigma_max] (sigma_max = maximum of
the stencil's Fourier symbol)."""
import math
import os

import numpy as np
import pytest

import richm_synth as synth
from oracle.operators import assemble_q1
from oracle.training import meta_output_map, mlp_forward
from paper_2412_08076_gb300 import meta

pytestmark = pytest.mark.usefixtures("built_lib")


def _layers(p, m=16):
    sizes = [(64, 2), (64,), (64, 64), (64,), (m + 1, 64), (m + 1,)]
    parts, off = [], 0
    for s in sizes:
        k = int(np.prod(s))
        parts.append(np.asarray(p[off:off + k], dtype=np.float64).reshape(s))
        off += k
    return [(parts[0], parts[1]), (parts[2], parts[3]), (parts[4], parts[5])]


def test_symbol_max_bounds_the_spectrum():
    rng = np.random.default_rng(3)
    for _ in range(6):
        eps, th = 10 ** rng.uniform(-3, 0), rng.uniform(0, math.pi)
        for n in (7, 20):
            lam = np.linalg.eigvalsh(assemble_q1(n, eps, th).toarray())
            assert lam.max() <= meta.symbol_max(eps, th) + 1e-12
    # and it is attained asymptotically: n = 40 gets within 1 %
    lam = np.linalg.eigvalsh(assemble_q1(40, 0.3, 1.0).toarray())
    assert lam.max() >= 0.99 * meta.symbol_max(0.3, 1.0)


def _certify(params, grid=6):
    insts = [synth.AnisoInstance(10 ** le, th, 255) for le in np.linspace(-3, 0, grid)
             for th in np.linspace(0, math.pi, grid, endpoint=False)]
    X = synth.meta_inputs(insts)
    o = mlp_forward(_layers(params), X)
    worst = 0.0
    for i, t in enumerate(insts):
        c, s = math.cos(t.theta), math.sin(t.theta)
        c11, c22 = c * c + t.eps * s * s, s * s + t.eps * c * c
        c12 = (1 - t.eps) * s * c
        ax, ay = (c22 - 2 * c11) / 3, (c11 - 2 * c22) / 3
        d1, d2 = -(c11 + c22) / 6 - c12 / 2, -(c11 + c22) / 6 + c12 / 2
        G = 4 * (c11 + c22) / 3 + 2 * (abs(ax) + abs(ay) + abs(d1) + abs(d2))
        w, a = meta_output_map(o[i:i + 1], [G], 16)
        smax = meta.symbol_max(t.eps, t.theta)
        lam = np.concatenate([np.geomspace(1e-7 * smax, 1e-2 * smax, 200), np.linspace(1e-2 * smax, smax, 3000)])
        worst = max(worst, meta.period_radius(w[0], a[0], lam).max())
    return worst


def test_initial_network_is_stable_on_every_spectrum():
    assert _certify(meta.init_params(16)) <= 1.0 + 1e-9


def test_fixed_momentum_network_outputs_beta_and_is_stable():
    # the benchmark's network: momentum held at 0.3 (its output row is constant), the
    # 16 weights trained from Leja-ordered Chebyshev weights on [1.2 G/30, 1.2 G]
    p0 = meta.init_params(16, beta=0.3, stretch=1.2, leja=True, fixed_beta=True)
    assert _certify(p0) <= 1.0 + 1e-9
    p, src = meta.load_params(16, variant="beta03")
    assert src == "trained"
    rng = np.random.default_rng(4)
    X = np.stack([rng.uniform(-3, 0, 50), rng.uniform(0, math.pi, 50)], axis=1)
    o = mlp_forward(_layers(p), X)
    beta = 1.0 / (1.0 + np.exp(-o[:, 16]))
    assert np.abs(beta - 0.3).max() <= 1e-6
    assert _certify(p) <= 1.0 + 1e-9


@pytest.mark.skipif(not os.path.exists(meta.trained_path(16)), reason="no trained parameters saved")
def test_trained_network_is_stable_on_every_spectrum():
    p, src = meta.load_params(16)
    assert src == "trained"
    assert _certify(p) <= 1.0 + 1e-9
