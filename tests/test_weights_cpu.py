"""The initial meta network gives a convergent NAG-Richardson(16) on every SPD spectrum in (0, G]."""
import math

import numpy as np
import pytest

from oracle.training import meta_output_map, mlp_forward
from paper_2412_08076_gb300 import meta

pytestmark = pytest.mark.usefixtures("built_lib")


def _period_radius(w, beta, lam):
    # per-mode 2x2 transfer of one NAG period on eigenvalue lam (A symmetric)
    P = np.tile(np.eye(2), (lam.size, 1, 1))
    for wi in w:
        mu = 1.0 - wi * lam
        T = np.zeros((lam.size, 2, 2))
        T[:, 0, 0] = mu * (1 + beta)
        T[:, 0, 1] = -mu * beta
        T[:, 1, 0] = 1.0
        P = T @ P
    return np.abs(np.linalg.eigvals(P)).max(axis=1)


def test_stretched_semi_iteration_weights_are_stable_with_momentum():
    w = meta.chebyshev_unit_weights(16)  # G * w_i
    lam = np.concatenate([np.geomspace(1e-8, 1e-2, 400), np.linspace(1e-2, 1.0, 4000)])
    rho = _period_radius(w, 0.3, lam)
    assert rho.max() <= 1.0 + 1e-12
    assert rho[lam > 0.05].max() < 0.9  # the upper spectrum is damped each period
    # the unstretched semi-iteration weights are not stable with this momentum
    w0 = meta.chebyshev_unit_weights(16, stretch=1.0)
    assert _period_radius(w0, 0.3, lam).max() > 1.5


def test_initial_network_outputs_the_stable_weights():
    m = 16
    p = meta.init_params(m, out_scale=0.0)
    sizes = [(64, 2), (64,), (64, 64), (64,), (m + 1, 64), (m + 1,)]
    parts, off = [], 0
    for s in sizes:
        k = int(np.prod(s))
        parts.append(p[off:off + k].astype(np.float64).reshape(s))
        off += k
    assert off == p.size == 5457
    layers = [(parts[0], parts[1]), (parts[2], parts[3]), (parts[4], parts[5])]
    X = np.array([[-3.0, 0.1], [0.0, 3.0], [-1.5, 1.0]])
    G = np.array([4.0, 5.3, 2.9])
    w, a = meta_output_map(mlp_forward(layers, X), G, m)
    np.testing.assert_allclose(w * G[:, None], np.tile(meta.chebyshev_unit_weights(m), (3, 1)), rtol=1e-6)
    np.testing.assert_allclose(a, 0.3, rtol=1e-6)
