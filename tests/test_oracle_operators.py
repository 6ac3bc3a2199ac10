"""Pins of the oracle's operators against facts that do not depend on its code."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.operators import (assemble_helmholtz, assemble_q1, diffusion_tensor,
                              gershgorin_max, helmholtz_wavenumber)


def _row_stencil(A, n, i, j):
    row = A.getrow(i * n + j).toarray().reshape(n, n)
    return row[i - 1:i + 2, j - 1:j + 2]


def test_diffusion_tensor_principal_axes():
    # C(eps, theta) has eigenvalue 1 along (cos t, sin t) and eps along (-sin t, cos t)
    for eps, th in [(1e-2, math.pi / 6), (0.3, 2.0), (1e-6, 0.1)]:
        C = diffusion_tensor(eps, th)
        d1 = np.array([math.cos(th), math.sin(th)])
        d2 = np.array([-math.sin(th), math.cos(th)])
        np.testing.assert_allclose(C @ d1, d1, atol=1e-15)
        np.testing.assert_allclose(C @ d2, eps * d2, atol=1e-15)


def test_q1_laplacian_textbook_stencil():
    # C = I: the bilinear-element Laplacian stencil is 1/3 [-1 -1 -1; -1 8 -1; -1 -1 -1]
    n = 7
    A = assemble_q1(n, 1.0, 0.37)
    st = _row_stencil(A, n, 3, 3)
    ref = np.full((3, 3), -1.0 / 3.0)
    ref[1, 1] = 8.0 / 3.0
    np.testing.assert_allclose(st, ref, atol=1e-14)


@pytest.mark.parametrize("eps,theta", [(1e-2, math.pi / 6), (0.5, 2.2), (1e-4, 1.0)])
def test_q1_exact_on_quadratics(eps, theta):
    # For u in {x^2, y^2, xy}, -div(C grad u) is the constant -2 c11, -2 c22, -2 c12 and
    # the Galerkin row at an interior node equals that constant times int(phi_i) = h^2.
    n = 9
    h = 1.0 / (n + 1)
    A = assemble_q1(n, eps, theta)
    C = diffusion_tensor(eps, theta)
    y, x = np.meshgrid((np.arange(n) + 1) * h, (np.arange(n) + 1) * h, indexing="ij")
    inner = np.zeros((n, n), bool)
    inner[1:-1, 1:-1] = True
    for u, c in [(x * x, C[0, 0]), (y * y, C[1, 1]), (x * y, C[0, 1])]:
        Au = (A @ u.ravel()).reshape(n, n)
        np.testing.assert_allclose(Au[inner], -2.0 * c * h * h, rtol=0, atol=1e-14)


def test_q1_theta0_separable_eigenvalues():
    # theta = 0: A = c11 K(x) M(y) + c22 M(x) K(y) with 1-D stiffness K = tridiag(-1,2,-1)
    # and mass M = tridiag(1,4,1)/6, so lam = c11 kap_j mu_k + c22 mu_j kap_k.
    n, eps = 15, 1e-2
    h = 1.0 / (n + 1)
    A = assemble_q1(n, eps, 0.0).toarray()
    s = np.sin(np.arange(1, n + 1) * math.pi * h / 2) ** 2
    kap, mu = 4 * s, 1 - 2 * s / 3
    lam = np.sort((1.0 * np.outer(kap, mu) + eps * np.outer(mu, kap)).ravel())
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(A)), lam, rtol=1e-12, atol=1e-13)


def test_q1_symmetry_periodicity_and_mirror():
    n = 8
    for eps, th in [(1e-3, 0.4), (0.2, 2.9)]:
        A = assemble_q1(n, eps, th)
        assert abs(A - A.T).max() < 1e-15
        assert abs(A - assemble_q1(n, eps, th + math.pi)).max() < 1e-14
        # mirroring x (j -> n-1-j) maps theta -> -theta
        P = sp.csr_matrix(np.kron(np.eye(n), np.fliplr(np.eye(n))))
        assert abs(P @ A @ P.T - assemble_q1(n, eps, -th)).max() < 1e-14


def test_q1_single_unknown():
    for eps, th in [(1.0, 0.0), (1e-2, 1.1)]:
        C = diffusion_tensor(eps, th)
        A = assemble_q1(1, eps, th).toarray()
        assert A.shape == (1, 1)
        np.testing.assert_allclose(A[0, 0], 4.0 * (C[0, 0] + C[1, 1]) / 3.0, rtol=1e-14)


def test_gershgorin_bounds_spectrum():
    for eps, th in [(1e-2, math.pi / 6), (1.0, 0.0), (1e-3, 2.0)]:
        A = assemble_q1(12, eps, th)
        assert np.linalg.eigvalsh(A.toarray()).max() <= gershgorin_max(A) + 1e-12


def test_gershgorin_hand_value():
    # eps = 1e-2, theta = pi/6: c11 = 0.7525, c22 = 0.2575, c12 = 0.99 sin(pi/6) cos(pi/6);
    # Q1 row (Sec. 2.4, eq. 18): centre 1.3466667, x-neighbours -0.4158333, y-neighbours
    # 0.0791667, corners -0.3826746 and 0.0460080, so an interior row's absolute sum is
    # 1.3466667 + 2 (0.4158333 + 0.0791667 + 0.3826746 + 0.0460080) = 3.1940319 (hand value)
    A = assemble_q1(15, 1e-2, math.pi / 6)
    assert abs(gershgorin_max(A) - 3.1940319) < 3e-7
    # theta = 0, eps = 1: the textbook stencil (8, -1 x 8) / 3 sums to 16/3
    assert abs(gershgorin_max(assemble_q1(6, 1.0, 0.0)) - 16.0 / 3.0) < 1e-13


def test_window_is_submatrix():
    n = 11
    A = assemble_q1(n, 1e-2, 0.8).toarray()
    for win in [(0, 5, 3, 11), (2, 9, 1, 6), (0, 11, 0, 11)]:
        i0, i1, j0, j1 = win
        idx = np.array([i * n + j for i in range(i0, i1) for j in range(j0, j1)])
        Aw = assemble_q1(n, 1e-2, 0.8, window=win).toarray()
        np.testing.assert_array_equal(Aw, A[np.ix_(idx, idx)])
    H = assemble_helmholtz(n, 17.0).toarray()
    win = (2, 9, 1, 6)
    idx = np.array([i * n + j for i in range(2, 9) for j in range(1, 6)])
    np.testing.assert_array_equal(assemble_helmholtz(n, 17.0, window=win).toarray(), H[np.ix_(idx, idx)])


def test_helmholtz_ghost_elimination():
    # Build the system with explicit ghost unknowns and the discrete boundary equations
    # -(u_1 - u_0)/h - i k u_0 = 0, then eliminate them by a Schur complement.
    n, k = 6, 9.0
    h = 1.0 / (n + 1)
    N = n + 2  # nodes 0..n+1 per direction; ghosts on the edges (corners unused)
    def gid(i, j):
        return i * N + j
    M = np.zeros((N * N, N * N), complex)
    interior = [(i, j) for i in range(1, n + 1) for j in range(1, n + 1)]
    ghosts = []
    for (i, j) in interior:
        r = gid(i, j)
        M[r, r] = (4 - (k * h) ** 2) / h ** 2
        for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
            M[r, gid(i + di, j + dj)] += -1 / h ** 2
    for i in range(1, n + 1):
        for (g, inner) in [((i, 0), (i, 1)), ((i, n + 1), (i, n)), ((0, i), (1, i)), ((n + 1, i), (n, i))]:
            r = gid(*g)
            ghosts.append(r)
            M[r, r] = 1 / h - 1j * k
            M[r, gid(*inner)] = -1 / h
    I = [gid(i, j) for (i, j) in interior]
    Gh = ghosts
    S = M[np.ix_(I, I)] - M[np.ix_(I, Gh)] @ np.linalg.solve(M[np.ix_(Gh, Gh)], M[np.ix_(Gh, I)])
    np.testing.assert_allclose(assemble_helmholtz(n, k).toarray(), S, rtol=1e-13, atol=1e-10)


def test_helmholtz_symmetric_and_poisson_limit():
    n = 9
    h = 1.0 / (n + 1)
    H = assemble_helmholtz(n, helmholtz_wavenumber(n))
    assert abs(H - H.T).max() < 1e-9  # complex symmetric, not Hermitian
    assert abs(H - H.conj().T).max() > 1.0
    P = assemble_helmholtz(n, 0.0, absorbing=False).toarray().real
    s = np.sin(np.arange(1, n + 1) * math.pi * h / 2) ** 2
    lam = np.sort((4 * np.add.outer(s, s) / h ** 2).ravel())
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(P)), lam, rtol=1e-12)


def test_helmholtz_wavenumber_ten_points():
    n = 2047
    k = helmholtz_wavenumber(n)
    assert abs(2 * math.pi / k - 10.0 / (n + 1)) < 1e-15


def test_sampled_sweeps_equal_full_grid():
    import richm_synth as synth
    from oracle.iterations import inner_steps
    from oracle.sampling import sampled_sweeps
    n, K = 23, 5
    rng = np.random.default_rng(1)
    X0 = rng.standard_normal((n, n))
    V0 = 0.1 * rng.standard_normal((n, n))
    F = synth.rhs_uniform(4, 0, n)
    w = rng.uniform(0.05, 0.4, 3)
    a = np.full(3, 0.3)
    pts = [(0, 0), (11, 11), (22, 3), (5, 17), (6, 6)]
    for op, A in [(("q1", 1e-2, 0.7), assemble_q1(n, 1e-2, 0.7)),
                  (("helmholtz", 40.0), assemble_helmholtz(n, 40.0))]:
        ww = w if op[0] == "q1" else w * (1.0 / (n + 1)) ** 2 / 4
        x, _ = inner_steps(A, F.ravel().astype(A.dtype), X0.ravel().astype(A.dtype),
                           V0.ravel().astype(A.dtype), ww, a, K=K, k_start=2)
        s = sampled_sweeps(op, n, X0.astype(A.dtype), V0.astype(A.dtype), F.astype(A.dtype),
                           ww, a, None, K, pts, k_start=2)
        np.testing.assert_allclose(s, [x.reshape(n, n)[p] for p in pts], rtol=1e-13, atol=1e-13)


def test_sponge_gamma_hand_values():
    # N = 128 (n = 127, h = 1/128), omega = 2 pi 10 (Table 9's first column), c = 1:
    # one wavelength L = 0.1 = 12.8 h, so gamma / omega = 1 - d / 12.8 with d the node's
    # distance to the boundary in grid spacings
    from oracle.operators import sponge_gamma
    n, om = 127, 2 * math.pi * 10
    g = sponge_gamma(n, om).reshape(n, n) / om
    assert abs(g[0, 0] - (1 - 1 / 12.8)) < 1e-14          # d = 1
    assert abs(g[0, 60] - (1 - 1 / 12.8)) < 1e-14         # an edge row, d = 1
    assert abs(g[11, 40] - (1 - 12 / 12.8)) < 1e-14       # d = 12: 0.0625
    assert g[12, 40] == 0.0 and g[63, 63] == 0.0          # d = 13 and the centre
    assert abs(g[126, 5] - (1 - 1 / 12.8)) < 1e-14        # last row, d = 1
    assert abs(g[5, 120] - (1 - 6 / 12.8)) < 1e-14        # d = min(6, 7) = 6


def test_sponge_operator_energy_identity():
    # the Laplacian and -k^2 parts are real symmetric, so Im(x^H A x) is the damping
    # energy sum_x gamma(x) omega / c^2 |x|^2, here summed node by node with the
    # distance taken from the node's coordinates
    from oracle.operators import assemble_helmholtz_sponge
    rng = np.random.default_rng(2)
    for n, om, c in [(15, 40.0, 1.0), (20, 25.0, 1.3), (7, 30.0, 1.0)]:
        A = assemble_helmholtz_sponge(n, om, c)
        h = 1.0 / (n + 1)
        x = rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n)
        E = 0.0
        for i in range(n):
            for j in range(n):
                yy, xx = (i + 1) * h, (j + 1) * h
                d = min(xx, 1 - xx, yy, 1 - yy)
                gam = om * max(0.0, 1.0 - d / (2 * math.pi * c / om))
                E += gam * om / c ** 2 * abs(x[i * n + j]) ** 2
        q = np.vdot(x, A @ x)
        assert abs(q.imag - E) <= 1e-10 * E
        Ah = (A + A.conj().T) / 2
        D = assemble_helmholtz(n, om / c, absorbing=False)
        assert abs(Ah - D).max() < 1e-9
        assert abs(A - A.T).max() < 1e-9  # complex symmetric
