"""Pins of the oracle's FGMRES: Krylov-space minimisation by brute force, exact and
polynomial preconditioners, restarts."""
import numpy as np
import scipy.sparse.linalg as spla

from oracle.krylov import fgmres, richardson_preconditioner
from oracle.operators import assemble_helmholtz_sponge, assemble_q1


def _system(n=5, seed=0):
    rng = np.random.default_rng(seed)
    A = assemble_helmholtz_sponge(n, 30.0)
    N = n * n
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    x0 = 0.1 * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
    return A, b, x0


def _krylov_min(AP, r0, j):
    """min over u in K_j(AP, r0) of ||r0 - AP u||: the columns r0, AP r0, ... formed
    explicitly (each scaled to unit length) and the least-squares problem solved directly."""
    K = [r0 / np.linalg.norm(r0)]
    for _ in range(j - 1):
        k = AP @ K[-1]
        K.append(k / np.linalg.norm(k))  # the same space; unit columns for conditioning
    K = np.stack(K, axis=1)
    c = np.linalg.lstsq(AP @ K, r0, rcond=None)[0]
    return K @ c, np.linalg.norm(r0 - AP @ (K @ c))


def test_identity_preconditioner_minimises_over_the_krylov_space():
    A, b, x0 = _system()
    Ad = A.toarray()
    r0 = b - Ad @ x0
    for j in range(1, 7):
        x, its, est = fgmres(A, b, x0, None, m=j, tol=0.0, max_iters=j)
        u, res = _krylov_min(Ad, r0, j)
        assert its == j + 1  # tol 0 is never reached
        np.testing.assert_allclose(np.linalg.norm(b - Ad @ x), res, rtol=1e-9)
        np.testing.assert_allclose(x, x0 + u, rtol=0, atol=1e-6 * np.abs(x0 + u).max())
        assert abs(est[-1] - res / np.linalg.norm(b)) <= 1e-9 * est[-1]


def test_exact_preconditioner_converges_in_one_step():
    A, b, x0 = _system(n=6, seed=1)
    lu = spla.splu(A.tocsc())
    x, its, est = fgmres(A, b, x0, lu.solve, m=20, tol=1e-12)
    assert its == 1
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b)


def test_polynomial_preconditioner_is_gmres_on_the_preconditioned_operator():
    # the NAG-Richardson(4) smoother is a fixed linear map P = p(A); FGMRES with it
    # minimises ||r0 - A P u|| over K_j(A P, r0) and returns x0 + P u
    n = 5
    A = assemble_q1(n, 1e-2, 0.4)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(n * n)
    x0 = np.zeros(n * n)
    G = abs(A).sum(axis=1).max()
    w = np.array([0.3, 0.9, 0.5, 1.3]) / G
    a = np.full(4, 0.3)
    M = richardson_preconditioner(A, w, a)
    P = np.stack([M(e) for e in np.eye(n * n)], axis=1)
    AP = A.toarray() @ P
    for j in range(1, 6):
        x, its, est = fgmres(A, b, x0, M, m=j, tol=0.0, max_iters=j)
        u, res = _krylov_min(AP, b, j)
        np.testing.assert_allclose(np.linalg.norm(b - A @ x), res, rtol=1e-9)
        np.testing.assert_allclose(x, P @ u, rtol=0, atol=1e-7 * np.abs(P @ u).max())


def test_restarted_cycles_each_minimise_over_their_own_space():
    A, b, x0 = _system(n=4, seed=2)
    Ad = A.toarray()
    x_ref = x0.copy()
    for _ in range(3):
        u, _ = _krylov_min(Ad, b - Ad @ x_ref, 3)
        x_ref = x_ref + u
    x, its, est = fgmres(A, b, x0, None, m=3, tol=0.0, max_iters=9)
    np.testing.assert_allclose(x, x_ref, rtol=0, atol=1e-7 * np.abs(x_ref).max())
    assert len(est) == 9
