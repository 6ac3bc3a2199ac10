"""Pins of the oracle's iterations: closed forms, exact solves, the paper's Table 2."""
import math
import os

import numpy as np
import pytest

import richm_synth as synth
from oracle.iterations import (chebyshev_weights, inner_steps, jacobi_binv, leja_order,
                               outer_iterations_to_tol, refined_steps, rel_residual,
                               semi_iteration_weights, ssor_binv)
from oracle.operators import assemble_q1, diffusion_tensor

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _theta0_modes(n, eps):
    """Sine modes and eigenvalues of the theta = 0 operator (separable closed form)."""
    h = 1.0 / (n + 1)
    C = diffusion_tensor(eps, 0.0)
    s = np.sin(np.arange(1, n + 1) * math.pi * h / 2) ** 2
    kap, mu = 4 * s, 1 - 2 * s / 3
    # eigenvalue for mode (p along y/rows, q along x/columns)
    lam = C[0, 0] * np.outer(mu, kap) + C[1, 1] * np.outer(kap, mu)
    grid = np.arange(1, n + 1) * h

    def mode(p, q):
        return np.outer(np.sin(p * math.pi * grid), np.sin(q * math.pi * grid)).ravel()
    return lam, mode


def test_richardson_period_is_the_printed_polynomial_form():
    # eqs. 3-5: one outer iteration of m sweeps maps u to T_m u + g with
    # T_m = (I - w_m A) ... (I - w_1 A) and g = (w_m + sum_j prod_{i>j} (I - w_i A) w_j) f,
    # formed here as dense matrix products, independently of the sweep loop
    rng = np.random.default_rng(5)
    for n, eps, theta, m in [(4, 1e-2, 0.7, 3), (5, 1.0, 2.0, 4), (3, 1e-4, 0.1, 5)]:
        A = assemble_q1(n, eps, theta).toarray()
        N = n * n
        w = rng.uniform(0.05, 0.4, m)
        u0 = rng.standard_normal(N)
        f = rng.standard_normal(N)
        I = np.eye(N)
        T = I.copy()
        for i in range(m):
            T = (I - w[i] * A) @ T
        G = w[m - 1] * I
        for j in range(m - 1):
            P = I.copy()
            for i in range(j + 1, m):
                P = (I - w[i] * A) @ P
            G = G + P * w[j]
        u, _ = inner_steps(assemble_q1(n, eps, theta), f, u0, None, w, K=m)
        np.testing.assert_allclose(u, T @ u0 + G @ f, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("eps", [1.0, 1e-2, 1e-5])
def test_sine_mode_contraction(eps):
    # b = 0, x0 = sine mode: x_K = prod_s (1 - w_{s mod m} lam) x0 (eqs. 3-5)
    n, m, K = 15, 8, 21
    A = assemble_q1(n, eps, 0.0)
    lam, mode = _theta0_modes(n, eps)
    w = semi_iteration_weights(lam.max() * 1.01, m)
    for p, q in [(1, 1), (3, 10), (15, 15), (7, 2)]:
        x0 = mode(p, q)
        x, _ = inner_steps(A, np.zeros_like(x0), x0, None, w, K=K, k_start=5)
        fac = np.prod([1 - w[(5 + s) % m] * lam[p - 1, q - 1] for s in range(K)])
        np.testing.assert_allclose(x, fac * x0, rtol=1e-11, atol=1e-13 * np.abs(x0).max())


def test_nag_mode_recurrence():
    # NAG (Table 1) on an eigenvector: x_{k+1} = (1 - w lam)((1 + a) x_k - a x_{k-1})
    n, m, K = 11, 4, 13
    A = assemble_q1(n, 1e-2, 0.0)
    lam, mode = _theta0_modes(n, 1e-2)
    w = np.array([0.3, 0.5, 0.2, 0.45])
    a = np.array([0.3, 0.1, 0.5, 0.2])
    for p, q in [(1, 2), (6, 6), (11, 3)]:
        x0 = mode(p, q)
        x, _ = inner_steps(A, np.zeros_like(x0), x0, None, w, a, K=K)
        L = lam[p - 1, q - 1]
        s_prev, s = 1.0, 1.0
        for k in range(K):
            s_prev, s = s, (1 - w[k % m] * L) * ((1 + a[k % m]) * s - a[k % m] * s_prev)
        np.testing.assert_allclose(x, s * x0, rtol=1e-11, atol=1e-13)


def _mode_transfer(w, a, at, lam, K, k_start=0):
    """State-space form of Table 1's MOM / NAG / NAGex rows on an eigenvector of A with
    eigenvalue lam (f = 0): the pair (u, v) of coefficients maps linearly per step,
        u~ = u + at_i v,  v' = a_i v - w_i lam u~,  u' = u + v'
    i.e. (u', v') = M_i (u, v) with M_i = [[1 - w_i lam, a_i - w_i lam at_i],
                                           [  - w_i lam, a_i - w_i lam at_i]].
    Returns the product M_{K-1} ... M_0 (a 2x2 matrix)."""
    m = len(w)
    P = np.eye(2)
    for s in range(K):
        i = (k_start + s) % m
        g = w[i] * lam
        c = a[i] - g * at[i]
        P = np.array([[1.0 - g, c], [-g, c]]) @ P
    return P


@pytest.mark.parametrize("kind", ["mom", "nagex"])
def test_lookahead_mode_transfer(kind):
    # Table 1's MOM (at = 0) and NAGex (at != a) rows on theta = 0 sine modes, with a
    # non-zero initial velocity: the oracle's (u, v) after K steps equal the product of
    # the per-step 2x2 transfer matrices applied to the mode's (u0, v0) coefficients.
    # Distinct a_i and at_i: a swapped pair (or a sign error in the look-ahead) moves the
    # result far outside the tolerance (checked below).
    n, m, K, k0 = 11, 5, 17, 3
    eps = 1e-2
    A = assemble_q1(n, eps, 0.0)
    lam, mode = _theta0_modes(n, eps)
    rng = np.random.default_rng(21)
    G = lam.max()
    w = rng.uniform(0.2, 1.2, m) / G
    a = rng.uniform(0.05, 0.6, m)
    at = np.zeros(m) if kind == "mom" else rng.uniform(0.3, 0.9, m)
    c_u, c_v = 1.0, -0.4
    for p, q in [(1, 2), (6, 6), (11, 3), (9, 10)]:
        L = lam[p - 1, q - 1]
        e = mode(p, q)
        u, v = inner_steps(A, np.zeros_like(e), c_u * e, c_v * e, w, a, at, K=K, k_start=k0)
        su, sv = _mode_transfer(w, a, at, L, K, k0) @ np.array([c_u, c_v])
        np.testing.assert_allclose(u, su * e, rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(v, sv * e, rtol=1e-11, atol=1e-13)
        # the pin discriminates: swapping a and at, or dropping the look-ahead, changes
        # the coefficient by far more than the tolerance
        if kind == "nagex":
            su_swap = (_mode_transfer(w, at, a, L, K, k0) @ np.array([c_u, c_v]))[0]
            su_nag = (_mode_transfer(w, a, a, L, K, k0) @ np.array([c_u, c_v]))[0]
            assert abs(su_swap - su) > 1e-6 * max(1.0, abs(su))
            assert abs(su_nag - su) > 1e-6 * max(1.0, abs(su))
        else:
            su_nag = (_mode_transfer(w, a, a, L, K, k0) @ np.array([c_u, c_v]))[0]
            assert abs(su_nag - su) > 1e-6 * max(1.0, abs(su))


def test_mom_is_heavy_ball_three_term_recurrence():
    # MOM-Richardson (Table 1, at = 0) on an eigenvector is Polyak's heavy-ball recurrence
    # x_{k+1} = (1 + a - w lam) x_k - a x_{k-1}, written here for the coefficient alone
    n, m, K = 9, 3, 14
    eps = 1.0
    A = assemble_q1(n, eps, 0.0)
    lam, mode = _theta0_modes(n, eps)
    w = np.array([0.21, 0.35, 0.5]) / lam.max() * 2
    a = np.array([0.4, 0.15, 0.3])
    for p, q in [(1, 1), (4, 8), (9, 9)]:
        L = lam[p - 1, q - 1]
        e = mode(p, q)
        x, _ = inner_steps(A, np.zeros_like(e), e, None, w, a, np.zeros(m), K=K)
        xm1, xk = 1.0, 1.0
        for k in range(K):
            i = k % m
            xm1, xk = xk, (1 + a[i] - w[i] * L) * xk - a[i] * xm1
        np.testing.assert_allclose(x, xk * e, rtol=1e-11, atol=1e-13)


def test_torch_unroll_lookahead_mode_transfer():
    # the training oracle's torch unroll (zero initial velocity) on the same modes
    import torch
    from oracle.training import to_torch_sparse, unrolled_nag
    n, m, K = 7, 4, 13
    eps = 1e-1
    A = assemble_q1(n, eps, 0.0)
    lam, mode = _theta0_modes(n, eps)
    rng = np.random.default_rng(8)
    w = rng.uniform(0.3, 1.4, m) / lam.max()
    a = rng.uniform(0.1, 0.5, m)
    for at in (np.zeros(m), rng.uniform(0.4, 0.8, m)):
        for p, q in [(2, 5), (7, 1)]:
            L = lam[p - 1, q - 1]
            e = mode(p, q)
            u = unrolled_nag(to_torch_sparse(A), torch.zeros(n * n, dtype=torch.float64), torch.from_numpy(e),
                             torch.from_numpy(w), torch.from_numpy(a), K, at=torch.from_numpy(at)).numpy()
            su = (_mode_transfer(w, a, at, L, K) @ np.array([1.0, 0.0]))[0]
            np.testing.assert_allclose(u, su * e, rtol=1e-11, atol=1e-13)


def test_momentum_zero_is_richardson_and_nagex_reductions():
    n = 9
    A = assemble_q1(n, 0.05, 0.7)
    rng = np.random.default_rng(0)
    f = rng.standard_normal(n * n)
    w = rng.uniform(0.05, 0.3, 5)
    x1, _ = inner_steps(A, f, np.zeros(n * n), None, w, K=17)
    x2, _ = inner_steps(A, f, np.zeros(n * n), None, w, np.zeros(5), K=17)
    np.testing.assert_array_equal(x1, x2)
    # NAGex with at = a is NAG
    a = rng.uniform(0.0, 0.5, 5)
    x3, _ = inner_steps(A, f, np.zeros(n * n), None, w, a, K=17)
    x4, _ = inner_steps(A, f, np.zeros(n * n), None, w, a, a.copy(), K=17)
    np.testing.assert_array_equal(x3, x4)


def test_chebyshev_closed_form_reduction():
    # One period with exact lmin/lmax scales the extreme eigenvectors by
    # +1/T_m(s) (lmin) and (-1)^m/T_m(s) (lmax), s = (lmax+lmin)/(lmax-lmin),
    # T_m(s) = cosh(m arccosh s); every other eigenvalue is reduced at least as much.
    n, eps = 15, 1e-2
    A = assemble_q1(n, eps, 0.0)
    lam, mode = _theta0_modes(n, eps)
    lmin, lmax = lam.min(), lam.max()
    pmin = np.unravel_index(lam.argmin(), lam.shape)
    pmax = np.unravel_index(lam.argmax(), lam.shape)
    for m in [3, 8, 16]:
        w = chebyshev_weights(lmax, lmin, m)
        Tm = math.cosh(m * math.acosh((lmax + lmin) / (lmax - lmin)))
        for (p, q), sign in [(pmin, 1.0), (pmax, (-1.0) ** m)]:
            x0 = mode(p + 1, q + 1)
            x, _ = inner_steps(A, np.zeros_like(x0), x0, None, w, K=m)
            # rounding inside a period is amplified by the large intermediate factors
            np.testing.assert_allclose(x, sign / Tm * x0, rtol=1e-7, atol=1e-8)
        rng = np.random.default_rng(m)
        for _ in range(5):
            p, q = rng.integers(1, n + 1, 2)
            x0 = mode(p, q)
            x, _ = inner_steps(A, np.zeros_like(x0), x0, None, w, K=m)
            assert np.linalg.norm(x) <= (1 / Tm) * np.linalg.norm(x0) * (1 + 1e-9)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("eps,theta", [(1.0, 0.0), (1e-2, math.pi / 6), (1e-4, 2.0)])
def test_direct_solve_small_grids(n, eps, theta):
    A = assemble_q1(n, eps, theta)
    f = synth.rhs_uniform(0, n, n).ravel()
    ev = np.linalg.eigvalsh(A.toarray())
    u_direct = np.linalg.solve(A.toarray(), f)
    w = chebyshev_weights(ev.max(), ev.min(), 8)
    k, u = outer_iterations_to_tol(A, f, w, tol=1e-13, max_outer=20000)
    assert k <= 20000
    np.testing.assert_allclose(u, u_direct, rtol=1e-11, atol=1e-11 * np.abs(u_direct).max())
    # NAG with a small momentum converges to the same solution
    k2, u2 = outer_iterations_to_tol(A, f, 0.6 * w, tol=1e-13, max_outer=40000, a=np.full(8, 0.2))
    assert k2 <= 40000
    np.testing.assert_allclose(u2, u_direct, rtol=1e-10, atol=1e-10 * np.abs(u_direct).max())


def test_jacobi_preconditioner_is_rescaled_weight():
    # Q1 with constant coefficients has a constant diagonal d, so D^{-1} = w/d.
    n = 10
    A = assemble_q1(n, 0.1, 1.2)
    f = synth.rhs_uniform(3, 0, n).ravel()
    d = A.diagonal()[0]
    assert np.all(A.diagonal() == d)
    w = np.array([0.5, 0.9, 0.7])
    a = np.array([0.2, 0.2, 0.2])
    x1, _ = inner_steps(A, f, np.zeros(n * n), None, w, a, K=11, Binv=jacobi_binv(A))
    x2, _ = inner_steps(A, f, np.zeros(n * n), None, w / d, a, K=11)
    np.testing.assert_allclose(x1, x2, rtol=1e-13, atol=1e-15)


def _sor_sweeps_by_loops(A, f, u, alpha):
    """One forward, then one backward point SOR sweep (in-place updates in the row-major
    numbering), written as plain loops over the points."""
    Ad = A.toarray()
    u = np.array(u, dtype=np.float64, copy=True)
    N = len(u)
    for order in (range(N), range(N - 1, -1, -1)):
        for p in order:
            sigma = Ad[p] @ u - Ad[p, p] * u[p]
            u[p] = (1.0 - alpha) * u[p] + alpha * (f[p] - sigma) / Ad[p, p]
    return u


@pytest.mark.parametrize("n,eps,theta,alpha", [(2, 1.0, 0.3, 1.0), (3, 1e-2, 1.0, 1.3), (5, 1e-3, 2.2, 0.7),
                                               (4, 1e-6, math.pi / 10, 1.9)])
def test_ssor_preconditioner_is_a_forward_and_a_backward_sor_sweep(n, eps, theta, alpha):
    A = assemble_q1(n, eps, theta)
    f = synth.rhs_uniform(5, n, n).ravel()
    u = synth.rhs_uniform(6, n, n).ravel()
    want = _sor_sweeps_by_loops(A, f, u, alpha)
    got = u + ssor_binv(A, alpha)(f - A @ u)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_ssor_of_a_diagonal_matrix_is_scaled_jacobi():
    import scipy.sparse as sp
    d = np.linspace(1.0, 3.0, 7)
    r = synth.rhs_uniform(7, 0, 7)[0]
    for alpha in (0.5, 1.0, 1.5):
        got = ssor_binv(sp.diags(d), alpha)(r)
        np.testing.assert_allclose(got, alpha * (2 - alpha) * r / d, rtol=1e-15)


@pytest.mark.parametrize("alpha", [0.6, 1.0, 1.8])
def test_ssor_preconditioner_is_spd_and_clusters_the_spectrum_in_0_1(alpha):
    n = 4
    A = assemble_q1(n, 1e-2, 0.9)
    Binv = ssor_binv(A, alpha)
    M = np.column_stack([Binv(e) for e in np.eye(n * n)])
    np.testing.assert_allclose(M, M.T, atol=1e-13 * np.abs(M).max())
    assert np.linalg.eigvalsh((M + M.T) / 2).min() > 0
    lam = np.linalg.eigvals(M @ A.toarray())
    assert np.abs(lam.imag).max() < 1e-10
    assert lam.real.min() > 0 and lam.real.max() <= 1 + 1e-12


def test_refinement_split_is_the_same_iteration():
    n = 17
    A = assemble_q1(n, 3e-2, 0.9)
    b = synth.rhs_uniform(2, 1, n).ravel()
    G = 4.0
    w = semi_iteration_weights(G, 16) * 0.6
    a = np.full(16, 0.3)
    for R in (64, 16, 7):
        x_split = refined_steps(A, b, np.zeros(n * n), 200, w, a, refine_every=R)
        x_plain, _ = inner_steps(A, b, np.zeros(n * n), None, w, a, K=200)
        np.testing.assert_allclose(x_split, x_plain, rtol=1e-12, atol=1e-12 * np.abs(x_plain).max())


def _golden_table2():
    rows = []
    with open(os.path.join(GOLDEN, "table2_chebyshev.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                meth, eps, it, band = line.split()
                rows.append((meth, float(eps), int(it), float(band)))
    return rows


@pytest.mark.parametrize("row", _golden_table2(), ids=lambda r: f"{r[0]}-{r[1]:g}")
def test_table2_chebyshev_rows(row):
    meth, eps, paper_it, band = row
    n = 63
    A = assemble_q1(n, eps, 0.0)
    lam, _ = _theta0_modes(n, eps)
    if meth == "cheb3":
        w = chebyshev_weights(lam.max(), lam.min(), 3)
    else:
        w = semi_iteration_weights(lam.max(), 3, 1.0 / 30.0)
    for seed in range(2):
        f = synth.rhs_normal(11, seed, n).ravel()
        k, u = outer_iterations_to_tol(A, f, w, tol=1e-6)
        assert rel_residual(A, f, u) < 1e-6
        assert abs(k - paper_it) <= band * paper_it, (meth, eps, seed, k, paper_it)


def _lex_best_order(z):
    """Brute force over all permutations: the first node of largest |z| (smallest index
    on ties), then the lexicographically largest sequence of distance products."""
    import itertools
    m = len(z)
    best, best_key = None, None
    for perm in itertools.permutations(range(m)):
        key = [abs(z[perm[0]])]
        for s in range(1, m):
            p = 1.0
            for j in perm[:s]:
                p *= abs(z[perm[s]] - z[j])
            key.append(p)
        if best_key is None or key > best_key:
            best, best_key = perm, key
    return list(best)


def test_leja_order_brute_force():
    rng = np.random.default_rng(4)
    for m in (1, 2, 3, 5, 6):
        for _ in range(4):
            w = 1.0 / rng.uniform(0.1, 3.0, m)
            assert list(leja_order(w)) == _lex_best_order(1.0 / w)
    # two nodes: the larger node first
    assert list(leja_order(np.array([1.0, 0.5]))) == [1, 0]


def test_leja_order_tames_partial_products():
    # The rounding made at step s of a period is carried by the product of the later
    # factors (1 - w_k lam). Chebyshev weights of eqs. 8-9 in index order (increasing w)
    # put the long steps last, so those suffix products reach ~5e5 on [0, G]; in Leja
    # order both the prefix and the suffix products stay below 10, and the period (the
    # whole product) is the same.
    G, m = 1.0, 16
    w = chebyshev_weights(G, G / 30.0, m)
    lam = np.linspace(0.0, G, 4001)

    def worst(order):
        order = list(order)
        out = []
        for seq in (order, order[::-1]):  # prefix, suffix products
            P = np.ones_like(lam)
            wst = 1.0
            for i in seq:
                P = P * (1.0 - w[i] * lam)
                wst = max(wst, np.abs(P).max())
            out.append(wst)
        return out, P
    (npre, nsuf), Pn = worst(range(m))
    (lpre, lsuf), Pl = worst(leja_order(w))
    np.testing.assert_allclose(Pl, Pn, rtol=1e-9, atol=1e-12)
    assert nsuf > 1e5 and max(lpre, lsuf) < 10.0, (npre, nsuf, lpre, lsuf)
