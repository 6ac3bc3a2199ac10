"""Richardson(m) and its momentum / preconditioned forms in FP64 (oracle; test only).

Every iteration here is written in the velocity form of Table 1 of the paper:

    u~ = u + at_i v                     (look-ahead; NAG: at = a, MOM: at = 0)
    v  = a_i v + w_i Binv (f - A u~)    (eq. 17 with Binv = I gives Table 1)
    u  = u + v

with i running over 1..m inside one outer iteration and u, v carried into the
next outer iteration. Plain Richardson(m) (eqs. 2-5) is a = at = 0. The inner
step with global index k uses weight index k mod m (0-based), i.e. the paper's
w_{(k mod m) + 1}. The initial velocity is zero unless given (reading: the
paper does not state v^0).
"""
from __future__ import annotations

import math

import numpy as np


def chebyshev_weights(lmax: float, lmin: float, m: int) -> np.ndarray:
    """Eqs. 8-9: w_i = 2 / (lmax + lmin + (lmax - lmin) x_i), x_i = cos((2i-1) pi / 2m).

    Pinned by: m sweeps on the lmin/lmax eigenvectors reduce them by
    1/T_m((lmax+lmin)/(lmax-lmin)) (closed form via cosh/arccosh, tests).
    """
    i = np.arange(1, m + 1)
    x = np.cos((2 * i - 1) * math.pi / (2 * m))
    return 2.0 / (lmax + lmin + (lmax - lmin) * x)


def semi_iteration_weights(lmax: float, m: int, alpha: float = 1.0 / 30.0) -> np.ndarray:
    """Chebyshev semi-iteration: eqs. 8-9 with lmin replaced by alpha * lmax (Sec. 2.1)."""
    return chebyshev_weights(lmax, alpha * lmax, m)


def leja_order(w) -> np.ndarray:
    """A Leja ordering of the steps of one period (reading: eqs. 8-9 fix the set of
    weights, not the order in which the m steps run; the order changes only how FP32
    rounding is amplified inside a period).

    The steps are ordered by their nodes z_i = 1/w_i, the roots of the period's residual
    polynomial prod_i (1 - w_i z): first the node of largest |z|, then repeatedly the
    node that maximises the product of its distances to the nodes already taken
    (Leja points of a discrete set, after Reichel, BIT 30 (1990) 332-346). Ties go to
    the smaller index. Returns the permutation: step s of the period uses original
    index perm[s].
    Pinned by: brute force over every choice on small sets, and the product bound of
    Leja points (tests).
    """
    z = 1.0 / np.asarray(w, dtype=np.float64)
    m = z.size
    left = list(range(m))
    first = max(left, key=lambda i: (abs(z[i]), -i))
    perm = [first]
    left.remove(first)
    while left:
        def score(i):
            p = 1.0
            for j in perm:  # in the order the nodes were taken (FP64)
                p *= abs(z[i] - z[j])
            return p
        best = left[0]
        for i in left[1:]:
            if score(i) > score(best):
                best = i
        perm.append(best)
        left.remove(best)
    return np.array(perm, dtype=np.int64)


def inner_steps(A, f, u, v, w, a=None, at=None, K=1, k_start=0, Binv=None):
    """K inner steps of the Table 1 iteration (NAGex form covers all rows).

    A: sparse (n^2 x n^2); f, u, v: flat arrays; w, a, at: length-m sequences
    (a=None means no momentum; at=None means at = a, i.e. NAG). Binv: optional
    callable r -> B^{-1} r (eq. 17). Returns (u, v) after the K steps.
    Pinned by: sine-mode contraction prod(1 - w_i lam) (a = 0) and the per-mode
    two-term recurrence (a != 0), dense direct solve for n <= 8 (tests).
    """
    m = len(w)
    u = np.array(u, dtype=np.result_type(u, f, 1.0), copy=True)
    v = np.zeros_like(u) if v is None else np.array(v, dtype=u.dtype, copy=True)
    for s in range(K):
        i = (k_start + s) % m
        ai = 0.0 if a is None else a[i]
        ati = ai if at is None else at[i]
        ut = u + ati * v
        r = f - A @ ut
        if Binv is not None:
            r = Binv(r)
        v = ai * v + w[i] * r
        u = u + v
    return u, v


def jacobi_binv(A):
    """B^{-1} = D^{-1}, the diagonal of A (the weighted-Jacobi preconditioner of eq. 17
    with its relaxation factor folded into w)."""
    d = A.diagonal()
    return lambda r: r / d


def ssor_binv(A, alpha):
    """B^{-1} = alpha (2 - alpha) (D - alpha U)^{-1} D (D - alpha L)^{-1}, the SSOR member
    of the stationary preconditioners listed after eq. 17 (A = D - L - U with D diagonal,
    -L and -U the strictly lower and upper triangles of A).

    Reading: the paper does not state the ordering of the unknowns; L and U are taken in
    the row-major (lexicographic) numbering in which A is assembled here. The two
    triangular solves are library routines (scipy), one step each.
    Pinned by: u + B^{-1}(f - A u) equals one forward and one backward point SOR sweep
    written as loops; a diagonal A gives alpha (2 - alpha) D^{-1}; B^{-1} is symmetric
    positive definite and the eigenvalues of B^{-1} A lie in (0, 1] for an SPD A and
    0 < alpha < 2 (tests).
    """
    import scipy.sparse as sp
    from scipy.sparse.linalg import spsolve_triangular
    A = sp.csr_matrix(A)
    d = A.diagonal()
    lower = sp.csr_matrix(sp.diags(d) + alpha * sp.tril(A, -1))  # D - alpha L
    upper = sp.csr_matrix(sp.diags(d) + alpha * sp.triu(A, 1))   # D - alpha U

    def apply(r):
        z = spsolve_triangular(lower, np.asarray(r, dtype=np.float64), lower=True)
        return alpha * (2.0 - alpha) * spsolve_triangular(upper, d * z, lower=False)
    return apply


def ssor_binv_matrix(A, alpha):
    """The SSOR B^{-1} of `ssor_binv` as a dense matrix (its columns are B^{-1} e_j);
    for small instances, where a matrix product is the plain way to differentiate
    through it."""
    apply = ssor_binv(A, alpha)
    N = A.shape[0]
    return np.stack([apply(np.eye(1, N, j).ravel()) for j in range(N)], axis=1)


def residual(A, f, u):
    """f - A u."""
    return f - A @ u


def rel_residual(A, f, u) -> float:
    """||f - A u||_2 / ||f||_2 (the quantity of eq. 15 and the stopping test, Sec. 2.4)."""
    return float(np.linalg.norm(f - A @ u) / np.linalg.norm(f))


def outer_iterations_to_tol(A, f, w, tol=1e-6, max_outer=100000, a=None, at=None, Binv=None):
    """Outer iterations (m inner steps each) from u0 = 0 until ||f-Au||/||f|| < tol.

    The test is made once per outer iteration (Sec. 2.4, "the iteration will stop if
    the relative residual is less than 1e-6"). Returns (count, u); count is
    max_outer + 1 if the tolerance was not reached. Pinned by: Table 2's two
    Chebyshev rows (tests/golden/table2_chebyshev.txt).
    """
    m = len(w)
    u = np.zeros_like(f, dtype=np.result_type(f, 1.0))
    v = np.zeros_like(u)
    fn = np.linalg.norm(f)
    for k in range(1, max_outer + 1):
        u, v = inner_steps(A, f, u, v, w, a, at, K=m, k_start=0, Binv=Binv)
        if np.linalg.norm(f - A @ u) / fn < tol:
            return k, u
    return max_outer + 1, u


def refined_steps(A, b, x, K, w, a=None, at=None, refine_every=64, Binv=None):
    """K inner steps written as an outer FP64 accumulation plus a correction iteration.

    Every ``refine_every`` steps: x += e, the correction's right-hand side becomes
    r = b - A x, e restarts from 0 and the velocity and weight index carry over.
    Reading: this split (an addition of this implementation for mixed precision) is
    the same affine iteration as ``inner_steps`` on x, so in exact arithmetic the
    two agree. Pinned by: agreement with ``inner_steps`` to 1e-12 (tests).
    """
    x = np.array(x, dtype=np.float64, copy=True)
    e = np.zeros_like(x)
    v = np.zeros_like(x)
    r = b - A @ x
    done = 0
    while done < K:
        steps = min(refine_every, K - done)
        e, v = inner_steps(A, r, e, v, w, a, at, K=steps, k_start=done, Binv=Binv)
        done += steps
        x = x + e
        e = np.zeros_like(x)
        r = b - A @ x
    return x
