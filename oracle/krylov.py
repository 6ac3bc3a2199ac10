"""Restarted flexible GMRES in FP64 / complex128 (oracle; test only).

Sec. 3.2 of the paper uses the multilevel solver with a NAG-Richardson(m) smoother as a
preconditioner of FGMRES restarted every 20 iterations (Table 9). This is FGMRES as
Saad states it (SIAM J. Sci. Comput. 14 (1993) 461-469): right preconditioning that
may change from one iteration to the next, x_m = x_0 + Z_m y_m with the
preconditioned vectors z_j kept, y_m the least-squares solution of the small
Hessenberg problem. Here the Arnoldi basis is orthogonalised by modified
Gram-Schmidt, the least-squares problem is solved by a library routine at every
iteration (its residual is the iteration's residual estimate), and the iteration
count is the number of Arnoldi steps until that estimate falls to tol * ||b||.
Pinned by: with the identity preconditioner every cycle minimises the residual over
the Krylov space (brute force on small systems); an exact preconditioner converges in
one step; a polynomial preconditioner p(A) gives GMRES on A p(A) (tests).
"""
from __future__ import annotations

import numpy as np


def fgmres(A, b, x0=None, M=None, m=20, tol=1e-6, max_iters=10000):
    """Solve A x = b. M: callable v -> z (the preconditioner of the iteration), or None
    for the identity. Returns (x, iterations, estimates) with estimates the relative
    residual estimate after every Arnoldi step, and iterations = max_iters + 1 if tol was
    not reached."""
    b = np.asarray(b)
    dt = np.result_type(b, A.dtype, 1.0)
    x = np.zeros(b.shape, dt) if x0 is None else np.array(x0, dtype=dt, copy=True)
    bn = np.linalg.norm(b)
    est = []
    its = 0
    while its < max_iters:
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta <= tol * bn:
            return x, its, est
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m), dt)
        y = None
        for j in range(m):
            z = V[j] if M is None else M(V[j])
            Z.append(z)
            w = A @ z
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            e1 = np.zeros(j + 2, dt)
            e1[0] = beta
            y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
            res = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y)
            its += 1
            est.append(res / bn)
            if res <= tol * bn or H[j + 1, j] == 0.0 or its >= max_iters:
                break
            V.append(w / H[j + 1, j])
        x = x + np.stack(Z, axis=1) @ y
        if est[-1] <= tol:
            return x, its, est
    return x, max_iters + 1, est


def richardson_preconditioner(A, w, a=None, at=None, K=None):
    """The NAG-Richardson(m) smoother as a preconditioner: z = K inner steps of the Table 1
    iteration on A z = v from z = 0 (zero velocity), K = len(w) by default."""
    from oracle.iterations import inner_steps
    K = len(w) if K is None else K

    def M(v):
        z, _ = inner_steps(A, v, np.zeros_like(v), None, w, a, at, K=K)
        return z
    return M
