"""Point samples of K sweeps on grids too large for the full oracle (oracle; test only).

A 9-point (or 5-point) stencil couples a point only to its Chebyshev-distance-1
neighbours, so after K sweeps the value at (i, j) depends only on the inputs
within distance K. Running the same Table 1 iteration on the sub-grid of radius K
around (i, j), with the operator block A[W, W] assembled on that window, gives
the exact value at (i, j) (windows clipped at the true boundary keep the true
boundary condition). Pinned by: equality with the full-grid run (tests).
"""
from __future__ import annotations

import numpy as np

from .iterations import inner_steps
from .operators import assemble_helmholtz, assemble_q1


def sampled_sweeps(op, n, X0, V0, F, w, a, at, K, points, k_start=0, jacobi=False):
    """Values at ``points`` after K inner steps from (X0, V0) with right-hand side F.

    op: ("q1", eps, theta) or ("helmholtz", k); X0, V0, F: (n, n) arrays (V0 may be
    None for zero velocity); w, a, at as in ``inner_steps``.
    """
    out = []
    for (i, j) in points:
        win = (max(0, i - K), min(n, i + K + 1), max(0, j - K), min(n, j + K + 1))
        i0, i1, j0, j1 = win
        if op[0] == "q1":
            A = assemble_q1(n, op[1], op[2], window=win)
        else:
            A = assemble_helmholtz(n, op[1], window=win)
        x = X0[i0:i1, j0:j1].ravel()
        v = None if V0 is None else V0[i0:i1, j0:j1].ravel()
        f = F[i0:i1, j0:j1].ravel()
        Binv = None
        if jacobi:
            d = A.diagonal()
            Binv = (lambda r, d=d: r / d)
        xK, _ = inner_steps(A, f, x, v, w, a, at, K=K, k_start=k_start, Binv=Binv)
        out.append(xK.reshape(i1 - i0, j1 - j0)[i - i0, j - j0])
    return np.array(out)
