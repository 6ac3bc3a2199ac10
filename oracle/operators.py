"""Discrete operators, assembled from their definitions (oracle; test only).

Grid convention: interior unknown (i, j), 0 <= i, j < n, sits at node
x = (j + 1) h, y = (i + 1) h with h = 1 / (n + 1); its flat index is i*n + j.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def diffusion_tensor(eps: float, theta: float) -> np.ndarray:
    """C = R(theta) diag(1, eps) R(theta)^T (Sec. 2.4, the matrix under eq. 18)."""
    c, s = math.cos(theta), math.sin(theta)
    R = np.array([[c, -s], [s, c]])
    return R @ np.diag([1.0, eps]) @ R.T


def q1_element_stiffness(C: np.ndarray) -> np.ndarray:
    """4x4 bilinear element matrix  K_ab = int grad(phi_a)^T C grad(phi_b)  on a square.

    Local nodes in (xi, eta) order (0,0), (1,0), (0,1), (1,1). Computed with the
    2x2 Gauss rule on the reference square; the element size cancels in 2-D
    (gradients scale by 1/h, the area by h^2). Pinned by: the 1/3[-1 -1 -1; -1 8 -1;
    -1 -1 -1] Laplacian stencil, exact action on x^2, y^2, xy (tests).
    """
    g = 0.5 / math.sqrt(3.0)
    pts = [0.5 - g, 0.5 + g]
    nodes = [(0, 0), (1, 0), (0, 1), (1, 1)]
    K = np.zeros((4, 4))
    for xi in pts:
        for eta in pts:
            grads = []
            for (a, b) in nodes:
                fx = xi if a else 1.0 - xi
                fy = eta if b else 1.0 - eta
                dfx = 1.0 if a else -1.0
                dfy = 1.0 if b else -1.0
                grads.append(np.array([dfx * fy, fx * dfy]))
            for p in range(4):
                for q in range(4):
                    K[p, q] += 0.25 * grads[p] @ C @ grads[q]
    return K


def assemble_q1(n: int, eps: float, theta: float, window=None) -> sp.csr_matrix:
    """Stiffness matrix of -div(C grad u) = f, u = 0 on the boundary (eq. 18, Sec. 2.4).

    Uniform (n+1) x (n+1) element mesh of the unit square, bilinear elements,
    Dirichlet nodes eliminated, so A has n^2 rows. Assembled element by element:
    every element adds its local matrix into the rows/columns of its interior nodes.
    ``window=(i0, i1, j0, j1)`` restricts rows and columns to the unknowns with
    i0 <= i < i1 and j0 <= j < j1 (the block A[W, W], flat index within the window).
    Pinned by: separable theta=0 eigenvalues, exact quadratic action, symmetry,
    Table 2 Chebyshev iteration counts (tests).
    """
    Ke = q1_element_stiffness(diffusion_tensor(eps, theta))
    N = n + 1
    if window is None:
        i0, i1, j0, j1 = 0, n, 0, n
    else:
        i0, i1, j0, j1 = window
    wi, wj = i1 - i0, j1 - j0
    # elements touching the window's nodes: element (ey, ex) spans nodes ey..ey+1
    # (node index = unknown index + 1)
    ey = np.arange(max(i0, 0), min(i1 + 1, N))
    ex = np.arange(max(j0, 0), min(j1 + 1, N))
    EY, EX = np.meshgrid(ey, ex, indexing="ij")
    EY = EY.ravel()
    EX = EX.ravel()
    local = [(0, 0), (1, 0), (0, 1), (1, 1)]  # (dx, dy)
    rows, cols, vals = [], [], []
    for p, (pdx, pdy) in enumerate(local):
        pi = EY + pdy - 1  # unknown row index of local node p
        pj = EX + pdx - 1
        okp = (pi >= i0) & (pi < i1) & (pj >= j0) & (pj < j1)
        for q, (qdx, qdy) in enumerate(local):
            qi = EY + qdy - 1
            qj = EX + qdx - 1
            ok = okp & (qi >= i0) & (qi < i1) & (qj >= j0) & (qj < j1)
            rows.append((pi[ok] - i0) * wj + (pj[ok] - j0))
            cols.append((qi[ok] - i0) * wj + (qj[ok] - j0))
            vals.append(np.full(int(ok.sum()), Ke[p, q]))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(wi * wj, wi * wj))
    return A.tocsr()


def helmholtz_wavenumber(n: int, points_per_wavelength: float = 10.0) -> float:
    """k with ``points_per_wavelength`` grid spacings per wavelength: 2 pi / (ppw h)."""
    h = 1.0 / (n + 1)
    return 2.0 * math.pi / (points_per_wavelength * h)


def assemble_helmholtz(n: int, k: float, absorbing: bool = True, window=None) -> sp.csr_matrix:
    """-Lap(u) - k^2 u, 5-point finite differences, h = 1/(n+1) (eq. 22).

    Interior rows follow eq. 22: (1/h^2)[0 -1 0; -1 4-k^2h^2 -1; 0 -1 0].
    With ``absorbing`` the boundary value next to each boundary-adjacent unknown
    is a ghost node eliminated through the first-order condition
    du/dn - i k u = 0, discretised one-sidedly as -(u_1 - u_0)/h - i k u_0 = 0,
    i.e. u_0 = u_1 / (1 - i k h) (time factor exp(-i omega t)); otherwise u_0 = 0
    (Dirichlet). Built row by row from the stencil. Pinned by: Schur-complement
    elimination of explicit ghost unknowns, complex symmetry, k=0 Dirichlet
    eigenvalues (tests).
    """
    h = 1.0 / (n + 1)
    if window is None:
        i0, i1, j0, j1 = 0, n, 0, n
    else:
        i0, i1, j0, j1 = window
    wi, wj = i1 - i0, j1 - j0
    ghost = (1.0 / (1.0 - 1j * k * h)) if absorbing else 0.0
    I, J = np.meshgrid(np.arange(i0, i1), np.arange(j0, j1), indexing="ij")
    I = I.ravel()
    J = J.ravel()
    me = (I - i0) * wj + (J - j0)
    diag = np.full(I.shape, (4.0 - (k * h) ** 2) / h ** 2, dtype=np.complex128)
    rows, cols, vals = [me], [me], [None]
    for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        ni, nj = I + di, J + dj
        inside = (ni >= 0) & (ni < n) & (nj >= 0) & (nj < n)
        # a neighbour outside the domain is a ghost/boundary node: eliminated
        diag = diag + np.where(inside, 0.0, -ghost / h ** 2)
        inw = inside & (ni >= i0) & (ni < i1) & (nj >= j0) & (nj < j1)
        rows.append(me[inw])
        cols.append((ni[inw] - i0) * wj + (nj[inw] - j0))
        vals.append(np.full(int(inw.sum()), -1.0 / h ** 2, dtype=np.complex128))
    vals[0] = diag
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(wi * wj, wi * wj))
    return A.tocsr()


def sponge_gamma(n: int, omega: float, c: float = 1.0, window=None) -> np.ndarray:
    """The damping mask gamma of eq. 21 at the interior nodes (row-major over the window).

    Readings: gamma rises linearly from 0 at depth L to omega on the boundary,
    gamma(x) = omega * max(0, 1 - d(x) / L), with d(x) the distance from node x to the
    boundary of the unit square and L = 2 pi c / omega one wavelength (the paper gives
    the layer's thickness, one wavelength, and the end values, not the profile); the
    wave speed c is constant. Pinned by: hand values (tests).
    """
    h = 1.0 / (n + 1)
    if window is None:
        i0, i1, j0, j1 = 0, n, 0, n
    else:
        i0, i1, j0, j1 = window
    I, J = np.meshgrid(np.arange(i0, i1), np.arange(j0, j1), indexing="ij")
    d = h * np.minimum(np.minimum(I + 1, n - I), np.minimum(J + 1, n - J))
    L = 2.0 * math.pi * c / omega
    return (omega * np.maximum(0.0, 1.0 - d / L)).ravel()


def assemble_helmholtz_sponge(n: int, omega: float, c: float = 1.0, window=None) -> sp.csr_matrix:
    """Eq. 21: -Lap(u) - k^2 u + i gamma omega / c^2 u = f, u = 0 on the boundary,
    k = omega / c, with the 5-point stencil of eq. 22 (h = 1/(n+1)) and the damping
    mask of `sponge_gamma` on the diagonal. Pinned by: Im(x^H A x) equals the
    mask-weighted energy sum over the nodes, computed node by node (tests); the
    Hermitian part is the Dirichlet Helmholtz operator.
    """
    k = omega / c
    A = assemble_helmholtz(n, k, absorbing=False, window=window)
    g = sponge_gamma(n, omega, c, window)
    return (A + sp.diags(1j * g * omega / c ** 2)).tocsr()


def gershgorin_max(A: sp.spmatrix) -> float:
    """max_i sum_j |a_ij|: an upper bound on the spectrum of symmetric A (used for lmax)."""
    return float(np.abs(A).sum(axis=1).max())
