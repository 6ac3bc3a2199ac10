"""Two-level step with a Fourier-domain correction (oracle; test only).

FNS-type iteration (eqs. 19-20): smoothing steps u += B(f - A u), then the
correction u += H (f - A u) with H = F T Lambda T* F^{-1}. This oracle takes
T = I and a given diagonal symbol S in place of Lambda, so the correction is
u += Re( IFFT2( S * FFT2(f - A u) ) ), with the unnormalised forward transform
and the 1/n^2-normalised inverse (numpy's convention). Reading: the residual is
real, so only the real part of the corrected field is added. The symbol's gradient
(for learning it, Algorithm 2's Meta-Lambda step) is taken with respect to the real and
imaginary parts of every entry of S.
"""
from __future__ import annotations

import numpy as np

from .iterations import inner_steps


def fourier_correction(A, f, u, S):
    """u + Re(ifft2(S * fft2(f - A u))) on an (n, n) grid (flat in, flat out).

    Pinned by: numpy's FFT against an explicit DFT matrix for n <= 33 and S = 0
    leaving u unchanged (tests).
    """
    n = S.shape[0]
    r = (f - A @ u).reshape(n, n)
    c = np.fft.ifft2(S * np.fft.fft2(r))
    return u + c.real.ravel()


def fourier_correction_vjp(A, f, u, S, g):
    """Reverse mode of ``fourier_correction`` for the learned symbol of Sec. 3.1.

    Given g = dL/du' for u' = u + Re(ifft2(S * fft2(f - A u))) (g real), returns
    (dS, du): dS[k] = dL/dRe S[k] + i dL/dIm S[k] (complex (n, n)) and du = dL/du (flat).
    With r = f - A u, R = fft2(r), G = fft2(g), n^2 the inverse transform's scale:
    u' changes by Re(sum_x' e^{2 pi i k.x'/n} R[k] dS[k]) / n^2 at x' for a change dS[k],
    whose inner product with g is Re(conj(G[k]) R[k] dS[k]) / n^2, which gives
    dS = conj(R) G / n^2; and the map r -> Re(ifft2(S * fft2(r))) has the transpose
    g -> Re(ifft2(conj(S) * fft2(g))) in the real inner product, so
    du = g - A^T Re(ifft2(conj(S) * G)) (A symmetric here).

    Pinned by: central finite differences of <g, u'> in Re S, Im S and u, and torch
    autograd of the forward on complex tensors (tests).
    """
    n = S.shape[0]
    r = (f - A @ u).reshape(n, n)
    R = np.fft.fft2(r)
    G = np.fft.fft2(np.asarray(g, dtype=np.float64).reshape(n, n))
    dS = np.conj(R) * G / (n * n)
    h = np.fft.ifft2(np.conj(S) * G).real.ravel()
    du = np.asarray(g, dtype=np.float64).ravel() - A.T @ h
    return dS, du


def two_level_cycle(A, f, u, w, S, Binv=None):
    """One cycle: len(w) Richardson(m) smoothing steps then one Fourier correction."""
    u, _ = inner_steps(A, f, u, None, w, K=len(w), Binv=Binv)
    return fourier_correction(A, f, u, S)
