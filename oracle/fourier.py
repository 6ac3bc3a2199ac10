"""Two-level step with a Fourier-domain correction (oracle; test only).

FNS-type iteration (eqs. 19-20): smoothing steps u += B(f - A u), then the
correction u += H (f - A u) with H = F T Lambda T* F^{-1}. This oracle takes
T = I and a given diagonal symbol S in place of Lambda, so the correction is
u += Re( IFFT2( S * FFT2(f - A u) ) ), with the unnormalised forward transform
and the 1/n^2-normalised inverse (numpy's convention). Reading: the residual is
real, so only the real part of the corrected field is added.
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


def two_level_cycle(A, f, u, w, S, Binv=None):
    """One cycle: len(w) Richardson(m) smoothing steps then one Fourier correction."""
    u, _ = inner_steps(A, f, u, None, w, K=len(w), Binv=Binv)
    return fourier_correction(A, f, u, S)
