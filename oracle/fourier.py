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


def transition_field(tau, n):
    """The real field t(x) of a banded transition T (reading: T mixes each frequency
    with its neighbours within a band, with the same kernel tau[d] for every frequency;
    tau is a (2w+1, 2w+1) array indexed by the offset d + w, Hermitian-symmetric,
    tau[-d] = conj(tau[d]), so that t is real): t(x) = sum_d tau[d] exp(2 pi i d.x / n)
    on the n x n grid (x = (row, column) indices)."""
    tau = np.asarray(tau, dtype=np.complex128)
    w = (tau.shape[0] - 1) // 2
    i = np.arange(n)
    t = np.zeros((n, n), dtype=np.complex128)
    for a in range(-w, w + 1):
        for c in range(-w, w + 1):
            t += tau[a + w, c + w] * np.exp(2j * np.pi * (a * i[:, None] + c * i[None, :]) / n)
    return t.real


def fourier_correction_t(A, f, u, S, t):
    """u + t * Re(ifft2(S * fft2(t * (f - A u)))): the correction H (f - A u) with
    H = F T S T* F^{-1} (eqs. 19-20) for a banded transition T given by its real field t
    (`transition_field`; a kernel convolving the spectrum is a pointwise product on the
    grid). Pinned by: equality with the explicit matrix product F T S T^H F^{-1} built from
    DFT matrices and the band matrix T for small n; t = 1 gives ``fourier_correction``
    (tests)."""
    n = S.shape[0]
    r = (f - A @ u).reshape(n, n)
    c = np.fft.ifft2(S * np.fft.fft2(t * r)).real
    return u + (t * c).ravel()


def fourier_correction_t_vjp(A, f, u, S, t, g):
    """Reverse mode of ``fourier_correction_t``: (dS, dt, du) for g = dL/du' (real).
    With q = t r, Q = fft2(q), p = Re(ifft2(S Q)) (so u' = u + t p), gh = t g and
    Gh = fft2(gh): dS = conj(Q) Gh / n^2, h = Re(ifft2(conj(S) Gh)) (the transpose of
    q -> p applied to gh), dt = g p + r h, du = g - A^T (t h).
    Pinned by: central finite differences in Re S, Im S, t and u (tests)."""
    n = S.shape[0]
    r = (f - A @ u).reshape(n, n)
    g = np.asarray(g, dtype=np.float64).reshape(n, n)
    Q = np.fft.fft2(t * r)
    p = np.fft.ifft2(S * Q).real
    Gh = np.fft.fft2(t * g)
    dS = np.conj(Q) * Gh / (n * n)
    h = np.fft.ifft2(np.conj(S) * Gh).real
    dt = g * p + r * h
    du = g.ravel() - A.T @ (t * h).ravel()
    return dS, dt, du


def symbol_from_stencil(q, o, n):
    """The FNS symbol of a few network outputs (reading: Meta-Lambda's architecture is not
    given; its output Lambda approximates the inverses of A's eigenvalues, here as the
    regularised inverse of a periodic 9-point symbol): p_m = q_m exp(o_m) (m < 5),
    delta = q_5 exp(o_5), sigma(k) = p0 + 2 p1 cos t2 + 2 p2 cos t1 + 2 p3 cos(t1 + t2)
    + 2 p4 cos(t1 - t2) with t = 2 pi k / n, and S = sigma / (sigma^2 + delta^2).
    Pinned by: for a Q1 stencil q and o = 0, sigma is the exact spectrum of the periodic
    extension of A (eigenvalues of the circulant matrix, tests); central differences of
    the reverse mode."""
    q = np.asarray(q, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    p = q[:5] * np.exp(o[:5])
    d = q[5] * np.exp(o[5])
    t = 2.0 * np.pi * np.arange(n) / n
    t1, t2 = np.meshgrid(t, t, indexing="ij")
    sig = p[0] + 2 * p[1] * np.cos(t2) + 2 * p[2] * np.cos(t1) + 2 * p[3] * np.cos(t1 + t2) \
        + 2 * p[4] * np.cos(t1 - t2)
    return (sig / (sig * sig + d * d)).astype(np.complex128)


def transition_band(tau9, n):
    """The transition field of the library's band parametrisation: tau9 = (tau_0, then
    (re, im) of the offsets (0,1), (1,0), (1,1), (1,-1)), the other half of the 3 x 3
    kernel by Hermitian symmetry; the field of `transition_field`."""
    t = np.asarray(tau9, dtype=np.float64)
    tau = np.zeros((3, 3), dtype=np.complex128)
    tau[1, 1] = t[0]
    for q, (a, c) in enumerate([(0, 1), (1, 0), (1, 1), (1, -1)]):
        v = t[1 + 2 * q] + 1j * t[2 + 2 * q]
        tau[a + 1, c + 1] = v
        tau[-a + 1, -c + 1] = np.conj(v)
    return transition_field(tau, n)


def two_level_cycle(A, f, u, w, S, Binv=None):
    """One cycle: len(w) Richardson(m) smoothing steps then one Fourier correction."""
    u, _ = inner_steps(A, f, u, None, w, K=len(w), Binv=Binv)
    return fourier_correction(A, f, u, S)
