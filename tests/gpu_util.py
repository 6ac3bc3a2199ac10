"""Helpers for the GPU parity tests: seeded inputs in, library buffers out.

Inputs come from richm_synth; they reach the device through the library's own
pack kernel and come back through its unpack kernel.
"""
from __future__ import annotations

import numpy as np
import torch

from paper_2412_08076_gb300 import richm


def make_op(instances, kind=richm.ANISO_Q1, k=0.0):
    return richm.Operator([(kind, t.n, getattr(t, "eps", 1.0), getattr(t, "theta", 0.0), k) for t in instances])


def to_dev(op, arrays, dtype):
    """List of (n, n) numpy arrays -> padded device buffer of `dtype`."""
    flat = np.concatenate([np.asarray(a).ravel() for a in arrays])
    t = torch.tensor(flat, dtype=richm.TORCH_DTYPE[dtype], device="cuda")
    return op.pack(t, dtype)


def from_dev(op, buf, dtype):
    """Padded device buffer -> list of (n, n) numpy arrays."""
    d = op.unpack(buf, dtype)
    d = (d.float() if d.dtype == torch.bfloat16 else d).cpu().numpy()
    out, off = [], 0
    for n in op.ns:
        out.append(d[off:off + n * n].reshape(n, n))
        off += n * n
    return out


def coef(arr, dtype):
    return torch.tensor(np.asarray(arr), dtype=richm.REAL_DTYPE[dtype], device="cuda").contiguous()


def nag_weights(G, m, beta=0.3, scale=1.6, alpha=1.0 / 30.0):
    """Chebyshev semi-iteration weights on [alpha c G, c G] (c = scale) and momentum beta.

    With beta = 0.3 and m = 16, c = 1.6 keeps every per-mode period transfer of the
    NAG iteration inside the unit disk on [0, G] (checked by tests/test_weights_cpu.py).
    """
    from oracle.iterations import chebyshev_weights
    G = np.atleast_1d(G)
    w = np.stack([chebyshev_weights(scale * g, alpha * scale * g, m) for g in G])
    a = np.full_like(w, beta)
    return w, a


def period_amplification(w, a, at, G, k_start, K, npts=4001):
    """max over lambda in [0, G] of the 2x2 per-mode transfer norm from sweep k+1 to K,
    for every k (FP32 rounding made at sweep k is carried by these factors)."""
    lam = np.linspace(0.0, G, npts)
    m = len(w)
    amps = np.zeros(K)
    # backward accumulation of the products
    P = np.tile(np.eye(2), (npts, 1, 1))
    for k in range(K - 1, -1, -1):
        amps[k] = np.linalg.norm(P, ord=2, axis=(1, 2)).max()
        i = (k_start + k) % m
        ai = a[i] if a is not None else 0.0
        ati = at[i] if at is not None else ai
        mu = 1.0 - w[i] * lam
        T = np.zeros((npts, 2, 2))
        T[:, 0, 0] = 1.0 + ai - w[i] * lam * (1.0 + ati)
        T[:, 0, 1] = -ai + w[i] * lam * ati
        T[:, 1, 0] = 1.0
        P = P @ T
    return amps


def fp32_bound(w, a, at, G, k_start, K, xmax, bmax, u=2.0 ** -24):
    """Rounding bound for K sweeps in a precision of unit roundoff u (FP32 by default)
    started from the same state as an exact run:
    16 u sum_k amp_k ((1+|a|+|at|) |x| + |w| (|b| + G (1+2|at|) |x|)), with amp_k the
    largest per-mode transfer norm from sweep k+1 to the end."""
    amps = period_amplification(w, a, at, G, k_start, K)
    tot = 0.0
    for k in range(K):
        i = (k_start + k) % len(w)
        ai = 0.0 if a is None else abs(a[i])
        ati = ai if at is None else abs(at[i])
        per = (1 + ai + ati) * xmax + abs(w[i]) * (bmax + G * (1 + 2 * ati) * xmax)
        tot += amps[k] * per
    return 16.0 * u * tot
