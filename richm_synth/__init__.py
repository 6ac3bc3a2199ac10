"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds random-number generation and workload recipes only; it
contains none of the solver's arithmetic (no stencil, weight or iteration).
All streams come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in counter form: the
i-th 64-bit output of stream ``key`` is ``mix64(key + (i + 1) * GOLDEN)``.

Grids follow one convention everywhere: a dense instance array has shape
``(n, n)``; row index ``i`` is the y coordinate (node ``y = (i + 1) h``) and
column index ``j`` the x coordinate (node ``x = (j + 1) h``), ``h = 1/(n + 1)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, *sub: int) -> int:
    """Derive a 64-bit stream key from a seed and sub-stream indices."""
    key = seed & _MASK64
    for s in sub:
        z = np.array([(key + (s + 1) * 0x9E3779B97F4A7C15) & _MASK64], dtype=np.uint64)
        key = int(_mix64(z)[0])
    return key


def splitmix64(key: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of SplitMix64 stream ``key`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(key & _MASK64) + i * GOLDEN
        return _mix64(z)


def uniform(key: int, count: int, lo: float = 0.0, hi: float = 1.0, start: int = 0) -> np.ndarray:
    """Doubles uniform in [lo, hi) from the top 53 bits of each output."""
    u = (splitmix64(key, count, start) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


# ----------------------------------------------------------------------------
# Workload recipes (shapes and distributions of the paper's test problems)
# ----------------------------------------------------------------------------

@dataclass(frozen=True)
class AnisoInstance:
    """One anisotropic diffusion instance: eps, theta, interior size n."""
    eps: float
    theta: float
    n: int


def rhs_uniform(seed: int, index: int, n: int) -> np.ndarray:
    """Right-hand side ``(n, n)`` uniform in [-1, 1) for instance ``index``."""
    return uniform(stream_key(seed, index), n * n, -1.0, 1.0).reshape(n, n)


def rhs_normal(seed: int, index: int, n: int) -> np.ndarray:
    """Right-hand side ``(n, n)`` ~ N(0, 1) (Box-Muller on two uniform streams)."""
    u1 = uniform(stream_key(seed, index, 0), n * n)
    u2 = uniform(stream_key(seed, index, 1), n * n)
    r = np.sqrt(-2.0 * np.log1p(-u1))
    return (r * np.cos(2.0 * math.pi * u2)).reshape(n, n)


def single_aniso(eps: float = 1e-2, theta: float = math.pi / 6, n: int = 63, seed: int = 0):
    """One instance with b ~ U[-1, 1] (the 63x63 FP64 Richardson(8) workload)."""
    return AnisoInstance(eps, theta, n), rhs_uniform(seed, 0, n)


def batched_aniso(batch: int = 256, sizes=(127, 255, 511), param_seed: int = 1,
                  log_eps=(-3.0, 0.0)) -> list[AnisoInstance]:
    """Instances with eps = 10^U[log_eps], theta ~ U[0, pi), n uniform from ``sizes``."""
    k = stream_key(param_seed)
    u = uniform(k, 3 * batch).reshape(batch, 3)
    out = []
    for b in range(batch):
        eps = 10.0 ** (log_eps[0] + (log_eps[1] - log_eps[0]) * u[b, 0])
        theta = math.pi * u[b, 1]
        n = int(sizes[min(int(u[b, 2] * len(sizes)), len(sizes) - 1)])
        out.append(AnisoInstance(float(eps), float(theta), n))
    return out


def batched_rhs(instances, seed: int = 2) -> list[np.ndarray]:
    """Per-instance right-hand sides uniform in [-1, 1)."""
    return [rhs_uniform(seed, b, inst.n) for b, inst in enumerate(instances)]


def fourier_symbol(n: int, seed: int = 3) -> np.ndarray:
    """Complex symbol ``(n, n)``: real part U[0, 1), imaginary part U[-0.1, 0.1)."""
    k = stream_key(seed)
    re = uniform(stream_key(k, 0), n * n, 0.0, 1.0)
    im = uniform(stream_key(k, 1), n * n, -0.1, 0.1)
    return (re + 1j * im).reshape(n, n)


def helmholtz_weights(m: int, h: float, seed: int = 4) -> np.ndarray:
    """Real weights (h^2 / 8) * U[0.5, 1.5) for m steps."""
    return (h * h / 8.0) * uniform(stream_key(seed), m, 0.5, 1.5)


def point_sources(n: int, count: int = 16, seed: int = 5) -> list[tuple[int, int]]:
    """Distinct interior (row, col) locations of unit point sources."""
    k = stream_key(seed)
    pts: list[tuple[int, int]] = []
    start = 0
    while len(pts) < count:
        u = uniform(k, 2, 0.0, 1.0, start=start)
        start += 2
        p = (min(int(u[0] * n), n - 1), min(int(u[1] * n), n - 1))
        if p not in pts:
            pts.append(p)
    return pts


def point_source_rhs(n: int, count: int = 16, seed: int = 5) -> np.ndarray:
    """``(count, n, n)`` complex right-hand sides, each a unit impulse."""
    out = np.zeros((count, n, n), dtype=np.complex128)
    for s, (i, j) in enumerate(point_sources(n, count, seed)):
        out[s, i, j] = 1.0
    return out


def meta_inputs(instances) -> np.ndarray:
    """Network inputs ``(batch, 2)``: (log10 eps, theta)."""
    return np.array([[math.log10(t.eps), t.theta] for t in instances], dtype=np.float64)


def mlp_init(layers=(2, 64, 64, 17), seed: int = 7) -> list[tuple[np.ndarray, np.ndarray]]:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases, row-major W[out][in]."""
    params = []
    for li, (fi, fo) in enumerate(zip(layers[:-1], layers[1:])):
        bound = 1.0 / math.sqrt(fi)
        w = uniform(stream_key(seed, li, 0), fo * fi, -bound, bound).reshape(fo, fi)
        b = uniform(stream_key(seed, li, 1), fo, -bound, bound)
        params.append((w, b))
    return params
