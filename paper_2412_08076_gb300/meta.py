"""Meta-network parameters: initialisation, storage and the weight map.

The meta network (Sec. 2.3) maps PDE parameters (log10 eps, theta) to the m
weights and the momentum of NAG-Richardson(m). Its output o maps to
w_i = exp(o_i) / G (G the instance's Gershgorin bound) and a = sigmoid(o_m).
The initial network is random in its hidden layers and starts its output layer
at the momentum-aware Chebyshev weights: eqs. 8-9 on [c G / 30, c G] with c = 1.6,
a stretch of the semi-iteration interval for which every per-mode period transfer
of NAG with a = 0.3 stays inside the unit disk on [0, G]. So an untrained network
already gives a convergent solver, and training only improves it.

The other output heads (Richardson, MOM, NAG and NAGex with per-step momenta) start
the same way: Chebyshev weights for Richardson (c = 1), and for the momentum heads
the smallest stretch c (in steps of 0.05) whose period transfers with momentum beta
stay in the unit disk, every a_i (and at_i) at beta.
"""
from __future__ import annotations

import math
import os

import numpy as np

HIDDEN = 64
STABLE_STRETCH = 1.6
SEMI_ALPHA = 1.0 / 30.0
PARAM_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "params")


def chebyshev_unit_weights(m: int, stretch: float = STABLE_STRETCH, alpha: float = SEMI_ALPHA) -> np.ndarray:
    """G * w_i for eqs. 8-9 on [alpha s G, s G] (independent of G), from the library's
    richm_chebyshev_weights with G = 1."""
    from . import richm
    return np.array(richm.chebyshev_weights(stretch, alpha * stretch, m))


HEAD_NAG_SHARED, HEAD_RICHARDSON, HEAD_MOM, HEAD_NAG, HEAD_NAGEX = 0, 1, 2, 3, 4


def head_outputs(head: int, m: int) -> int:
    return {HEAD_NAG_SHARED: m + 1, HEAD_RICHARDSON: m, HEAD_MOM: 2 * m, HEAD_NAG: 2 * m, HEAD_NAGEX: 3 * m}[head]


def stable_stretch(m: int, beta: float, lookahead: bool, step: float = 0.05, top: float = 4.0) -> float:
    """Smallest c = 1 + k step for which the period transfer of Chebyshev weights on
    [c/30, c] with momentum beta (look-ahead beta for NAG, 0 for MOM) has spectral
    radius <= 1 at every eigenvalue of [0, 1]."""
    lam = np.linspace(0.0, 1.0, 4001)
    for k in range(int(round((top - 1.0) / step)) + 1):
        c = 1.0 + k * step
        r = period_radius(chebyshev_unit_weights(m, c), beta, lam, beta if lookahead else 0.0)
        if r.max() <= 1.0 + 1e-12:
            return c
    raise ValueError(f"no stable stretch up to {top} for m = {m}, beta = {beta}")


def init_params(m: int = 16, beta: float = 0.3, seed: int = 7, out_scale: float = 0.01,
                head: int = HEAD_NAG_SHARED, stretch: float = STABLE_STRETCH, leja: bool = False,
                fixed_beta: bool = False) -> np.ndarray:
    """Flat FP32 parameter vector in the library's order (W1, b1, W2, b2, W3, b3).

    Shared-momentum head options: `stretch` of the Chebyshev interval, `leja` to start the
    weights in the library's Leja step order (richm_leja_order) instead of index order,
    and `fixed_beta` to make the momentum output the constant `beta` (its weight row
    zero; training then leaves it untouched, see train.Trainer)."""
    import richm_synth as synth  # seeded generator shared by every consumer
    layers = synth.mlp_init((2, HIDDEN, HIDDEN, head_outputs(head, m)), seed=seed)
    W3, b3 = layers[2]
    W3 = W3 * out_scale
    logit = math.log(beta / (1.0 - beta))
    if head == HEAD_NAG_SHARED:
        unit = chebyshev_unit_weights(m, stretch)
        if leja:
            from . import richm
            unit = unit[richm.leja_order(unit)]
        b3 = np.concatenate([np.log(unit), [logit]])
        if fixed_beta:
            W3 = np.array(W3, copy=True)
            W3[m, :] = 0.0
    elif head == HEAD_RICHARDSON:
        b3 = np.log(chebyshev_unit_weights(m, 1.0))
    else:
        c = stable_stretch(m, beta, head != HEAD_MOM)
        moms = (2 if head == HEAD_NAGEX else 1) * m
        b3 = np.concatenate([np.log(chebyshev_unit_weights(m, c)), np.full(moms, logit)])
    layers[2] = (W3, b3)
    flat = []
    for W, b in layers:
        flat.append(np.asarray(W, dtype=np.float64).ravel())
        flat.append(np.asarray(b, dtype=np.float64).ravel())
    return np.concatenate(flat).astype(np.float32)


def trained_path(m: int, head: int = HEAD_NAG_SHARED, precond: int = 0, variant: str = "") -> str:
    """Where the trained network of a head is kept; variant "beta03" is the m = 16 network
    trained with its momentum held at 0.3."""
    if head == HEAD_NAG_SHARED and precond == 0:
        return os.path.join(PARAM_DIR, f"meta_m{m}{'_' + variant if variant else ''}.npy")
    return os.path.join(PARAM_DIR, f"meta_m{m}_head{head}_precond{precond}.npy")


def load_params(m: int = 16, prefer_trained: bool = True, head: int = HEAD_NAG_SHARED,
                precond: int = 0, variant: str = "") -> tuple[np.ndarray, str]:
    """(params, source): the trained network if one was saved, else the initial one."""
    p = trained_path(m, head, precond, variant)
    if prefer_trained and os.path.exists(p):
        return np.load(p).astype(np.float32), "trained"
    return init_params(m, head=head), "initial"


def symbol_max(eps: float, theta: float, grid: int = 513) -> float:
    """Upper bound on the Q1 operator's spectrum: the maximum of the library's stencil's
    Fourier symbol c + 2 ax cos x + 2 ay cos y + 2 d1 cos(x + y) + 2 d2 cos(x - y) over
    x in [0, pi], y in [-pi, pi] (a symmetric Toeplitz-block-Toeplitz matrix's
    eigenvalues lie within the range of its symbol)."""
    from . import richm
    cen, ax, ay, d1, d2, _ = richm.q1_stencil(eps, theta)  # the library's stencil (host)
    x = np.linspace(0.0, math.pi, grid)
    y = np.linspace(-math.pi, math.pi, 2 * grid - 1)
    X, Y = np.meshgrid(x, y, indexing="ij")
    S = cen + 2 * ax * np.cos(X) + 2 * ay * np.cos(Y) + 2 * d1 * np.cos(X + Y) + 2 * d2 * np.cos(X - Y)
    return float(S.max())


def period_radius(w, beta: float, lam, lookahead: float | None = None) -> np.ndarray:
    """Spectral radius of one period's 2x2 per-mode transfer at each eigenvalue lam
    (A symmetric, so every eigenvector evolves independently) for the Table 1 step
    e' = e + beta (e - e_prev) - w lam (e + at (e - e_prev)), at = `lookahead`
    (default beta: NAG; 0: MOM)."""
    at = beta if lookahead is None else lookahead
    lam = np.asarray(lam, dtype=np.float64)
    P = np.tile(np.eye(2), (lam.size, 1, 1))
    for wi in w:
        T = np.zeros((lam.size, 2, 2))
        T[:, 0, 0] = 1.0 + beta - wi * lam * (1.0 + at)
        T[:, 0, 1] = -beta + wi * lam * at
        T[:, 1, 0] = 1.0
        P = T @ P
    return np.abs(np.linalg.eigvals(P)).max(axis=1)
