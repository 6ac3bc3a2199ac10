"""Meta-omega of the Helmholtz smoother (Sec. 3.2, Table 9).

The library's meta MLP 2 -> 64 -> 64 -> (m + 1) maps an instance's (k h, log2(n + 1) / 10)
to the m weights w_i = exp(o_i) / G (the log-omega parametrisation: the network
outputs log-weights, so the weights stay positive) and one momentum sigmoid(o_m) of the
NAG-Richardson(m) smoother that preconditions FGMRES(20). Training follows Algorithm 1
on complex64 sweeps: K sweeps from z = 0 with right-hand side b give z = M b with
M = p(A) the preconditioner, the loss is the mean log relative residual
ln(||b - A M b|| / ||b||) over a batch of random right-hand sides, and its gradient
comes from the library's complex adjoint sweep (A^H = conj(A)) and the meta network's
backward kernel, with the library's Adam step. The WANS multigrid around the smoother
is not built; the trained smoother is used alone as the FGMRES preconditioner.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import richm


def instance_inputs(specs) -> np.ndarray:
    """Network inputs [B][2] of Helmholtz instances given as (kind, n, k)."""
    return np.array([[k / (n + 1), math.log2(n + 1) / 10.0] for (_, n, k) in specs], dtype=np.float32)


class SmootherNet:
    """Meta-omega for NAG-Richardson(m) on Helmholtz problems (shared-momentum head).
    Initial network: the Chebyshev weights of eqs. 8-9 on [lo G, G] (G the instance's
    Gershgorin bound) and momentum `beta`, with a small output layer so that the
    network starts near them for every input."""

    def __init__(self, m: int = 5, K: int = 5, beta: float = 0.3, lo: float = 0.25, seed: int = 11,
                 out_scale: float = 1e-3):
        import richm_synth as synth  # seeded initialisation shared with the other networks
        layers = synth.mlp_init((2, 64, 64, m + 1), seed=seed)
        W3, _ = layers[2]
        unit = np.array(richm.chebyshev_weights(1.0, lo, m))
        b3 = np.concatenate([np.log(unit), [math.log(beta / (1.0 - beta))]])
        layers[2] = (np.asarray(W3) * out_scale, b3)
        self.P = torch.tensor(richm.pack_mlp_params(layers), dtype=torch.float32, device="cuda")
        self.m1 = torch.zeros_like(self.P)
        self.m2 = torch.zeros_like(self.P)
        self.t = 0
        self.m, self.K = m, K

    def coefficients(self, X: torch.Tensor, G: torch.Tensor):
        """(w, a, activations) for inputs X [B][2] and Gershgorin bounds G [B]."""
        acts = torch.empty(richm.meta_acts_size(X.shape[0], self.m), dtype=torch.float32, device="cuda")
        w, a, _ = richm.meta_forward_head(self.P, X, G, self.m, richm.HEAD_NAG_SHARED, acts)
        return w, a, acts

    def loss_and_grads(self, op: richm.Operator, X: torch.Tensor, G: torch.Tensor, B: torch.Tensor):
        """Loss (device FP64 scalar) and the parameter gradient for a batch of padded
        complex64 right-hand sides B (one per instance of op)."""
        m, K = self.m, self.K
        w, a, acts = self.coefficients(X, G)
        ck = torch.zeros(op.checkpoint_elems(K, K), dtype=torch.complex64, device="cuda")
        X0, XK, gK = op.zeros(richm.C64), op.zeros(richm.C64), op.zeros(richm.C64)
        op.forward_checkpointed(richm.C64, X0, B, w, a, None, m, K, K, 0, ck, XK)
        loss = op.loss_log_residual(richm.C64, XK, B, gK)
        gw, ga = torch.zeros_like(w), torch.zeros_like(a)
        op.sweeps_adjoint(richm.C64, ck, K, B, gK, w, a, None, m, K, 0, gw, ga, None, None)
        g = richm.meta_backward(self.P, X, G, acts, m, gw, ga)
        return loss, g

    def step(self, op, X, G, B, lr: float):
        loss, g = self.loss_and_grads(op, X, G, B)
        self.t += 1
        richm.adam_step(self.P, g, self.m1, self.m2, self.t, lr=lr)
        return loss


def random_rhs(op: richm.Operator, specs, seed: int) -> torch.Tensor:
    """Padded complex64 right-hand sides with real and imaginary parts uniform in [-1, 1)."""
    import richm_synth as synth
    parts = [(synth.rhs_uniform(seed, i, n) + 1j * synth.rhs_uniform(seed + 1, i, n)).ravel()
             for i, (_, n, _) in enumerate(specs)]
    t = torch.tensor(np.concatenate(parts).astype(np.complex64), device="cuda")
    return op.pack(t, richm.C64)


def train(net: SmootherNet, specs, steps: int = 200, lr: float = 3e-3, seed: int = 40, log=None):
    """Algorithm 1's loop over fresh random right-hand sides each step (instances of
    `specs`, one operator); returns the loss history."""
    op = richm.Operator([(kind, n, 1.0, 0.0, k) for kind, n, k in specs])
    X = torch.tensor(instance_inputs(specs), device="cuda")
    G = torch.tensor(np.array(op.gershgorin()), dtype=torch.float32, device="cuda")
    hist = []
    for s in range(steps):
        B = random_rhs(op, specs, seed + 2 * s)
        hist.append(float(net.step(op, X, G, B, lr).item()))
        if log and (s % 50 == 0 or s == steps - 1):
            log(f"step {s}: loss {hist[-1]:.4f}")
    op.close()
    return hist
