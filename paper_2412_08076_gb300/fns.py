"""Richardson(m)-FNS (Sec. 3.1): M smoothing sweeps of Richardson(m) per outer iteration
(eq. 19 with the Richardson(m) smoother in place of B), then the Fourier neural
iteration (eq. 20) with T = I and a symbol S shared by the instances of a batch:
  x <- x + Re(IFFT2(S .* FFT2(b - A x))).
Every step runs in the library's kernels (richm_apply_sweeps, richm_fourier_correction,
richm_forward_checkpointed, richm_sweeps_adjoint, richm_fourier_correction_vjp,
richm_loss_log_residual, richm_adam_step); this module only sequences the calls.

Training (Algorithm 2, alternating optimisation) with the parameters held directly: the
symbol S (complex [n][n], in place of the Meta-Lambda network's output, since the FNO
architecture of that network is not given) and the smoother's m weights per instance (in
place of Meta-omega's output). `FNS.loss_and_grads` unrolls C outer iterations from x = 0
and returns the log-residual loss (eq. 15) with its gradients in S and in the weights;
`train_alternating` runs Algorithm 2's schedule: the symbol alone with the weights fixed
at their initial value, then weights and symbol in turn.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import richm


def periodic_inverse_symbol(coef, n: int, delta: float = 0.0) -> np.ndarray:
    """S(k) = 1 / lambda(k) for the periodic extension of a Q1 stencil (coef: centre,
    x-neighbour, y-neighbour, corner (+1, +1), corner (+1, -1), as Operator.stencil
    gives them): lambda(k) = c + 2 ax cos t2 + 2 ay cos t1 + 2 d1 cos(t1 + t2)
    + 2 d2 cos(t1 - t2), t = 2 pi k / n. lambda(0) = 0 (the rows sum to zero), so the
    inverse is regularised as lambda / (lambda^2 + delta^2) (delta defaults to 1e-3 of
    the largest |lambda|)."""
    c, ax, ay, d1, d2 = (float(v) for v in coef[:5])
    t = 2.0 * math.pi * np.arange(n) / n
    t1, t2 = np.meshgrid(t, t, indexing="ij")
    lam = c + 2 * ax * np.cos(t2) + 2 * ay * np.cos(t1) + 2 * d1 * np.cos(t1 + t2) + 2 * d2 * np.cos(t1 - t2)
    if delta <= 0.0:
        delta = 1e-3 * float(np.abs(lam).max())
    return (lam / (lam * lam + delta * delta)).astype(np.complex128)


class FNS:
    """Richardson(m)-FNS on an operator of Q1 instances of one size (FP32 state)."""

    def __init__(self, op: richm.Operator, w: torch.Tensor, m: int, M: int, symbol: torch.Tensor, precond: int = 1):
        self.op, self.w, self.m, self.M, self.S, self.precond = op, w, m, M, symbol, precond
        self.n = op.ns[0]

    def outer(self, x, b):
        """One outer iteration in place: M smoothing sweeps, then the Fourier correction."""
        self.op.apply_sweeps(richm.F32, x, None, b, self.w, K=self.M, m=self.m, precond=self.precond, fuse=1)
        self.op.fourier_correction(x, b, self.S)

    def iterations(self, b, tol=1e-6, max_outer=2000):
        """Outer iterations from x = 0 until every instance's relative residual is <= tol
        (checked after each outer iteration); [batch] counts, None where not reached."""
        op = self.op
        x = op.zeros(richm.F32)
        count = [None] * op.batch
        for it in range(1, max_outer + 1):
            self.outer(x, b)
            rel = op.residual_norm(richm.F32, x, b)[2].cpu().numpy()
            for i, r in enumerate(rel):
                if count[i] is None and r <= tol:
                    count[i] = it
            if all(c is not None for c in count) or not np.all(np.isfinite(rel)):
                break
        return count

    def loss_and_grads(self, b, C: int):
        """Log-residual loss after C outer iterations from x = 0, with dL/dS (complex64
        [n][n]) and dL/dw ([batch][m]); the smoothing is recomputed from one checkpoint
        per outer iteration in the adjoint."""
        op, M, m = self.op, self.M, self.m
        elems = op.checkpoint_elems(M, M)
        # zeroed: the forward writes the slots' interior rows only, and xK is a copy of a slot
        ckpts = [torch.zeros(elems, dtype=torch.float32, device="cuda") for _ in range(C)]
        xs = [op.zeros(richm.F32) for _ in range(C)]
        x = op.zeros(richm.F32)
        for c in range(C):
            op.forward_checkpointed(richm.F32, x, b, self.w, None, None, m, M, M, self.precond, ckpts[c], xs[c])
            x = xs[c].clone()
            op.fourier_correction(x, b, self.S)
        g = op.zeros(richm.F32)
        loss = op.loss_log_residual(richm.F32, x, b, g)
        dS = torch.zeros((self.n, self.n), dtype=torch.complex64, device="cuda")
        gw = torch.zeros_like(self.w)
        dS_c = torch.empty_like(dS)
        gw_c = torch.empty_like(self.w)
        g0 = op.zeros(richm.F32)
        for c in reversed(range(C)):
            op.fourier_correction_vjp(xs[c], b, g, self.S, dsymbol=dS_c, g_x=g)
            dS += dS_c
            op.sweeps_adjoint(richm.F32, ckpts[c], M, b, g, self.w, None, None, m, M, self.precond, g_w=gw_c,
                              g_x0=g0)
            gw += gw_c
            g, g0 = g0, g
        return loss, dS, gw


def train_alternating(fns: FNS, batches, C=2, rounds=3, steps=100, lr_symbol=1e-2, lr_w=1e-3, log=None):
    """Algorithm 2 with directly held parameters: `steps` Adam steps on the symbol with the
    weights frozen, then `rounds` times: weights alone, symbol alone. batches: list of
    right-hand-side buffers (padded, F32), taken in turn. Returns the loss history."""
    S_real = torch.view_as_real(fns.S)  # float32 [n][n][2], shares storage with S
    state = {"S": [torch.zeros_like(S_real), torch.zeros_like(S_real), 0],
             "w": [torch.zeros_like(fns.w), torch.zeros_like(fns.w), 0]}
    hist = []

    def run(which, nsteps, lr):
        for s in range(nsteps):
            b = batches[len(hist) % len(batches)]
            loss, dS, gw = fns.loss_and_grads(b, C)
            st = state[which]
            st[2] += 1
            if which == "S":
                richm.adam_step(S_real, torch.view_as_real(dS).contiguous(), st[0], st[1], st[2], lr=lr)
            else:
                richm.adam_step(fns.w, gw, st[0], st[1], st[2], lr=lr)
            hist.append(float(loss.item()))
        if log:
            log(f"  {which}: loss {hist[-nsteps]:.3f} -> {hist[-1]:.3f}")

    run("S", steps, lr_symbol)
    for _ in range(rounds):
        run("w", steps, lr_w)
        run("S", steps, lr_symbol)
    return hist
