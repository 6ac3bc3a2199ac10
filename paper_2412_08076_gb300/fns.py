"""Richardson(m)-FNS (Sec. 3.1): M smoothing sweeps of Richardson(m) per outer iteration
(eq. 19 with the Richardson(m) smoother in place of B), then the Fourier neural
iteration (eq. 20), H = F T S T^* F^{-1}, with a symbol S and a banded transition T
(applied as its real field t on the grid; t = 1 is T = I) shared by the instances of a
batch:
  x <- x + t .* Re(IFFT2(S .* FFT2(t .* (b - A x)))).
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

`MetaFNS` trains the three networks of Algorithm 2 through the library's kernels:
Meta-omega (the meta MLP with the Richardson head: m weights per instance), Meta-Lambda and
Meta-T (the meta MLP with the identity head: 6 and 9 outputs, turned into the symbol and
the transition field by richm_symbol_from_stencil and richm_transition_from_band). All
three take (lg eps, theta); the architectures of the paper's FNO and CNN are not given,
so these small maps stand in for them. `train_algorithm2` runs the alternating schedule
over batches of several (eps, theta).
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
    """Richardson(m)-FNS on an operator of Q1 instances of one size (FP32 state);
    transition: the field t (FP32 [n][n]) of the transition T, or None for T = I."""

    def __init__(self, op: richm.Operator, w: torch.Tensor, m: int, M: int, symbol: torch.Tensor, precond: int = 1,
                 transition: torch.Tensor | None = None):
        self.op, self.w, self.m, self.M, self.S, self.precond = op, w, m, M, symbol, precond
        self.t = transition
        self.n = op.ns[0]

    def outer(self, x, b):
        """One outer iteration in place: M smoothing sweeps, then the Fourier correction."""
        self.op.apply_sweeps(richm.F32, x, None, b, self.w, K=self.M, m=self.m, precond=self.precond, fuse=1)
        self.op.fourier_correction(x, b, self.S, transition=self.t)

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

    def loss_and_grads(self, b, C: int, want_dt: bool = False):
        """Log-residual loss after C outer iterations from x = 0, with dL/dS (complex64
        [n][n]) and dL/dw ([batch][m]), and with want_dt (a transition given) dL/dt
        ([n][n]) as a fourth value; the smoothing is recomputed from one checkpoint per
        outer iteration in the adjoint."""
        op, M, m = self.op, self.M, self.m
        elems = op.checkpoint_elems(M, M)
        # zeroed: the forward writes the slots' interior rows only, and xK is a copy of a slot
        ckpts = [torch.zeros(elems, dtype=torch.float32, device="cuda") for _ in range(C)]
        xs = [op.zeros(richm.F32) for _ in range(C)]
        x = op.zeros(richm.F32)
        for c in range(C):
            op.forward_checkpointed(richm.F32, x, b, self.w, None, None, m, M, M, self.precond, ckpts[c], xs[c])
            x = xs[c].clone()
            op.fourier_correction(x, b, self.S, transition=self.t)
        g = op.zeros(richm.F32)
        loss = op.loss_log_residual(richm.F32, x, b, g)
        dS = torch.zeros((self.n, self.n), dtype=torch.complex64, device="cuda")
        gw = torch.zeros_like(self.w)
        dS_c = torch.empty_like(dS)
        gw_c = torch.empty_like(self.w)
        dt = torch.zeros((self.n, self.n), dtype=torch.float32, device="cuda") if want_dt else None
        dt_c = torch.empty_like(dt) if want_dt else None
        g0 = op.zeros(richm.F32)
        for c in reversed(range(C)):
            if self.t is None:
                op.fourier_correction_vjp(xs[c], b, g, self.S, dsymbol=dS_c, g_x=g)
            else:
                op.fourier_correction_t_vjp(xs[c], b, g, self.S, self.t, dsymbol=dS_c, dtransition=dt_c, g_x=g)
                if want_dt:
                    dt += dt_c
            dS += dS_c
            op.sweeps_adjoint(richm.F32, ckpts[c], M, b, g, self.w, None, None, m, M, self.precond, g_w=gw_c,
                              g_x0=g0)
            gw += gw_c
            g, g0 = g0, g
        if want_dt:
            return loss, dS, gw, dt
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


class MetaFNS:
    """Richardson(m)-FNS with the three meta networks of Algorithm 2 (Sec. 3.1), each an
    MLP 2 -> 64 -> 64 -> nout on (lg eps, theta) run by the library's meta kernels:
      Meta-omega: the Richardson head, m weights w_i = exp(o_i) (the Jacobi-preconditioned
                  spectrum lies in (0, 2], so no further scale);
      Meta-Lambda: the identity head, 6 outputs, the symbol richm_symbol_from_stencil maps
                  them to (the instance's Q1 stencil scaled by exp(o), regularised inverse);
      Meta-T:     the identity head, 9 outputs, the band kernel richm_transition_from_band
                  maps to the transition field.
    A batch holds instances of one (eps, theta) (the symbol and the transition are shared
    by the batch); the networks make one evaluation per batch. Initialisation: Meta-omega
    at w = 0.5 (Algorithm 2's omega^(0)), Meta-Lambda at the periodic inverse of the
    instance's stencil with delta = delta0 q_0, Meta-T at t = 1 (T = I)."""

    def __init__(self, m: int = 10, M: int = 10, seed: int = 7, delta0: float = 1e-2, use_t: bool = True):
        import richm_synth as synth
        from . import meta as meta_mod  # noqa: F401 (the parameter layout is the library's)
        self.m, self.M, self.delta0, self.use_t = m, M, delta0, use_t
        self.P = {}
        for name, nout, bias in (("w", m, [math.log(0.5)] * m), ("lam", 6, [0.0] * 6),
                                 ("t", 9, [1.0] + [0.0] * 8)):
            layers = synth.mlp_init((2, 64, 64, nout), seed=seed + len(self.P))
            W3, b3 = layers[2]
            layers[2] = (np.asarray(W3) * 1e-3, np.asarray(bias, dtype=np.float64))
            flat = np.concatenate([np.concatenate([np.asarray(W, np.float64).ravel(), np.asarray(b, np.float64)])
                                   for W, b in layers]).astype(np.float32)
            self.P[name] = torch.tensor(flat, device="cuda")
        self.adam = {k: [torch.zeros_like(v), torch.zeros_like(v), 0] for k, v in self.P.items()}
        self.frozen_w = True  # Algorithm 2 starts with Meta-omega frozen at omega^(0)

    def _q(self, op):
        c = op.stencil(0)
        return [c[0], c[1], c[2], c[3], c[4], self.delta0 * c[0]]

    def fields(self, op, X1, XB):
        """(w [B][m], symbol, transition or None, activations) for a batch: X1 [1][2] the
        batch's (lg eps, theta), XB [B][2] per instance."""
        B, n = op.batch, op.ns[0]
        ones1 = torch.ones(1, dtype=torch.float32, device="cuda")
        onesB = torch.ones(B, dtype=torch.float32, device="cuda")
        acts = {"w": torch.empty(richm.meta_acts_size(B, self.m, richm.HEAD_RICHARDSON), device="cuda"),
                "lam": torch.empty(richm.meta_acts_size(1, 6, richm.HEAD_RAW), device="cuda"),
                "t": torch.empty(richm.meta_acts_size(1, 9, richm.HEAD_RAW), device="cuda")}
        if self.frozen_w:
            w = torch.full((B, self.m), 0.5, dtype=torch.float32, device="cuda")
        else:
            w, _, _ = richm.meta_forward_head(self.P["w"], XB, onesB, self.m, richm.HEAD_RICHARDSON, acts["w"])
        o_lam, _, _ = richm.meta_forward_head(self.P["lam"], X1, ones1, 6, richm.HEAD_RAW, acts["lam"])
        S = richm.symbol_from_stencil(n, self._q(op), o_lam)
        t, o_t = None, None
        if self.use_t:
            o_t, _, _ = richm.meta_forward_head(self.P["t"], X1, ones1, 9, richm.HEAD_RAW, acts["t"])
            t = richm.transition_from_band(n, o_t)
        return w, S, t, (o_lam, o_t, acts)

    def loss_and_grads(self, op, b, X1, XB, C: int, which: str):
        """The log-residual loss after C outer iterations and the parameter gradients of the
        networks being trained (which = "w" or "lam_t")."""
        n = op.ns[0]
        w, S, t, (o_lam, o_t, acts) = self.fields(op, X1, XB)
        f = FNS(op, w, self.m, self.M, S, precond=1, transition=t)
        out = f.loss_and_grads(b, C, want_dt=t is not None)
        loss, dS, gw = out[0], out[1], out[2]
        grads = {}
        ones1 = torch.ones(1, dtype=torch.float32, device="cuda")
        if which == "w":
            B = op.batch
            onesB = torch.ones(B, dtype=torch.float32, device="cuda")
            grads["w"] = richm.meta_backward(self.P["w"], XB, onesB, acts["w"], self.m, gw, None,
                                             head=richm.HEAD_RICHARDSON)
        else:
            d_lam = richm.symbol_from_stencil_vjp(n, self._q(op), o_lam, dS).reshape(1, 6)
            grads["lam"] = richm.meta_backward(self.P["lam"], X1, ones1, acts["lam"], 6, d_lam, None,
                                               head=richm.HEAD_RAW)
            if t is not None:
                d_tau = richm.transition_from_band_vjp(n, out[3]).reshape(1, 9)
                grads["t"] = richm.meta_backward(self.P["t"], X1, ones1, acts["t"], 9, d_tau, None,
                                                 head=richm.HEAD_RAW)
        return loss, grads

    def step(self, op, b, X1, XB, C, which, lr):
        loss, grads = self.loss_and_grads(op, b, X1, XB, C, which)
        for k, g in grads.items():
            st = self.adam[k]
            st[2] += 1
            richm.adam_step(self.P[k], g, st[0], st[1], st[2], lr=lr)
        return loss

    def iterations(self, op, b, X1, XB, tol=1e-2, max_outer=500):
        w, S, t, _ = self.fields(op, X1, XB)
        return FNS(op, w, self.m, self.M, S, precond=1, transition=t).iterations(b, tol=tol, max_outer=max_outer)


def train_algorithm2(net: MetaFNS, batches, C=2, cycles=2, steps=40, lr=2e-3, log=None):
    """Algorithm 2: Meta-omega frozen at omega^(0) while Meta-Lambda and Meta-T train for
    `steps`, then `cycles` times: Meta-omega alone, then Meta-Lambda and Meta-T. batches:
    list of (op, b, X1, XB), one (eps, theta) each, taken in turn. Returns the loss history."""
    hist = []

    def run(which):
        for s in range(steps):
            op, b, X1, XB = batches[len(hist) % len(batches)]
            hist.append(float(net.step(op, b, X1, XB, C, which, lr).item()))
        if log:
            log(f"  {which}: loss {hist[-steps]:.3f} -> {hist[-1]:.3f}")

    net.frozen_w = True
    run("lam_t")
    net.frozen_w = False
    for _ in range(cycles):
        run("w")
        run("lam_t")
    return hist


def table5_analogue(n: int = 63, classes=((1.0, 0.0), (1e-2, 0.0), (1e-4, 0.0), (1e-2, math.pi / 6), (1e-4, math.pi / 3)),
                    B: int = 8, m: int = 4, M: int = 10, C: int = 2, cycles: int = 2, steps: int = 150,
                    lr: float = 2e-3, tol: float = 1e-6, max_outer: int = 3000, log=None):
    """Outer iterations of Richardson(m)-FNS to `tol` (the count of Tables 5-7) on classes
    of (eps, theta) at n x n, Jacobi-preconditioned smoother with M sweeps per outer
    iteration, for: the smoother alone (weights 0.5, no correction); the initial networks
    (the stencil's periodic inverse, T = I); the networks trained by Algorithm 2 with
    T = I; and trained with the banded transition. Training: B right-hand sides N(0, I)
    per class, the classes taken in turn; counting: B others. Returns {row: {class: mean
    count (None where some instance did not reach tol)}}."""
    import richm_synth as synth
    batches, evals = [], []
    for k, (eps, th) in enumerate(classes):
        insts = [synth.AnisoInstance(eps, th, n)] * B
        op = richm.Operator([(richm.ANISO_Q1, t.n, t.eps, t.theta, 0.0) for t in insts])
        mk = lambda seed: op.pack(torch.tensor(np.concatenate(
            [synth.rhs_normal(seed, i, n).ravel() for i in range(B)]), dtype=torch.float32, device="cuda"), richm.F32)
        X = torch.tensor(synth.meta_inputs(insts), dtype=torch.float32, device="cuda")
        batches.append((op, mk(300 + k), X[:1].contiguous(), X))
        evals.append((op, mk(400 + k), X[:1].contiguous(), X))

    def mean_count(counts):
        return None if any(c is None for c in counts) else float(np.mean(counts))

    out = {}
    row = {}
    for (eps, th), (op, b, X1, XB) in zip(classes, evals):
        S0 = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
        f = FNS(op, torch.full((op.batch, m), 0.5, device="cuda"), m, M, S0, precond=1)
        row[f"{eps:g},{th:.3f}"] = mean_count(f.iterations(b, tol=tol, max_outer=max_outer))
    out["smoother_alone"] = row
    for name, use_t, train in (("initial_networks", False, False), ("trained_T_identity", False, True),
                               ("trained_with_T", True, True)):
        net = MetaFNS(m=m, M=M, use_t=use_t)
        if train:
            hist = train_algorithm2(net, batches, C=C, cycles=cycles, steps=steps, lr=lr)
            if log:
                log(f"{name}: loss {np.mean(hist[:len(classes)]):.3f} -> {np.mean(hist[-len(classes):]):.3f}")
        row = {}
        for (eps, th), (op, b, X1, XB) in zip(classes, evals):
            row[f"{eps:g},{th:.3f}"] = mean_count(net.iterations(op, b, X1, XB, tol=tol, max_outer=max_outer))
        out[name] = row
    return out


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Richardson(m)-FNS outer-iteration counts (Tables 5-7 analogue)")
    ap.add_argument("--n", type=int, default=63)
    ap.add_argument("--steps", type=int, default=150)
    ap.add_argument("--cycles", type=int, default=2)
    ap.add_argument("--tol", type=float, default=1e-4)
    args = ap.parse_args()
    print(json.dumps(table5_analogue(n=args.n, steps=args.steps, cycles=args.cycles, tol=args.tol, log=print)))
