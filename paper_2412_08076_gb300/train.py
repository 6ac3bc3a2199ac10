"""Meta-network training on the GPU through the library's kernels (Algorithm 1).

Each step: w, a = Meta(theta; mu) (library forward), K NAG sweeps from x0 = 0 with
checkpoints (library forward), loss = mean log relative residual and its gradient
(library), adjoint sweeps (library), network backward and Adam (library). Python only
sequences the calls. The network's head selects the Table 1 method (Richardson, MOM,
NAG, NAGex; shared or per-step momenta) and --precond 2 the SSOR preconditioner. The
committed m = 16 networks come from two stages each (the first stage's output is not kept):
  python -m paper_2412_08076_gb300.train --steps 1500 --out stage1.npy
  python -m paper_2412_08076_gb300.train --finetune-from stage1.npy --out paper_2412_08076_gb300/params/meta_m16.npy
and, with the momentum held at 0.3 and Leja-ordered initial weights (the benchmark's network),
three stages:
  python -m paper_2412_08076_gb300.train --steps 1500 --fixed-beta 0.3 --stretch 1.2 --leja --out stage1.npy
  python -m paper_2412_08076_gb300.train --finetune-from stage1.npy --fixed-beta 0.3 --stop 750 --out stage2.npy
  python -m paper_2412_08076_gb300.train --hard-from stage2.npy \
      --out paper_2412_08076_gb300/params/meta_m16_beta03.npy
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np
import torch

from . import meta as meta_mod
from . import richm


class Batch:
    """One minibatch: operator, padded FP32 right-hand sides, network inputs."""

    def __init__(self, insts, seed, normal_rhs=False):
        import richm_synth as synth
        self.insts = insts
        self.op = richm.Operator([(richm.ANISO_Q1, t.n, t.eps, t.theta, 0.0) for t in insts])
        gen = synth.rhs_normal if normal_rhs else synth.rhs_uniform
        rhs = [gen(seed, i, t.n) for i, t in enumerate(insts)]
        dense = torch.tensor(np.concatenate([r.ravel() for r in rhs]), dtype=torch.float32, device="cuda")
        self.b = self.op.pack(dense, richm.F32)
        self.X = torch.tensor(synth.meta_inputs(insts), dtype=torch.float32, device="cuda")
        self.G = torch.tensor(self.op.gershgorin(), dtype=torch.float32, device="cuda")


class Trainer:
    """Algorithm 1 on the GPU: meta forward, K checkpointed sweeps, loss, adjoint sweeps,
    meta backward, Adam. precond 2 trains the SSOR-preconditioned iteration (relaxation
    factor `relax`); its weights are then scaled by 1 instead of the Gershgorin bound,
    since the spectrum of B^{-1} A lies in (0, 1]."""

    def __init__(self, params: np.ndarray, m=16, K=64, every=8, lr=2e-3, precond=0, relax=1.0,
                 head=richm.HEAD_NAG_SHARED, fixed_beta=False):
        self.m, self.K, self.every, self.lr = m, K, every, lr
        self.fixed_beta = fixed_beta  # the momentum output gets no gradient (held at its initial value)
        self.precond, self.relax, self.head = precond, relax, head
        self.P = torch.tensor(params, dtype=torch.float32, device="cuda")
        self.m1 = torch.zeros_like(self.P)
        self.m2 = torch.zeros_like(self.P)
        self.t = 0
        self.ws = {}

    def _work(self, batch: Batch):
        key = id(batch)
        if key not in self.ws:
            op = batch.op
            B = op.batch
            self.ws[key] = dict(
                ck=torch.empty(op.checkpoint_elems(self.K, self.every), dtype=torch.float32, device="cuda"),
                x0=op.zeros(richm.F32), xK=op.zeros(richm.F32), g=op.zeros(richm.F32),
                work=op.workspace(op._ws("richm_adjoint_workspace", richm.F32, self.every)),
                acts=torch.empty(richm.meta_acts_size(B, self.m, self.head), dtype=torch.float32, device="cuda"),
                gw=torch.empty(B, self.m, dtype=torch.float32, device="cuda"),
                ga=torch.zeros(B, self.m, dtype=torch.float32, device="cuda"),
                gat=torch.zeros(B, self.m, dtype=torch.float32, device="cuda"),
                gP=torch.empty(self.P.numel(), dtype=torch.float32, device="cuda"),
                mwork=torch.empty(B * self.P.numel() * 4, dtype=torch.uint8, device="cuda"),
            )
        return self.ws[key]

    def loss_and_grad(self, batch: Batch):
        """Loss (device FP64 scalar) and parameter gradient (device FP32)."""
        W = self._work(batch)
        op = batch.op
        G = self.scale(batch)
        w, a, at = richm.meta_forward_head(self.P, batch.X, G, self.m, self.head, W["acts"])
        op.forward_checkpointed(richm.F32, W["x0"], batch.b, w, a, at, self.m, self.K, self.every, self.precond,
                                W["ck"], W["xK"], work=W["work"], relax=self.relax)
        loss = op.loss_log_residual(richm.F32, W["xK"], batch.b, W["g"], work=W["work"])
        gat = W["gat"] if self.head == richm.HEAD_NAGEX else None
        op.sweeps_adjoint(richm.F32, W["ck"], self.every, batch.b, W["g"], w, a, at, self.m, self.K, self.precond,
                          W["gw"], W["ga"] if a is not None else None, gat, None, work=W["work"], relax=self.relax)
        if self.fixed_beta and a is not None:
            W["ga"].zero_()
        gP = richm.meta_backward(self.P, batch.X, G, W["acts"], self.m, W["gw"], W["ga"], W["gP"], W["mwork"],
                                 head=self.head, g_alpha_t=gat)
        return loss, gP

    def scale(self, batch: Batch):
        """The per-instance spectral scale G of the output map w_i = exp(o_i) / G."""
        return torch.ones_like(batch.G) if self.precond == 2 else batch.G

    def step(self, batch: Batch, lr: float | None = None):
        loss, gP = self.loss_and_grad(batch)
        self.t += 1
        richm.adam_step(self.P, gP, self.m1, self.m2, self.t, lr=self.lr if lr is None else lr)
        return loss

    def params(self) -> np.ndarray:
        return self.P.detach().cpu().numpy()


def make_batches(nbatches=8, B=64, n=255, seed=1000, log_eps=(-3.0, 0.0), normal_rhs=False):
    import richm_synth as synth
    out = []
    for j in range(nbatches):
        insts = synth.batched_aniso(B, sizes=(n,), param_seed=seed + j, log_eps=log_eps)
        out.append(Batch(insts, seed=seed + 500 + j, normal_rhs=normal_rhs))
    return out


def train(steps=1000, lr=2e-3, nbatches=8, n=255, log_every=100, verbose=True, K=64, fixed_beta=None,
          stretch=meta_mod.STABLE_STRETCH, leja=False):
    """Algorithm 1 with the config-3 workload (64 instances of n x n per batch, K = 64,
    checkpoints every 8) from the initial network; cosine-decayed Adam step size.
    fixed_beta: hold the momentum at this value (the network's momentum output is the
    constant, untrained). stretch, leja: the initial weights (meta.init_params).
    Deterministic: seeded data, fixed-order kernels. Returns (params, loss history)."""
    if fixed_beta is None and stretch == meta_mod.STABLE_STRETCH and not leja:
        params, _ = meta_mod.load_params(16, prefer_trained=False)
    else:
        params = meta_mod.init_params(16, beta=0.3 if fixed_beta is None else fixed_beta, stretch=stretch,
                                      leja=leja, fixed_beta=fixed_beta is not None)
    tr = Trainer(params, K=K, lr=lr, fixed_beta=fixed_beta is not None)
    batches = make_batches(nbatches, n=n)
    hist = []
    t0 = time.time()
    for s in range(steps):
        lr_s = lr * 0.5 * (1.0 + math.cos(math.pi * s / max(1, steps)))
        loss = tr.step(batches[s % len(batches)], lr=lr_s)
        if s % log_every == 0 or s == steps - 1:
            hist.append((s, float(loss.item())))
            if verbose:
                print(f"step {s:5d} loss {hist[-1][1]:.4f} ({time.time() - t0:.1f} s)", flush=True)
    return tr.params(), hist


def finetune(params, steps=2000, stop=1250, K=128, lr=1e-3, log_every=250, verbose=True, fixed_beta=False,
             save_every=0, save_prefix=None):
    """Second training stage of the committed m = 16 network: from `params`, alternate
    batches of 64 x 255^2 and 32 x 511^2 instances (seeds 7000 and 7100, four of each),
    K = 128 unrolled sweeps, checkpoints every 8, Adam with a cosine step size over
    `steps`, stopped after `stop` steps. The stop was chosen among the checkpoints every
    250 steps as one whose weights keep every per-mode period transfer in the unit disk
    on a dense (eps, theta) grid and on 3 000 random points of the training range (the
    checks of tests/test_meta_stability_cpu.py) and that converged on every instance of
    four 256-instance batches; later checkpoints of this run lowered the loss further but
    left a few (eps, theta) with a transfer radius above 1 and a diverging instance."""
    tr = Trainer(params, K=K, every=8, lr=lr, fixed_beta=fixed_beta)
    b255 = make_batches(4, B=64, n=255, seed=7000)
    b511 = make_batches(4, B=32, n=511, seed=7100)
    hist = []
    for s in range(stop):
        lr_s = lr * 0.5 * (1.0 + math.cos(math.pi * s / max(1, steps)))
        loss = tr.step(b511[s % 4] if s % 2 else b255[s % 4], lr=lr_s)
        if (s + 1) % log_every == 0:
            hist.append((s + 1, float(loss.item())))
            if verbose:
                print(f"step {s + 1:5d} loss {hist[-1][1]:.4f}", flush=True)
        if save_every and save_prefix and (s + 1) % save_every == 0:
            np.save(f"{save_prefix}_{s + 1}.npy", tr.params())
    return tr.params(), hist


def finetune_hard(params, steps=600, K=256, lr=3e-4, log_every=100, verbose=True, fixed_beta=True):
    """Third training stage of the benchmark's network: from `params`, K = 256 unrolled
    sweeps (checkpoints every 8) on batches that cycle through 32 x 511^2 instances with
    eps in 10^[-3, -2] (the slowest to converge; seeds 8100..8103), 32 x 511^2 over the
    whole range (8200..8203) and 64 x 255^2 (8300..8303), Adam with a cosine step size over
    `steps`. The longer unroll weighs the slow modes of the hardest instances, which
    decide the time to tolerance of a batch; the result keeps every per-mode period
    transfer in the unit disk (tests/test_meta_stability_cpu.py) and converged on twelve
    256-instance batches (seeds 1-12), 11-12 % faster than the second stage on each."""
    tr = Trainer(params, K=K, every=8, lr=lr, fixed_beta=fixed_beta)
    sets = [make_batches(4, B=32, n=511, seed=8100, log_eps=(-3.0, -2.0)),
            make_batches(4, B=32, n=511, seed=8200),
            make_batches(4, B=64, n=255, seed=8300)]
    hist = []
    for s in range(steps):
        lr_s = lr * 0.5 * (1.0 + math.cos(math.pi * s / steps))
        loss = tr.step(sets[s % 3][(s // 3) % 4], lr=lr_s)
        if (s + 1) % log_every == 0:
            hist.append((s + 1, float(loss.item())))
            if verbose:
                print(f"step {s + 1:5d} loss {hist[-1][1]:.4f}", flush=True)
    return tr.params(), hist


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--batches", type=int, default=8)
    ap.add_argument("--n", type=int, default=255)
    ap.add_argument("--K", type=int, default=64, help="unrolled sweeps per loss evaluation")
    ap.add_argument("--out", default=None, help="where to save the parameters (.npy)")
    ap.add_argument("--finetune-from", default=None,
                    help="run the second stage (finetune) from these parameters instead of training from scratch")
    ap.add_argument("--fixed-beta", type=float, default=None, help="hold the momentum at this value")
    ap.add_argument("--stretch", type=float, default=meta_mod.STABLE_STRETCH, help="initial Chebyshev stretch")
    ap.add_argument("--leja", action="store_true", help="initial weights in Leja step order")
    ap.add_argument("--stop", type=int, default=1250, help="finetune: stop after this many steps")
    ap.add_argument("--save-every", type=int, default=0, help="finetune: save parameters every this many steps")
    ap.add_argument("--hard-from", default=None,
                    help="run the third stage (finetune_hard, K = 256 on the hardest instances) from these parameters")
    args = ap.parse_args(argv)
    if args.hard_from:
        params, hist = finetune_hard(np.load(args.hard_from).astype(np.float32))
    elif args.finetune_from:
        params, hist = finetune(np.load(args.finetune_from).astype(np.float32), stop=args.stop,
                                fixed_beta=args.fixed_beta is not None, save_every=args.save_every,
                                save_prefix=args.out[:-4] if args.out and args.save_every else None)
    else:
        params, hist = train(args.steps, args.lr, args.batches, args.n, K=args.K, fixed_beta=args.fixed_beta,
                             stretch=args.stretch, leja=args.leja)
    if args.out:
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        np.save(args.out, params)
    return hist


if __name__ == "__main__":
    main()
