"""The single-level neural-solver experiments of Sec. 2.4 (Tables 2-4) on this library.

Trains the meta network (Algorithm 1, all steps in the library's kernels) for the
Table 1 methods with m = 3, Richardson(3), MOM-, NAG- and NAGex-Richardson(3), and
NAGex-Richardson(3) with the SSOR preconditioner, on synthetic data drawn like the
paper's training set: N = 64 elements per side (63^2 unknowns), eps log-uniform on
[1e-6, 1], theta uniform on [0, pi), f ~ N(0, I). Then counts outer iterations (m sweeps
each, zero initial guess, residual test once per outer iteration) to a relative
residual of 1e-6:
  Table 2: theta = 0, N = 64, eps in {1, 1e-2, 1e-4, 1e-6, 1e-8}, every method;
  Table 3: eps = 1e-6, N = 64, theta in {0, pi/6, ..., pi}, NAGex + SSOR;
  Table 4: eps = 1e-6, theta = pi/10, N in {32, ..., 512}, NAGex + SSOR.
The networks are ours (trained here on synthetic data), not the paper's, so the counts
are a qualitative comparison. Each momentum head starts at a = 0.3 where a stable
initial stretch exists for m = 3 (NAG, NAGex), else at 0.1 (MOM). At test time the
network input lg eps is clamped to the training range [-6, 0] (eps = 1e-8 lies outside
it). The solves run in FP64 (richm_solve with an FP64 inner state, a residual check
every m sweeps), so a count is exact for the weights given.
Usage:
  python -m paper_2412_08076_gb300.single_level --steps 2000 [--save paper_2412_08076_gb300/params]
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
from .train import Batch, Trainer

M = 3
TOL = 1e-6
RELAX = 1.0  # SSOR relaxation factor (symmetric Gauss-Seidel)

# (row label, head, precond)
METHODS = [
    ("Richardson(3)-NS", richm.HEAD_RICHARDSON, 0),
    ("MOM-Richardson(3)-NS", richm.HEAD_MOM, 0),
    ("NAG-Richardson(3)-NS", richm.HEAD_NAG, 0),
    ("NAGex-Richardson(3)-NS", richm.HEAD_NAGEX, 0),
    ("NAGex-Richardson(3)-NS (SSOR)", richm.HEAD_NAGEX, 2),
]


def training_batches(nbatches=16, B=64, seed=6400):
    import richm_synth as synth
    out = []
    for j in range(nbatches):
        insts = synth.batched_aniso(B, sizes=(63,), param_seed=seed + j, log_eps=LOG_EPS_RANGE)
        out.append(Batch(insts, seed=seed + 500 + j, normal_rhs=True))
    return out


LOG_EPS_RANGE = (-6.0, 0.0)


def initial_momentum(head):
    """0.3 if the head's initial weights can be made stable with it at m = 3, else 0.1."""
    if head in (richm.HEAD_RICHARDSON, richm.HEAD_NAG_SHARED):
        return 0.3
    try:
        meta_mod.stable_stretch(M, 0.3, head != richm.HEAD_MOM)
        return 0.3
    except ValueError:
        return 0.1


def train_method(head, precond, steps, batches, K=48, lr=3e-3, beta=None, log=print):
    beta = initial_momentum(head) if beta is None else beta
    params = meta_mod.init_params(M, beta=beta, head=head)
    tr = Trainer(params, m=M, K=K, every=8, lr=lr, precond=precond, relax=RELAX, head=head)
    first = last = None
    t0 = time.time()
    for s in range(steps):
        lr_s = lr * 0.5 * (1.0 + math.cos(math.pi * s / max(1, steps)))
        L = tr.step(batches[s % len(batches)], lr=lr_s)
        if s == 0:
            first = float(L.item())
    torch.cuda.synchronize()
    last = float(tr.loss_and_grad(batches[0])[0].item())
    log(f"  trained head {head} precond {precond}: loss {first:.3f} -> {last:.3f} "
        f"({steps} steps, {(time.time() - t0) / max(1, steps) * 1e3:.1f} ms/step)")
    return tr.params(), (first, last)


def iterations(params, head, precond, cases, max_outer=200000, seed=6464):
    """Outer iterations to TOL for each (eps, theta, n) of `cases` (one batched solve)."""
    import richm_synth as synth
    insts = [synth.AnisoInstance(eps, theta, n) for eps, theta, n in cases]
    op = richm.Operator([(richm.ANISO_Q1, t.n, t.eps, t.theta, 0.0) for t in insts])
    X = synth.meta_inputs(insts)
    X[:, 0] = np.clip(X[:, 0], *LOG_EPS_RANGE)
    X = torch.tensor(X, dtype=torch.float32, device="cuda")
    G = torch.ones(len(insts), dtype=torch.float32, device="cuda") if precond == 2 else \
        torch.tensor(op.gershgorin(), dtype=torch.float32, device="cuda")
    P = torch.tensor(params, dtype=torch.float32, device="cuda")
    w, a, at = richm.meta_forward_head(P, X, G, M, head)
    to64 = (lambda t: None if t is None else t.double().contiguous())
    rhs = [synth.rhs_normal(seed, i, t.n) for i, t in enumerate(insts)]
    b = op.pack(torch.tensor(np.concatenate([r.ravel() for r in rhs]), device="cuda"), richm.F64)
    x = op.zeros(richm.F64)
    opts = op.solve_opts(M, tol=TOL, max_sweeps=M * max_outer, refine_every=M, inner=richm.F64, precond=precond,
                         fuse=1, relax=RELAX)
    st, info = op.solve(b, x, to64(w), to64(a), to64(at), opts)
    out = []
    for sweeps, rel, status in info:
        out.append(sweeps // M if status == richm.OK else None)
    return out


def fmt(v):
    return "-" if v is None else str(v)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--K", type=int, default=48)
    ap.add_argument("--save", default=None, help="directory to save the trained networks in (file names as "
                                                 "meta.trained_path)")
    args = ap.parse_args(argv)
    batches = training_batches()
    eps_list = [1.0, 1e-2, 1e-4, 1e-6, 1e-8]
    table2_cases = [(e, 0.0, 63) for e in eps_list]
    thetas = [k * math.pi / 6 for k in range(7)]
    table3_cases = [(1e-6, t, 63) for t in thetas]
    sizes = [32, 64, 128, 256, 512]
    table4_cases = [(1e-6, math.pi / 10, N - 1) for N in sizes]
    rows = []
    trained = {}
    for label, head, precond in METHODS:
        print(label, flush=True)
        params, losses = train_method(head, precond, args.steps, batches, K=args.K)
        trained[(head, precond)] = params
        if args.save:
            os.makedirs(args.save, exist_ok=True)
            np.save(os.path.join(args.save, os.path.basename(meta_mod.trained_path(M, head, precond))), params)
        init = iterations(meta_mod.init_params(M, beta=initial_momentum(head), head=head), head, precond,
                          table2_cases)
        its = iterations(params, head, precond, table2_cases)
        rows.append((label, its, init, losses))
    print()
    print("Table 2 (theta = 0, N = 64): outer iterations to 1e-6; trained network (initial network)")
    print("| solver | " + " | ".join(f"eps={e:g}" for e in eps_list) + " | loss first -> last |")
    print("|---|" + "---|" * (len(eps_list) + 1))
    for label, its, init, (l0, l1) in rows:
        cells = [f"{fmt(v)} ({fmt(u)})" for v, u in zip(its, init)]
        print(f"| {label} | " + " | ".join(cells) + f" | {l0:.2f} -> {l1:.2f} |")
    p = trained[(richm.HEAD_NAGEX, 2)]
    t3 = iterations(p, richm.HEAD_NAGEX, 2, table3_cases)
    print()
    print("Table 3 (NAGex-Richardson(3)-NS with SSOR, eps = 1e-6, N = 64)")
    print("| theta | " + " | ".join(f"{k}pi/6" for k in range(7)) + " |")
    print("|---|" + "---|" * 7)
    print("| iterations | " + " | ".join(fmt(v) for v in t3) + " |")
    t4 = iterations(p, richm.HEAD_NAGEX, 2, table4_cases)
    print()
    print("Table 4 (NAGex-Richardson(3)-NS with SSOR, eps = 1e-6, theta = pi/10)")
    print("| N | " + " | ".join(str(N) for N in sizes) + " |")
    print("|---|" + "---|" * len(sizes))
    print("| iterations | " + " | ".join(fmt(v) for v in t4) + " |")


if __name__ == "__main__":
    main()
