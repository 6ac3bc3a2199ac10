"""Meta-network training on the GPU (Algorithm 1) through the library's kernels only,
and what the trained network gains over the solver without it (the momentum-aware
Chebyshev weights the untrained network starts from)."""
import numpy as np
import pytest
import torch

import richm_synth as synth
from paper_2412_08076_gb300 import meta, richm
from paper_2412_08076_gb300.train import Trainer, make_batches

pytestmark = pytest.mark.gpu


def _sweeps_to_tol(params, insts, tol=1e-8):
    op = richm.Operator([(richm.ANISO_Q1, t.n, t.eps, t.theta, 0.0) for t in insts])
    X = torch.tensor(synth.meta_inputs(insts), dtype=torch.float32, device="cuda")
    G = torch.tensor(op.gershgorin(), dtype=torch.float32, device="cuda")
    P = torch.tensor(params, dtype=torch.float32, device="cuda")
    w, a = richm.meta_forward(P, X, G, 16)
    rhs = synth.batched_rhs(insts, seed=77)
    B = op.pack(torch.tensor(np.concatenate([r.ravel() for r in rhs]), device="cuda"), richm.F64)
    x = op.zeros(richm.F64)
    st, info = op.solve(B, x, w, a, None, op.solve_opts(16, tol=tol, max_sweeps=2_000_000))
    assert st == richm.OK, info
    return np.array([s for s, _, _ in info], dtype=float)


def test_training_lowers_the_loss_and_the_sweeps_to_tolerance():
    p0 = meta.init_params(16)
    tr = Trainer(p0, lr=2e-3)
    batches = make_batches(4, B=32, n=63, seed=3000)
    first = float(tr.loss_and_grad(batches[0])[0].item())
    for s in range(120):
        tr.step(batches[s % 4])
    last = float(tr.loss_and_grad(batches[0])[0].item())
    assert last < first - 0.2, (first, last)
    held = synth.batched_aniso(16, (63, 127), param_seed=4243)
    s0 = _sweeps_to_tol(p0, held)
    s1 = _sweeps_to_tol(tr.params(), held)
    assert np.median(s1) <= 0.8 * np.median(s0), (np.median(s0), np.median(s1))


def _ssor_sweeps_to_tol(params, insts, relax, tol=1e-8):
    op = richm.Operator([(richm.ANISO_Q1, t.n, t.eps, t.theta, 0.0) for t in insts])
    X = torch.tensor(synth.meta_inputs(insts), dtype=torch.float32, device="cuda")
    G = torch.ones(len(insts), dtype=torch.float32, device="cuda")
    P = torch.tensor(params, dtype=torch.float32, device="cuda")
    w, a = richm.meta_forward(P, X, G, 16)
    rhs = synth.batched_rhs(insts, seed=77)
    B = op.pack(torch.tensor(np.concatenate([r.ravel() for r in rhs]), device="cuda"), richm.F64)
    x = op.zeros(richm.F64)
    st, info = op.solve(B, x, w, a, None, op.solve_opts(16, tol=tol, max_sweeps=400_000, precond=2, fuse=1,
                                                        relax=relax))
    assert st == richm.OK, info
    return np.array([s for s, _, _ in info], dtype=float)


def test_ssor_training_lowers_the_loss():
    # Algorithm 1 for the SSOR-preconditioned NAG iteration (weights scaled by 1: the
    # spectrum of B^{-1} A lies in (0, 1]); gradients through the SSOR adjoint
    relax = 1.0
    p0 = meta.init_params(16)
    tr = Trainer(p0, lr=2e-3, K=32, every=8, precond=2, relax=relax)
    batches = make_batches(4, B=32, n=63, seed=3000)
    first = float(tr.loss_and_grad(batches[0])[0].item())
    for s in range(60):
        tr.step(batches[s % 4])
    last = float(tr.loss_and_grad(batches[0])[0].item())
    assert np.isfinite(last) and last < first - 0.1, (first, last)
    held = synth.batched_aniso(8, (63,), param_seed=4243)
    s0 = _ssor_sweeps_to_tol(p0, held, relax)
    s1 = _ssor_sweeps_to_tol(tr.params(), held, relax)
    print("SSOR sweeps to 1e-8 before/after training (median):", np.median(s0), np.median(s1))
    assert np.median(s1) <= np.median(s0), (np.median(s0), np.median(s1))
