"""Benchmark: batched NAG-Richardson(m) with FP64 refinement on synthetic anisotropic Q1 instances.

Workload (the batched NAG configuration): 256 instances of -div(C grad u) = f (bilinear
elements), eps = 10^U[-3, 0], theta ~ U[0, pi), n drawn from {127, 255, 511},
right-hand sides U[-1, 1]; NAG-Richardson(16) with beta = 0.3 and the 16 weights of each
instance from the meta network; FP32 sweeps (fused passes of 8), FP64 refinement every 64
sweeps. One step = the whole hot path over the batch: the meta network's weight supply
and the solve of every instance from x = 0 to relative residual 1e-10. value = the
dof-sweeps performed / the time of the timed steps; ms_per_step = the time to 1e-10.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0). Under torchrun each rank solves its own batch of the
same shape (weak scaling); no collective touches the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "batched Richardson(m) Gdof-sweeps/s, time to 1e-10 rel residual, % HBM peak"
UNIT = "Gdof-sweeps/s"
M, BETA, REFINE, TOL = 16, 0.3, 64, 1e-10
# A longer refinement interval (measured beside the headline): the momentum is carried
# across refinements, so the interval changes only where FP32 rounding is corrected.
REFINE_LONG = 256
# The solver stops at FP64 residual <= TOL * (1 - 1e-3): two independent FP64
# evaluations of ||b - A x|| / ||b|| near 1e-10 (the library's stencil and the
# oracle's assembled matrix) differ by ~1e-5 relative, so the margin makes the
# oracle's own recompute land at or below TOL too.
SOLVE_TOL = TOL * (1.0 - 1e-3)
SIZES = (127, 255, 511)
BATCH = 256
# the meta network trained with its momentum held at BETA (meta.trained_path variant)
META_VARIANT = "beta03"


def workload_config(batch=BATCH):
    return {
        "workload": f"{batch} anisotropic Q1 (bilinear FEM) instances, n in {{127,255,511}}, "
                    "eps=10^U[-3,0], theta~U[0,pi), b~U[-1,1]; NAG-Richardson(16), beta=0.3, weights from the "
                    f"meta MLP 2-64-64-17; FP32 sweeps, FP64 refinement every {REFINE} sweeps; "
                    "one step = weight supply + solve of every instance from x=0 to rel. residual 1e-10",
        "instances": batch,
        "m": M,
        "beta": BETA,
        "refine_every": REFINE,
        "l2": "inputs larger than L2 (state ~0.47 GB FP32 + 0.71 GB FP64 > 129 MB): no flush",
    }


# ---------------------------------------------------------------- distributed helpers

def dist_env():
    """(rank, world) from torchrun's environment, (0, 1) otherwise."""
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def shard_seed(rank: int) -> int:
    """Instance-parameter seed of a rank's batch (rank 0 = the canonical batch)."""
    return 1 + rank


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Max of a per-rank float over the process group (timing only)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle legs

def oracle_sample_rate(instances, seconds: float = 12.0, sweeps_per_chunk: int = 4):
    """FP64 oracle NAG sweeps on one instance of each grid size, until `seconds` pass.

    Returns (Gdof-sweeps/s, description). The oracle is timed as it stands
    (scipy sparse mat-vec per sweep, one host thread)."""
    import numpy as np

    import richm_synth as synth
    from oracle.iterations import inner_steps, semi_iteration_weights
    from oracle.operators import assemble_q1, gershgorin_max
    picked = {}
    for i, t in enumerate(instances):
        if t.n not in picked:
            picked[t.n] = (i, t)
    cases = []
    for n, (i, t) in sorted(picked.items()):
        A = assemble_q1(t.n, t.eps, t.theta)
        G = gershgorin_max(A)
        w = semi_iteration_weights(1.6 * G, M)
        a = np.full(M, BETA)
        cases.append((A, synth.rhs_uniform(2, i, t.n).ravel(), w, a, t.n))
    dofs = 0
    t0 = time.perf_counter()
    done = 0
    while True:
        for A, f, w, a, n in cases:
            inner_steps(A, f, np.zeros(n * n), None, w, a, K=sweeps_per_chunk, k_start=done)
            dofs += n * n * sweeps_per_chunk
        done += sweeps_per_chunk
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    desc = (f"{done} NAG sweeps on one instance of each n in {sorted(picked)} "
            f"({sum(c[4] ** 2 for c in cases)} dofs), FP64 scipy CSR mat-vec, {el:.1f} s")
    return dofs / el / 1e9, desc


def oracle_other_configs():
    """The oracle (one host thread, as it stands) on the other configurations' shapes:
    400 FP64 Richardson(8) sweeps on the 63^2 instance (eps 1e-2, theta pi/6) and 8
    complex NAG-Richardson(8) sweeps on one 2047^2 Helmholtz instance with the absorbing
    boundary (k for 10 points per wavelength)."""
    import numpy as np

    import richm_synth as synth
    from oracle.iterations import chebyshev_weights, inner_steps
    from oracle.operators import assemble_helmholtz, assemble_q1, gershgorin_max, helmholtz_wavenumber
    out = {}
    A = assemble_q1(63, 1e-2, math.pi / 6)
    G = gershgorin_max(A)
    w = chebyshev_weights(G, G / 30.0, 8)
    f = synth.rhs_uniform(0, 0, 63).ravel()
    t0 = time.perf_counter()
    inner_steps(A, f, np.zeros_like(f), None, w, K=400)
    el = time.perf_counter() - t0
    out["fp64_63sq_richardson8_400_sweeps"] = {"seconds": el, "us_per_sweep": 1e6 * el / 400,
                                                "gdof_sweeps_per_s": 63 * 63 * 400 / el / 1e9}
    n = 2047
    t0 = time.perf_counter()
    H = assemble_helmholtz(n, helmholtz_wavenumber(n, 10.0), absorbing=True).tocsr()
    t_asm = time.perf_counter() - t0
    h2 = 1.0 / (n + 1) ** 2
    wv = (h2 / 8.0) * np.linspace(0.5, 1.5, 8)
    b = np.zeros(n * n, np.complex128)
    b[(n // 2) * n + n // 3] = 1.0
    t0 = time.perf_counter()
    inner_steps(H, b, np.zeros_like(b), None, wv, np.full(8, 0.3), K=8)
    el = time.perf_counter() - t0
    out["helmholtz_2047sq_c128_8_sweeps"] = {"seconds": el, "assembly_seconds": t_asm,
                                              "gdof_sweeps_per_s": n * n * 8 / el / 1e9}
    return out


def _oracle_worker_init():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def _oracle_worker(job):
    """One process of the all-cores oracle leg: NAG sweeps on one instance for `seconds`."""
    n, eps, theta, index, seconds = job
    import numpy as np

    import richm_synth as synth
    from oracle.iterations import inner_steps, semi_iteration_weights
    from oracle.operators import assemble_q1, gershgorin_max
    A = assemble_q1(n, eps, theta)
    w = semi_iteration_weights(1.6 * gershgorin_max(A), M)
    a = np.full(M, BETA)
    f = synth.rhs_uniform(2, index, n).ravel()
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < seconds:
        inner_steps(A, f, np.zeros(n * n), None, w, a, K=4, k_start=done)
        done += 4
    return n * n * done, time.perf_counter() - t0


def oracle_all_cores_rate(instances, seconds: float = 8.0):
    """The oracle on every host core at once: one spawned process per core, each sweeping
    one instance (the sizes taken in turn) for `seconds`; returns (Gdof-sweeps/s over all
    processes, processes, description)."""
    import multiprocessing as mp
    procs = os.cpu_count() or 1
    picked = {}
    for i, t in enumerate(instances):
        picked.setdefault(t.n, (i, t))
    sizes = sorted(picked)
    jobs = []
    for k in range(procs):
        i, t = picked[sizes[k % len(sizes)]]
        jobs.append((t.n, t.eps, t.theta, i, seconds))
    with mp.get_context("spawn").Pool(procs, initializer=_oracle_worker_init) as pool:
        res = pool.map(_oracle_worker, jobs)
    dofs = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    desc = (f"{procs} processes (one per host core), each NAG sweeps on one instance of n in {sizes} "
            f"(taken in turn), FP64 scipy CSR mat-vec, {el:.1f} s")
    return dofs / el / 1e9, procs, desc


def kernel_traffic(kind: str, dofs: int):
    """DRAM bytes per launch from the committed ncu summary of this kernel
    (profiles/traffic.txt: kind, sha256 of its sources, bytes per unknown, sources),
    scaled by unknowns; None when the sources changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        parts = ln.split()
        if len(parts) < 4 or parts[0] != kind:
            continue
        h = hashlib.sha256()
        for f in parts[3:]:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        return float(parts[2]) * dofs if h.hexdigest() == parts[1] else None
    return None


def secondary_workloads(dev):
    """Bounded measurements of the other four workloads (not part of the headline)."""
    import numpy as np
    import torch

    import richm_synth as synth
    from paper_2412_08076_gb300 import richm
    from paper_2412_08076_gb300 import meta as meta_mod
    from paper_2412_08076_gb300.train import Trainer, make_batches
    out = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    # 63^2 FP64 Richardson(8), Chebyshev weights from Gershgorin, lmin = lmax/30:
    # 400 sweeps, one launch each, with the residual after every sweep
    inst, b = synth.single_aniso()
    op = richm.Operator([(richm.ANISO_Q1, inst.n, inst.eps, inst.theta, 0.0)])
    G = op.gershgorin()[0]
    w = torch.tensor([richm.chebyshev_weights(G, G / 30.0, 8)], dtype=torch.float64, device=dev)
    B = op.pack(torch.tensor(b.ravel(), device=dev), richm.F64)
    X = op.zeros(richm.F64)
    ws = op.workspace(op._ws("richm_sweeps_workspace", richm.F64))
    rw = op.workspace(op._ws("richm_residual_workspace"))
    hist = torch.empty(400, dtype=torch.float64, device=dev)

    def run400():
        for k in range(400):
            op.apply_sweeps(richm.F64, X, None, B, w, K=1, m=8, k_start=k, work=ws)
            hist[k:k + 1] = op.residual_norm(richm.F64, X, B, work=rw)[2]

    run400()  # warm-up: tile maps and allocations happen outside the timed region
    torch.cuda.synchronize()
    X.zero_()
    e0, e1 = ev(), ev()
    e0.record()
    run400()
    e1.record()
    torch.cuda.synchronize()
    eager_us = 1e3 * e0.elapsed_time(e1) / 400
    # the same 800 launches captured once as a CUDA graph (the launch latency of a
    # 3969-unknown problem otherwise dominates)
    graph_us = None
    try:
        g = torch.cuda.CUDAGraph()
        X.zero_()
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            run400()
        X.zero_()
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        graph_us = 1e3 * e0.elapsed_time(e1) / 400
    except Exception as exc:  # capture is an optimisation of this measurement only
        print(f"note: CUDA graph capture of the 63^2 loop failed ({exc})", file=sys.stderr)
    out["fp64_63sq_richardson8"] = {"sweeps": 400, "us_per_sweep_with_residual": eager_us,
                                    "us_per_sweep_with_residual_graph": graph_us,
                                    "rel_res_after_400": float(hist[-1].item()),
                                    "note": "latency-bound (3969 unknowns): one sweep and one residual norm "
                                            "per step; parity vs oracle in tests"}
    op.close()

    # training step: meta forward, 64 checkpointed NAG sweeps on 64 x 255^2, loss,
    # adjoint, meta backward, Adam
    params, _ = meta_mod.load_params(16, prefer_trained=False)
    tr = Trainer(params)
    batches = make_batches(2, n=255, seed=1000)
    for j in range(3):
        tr.step(batches[j % 2])
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record()
    for j in range(10):
        tr.step(batches[j % 2])
    e1.record()
    torch.cuda.synchronize()
    out["training_step_64x255sq_K64"] = {"ms_per_step": e0.elapsed_time(e1) / 10,
                                         "note": "gradient checks vs oracle and finite differences in tests"}

    # two-level cycle on 32 x 1023^2: 8 FP32 Richardson sweeps + Fourier correction +
    # FP64 refinement
    n, nb = 1023, 32
    op = richm.Operator([(richm.ANISO_Q1, n, 1e-4, math.pi / 3, 0.0)] * nb)
    G = op.gershgorin()[0]
    w8 = torch.tensor([richm.chebyshev_weights(G, G / 30.0, 8)] * nb, dtype=torch.float32, device=dev)
    S = torch.tensor(synth.fourier_symbol(n, seed=3).astype(np.complex64), device=dev)
    rhs = np.concatenate([synth.rhs_uniform(40, i, n).ravel() for i in range(nb)])
    B64 = op.pack(torch.tensor(rhs, device=dev), richm.F64)
    X64 = op.zeros(richm.F64)
    E = op.zeros(richm.F32)
    R = op.zeros(richm.F32)
    fw = op.workspace(op._ws("richm_fourier_workspace"))
    ws = op.workspace(op._ws("richm_sweeps_workspace", richm.F32))
    rw = op.workspace(op._ws("richm_residual_workspace"))
    rel = op.refine(X64, B64, None, None, richm.F32, R, work=rw)

    def cycle():
        op.apply_sweeps(richm.F32, E, None, R, w8, K=8, m=8, fuse=8, work=ws)  # one 8-sweep pass
        op.fourier_correction(E, R, S, work=fw)
        return op.refine(X64, B64, E, None, richm.F32, R, work=rw)

    cycle()
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record()
    for _ in range(5):
        rel = cycle()
    e1.record()
    torch.cuda.synchronize()
    out["two_level_32x1023sq"] = {"ms_per_cycle": e0.elapsed_time(e1) / 5,
                                  "gdof_sweeps_per_s": nb * n * n * 8 / (e0.elapsed_time(e1) / 5e3) / 1e9,
                                  "note": "random symbol: parity only (vs oracle in tests)"}
    op.close()

    # SSOR-preconditioned NAG-Richardson(16) against the Jacobi-preconditioned one on the
    # setting of the paper's SSOR tables (eps = 1e-6, theta = pi/10), 152 instances of
    # 255^2 (one warp per instance for the triangular solves): the same weight recipe
    # (momentum-aware Chebyshev semi-iteration, beta = 0.3) on each preconditioned
    # spectrum bound, (0, 1] for SSOR and (0, G/d] for Jacobi; FP32 sweeps, FP64
    # refinement every 64 sweeps, to 1e-10
    n, nb = 255, 152
    op = richm.Operator([(richm.ANISO_Q1, n, 1e-6, math.pi / 10, 0.0)] * nb)
    G = op.gershgorin()[0]
    dgl = op.stencil(0)[0]
    rhs = np.concatenate([synth.rhs_uniform(46, i, n).ravel() for i in range(nb)])
    B64 = op.pack(torch.tensor(rhs, device=dev), richm.F64)
    res = {}
    for name, pc, bound, relax in (("ssor", 2, 1.0, 1.5), ("jacobi", 1, G / dgl, 1.0)):
        wv = np.array(richm.chebyshev_weights(1.6 * bound, 1.6 * bound / 30.0, 16))
        wt = torch.tensor(np.tile(wv, (nb, 1)), dtype=torch.float32, device=dev)
        at_ = torch.full_like(wt, 0.3)
        o = op.solve_opts(16, tol=SOLVE_TOL, max_sweeps=400000, refine_every=64, inner=richm.F32, precond=pc,
                          fuse=1 if pc == 2 else 0, relax=relax)
        X = op.zeros(richm.F64)
        t0, t1 = ev(), ev()
        t0.record()
        st_, info_ = op.solve(B64, X, wt, at_, None, o)
        t1.record()
        torch.cuda.synchronize()
        sw_ = max(sw for sw, _, _ in info_)
        res[name] = {"status": int(st_), "max_sweeps": int(sw_), "seconds": t0.elapsed_time(t1) / 1e3,
                     "worst_rel_res": max(r for _, r, _ in info_),
                     "gdof_sweeps_per_s": nb * n * n * sw_ / (t0.elapsed_time(t1) / 1e3) / 1e9}
    res["sweep_ratio_jacobi_over_ssor"] = res["jacobi"]["max_sweeps"] / max(1, res["ssor"]["max_sweeps"])
    res["note"] = ("SSOR: one warp per instance walks the rows (scan of the row recurrence), latency-bound; "
                   "parity vs oracle in tests/test_gpu_ssor.py")
    out["ssor_vs_jacobi_152x255sq_eps1e-6"] = res
    op.close()

    # Helmholtz: 16 x 2047^2 complex64, NAG m = 8, seeded weights, 128 sweeps (the
    # library's default pass length for complex64: 4 fused sweeps)
    n, nb = 2047, 16
    k = 2 * math.pi * (n + 1) / 10
    op = richm.Operator([(richm.HELMHOLTZ_FD5_ABC, n, 1.0, 0.0, k)] * nb)
    h = 1.0 / (n + 1)
    wh = torch.tensor(np.tile(synth.helmholtz_weights(8, h, seed=4), (nb, 1)), dtype=torch.float32, device=dev)
    ah = torch.full_like(wh, 0.3)
    src = np.zeros((nb, n * n), np.complex64)
    for s_, (i, j) in enumerate(synth.point_sources(n, nb, seed=5)):
        src[s_, i * n + j] = 1.0
    Bc = op.pack(torch.tensor(src.ravel(), device=dev), richm.C64)
    Xc, XPc = op.zeros(richm.C64), op.zeros(richm.C64)
    ws = op.workspace(op._ws("richm_sweeps_workspace", richm.C64))
    op.apply_sweeps(richm.C64, Xc, XPc, Bc, wh, ah, None, K=8, m=8, work=ws)
    Xc.zero_()
    XPc.zero_()
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record()
    op.apply_sweeps(richm.C64, Xc, XPc, Bc, wh, ah, None, K=128, m=8, work=ws)
    e1.record()
    torch.cuda.synchronize()
    _, _, relh = op.residual_norm(richm.C64, Xc, Bc)
    out["table9_analogue_fgmres20_sponge"] = table9_analogue(dev)
    out["helmholtz_16x2047sq_c64"] = {"ms_128_sweeps": e0.elapsed_time(e1),
                                      "gdof_sweeps_per_s": nb * n * n * 128 / (e0.elapsed_time(e1) / 1e3) / 1e9,
                                      "rel_res_after_128_max": float(relh.max().item()),
                                      "rel_res_after_128_min": float(relh.min().item()),
                                      "note": "fused passes of 4 complex sweeps (64-column tiles); oracle residual "
                                              "check in tests. The seeded weights (h^2/8) U[0.5, 1.5) with momentum "
                                              "0.3 do not converge on this indefinite operator: the residual grows "
                                              "over the 128 sweeps (a throughput workload, as the configuration "
                                              "states)"}
    op.close()
    return out


def table9_analogue(dev, sizes=(128, 256, 512), batch=4, tol=1e-6, max_iters=3000):
    """FGMRES(20) on the sponge-layer Helmholtz problem of eq. 21 at Table 9's grids
    (h = 1/N, omega/2pi = 10 N/128, c = 1), preconditioned by 5 sweeps of Richardson(5) or
    NAG-Richardson(5) (Chebyshev weights of eqs. 8-9 on the upper spectrum [G/4, G], G the
    Gershgorin bound; NAG with beta = 0.3 on the interval stretched by 1.6), by 5 sweeps of
    NAG-Richardson(5) with log-weights and momentum from a Meta-omega network trained here
    (paper_2412_08076_gb300.helmholtz), or by nothing; each with the complex128 Arnoldi basis
    and with the complex64 one (`complex64_basis`).
    The WANS multigrid and ADR parts are not built (their networks and data are not
    available), so the counts are for the smoother alone as the preconditioner. Right-hand
    sides: unit point sources at seeded interior points."""
    import numpy as np
    import torch

    import richm_synth as synth
    from paper_2412_08076_gb300 import richm
    from paper_2412_08076_gb300 import helmholtz as hz
    out = {}
    # Meta-omega: one network for the three grids, trained on random right-hand sides
    specs = [(richm.HELMHOLTZ_FD5_SPONGE, N - 1, 2 * math.pi * 10 * N / 128) for N in sizes for _ in range(2)]
    net = hz.SmootherNet(m=5, K=5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = hz.train(net, specs, steps=300, lr=3e-3)
    torch.cuda.synchronize()
    out["meta_omega_training"] = {"steps": 300, "seconds": time.perf_counter() - t0, "loss_first": hist[0],
                                  "loss_last": hist[-1], "instances": len(specs),
                                  "note": "log-weights and momentum of NAG-Richardson(5) from the meta MLP, "
                                          "complex64 sweeps, complex adjoint, Adam 3e-3"}
    for N in sizes:
        n = N - 1
        om = 2 * math.pi * 10 * N / 128
        op = richm.Operator([(richm.HELMHOLTZ_FD5_SPONGE, n, 1.0, 0.0, om)] * batch)
        G = op.gershgorin()[0]
        src = np.zeros((batch, n * n), np.complex128)
        for s_, (i, j) in enumerate(synth.point_sources(n, batch, seed=6)):
            src[s_, i * n + j] = 1.0
        B = op.pack(torch.tensor(src.ravel(), device=dev), richm.C128)
        row = {"omega_over_2pi": om / (2 * math.pi)}
        for name, beta, stretch in (("none", None, 1.0), ("richardson5", None, 1.0), ("nag_richardson5", 0.3, 1.6),
                                    ("meta_omega_nag5", None, 1.0)):
            X = op.zeros(richm.C128)
            if name == "none":
                w = a = None
                sweeps = 0
            elif name == "meta_omega_nag5":
                Xin = torch.tensor(hz.instance_inputs([(richm.HELMHOLTZ_FD5_SPONGE, n, om)] * batch), device=dev)
                Gt = torch.full((batch,), G, dtype=torch.float32, device=dev)
                w, a, _ = net.coefficients(Xin, Gt)
                sweeps = 5
            else:
                wv = np.array(richm.chebyshev_weights(stretch * G, stretch * G / 4.0, 5))
                w = torch.tensor(np.tile(wv, (batch, 1)), dtype=torch.float32, device=dev)
                a = torch.full_like(w, beta) if beta is not None else None
                sweeps = 5
            res = {}
            for basis in (richm.C128, richm.C64):
                X = op.zeros(richm.C128)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, info = op.fgmres(B, X, w, a, None, restart=20, tol=tol, max_iters=max_iters, m=5, sweeps=sweeps,
                                     inner=richm.C64, basis=basis)
                el = time.perf_counter() - t0
                its = [i_ for i_, _, _ in info]
                res[basis] = {"iterations_mean": float(np.mean(its)), "iterations_max": int(max(its)),
                              "converged": sum(1 for *_, s_ in info if s_ == richm.OK), "seconds": el,
                              "worst_rel_res": max(r for _, r, _ in info)}
            row[name] = dict(res[richm.C128], complex64_basis=res[richm.C64])
        out[f"N{N}"] = row
        op.close()
    return out


def run_reference(args):
    """The oracle as the reference arm: same metric and workload, bounded samples."""
    rank, world = dist_env()
    if rank != 0:
        return 0
    import richm_synth as synth
    insts = synth.batched_aniso(BATCH, SIZES, param_seed=shard_seed(0))
    per_step = min(5.0, max(1.0, 90.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample_rate(insts, seconds=per_step)
    rates = []
    t0 = time.perf_counter()
    desc = ""
    for _ in range(args.steps):
        r, desc = oracle_sample_rate(insts, seconds=per_step)
        rates.append(r)
    el = time.perf_counter() - t0
    value = statistics.mean(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * el / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "per step: " + desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm

def build_batch(seed: int):
    import numpy as np
    import torch

    import richm_synth as synth
    from paper_2412_08076_gb300 import richm
    insts = synth.batched_aniso(BATCH, SIZES, param_seed=seed)
    op = richm.Operator([(richm.ANISO_Q1, t.n, t.eps, t.theta, 0.0) for t in insts])
    rhs = synth.batched_rhs(insts, seed=2 if seed == 1 else 100 + seed)
    dense = torch.tensor(np.concatenate([r.ravel() for r in rhs]), dtype=torch.float64)
    return insts, op, rhs, dense


def meta_inputs(op, insts, params):
    """Device inputs of the meta network: (log10 eps, theta), Gershgorin bounds, parameters."""
    import numpy as np
    import torch

    import richm_synth as synth
    from paper_2412_08076_gb300 import richm
    X = torch.tensor(synth.meta_inputs(insts), dtype=torch.float32, device="cuda")
    G = torch.tensor(op.gershgorin(), dtype=torch.float32, device="cuda")
    P = torch.tensor(params, dtype=torch.float32, device="cuda")
    return X, G, P


def _timed(stream, fn):
    """(result, ms) of fn() bracketed by CUDA events on `stream`."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return r, e0.elapsed_time(e1)


def oracle_check(op, X, insts, rhs, per_size=4):
    """Relative residuals of a sample of solutions (per_size of each grid size),
    recomputed by the FP64 oracle from its own assembled matrices."""
    import numpy as np

    from oracle.operators import assemble_q1
    from paper_2412_08076_gb300 import richm
    xs_h = op.unpack(X, richm.F64).cpu().numpy()
    offs = np.cumsum([0] + [t.n * t.n for t in insts])
    checked, worst, per_n = 0, 0.0, {}
    for i, t in enumerate(insts):
        if per_n.get(t.n, 0) >= per_size:
            continue
        per_n[t.n] = per_n.get(t.n, 0) + 1
        A = assemble_q1(t.n, t.eps, t.theta)
        r = np.linalg.norm(rhs[i].ravel() - A @ xs_h[offs[i]:offs[i + 1]]) / np.linalg.norm(rhs[i])
        worst = max(worst, float(r))
        checked += 1
    return checked, worst


def plain_fp64_baseline(op, insts, rhs, w, a, sweeps, dev):
    """The plain single-instance FP64 GPU sweep (one instance per call, one sweep per
    launch, no graph, same weights, momentum and tolerance): one full solve to 1e-10 of
    one instance of each grid size, timed; the batch's time is those solves plus the
    other instances extrapolated from the measured time per sweep of their size."""
    import torch

    from paper_2412_08076_gb300 import richm
    solved, per_sweep = {}, {}
    for i, t in enumerate(insts):
        if t.n in solved:
            continue
        op1 = richm.Operator([(richm.ANISO_Q1, t.n, t.eps, t.theta, 0.0)])
        b1 = op1.pack(torch.tensor(rhs[i].ravel(), device=dev), richm.F64)
        x1 = op1.zeros(richm.F64)
        w1 = w[i:i + 1].double().contiguous()
        a1 = a[i:i + 1].double().contiguous()
        o1 = op1.solve_opts(M, tol=SOLVE_TOL, max_sweeps=10 ** 7, refine_every=REFINE, inner=richm.F64, use_graph=0,
                            fuse=1)
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        st1, info1 = op1.solve(b1, x1, w1, a1, None, o1)
        el = time.perf_counter() - c0
        solved[t.n] = {"instance": i, "seconds": el, "sweeps": int(info1[0][0]), "status": int(st1),
                       "rel_res": float(info1[0][1])}
        per_sweep[t.n] = el / max(1, info1[0][0])
        op1.close()
    total = sum(v["seconds"] for v in solved.values())
    done = {v["instance"] for v in solved.values()}
    total += sum(per_sweep[t.n] * s for i, (s, t) in enumerate(zip(sweeps, insts)) if i not in done)
    return {"seconds_measured_plus_extrapolated": total, "measured_solves": {str(k): v for k, v in solved.items()},
            "per_sweep_s": {str(k): v for k, v in per_sweep.items()},
            "note": "one full FP64 solve per grid size measured; the other instances extrapolated from the "
                    "measured time per sweep of their size"}


def run_ours(args):
    import numpy as np
    import torch

    from paper_2412_08076_gb300 import meta as meta_mod
    from paper_2412_08076_gb300 import richm

    rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    insts, op, rhs, dense_b = build_batch(shard_seed(rank))
    dofs = sum(t.n * t.n for t in insts)
    params, psrc = meta_mod.load_params(M, variant=META_VARIANT)
    X, G, P = meta_inputs(op, insts, params)
    B64 = op.pack(dense_b.to(dev), richm.F64)
    w, a = richm.meta_forward(P, X, G, M)
    torch.cuda.synchronize()
    beta_seen = float(a.min().item()), float(a.max().item())
    fuse, tune_ms = op.autotune(M, momentum=True)
    opts = op.solve_opts(M, tol=SOLVE_TOL, max_sweeps=10 ** 7, refine_every=REFINE, inner=richm.F32, use_graph=1,
                         fuse=fuse)
    stream = torch.cuda.current_stream()
    lib = richm.load()

    def weight_supply():
        richm._check(lib.richm_meta_forward(richm._ptr(P), richm._ptr(X), richm._ptr(G), len(insts), M,
                                            richm.HEAD_NAG_SHARED, richm._ptr(w), richm._ptr(a), None, None,
                                            richm._stream(stream)), "richm_meta_forward")

    # one step: the weight supply and the solve of the whole batch to tolerance
    Xs = op.zeros(richm.F64)
    wsolve = op.workspace(op._ws("richm_solve_workspace", richm.C.byref(opts)))

    def step():
        weight_supply()
        Xs.zero_()  # every step solves from x = 0
        return op.solve(B64, Xs, w, a, None, opts, work=wsolve)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    infos = []
    for _ in range(args.steps):
        infos.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    st, info = infos[-1]
    sweeps = [sw for sw, _, _ in info]
    step_dof_sweeps = float(sum(sw * t.n * t.n for sw, t in zip(sweeps, insts)))
    t_max_ms = max_over_ranks(ms, world, dev)
    total = sum_over_ranks(step_dof_sweeps * args.steps, world, dev)
    value = total / (t_max_ms / 1e3) / 1e9
    # launches per step: the meta forward, the solver's start (zero start, reduction) and
    # per cycle refine_every / fuse fused passes, the refinement and the reduction
    cycles = int(math.ceil(max(sweeps) / REFINE))
    launches_per_step = 1 + 2 + cycles * (REFINE // fuse + 2)
    checked, worst = oracle_check(op, Xs, insts, rhs)
    ttt = {"seconds": t_max_ms / args.steps / 1e3, "status": int(st),
           "converged": sum(1 for _, _, s_ in info if s_ == richm.OK), "instances": len(insts),
           "max_sweeps": int(max(sweeps)), "mean_sweeps": float(np.mean(sweeps)), "dof_sweeps": step_dof_sweeps,
           "oracle_checked": checked, "oracle_worst_rel_res": worst,
           "beta_from_network": list(beta_seen), "meta_params": psrc}

    # -- refinement cycles with every instance active (tol = 0), both intervals: the
    #    throughput of whole cycles without the convergence tail
    cycle_tp = {}
    for refine in (REFINE, REFINE_LONG):
        o_tp = op.solve_opts(M, tol=0.0, max_sweeps=10 ** 8, refine_every=refine, inner=richm.F32, use_graph=1,
                             fuse=fuse)
        S = richm.Solver(op, o_tp, w, a)
        S.start(B64, op.zeros(richm.F64))
        nc = max(4, 4096 // refine)
        S.step(4, sync=True)
        _, cms = _timed(stream, lambda: S.step(nc, sync=False))
        cycle_tp[f"refine_every_{refine}"] = {"ms_per_cycle": cms / nc,
                                              "gdof_sweeps_per_s": dofs * refine * nc / (cms / 1e3) / 1e9}
        S.close()
    # the earlier network (momentum output ~0.645, trained without the momentum held)
    # with refinement every 256 sweeps, for comparison
    alt = None
    if not args.no_secondary:
        p_alt, src_alt = meta_mod.load_params(M)
        _, _, P_alt = meta_inputs(op, insts, p_alt)
        w_alt, a_alt = richm.meta_forward(P_alt, X, G, M)
        o_alt = op.solve_opts(M, tol=SOLVE_TOL, max_sweeps=10 ** 7, refine_every=REFINE_LONG, inner=richm.F32,
                              use_graph=1, fuse=fuse)
        Xa = op.zeros(richm.F64)
        (st_a, info_a), ams = _timed(stream, lambda: op.solve(B64, Xa, w_alt, a_alt, None, o_alt))
        sw_a = [s_ for s_, _, _ in info_a]
        alt = {"seconds": ams / 1e3, "status": int(st_a), "max_sweeps": int(max(sw_a)),
               "beta": float(a_alt[0, 0].item()), "refine_every": REFINE_LONG,
               "gdof_sweeps_per_s": sum(s_ * t.n * t.n for s_, t in zip(sw_a, insts)) / (ams / 1e3) / 1e9,
               "note": "meta network trained with its momentum free (it settles near 0.645), refinement every "
                       f"{REFINE_LONG} sweeps: not the stated configuration"}

    # the headline solve with each refinement residual formed in FP64 arithmetic instead of
    # the library's default 64-bit fixed point (which is at least as accurate)
    fp64r = None
    if not args.no_secondary:
        o64 = op.solve_opts(M, tol=SOLVE_TOL, max_sweeps=10 ** 7, refine_every=REFINE, inner=richm.F32, use_graph=1,
                            fuse=fuse, fp64_residual=1)
        X64 = op.zeros(richm.F64)
        op.solve(B64, X64, w, a, None, o64)  # warms the session's graphs
        X64.zero_()
        (st64, info64), ms64 = _timed(stream, lambda: op.solve(B64, X64, w, a, None, o64))
        sw64 = [s_ for s_, _, _ in info64]
        fp64r = {"seconds": ms64 / 1e3, "status": int(st64), "max_sweeps": int(max(sw64)),
                 "converged": sum(1 for _, _, s_ in info64 if s_ == richm.OK),
                 "gdof_sweeps_per_s": sum(s_ * t.n * t.n for s_, t in zip(sw64, insts)) / (ms64 / 1e3) / 1e9,
                 "note": "fp64_residual = 1: the refinement's r = b - A x in FP64 arithmetic (GB300 runs FP64 at "
                         "~1/70 of its FP32 rate); the headline value uses the fixed-point form"}

    # -- dominant kernel (the fused FP32 NAG pass) and the one-sweep kernel: launch
    #    durations by CUDA events on the launching stream
    xs = op.zeros(richm.F32)
    xps = op.zeros(richm.F32)
    b32 = op.zeros(richm.F32)
    b32.copy_(B64.to(torch.float32))
    ws = op.workspace(op._ws("richm_sweeps_workspace", richm.F32))

    def launch_ms(f, K=192, reps=3):
        op.apply_sweeps(richm.F32, xs, xps, b32, w, a, None, K=K, m=M, fuse=f, work=ws)
        torch.cuda.synchronize()

        def run():
            for _ in range(reps):
                op.apply_sweeps(richm.F32, xs, xps, b32, w, a, None, K=K, m=M, fuse=f, work=ws)
        _, t = _timed(stream, run)
        return t / (reps * K // f)

    one_ms = launch_ms(1)
    one_gbs = 16.0 * dofs / (one_ms / 1e3) / 1e9  # read x_k, x_{k-1}, b; write x_{k+1}
    if fuse == 1:
        roof = {"bound": "hbm", "achieved": one_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": one_gbs / hbm_peak,
                "traffic": kernel_traffic("sweep1", dofs), "kernel": "sweep1_kernel<float,NAG>",
                "alg_bytes_per_launch": 16.0 * dofs, "launch_ms": one_ms, "sweeps_per_launch": 1,
                "peak_source": f"{peak_src} hbm_gbs"}
    else:
        fused_ms = launch_ms(fuse)
        kname = (f"sweepT8_kernel<NAG> (8 FP32 NAG sweeps per launch, temporal blocking)"
                 if fuse == 8 else f"sweepT_kernel<{fuse},NAG> ({fuse} FP32 NAG sweeps per launch, temporal blocking)")
        # algorithmic bytes of a pass: read x_k, x_{k-1}, b, write x_{k+T}, x_{k+T-1}
        # (20 B per unknown, 20/T B per dof-sweep); the binding roof at T = 8 is HBM's
        # (HBM: 6768 / 2.5 = 2707 Gdof-sweeps/s; FP32 pipe: 80.5 TFLOP/s / 19 = 4237)
        alg = 20.0 * dofs
        gbs = alg / (fused_ms / 1e3) / 1e9
        sm_ghz = (clk.get("sm_mhz") or 2070.0) / 1e3
        fp32_peak = sms * 128 * 2 * sm_ghz / 1e3  # TFLOP/s
        flops = 19.0 * dofs * fuse
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "traffic": kernel_traffic(f"sweepT{fuse}", dofs), "kernel": kname, "alg_bytes_per_launch": alg,
                "launch_ms": fused_ms, "sweeps_per_launch": fuse, "peak_source": f"{peak_src} hbm_gbs",
                "gdof_sweeps_per_s": dofs * fuse / (fused_ms / 1e3) / 1e9,
                "alu_view": {"alg_flops_per_launch": flops, "achieved_tflops": flops / (fused_ms / 1e3) / 1e12,
                             "derived_fp32_peak_tflops": fp32_peak,
                             "frac": flops / (fused_ms / 1e3) / 1e12 / fp32_peak,
                             "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 x {sm_ghz:.3f} GHz (sampled)"},
                "one_sweep_kernel": {"kernel": "sweep1_kernel<float,NAG>", "launch_ms": one_ms,
                                     "achieved_gbs": one_gbs, "frac_of_measured_hbm": one_gbs / hbm_peak}}
        try:
            fma = {"fp32": richm.fma_peak(richm.FMA_F32), "fp32x2": richm.fma_peak(richm.FMA_F32X2),
                   "fp64": richm.fma_peak(richm.FMA_F64), "unit": "TFLOP/s"}
            best = max(fma["fp32"], fma["fp32x2"])
            fma["frac_of_measured_fp32"] = flops / (fused_ms / 1e3) / 1e12 / best if best > 0 else None
            roof["alu_view"]["fma_microbenchmark"] = fma
        except Exception as exc:  # a diagnostic: never costs the bench line
            roof["alu_view"]["fma_microbenchmark"] = {"error": str(exc)[:200]}

    # -- e2e: the call a user makes with host buffers: richm_solve_host copies b from
    #    pinned host memory, packs, solves every instance to tolerance from x = 0,
    #    unpacks and copies x back (synchronous); value = dof-sweeps done / wall time
    hb = dense_b.pin_memory()
    hx = torch.empty(op.dense_elems(), dtype=torch.float64).pin_memory()
    e2e_runs = []
    e2e_clocks = ClockSampler(torch.cuda.current_device())
    for rep in range(1 + max(1, args.e2e_runs)):
        torch.cuda.synchronize()
        if rep == 1:
            e2e_clocks.start()
        c0 = time.perf_counter()
        weight_supply()
        st_e, info_e = op.solve_host(hb, hx, w, a, None, opts)
        el = time.perf_counter() - c0
        if rep > 0:  # the first call warms the host path
            e2e_runs.append((el, sum(sw * t.n * t.n for (sw, _, _), t in zip(info_e, insts)), st_e))
    e2e_clk = e2e_clocks.stop()
    e2e_s = sum(r[0] for r in e2e_runs) / len(e2e_runs)
    e2e_val = sum(r[1] for r in e2e_runs) / sum(r[0] for r in e2e_runs) / 1e9

    plain = None
    if not args.no_solve:
        plain = plain_fp64_baseline(op, insts, rhs, w, a, sweeps, dev)
        plain["speedup_of_the_batched_solve"] = plain["seconds_measured_plus_extrapolated"] / ttt["seconds"]

    fuse_rows = op.tuned()[1]
    workloads = None if args.no_secondary else secondary_workloads(dev)
    # -- experiment: bfloat16 storage of the inner iterate (FP32 arithmetic, FP64 refinement)
    bf16 = None
    if not args.no_solve:
        xb16 = op.zeros(richm.BF16)
        xpb16 = op.zeros(richm.BF16)
        wsb = op.workspace(op._ws("richm_sweeps_workspace", richm.BF16))
        op.apply_sweeps(richm.BF16, xb16, xpb16, b32, w, a, None, K=192, m=M, fuse=fuse, work=wsb)
        torch.cuda.synchronize()

        def runb():
            for _ in range(3):
                op.apply_sweeps(richm.BF16, xb16, xpb16, b32, w, a, None, K=192, m=M, fuse=fuse, work=wsb)
        _, bms = _timed(stream, runb)
        bf_ms = bms / (3 * 192 // fuse)
        ob = op.solve_opts(M, tol=SOLVE_TOL, max_sweeps=10 ** 6, refine_every=REFINE, inner=richm.BF16, use_graph=1,
                           fuse=fuse)
        Xb = op.zeros(richm.F64)
        (st_b, info_b), sbms = _timed(stream, lambda: op.solve(B64, Xb, w, a, None, ob))
        nb_chk, worst_b = oracle_check(op, Xb, insts, rhs, per_size=1)
        bf16 = {"fused_launch_ms": bf_ms, "fused_gdof_sweeps_per_s": dofs * fuse / (bf_ms / 1e3) / 1e9,
                "fp32_fused_gdof_sweeps_per_s": roof.get("gdof_sweeps_per_s"),
                "solve_seconds": sbms / 1e3, "status": int(st_b),
                "converged": sum(1 for _, _, s_ in info_b if s_ == richm.OK),
                "max_sweeps": int(max(sw_ for sw_, _, _ in info_b)), "oracle_checked": nb_chk,
                "oracle_worst_rel_res": worst_b,
                "note": "bfloat16 inner state (x_k, x_{k-1} and the correction stored as bf16), FP32 arithmetic "
                        f"and rhs, FP64 refinement every {REFINE} sweeps; an experiment, not the headline"}

    line = None
    if rank == 0:
        cpu_rate, cpu_desc = oracle_sample_rate(insts, seconds=args.cpu_seconds)
        all_rate, all_procs, all_desc = oracle_all_cores_rate(insts, seconds=min(8.0, args.cpu_seconds))
        other_cpu = oracle_other_configs() if args.cpu_seconds >= 5 else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(), dofs_per_rank=dofs, meta_params=psrc, sweeps_per_pass=fuse,
                           fused_tile_rows=fuse_rows, autotune_ms_per_sweep=tune_ms, solve_tol=SOLVE_TOL),
            "roofline": roof,
            "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": cpu_desc,
                             "host_cores": os.cpu_count()},
            "cpu_baseline_all_cores": {"value": all_rate, "unit": UNIT, "cores": all_procs, "kind": "oracle",
                                       "sample": all_desc},
            "cpu_oracle_other_configs": other_cpu,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(dense_b.numel() * 8),
                    "d2h_bytes_per_step": int(hx.numel() * 8), "seconds_per_call": e2e_s,
                    "seconds_each": [round(r[0], 4) for r in e2e_runs],
                    "statuses": [r[2] for r in e2e_runs], "clocks": e2e_clk,
                    "note": "one step = the weight supply and one richm_solve_host call: pinned H2D of b, pack, "
                            "solve every instance to 1e-10 from x = 0 (FP32 sweeps + FP64 refinement), unpack, "
                            "D2H of x; value = dof-sweeps performed / wall time"},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
            "time_to_tol": ttt,
            "cycle_throughput_all_active": cycle_tp,
            "plain_fp64_gpu_sweep": plain,
            "network_free_momentum_refine256": alt,
            "refinement_residual_fp64_arithmetic": fp64r,
            "workloads": workloads,
            "bf16_state_experiment": bf16,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- profiling cases

# the sources a kernel is compiled from (its translation unit and the shared device
# header; kernels.cuh only declares host launchers)
TRAFFIC_SOURCES = {
    "sweep1": ["paper_2412_08076_gb300/csrc/sweep.cu", "paper_2412_08076_gb300/csrc/common.cuh"],
    "sweepT4": ["paper_2412_08076_gb300/csrc/sweep_fused.cu", "paper_2412_08076_gb300/csrc/common.cuh"],
    "sweepT8": ["paper_2412_08076_gb300/csrc/sweep_fused.cu", "paper_2412_08076_gb300/csrc/common.cuh"],
    "refine": ["paper_2412_08076_gb300/csrc/solve.cu", "paper_2412_08076_gb300/csrc/common.cuh"],
}


def record_traffic(report: str, kind: str, unknowns: int) -> float:
    """Read dram__bytes_read/write.sum of the captured launch from an ncu report and
    store DRAM bytes per unknown in profiles/traffic.txt with a hash of the kernel's
    sources (the bench reports traffic only while the hash still matches)."""
    import csv
    import hashlib
    out = subprocess.run(["ncu", "-i", report, "--page", "raw", "--csv"], capture_output=True, text=True,
                         check=True).stdout
    rows = list(csv.reader(out.splitlines()))
    hdr, units, data = rows[0], rows[1], rows[2]
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    tot = 0.0
    if "dram__bytes_read.sum" in hdr:
        for name in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            i = hdr.index(name)
            tot += float(data[i].replace(",", "")) * scale[units[i]]
    else:  # a capture by sections: the DRAM byte rate times the launch's duration
        i = hdr.index("dram__bytes.sum.per_second")
        rate = float(data[i].replace(",", "")) * {"byte/s": 1.0, "Kbyte/s": 1e3, "Mbyte/s": 1e6,
                                                   "Gbyte/s": 1e9, "Tbyte/s": 1e12}[units[i]]
        j = hdr.index("gpu__time_duration.sum")
        dur = float(data[j].replace(",", "")) * {"nsecond": 1e-9, "ns": 1e-9, "usecond": 1e-6, "us": 1e-6, "msecond": 1e-3, "ms": 1e-3}[units[j]]
        tot = rate * dur
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES[kind]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    lines = []
    if os.path.exists(path):
        lines = [ln for ln in open(path).read().splitlines() if ln and not ln.startswith(kind + " ")]
    per = tot / unknowns
    lines.append(f"{kind} {h.hexdigest()} {per:.6f} {' '.join(TRAFFIC_SOURCES[kind])}")
    with open(path, "w") as fh:
        fh.write("\n".join(sorted(lines)) + "\n")
    return per


def run_profile_case(args):
    """A small fixed workload for capturing one kernel family with ncu: a few FP32 NAG
    sweeps (or solver cycles, adjoint steps, complex Helmholtz or SSOR sweeps) on a batch
    of identical-size anisotropic instances, large enough that the state exceeds L2 and
    small enough (a few hundred MB) for a short capture."""
    import numpy as np
    import torch

    import richm_synth as synth
    from paper_2412_08076_gb300 import richm
    m = 16
    what = args.profile
    if what == "bench_cycles":
        # the benchmark's batch, network and settings: the weight supply, the solver's start
        # and `sweeps` / 64 refinement cycles (plain launches, no graph)
        from paper_2412_08076_gb300 import meta as meta_mod
        insts, op, rhs, dense_b = build_batch(1)
        params, _ = meta_mod.load_params(M, variant=META_VARIANT)
        X, G, P = meta_inputs(op, insts, params)
        w, a = richm.meta_forward(P, X, G, M)
        op.set_tuning(8, 128)
        B64 = op.pack(dense_b.cuda(), richm.F64)
        S = richm.Solver(op, op.solve_opts(M, tol=SOLVE_TOL, max_sweeps=10 ** 7, refine_every=REFINE,
                                           inner=richm.F32, use_graph=0, fuse=8), w, a)
        S.start(B64, op.zeros(richm.F64))
        S.step(max(1, args.sweeps // REFINE), sync=True)
        S.close()
        torch.cuda.synchronize()
        return 0
    if what in ("fgmres", "adjoint_cx"):
        # Table 9's largest grid (N = 512, sponge layer): FGMRES(20) preconditioned by 5 NAG
        # sweeps (`sweeps` bounds the iterations), or one Meta-omega training step (forward
        # and complex adjoint of 5 complex64 sweeps on random right-hand sides)
        from paper_2412_08076_gb300 import helmholtz as hz
        N = args.n + 1
        spec = (richm.HELMHOLTZ_FD5_SPONGE, args.n, 2 * math.pi * 10 * N / 128)
        op = richm.Operator([(kind, n_, 1.0, 0.0, k) for kind, n_, k in [spec] * args.batch])
        net = hz.SmootherNet(m=5, K=5)
        X = torch.tensor(hz.instance_inputs([spec] * args.batch), device="cuda")
        G = torch.tensor(np.array(op.gershgorin()), dtype=torch.float32, device="cuda")
        B = hz.random_rhs(op, [spec] * args.batch, 77)
        if what == "adjoint_cx":
            net.loss_and_grads(op, X, G, B)
        else:
            w, a, _ = net.coefficients(X, G)
            B128 = op.pack(op.unpack(B, richm.C64).to(torch.complex128), richm.C128)
            op.fgmres(B128, op.zeros(richm.C128), w, a, None, restart=20, tol=1e-6, max_iters=args.sweeps, m=5,
                      sweeps=5, inner=richm.C64, basis=richm.C64 if args.basis == "c64" else richm.C128)
        torch.cuda.synchronize()
        return 0
    insts = synth.batched_aniso(args.batch, sizes=(args.n,), param_seed=1)
    if what == "helmholtz":
        k = 2 * math.pi * (args.n + 1) / 10
        op = richm.Operator([(richm.HELMHOLTZ_FD5_ABC, args.n, 1.0, 0.0, k)] * args.batch)
        dt = richm.C64
        w = torch.full((args.batch, 8), 1.0 / (8 * (args.n + 1) ** 2), device="cuda")
        a = torch.full((args.batch, 8), 0.3, device="cuda")
        x, xp, b = op.zeros(dt), op.zeros(dt), op.zeros(dt)
        b.fill_(1.0)
        op.apply_sweeps(dt, x, xp, b, w, a, None, K=args.sweeps, m=8, fuse=args.fuse)
        torch.cuda.synchronize()
        return 0
    op = richm.Operator([(richm.ANISO_Q1, t.n, t.eps, t.theta, 0.0) for t in insts])
    G = np.array(op.gershgorin())
    unit = np.array(richm.chebyshev_weights(1.6, 1.6 / 30.0, m))
    w = torch.tensor(unit[None, :] / G[:, None], dtype=torch.float32, device="cuda")
    a = torch.full_like(w, 0.3)
    dense = torch.tensor(np.concatenate([synth.rhs_uniform(2, i, t.n).ravel() for i, t in enumerate(insts)]),
                         device="cuda")
    if what == "sweep":
        b = op.pack(dense.float(), richm.F32)
        x, xp = op.zeros(richm.F32), op.zeros(richm.F32)
        op.apply_sweeps(richm.F32, x, xp, b, w, a, None, K=args.sweeps, m=m, fuse=args.fuse)
    elif what == "ssor":
        # SSOR-preconditioned NAG sweeps (B^{-1} A has its spectrum in (0, 1])
        b = op.pack(dense.float(), richm.F32)
        x, xp = op.zeros(richm.F32), op.zeros(richm.F32)
        ws_ = torch.tensor(np.tile(unit, (args.batch, 1)), dtype=torch.float32, device="cuda")
        op.apply_sweeps(richm.F32, x, xp, b, ws_, a, None, K=args.sweeps, m=m, precond=2, relax=1.5)
    elif what == "cycle":
        b = op.pack(dense, richm.F64)
        x = op.zeros(richm.F64)
        S = richm.Solver(op, op.solve_opts(m, tol=1e-10, max_sweeps=10 ** 8, fuse=args.fuse), w, a)
        S.start(b, x)
        S.step(max(1, args.sweeps // 64), sync=True)
        S.close()
    else:  # adjoint
        b = op.pack(dense.float(), richm.F32)
        K, every = 16, 8
        ck = torch.empty(op.checkpoint_elems(K, every), dtype=torch.float32, device="cuda")
        xK, g = op.zeros(richm.F32), op.zeros(richm.F32)
        x0 = op.zeros(richm.F32)
        op.forward_checkpointed(richm.F32, x0, b, w, a, None, m, K, every, 0, ck, xK)
        op.loss_log_residual(richm.F32, xK, b, g)
        gw, ga = torch.zeros_like(w), torch.zeros_like(a)
        op.sweeps_adjoint(richm.F32, ck, every, b, g, w, a, None, m, K, 0, gw, ga, None, None)
    torch.cuda.synchronize()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-solve", action="store_true", help="skip the time-to-tolerance solve")
    ap.add_argument("--no-secondary", action="store_true", help="skip the other workloads' measurements")
    ap.add_argument("--e2e-runs", type=int, default=4, help="timed richm_solve_host calls")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--profile", choices=["sweep", "cycle", "adjoint", "helmholtz", "ssor", "bench_cycles", "fgmres",
                                          "adjoint_cx"], default=None,
                    help="run a small fixed workload of one kernel family for an ncu capture instead of the bench")
    ap.add_argument("--batch", type=int, default=32, help="--profile: instances")
    ap.add_argument("--basis", choices=["c128", "c64"], default="c128", help="--profile fgmres: the Arnoldi basis")
    ap.add_argument("--n", type=int, default=511, help="--profile: grid size")
    ap.add_argument("--sweeps", type=int, default=6, help="--profile: sweeps")
    ap.add_argument("--fuse", type=int, default=1, help="--profile: sweeps per pass")
    ap.add_argument("--record-traffic", metavar="NCU_REPORT", default=None,
                    help="store the report's DRAM bytes per unknown (--kind, --batch x --n^2 unknowns) in "
                         "profiles/traffic.txt and exit")
    ap.add_argument("--kind", default="sweepT8", choices=sorted(TRAFFIC_SOURCES))
    args = ap.parse_args(argv)
    if args.record_traffic:
        per = record_traffic(args.record_traffic, args.kind, args.batch * args.n * args.n)
        print(f"{args.kind}: {per:.3f} DRAM bytes per unknown per launch")
        return 0
    if args.profile:
        return run_profile_case(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
