"""Small, fixed workloads for profiling one kernel family with ncu.

  python -m paper_2412_08076_gb300.profile_case --what sweep --batch 32 --n 511 --sweeps 6
runs a few FP32 NAG sweeps (or solver cycles with --what cycle) on a batch of
identical-size anisotropic instances: large enough that the state exceeds L2,
small enough (a few hundred MB) for a short capture.
"""
from __future__ import annotations

import argparse
import math

import numpy as np
import torch

from . import meta as meta_mod
from . import richm


# the sources a kernel is compiled from (its translation unit and the shared device
# header; kernels.cuh only declares host launchers)
TRAFFIC_SOURCES = {
    "sweep1": ["paper_2412_08076_gb300/csrc/sweep.cu", "paper_2412_08076_gb300/csrc/common.cuh"],
    "sweepT4": ["paper_2412_08076_gb300/csrc/sweep_fused.cu", "paper_2412_08076_gb300/csrc/common.cuh"],
    "sweepT8": ["paper_2412_08076_gb300/csrc/sweep_fused.cu", "paper_2412_08076_gb300/csrc/common.cuh"],
    "refine": ["paper_2412_08076_gb300/csrc/solve.cu", "paper_2412_08076_gb300/csrc/common.cuh"],
}


def record_traffic(report: str, kind: str, unknowns: int, root: str) -> float:
    """Read dram__bytes_read/write.sum of the captured launch from an ncu report and
    store DRAM bytes per unknown in profiles/traffic.txt with a hash of the kernel's
    sources (bench.py reports traffic only while the hash still matches)."""
    import csv
    import hashlib
    import os
    import subprocess
    out = subprocess.run(["ncu", "-i", report, "--page", "raw", "--csv"], capture_output=True, text=True,
                         check=True).stdout
    rows = list(csv.reader(out.splitlines()))
    hdr, units, data = rows[0], rows[1], rows[2]
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    tot = 0.0
    for name in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
        i = hdr.index(name)
        tot += float(data[i].replace(",", "")) * scale[units[i]]
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES[kind]:
        with open(os.path.join(root, f), "rb") as fh:
            h.update(fh.read())
    path = os.path.join(root, "profiles", "traffic.txt")
    lines = []
    if os.path.exists(path):
        lines = [ln for ln in open(path).read().splitlines() if ln and not ln.startswith(kind + " ")]
    per = tot / unknowns
    lines.append(f"{kind} {h.hexdigest()} {per:.6f} {' '.join(TRAFFIC_SOURCES[kind])}")
    with open(path, "w") as fh:
        fh.write("\n".join(sorted(lines)) + "\n")
    return per


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--what", choices=["sweep", "cycle", "adjoint", "helmholtz", "ssor"], default="sweep")
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--n", type=int, default=511)
    ap.add_argument("--sweeps", type=int, default=6)
    ap.add_argument("--fuse", type=int, default=1)
    ap.add_argument("--record-traffic", metavar="NCU_REPORT", default=None,
                    help="store the report's DRAM bytes per unknown in profiles/traffic.txt and exit")
    ap.add_argument("--kind", default="sweepT8")
    args = ap.parse_args(argv)
    if args.record_traffic:
        import os
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        per = record_traffic(args.record_traffic, args.kind, args.batch * args.n * args.n, root)
        print(f"{args.kind}: {per:.3f} DRAM bytes per unknown per launch")
        return
    import richm_synth as synth
    m = 16
    insts = synth.batched_aniso(args.batch, sizes=(args.n,), param_seed=1)
    if args.what == "helmholtz":
        k = 2 * math.pi * (args.n + 1) / 10
        op = richm.Operator([(richm.HELMHOLTZ_FD5_ABC, args.n, 1.0, 0.0, k)] * args.batch)
        dt = richm.C64
        w = torch.full((args.batch, 8), 1.0 / (8 * (args.n + 1) ** 2), device="cuda")
        a = torch.full((args.batch, 8), 0.3, device="cuda")
        x, xp, b = op.zeros(dt), op.zeros(dt), op.zeros(dt)
        b.fill_(1.0)
        op.apply_sweeps(dt, x, xp, b, w, a, None, K=args.sweeps, m=8, fuse=args.fuse)
        torch.cuda.synchronize()
        return
    op = richm.Operator([(richm.ANISO_Q1, t.n, t.eps, t.theta, 0.0) for t in insts])
    G = np.array(op.gershgorin())
    wn = meta_mod.chebyshev_unit_weights(m)[None, :] / G[:, None]
    w = torch.tensor(wn, dtype=torch.float32, device="cuda")
    a = torch.full_like(w, 0.3)
    dense = torch.tensor(np.concatenate([synth.rhs_uniform(2, i, t.n).ravel() for i, t in enumerate(insts)]),
                         device="cuda")
    if args.what == "sweep":
        b = op.pack(dense.float(), richm.F32)
        x, xp = op.zeros(richm.F32), op.zeros(richm.F32)
        op.apply_sweeps(richm.F32, x, xp, b, w, a, None, K=args.sweeps, m=m, fuse=args.fuse)
    elif args.what == "ssor":
        # SSOR-preconditioned NAG sweeps (B^{-1} A has its spectrum in (0, 1])
        b = op.pack(dense.float(), richm.F32)
        x, xp = op.zeros(richm.F32), op.zeros(richm.F32)
        ws = torch.tensor(meta_mod.chebyshev_unit_weights(m)[None, :].repeat(args.batch, 0), dtype=torch.float32,
                          device="cuda")
        op.apply_sweeps(richm.F32, x, xp, b, ws, a, None, K=args.sweeps, m=m, precond=2, relax=1.5)
    elif args.what == "cycle":
        b = op.pack(dense, richm.F64)
        x = op.zeros(richm.F64)
        S = richm.Solver(op, op.solve_opts(m, tol=1e-10, max_sweeps=10**8, fuse=args.fuse), w, a)
        S.start(b, x)
        S.step(max(1, args.sweeps // 64), sync=True)
        S.close()
    else:
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


if __name__ == "__main__":
    main()
