"""Host-side logic of bench.py: rank sharding and max/sum over ranks (gloo, 2 ranks on CPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shard_seeds_distinct_and_rank0_canonical():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.shard_seed(0) == 1
    assert len({bench.shard_seed(r) for r in range(8)}) == 8


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w = bench.dist_env()
    mx = bench.max_over_ranks(10.0 + r, w)
    sm = bench.sum_over_ranks(100.0 * (r + 1), w)
    dist.barrier()
    dist.destroy_process_group()
    with open(out + f".{rank}", "w") as fh:
        json.dump({"rank": r, "world": w, "max": mx, "sum": sm}, fh)


def test_max_and_sum_over_two_gloo_ranks(tmp_path):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = 29500 + os.getpid() % 1000
    out = str(tmp_path / "res")
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        res = json.load(open(out + f".{r}"))
        assert res["world"] == 2 and res["rank"] == r
        assert res["max"] == 11.0 and res["sum"] == 300.0


def test_weak_scaling_value_arithmetic():
    # value = (all ranks' dof-sweeps) / (max over ranks of the time); one step solves a
    # rank's batch to tolerance, so its dof-sweeps are sum_b sweeps_b n_b^2
    sys.path.insert(0, ROOT)
    import bench
    assert (bench.M, bench.BETA, bench.REFINE, bench.TOL) == (16, 0.3, 64, 1e-10)  # the stated configuration
    per_step = [3.0e9, 2.0e9]  # two ranks' dof-sweeps per solve
    steps, ms_max = 10, 4000.0
    v = sum(per_step) * steps / (ms_max / 1e3) / 1e9
    assert abs(v - 12.5) < 1e-12
