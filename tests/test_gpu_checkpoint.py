"""Checkpoint and resume of a solver session: an image saved between steps, restored
into a new session (in this process or in another one), continues with the same bits
as the uninterrupted session; images that do not match the session are refused."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import richm_synth as synth
from gpu_util import coef, make_op, nag_weights, to_dev
from oracle.operators import assemble_q1, gershgorin_max
from paper_2412_08076_gb300 import richm

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SIZES = [17, 40, 63, 130]
MODES = {"fused": dict(refine_every=64, inner=richm.F32, fuse=8),
         "fp64": dict(refine_every=16, inner=richm.F64, fuse=1)}


def _setup(mode, sizes=SIZES, wscale=1.0):
    insts = [synth.AnisoInstance(10 ** (-0.7 * i), 0.4 + 0.5 * i, n) for i, n in enumerate(sizes)]
    op = make_op(insts)
    G = np.array([gershgorin_max(assemble_q1(t.n, t.eps, t.theta)) for t in insts])
    w, a = nag_weights(G, 16)
    rd = richm.F64 if MODES[mode]["inner"] == richm.F64 else richm.F32
    W, A = coef(w * wscale, rd), coef(a, rd)
    B = to_dev(op, [synth.rhs_uniform(2, i, t.n) for i, t in enumerate(insts)], richm.F64)
    opts = op.solve_opts(16, tol=1e-10, max_sweeps=10 ** 6, use_graph=1, **MODES[mode])
    return op, W, A, B, opts


# run in a fresh process: rebuild the same session, resume from the image, continue
CHILD = r'''
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import numpy as np, torch
import test_gpu_checkpoint as T
from paper_2412_08076_gb300 import richm
op, W, A, B, opts = T._setup({mode!r})
X = torch.full((op.elems,), -3.0, dtype=torch.float64, device="cuda")
S = richm.Solver(op, opts, W, A)
with open({img!r}, "rb") as fh:
    S.resume(B, X, fh.read())
S.step({cycles})
st, info = S.finish()
np.save({out!r}, X.cpu().numpy())
np.save({out!r}.replace(".npy", "_info.npy"), np.array([[i[0], i[1], i[2]] for i in info], dtype=np.float64))
'''


def _run_to(S, B, X, first, then):
    S.start(B, X)
    S.step(first)
    img = S.save()
    S.step(then)
    st, info = S.finish()
    return img, X.cpu().numpy(), info


@pytest.mark.parametrize("mode", ["fused", "fp64"])
def test_resume_in_a_new_session_continues_bit_for_bit(mode):
    op, W, A, B, opts = _setup(mode)
    X1 = op.zeros(richm.F64)
    S1 = richm.Solver(op, opts, W, A)
    img, x1, info1 = _run_to(S1, B, X1, 3, 150)
    X2 = torch.full_like(X1, 7.0)  # the image overwrites every element, padding included
    S2 = richm.Solver(op, opts, W, A)
    S2.resume(B, X2, img)
    S2.step(150)
    st2, info2 = S2.finish()
    assert info2 == info1
    np.testing.assert_array_equal(X2.cpu().numpy(), x1)
    # the image of the resumed session at the same point is the saved one
    S3 = richm.Solver(op, opts, W, A)
    X3 = op.zeros(richm.F64)
    S3.resume(B, X3, img)
    assert S3.save() == img
    for S in (S1, S2, S3):
        S.close()


def test_resume_in_another_process(tmp_path):
    mode = "fused"
    op, W, A, B, opts = _setup(mode)
    X1 = op.zeros(richm.F64)
    S1 = richm.Solver(op, opts, W, A)
    img, x1, info1 = _run_to(S1, B, X1, 2, 60)
    S1.close()
    path = str(tmp_path / "solver.img")
    with open(path, "wb") as fh:
        fh.write(img)
    out = str(tmp_path / "x.npy")
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), mode=mode, img=path, cycles=60, out=out)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    np.testing.assert_array_equal(np.load(out), x1)
    info2 = np.load(out.replace(".npy", "_info.npy"))
    np.testing.assert_array_equal(info2, np.array([[i[0], i[1], i[2]] for i in info1], dtype=np.float64))


def test_mismatched_images_are_refused():
    op, W, A, B, opts = _setup("fused")
    S = richm.Solver(op, opts, W, A)
    with pytest.raises(richm.RichmError):
        S.save()  # not started
    X = op.zeros(richm.F64)
    S.start(B, X)
    S.step(1)
    img = S.save()
    x_before = X.cpu().numpy()
    # other weights
    op2, W2, A2, B2, opts2 = _setup("fused", wscale=1.01)
    S2 = richm.Solver(op2, opts2, W2, A2)
    X2 = op2.zeros(richm.F64)
    with pytest.raises(richm.RichmError, match="weights"):
        S2.resume(B2, X2, img)
    # other options
    opts3 = op.solve_opts(16, tol=1e-10, max_sweeps=10 ** 6, use_graph=1, refine_every=128, inner=richm.F32, fuse=8)
    S3 = richm.Solver(op, opts3, W, A)
    with pytest.raises(richm.RichmError, match="options"):
        S3.resume(B, op.zeros(richm.F64), img)
    # the other refinement residual form
    opts3b = op.solve_opts(16, tol=1e-10, max_sweeps=10 ** 6, use_graph=1, refine_every=64, inner=richm.F32, fuse=8,
                           fp64_residual=1)
    S3b = richm.Solver(op, opts3b, W, A)
    with pytest.raises(richm.RichmError, match="options"):
        S3b.resume(B, op.zeros(richm.F64), img)
    S3b.close()
    # other instances
    op4, W4, A4, B4, opts4 = _setup("fused", sizes=[17, 40, 63, 129])
    S4 = richm.Solver(op4, opts4, W4, A4)
    with pytest.raises(richm.RichmError):
        S4.resume(B4, op4.zeros(richm.F64), img)
    # truncated or damaged images
    S5 = richm.Solver(op, opts, W, A)
    X5 = op.zeros(richm.F64)
    with pytest.raises(richm.RichmError):
        S5.resume(B, X5, img[:-8])
    with pytest.raises(richm.RichmError):
        S5.resume(B, X5, b"RICHMSV2" + img[8:])
    assert not X5.any()  # nothing restored
    np.testing.assert_array_equal(X.cpu().numpy(), x_before)
    for s in (S, S2, S3, S4, S5):
        s.close()


def test_resume_at_the_benchmark_size():
    # the benchmark's batch (256 instances, 27 M unknowns), network and settings: an image
    # saved after 20 refinement cycles and resumed in a new session continues with the
    # same bits as the uninterrupted session after 20 more
    import bench
    from paper_2412_08076_gb300 import meta as meta_mod
    insts, op, rhs, dense_b = bench.build_batch(1)
    params, _ = meta_mod.load_params(bench.M, variant=bench.META_VARIANT)
    X, G, P = bench.meta_inputs(op, insts, params)
    w, a = richm.meta_forward(P, X, G, bench.M)
    B = op.pack(dense_b.cuda(), richm.F64)
    opts = op.solve_opts(bench.M, tol=bench.SOLVE_TOL, max_sweeps=10 ** 7, refine_every=bench.REFINE,
                         inner=richm.F32, use_graph=1, fuse=8)
    X1 = op.zeros(richm.F64)
    S1 = richm.Solver(op, opts, w, a)
    img, x1, info1 = _run_to(S1, B, X1, 20, 20)
    S1.close()
    X2 = torch.full_like(X1, 1.0)
    S2 = richm.Solver(op, opts, w, a)
    S2.resume(B, X2, img)
    del img
    S2.step(20)
    st2, info2 = S2.finish()
    assert info2 == info1
    assert torch.equal(X2, torch.tensor(x1, device="cuda"))
    S2.close()
