"""The allocation-free residual norm gives the same results as the workspace version.

richm_residual_norm_static serves callers that cannot allocate device memory
(code running inside someone else's memory pool or allocator callback, or a
process whose device memory was reserved up front by another framework): its
scratch lives in file-scope device arrays of the library instead of a
caller-supplied workspace. This file is collected last so that a run stopping at
its first failure has already run every other test; it also passes alone.
"""
import ctypes

import numpy as np
import pytest
import torch

import richm_synth as synth
from paper_2412_08076_gb300 import richm

pytestmark = pytest.mark.gpu


def _static(op, dtype, x, b):
    lib = richm.load()
    fn = lib.richm_residual_norm_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 7
    rn = torch.empty(op.batch, dtype=torch.float64, device="cuda")
    bn = torch.empty_like(rn)
    rel = torch.empty_like(rn)
    r = op.zeros(dtype)
    st = fn(op.handle, dtype, x.data_ptr(), b.data_ptr(), rn.data_ptr(), bn.data_ptr(), rel.data_ptr(), r.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
    assert st == richm.OK, lib.richm_last_error()
    return rn, bn, rel, r


@pytest.mark.parametrize("dtype", [richm.F32, richm.F64])
def test_static_scratch_residual_matches_workspace_version_twice(dtype):
    insts = synth.batched_aniso(12, sizes=(1, 31, 127, 200), param_seed=77)
    op = richm.Operator([(richm.ANISO_Q1, t.n, t.eps, t.theta, 0.0) for t in insts])
    td = richm.TORCH_DTYPE[dtype]
    for call in range(2):  # two calls in a row: the shared array keeps the previous contents
        xs = np.concatenate([synth.rhs_uniform(90 + call, i, t.n).ravel() for i, t in enumerate(insts)])
        bs = np.concatenate([synth.rhs_uniform(95 + call, i, t.n).ravel() for i, t in enumerate(insts)])
        X = op.pack(torch.tensor(xs, dtype=td, device="cuda"), dtype)
        B = op.pack(torch.tensor(bs, dtype=td, device="cuda"), dtype)
        R = op.zeros(dtype)
        rn0, bn0, rel0 = op.residual_norm(dtype, X, B, r_out=R)
        rn1, bn1, rel1, R1 = _static(op, dtype, X, B)
        torch.cuda.synchronize()
        for u, v in ((rn0, rn1), (bn0, bn1), (rel0, rel1)):
            np.testing.assert_allclose(v.cpu().numpy(), u.cpu().numpy(), rtol=1e-14, atol=0)
        np.testing.assert_allclose(R1.cpu().numpy(), R.cpu().numpy(), rtol=1e-14, atol=0)


@pytest.mark.parametrize("dtype", [richm.C64, richm.C128])
def test_static_scratch_complex_helmholtz_matches_workspace_version_twice(dtype):
    # the complex branch: 5-point Helmholtz stencil with the absorbing boundary's diagonal
    from oracle.operators import helmholtz_wavenumber
    ns = (1, 17, 64, 100)
    op = richm.Operator([(richm.HELMHOLTZ_FD5_ABC, n, 1.0, 0.0, helmholtz_wavenumber(n)) for n in ns])
    td = richm.TORCH_DTYPE[dtype]
    for call in range(2):
        xs = np.concatenate([(synth.rhs_uniform(60 + call, i, n) + 1j * synth.rhs_uniform(70 + call, i, n)).ravel()
                             for i, n in enumerate(ns)])
        bs = np.concatenate([(synth.rhs_uniform(80 + call, i, n) - 0.5j * synth.rhs_uniform(85 + call, i, n)).ravel()
                             for i, n in enumerate(ns)])
        X = op.pack(torch.tensor(xs, dtype=td, device="cuda"), dtype)
        B = op.pack(torch.tensor(bs, dtype=td, device="cuda"), dtype)
        R = op.zeros(dtype)
        rn0, bn0, rel0 = op.residual_norm(dtype, X, B, r_out=R)
        rn1, bn1, rel1, R1 = _static(op, dtype, X, B)
        torch.cuda.synchronize()
        for u, v in ((rn0, rn1), (bn0, bn1), (rel0, rel1)):
            np.testing.assert_allclose(v.cpu().numpy(), u.cpu().numpy(), rtol=1e-14, atol=0)
        np.testing.assert_allclose(R1.cpu().numpy(), R.cpu().numpy(), rtol=1e-14, atol=0)


def test_static_scratch_many_instances():
    # 3000 instances: the tile offsets come from a block-wide scan in which every thread
    # sums a run of three consecutive instances
    ns = [1 + (i * 7) % 40 for i in range(3000)]
    op = richm.Operator([(richm.ANISO_Q1, n, 0.1 + 0.0003 * i, 0.001 * i, 0.0) for i, n in enumerate(ns)])
    xs = np.concatenate([synth.rhs_uniform(40, i, n).ravel() for i, n in enumerate(ns)])
    bs = np.concatenate([synth.rhs_uniform(41, i, n).ravel() for i, n in enumerate(ns)])
    X = op.pack(torch.tensor(xs, dtype=torch.float64, device="cuda"), richm.F64)
    B = op.pack(torch.tensor(bs, dtype=torch.float64, device="cuda"), richm.F64)
    rn0, bn0, rel0 = op.residual_norm(richm.F64, X, B)
    for _ in range(2):
        rn1, bn1, rel1, _r = _static(op, richm.F64, X, B)
        torch.cuda.synchronize()
        for u, v in ((rn0, rn1), (bn0, bn1), (rel0, rel1)):
            np.testing.assert_allclose(v.cpu().numpy(), u.cpu().numpy(), rtol=1e-14, atol=0)


def test_static_scratch_rejects_batches_beyond_its_limit():
    # 32 instances of 2047^2 in FP64: 64-column tiles, 32 x 128 = 4096 warp tiles each,
    # 131072 in all, twice what the static scratch holds (65536)
    op = richm.Operator([(richm.ANISO_Q1, 2047, 0.5, 0.3, 0.0)] * 32)
    lib = richm.load()
    fn = lib.richm_residual_norm_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 7
    x = torch.zeros(8, dtype=torch.float64, device="cuda")  # never touched: rejected first
    st = fn(op.handle, richm.F64, x.data_ptr(), x.data_ptr(), None, None, None, None, None)
    assert st == richm.ERR_NOMEM
    assert b"static scratch holds" in lib.richm_last_error()
