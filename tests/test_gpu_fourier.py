"""GPU Fourier-domain correction (eqs. 19-20 with T = I) against the oracle."""
import numpy as np
import pytest

import richm_synth as synth
from gpu_util import from_dev, make_op, to_dev
from oracle.fourier import fourier_correction
from oracle.operators import assemble_q1
from paper_2412_08076_gb300 import richm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,batch", [(33, 3), (63, 2), (1, 1)])
def test_fourier_correction_matches_oracle(n, batch):
    import torch
    insts = [synth.AnisoInstance(1e-4, np.pi / 3, n)] * batch
    op = make_op(insts)
    A = assemble_q1(n, 1e-4, np.pi / 3)
    S = synth.fourier_symbol(n, seed=3)
    us = [(0.3 * synth.rhs_uniform(8, i, n)).astype(np.float32).astype(np.float64) for i in range(batch)]
    fs = [synth.rhs_uniform(9, i, n).astype(np.float32).astype(np.float64) for i in range(batch)]
    U, F = to_dev(op, us, richm.F32), to_dev(op, fs, richm.F32)
    St = torch.tensor(S.astype(np.complex64), device="cuda")
    op.fourier_correction(U, F, St)
    got = from_dev(op, U, richm.F32)
    S32 = S.astype(np.complex64).astype(np.complex128)
    for i in range(batch):
        ref = fourier_correction(A, fs[i].ravel(), us[i].ravel(), S32)
        assert np.linalg.norm(got[i].ravel() - ref) <= 1e-5 * np.linalg.norm(ref)
