"""The C-ABI library builds, loads and exports every entry point the header declares.

No GPU is needed: only host-side entries (weights, counts, argument validation)
are called here.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


@pytest.fixture(scope="module")
def clib():
    from paper_2412_08076_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def _declared():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(richm_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["richm_operator_create", "richm_apply_sweeps", "richm_residual_norm", "richm_solve",
                     "richm_sweeps_adjoint", "richm_meta_forward", "richm_fourier_correction"]:
        assert required in names
    assert len(names) >= 30


def test_every_declared_symbol_is_exported(clib):
    missing = [n for n in _declared() if not hasattr(clib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2412_08076_gb300 import richm
    missing = [n for n in _declared() if n not in richm._SIGS]
    assert not missing, missing


def test_chebyshev_weights_match_oracle(clib):
    from oracle.iterations import chebyshev_weights
    f = clib.richm_chebyshev_weights
    f.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    for lmax, lmin, m in [(4.0, 0.01, 3), (3.19, 3.19 / 30, 8), (5.3, 1e-4, 16)]:
        out = (ctypes.c_double * m)()
        assert f(lmax, lmin, m, out) == 0
        np.testing.assert_allclose(list(out), chebyshev_weights(lmax, lmin, m), rtol=1e-15)
    out = (ctypes.c_double * 3)()
    assert f(1.0, 2.0, 3, out) == 1  # lmin > lmax
    assert f(1.0, 0.5, 0, out) == 1  # m = 0


def test_meta_param_count_and_version(clib):
    c = ctypes.c_int()
    clib.richm_meta_param_count.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    assert clib.richm_meta_param_count(16, 0, ctypes.byref(c)) == 0
    assert c.value == 2 * 64 + 64 + 64 * 64 + 64 + 17 * 64 + 17 == 5457
    base = 2 * 64 + 64 + 64 * 64 + 64
    for head, nout in ((1, 16), (2, 32), (3, 32), (4, 48), (5, 16)):
        assert clib.richm_meta_param_count(16, head, ctypes.byref(c)) == 0
        assert c.value == base + 65 * nout
    assert clib.richm_meta_param_count(0, 0, ctypes.byref(c)) == 1
    assert clib.richm_meta_param_count(22, 4, ctypes.byref(c)) == 1  # 66 outputs > 64
    assert clib.richm_meta_param_count(21, 4, ctypes.byref(c)) == 0
    assert clib.richm_meta_param_count(64, 5, ctypes.byref(c)) == 0  # raw head: m outputs
    assert clib.richm_meta_param_count(3, 6, ctypes.byref(c)) == 1   # unknown head
    clib.richm_version.restype = ctypes.c_char_p
    assert b"richm" in clib.richm_version()


def test_argument_errors_before_any_device_work(clib):
    from paper_2412_08076_gb300 import richm
    lib = richm.load()
    h = ctypes.c_void_p()
    arr = (richm.richm_pde * 1)(richm.richm_pde(0, 0, 0.5, 0.0, 0.0))
    assert lib.richm_operator_create(arr, 1, ctypes.byref(h)) == richm.ERR_ARG
    assert b"n = 0" in lib.richm_last_error()
    arr = (richm.richm_pde * 1)(richm.richm_pde(0, 10, 2.0, 0.0, 0.0))
    assert lib.richm_operator_create(arr, 1, ctypes.byref(h)) == richm.ERR_ARG
    arr = (richm.richm_pde * 1)(richm.richm_pde(7, 10, 0.5, 0.0, 0.0))
    assert lib.richm_operator_create(arr, 1, ctypes.byref(h)) == richm.ERR_ARG
    assert lib.richm_operator_create(arr, 0, ctypes.byref(h)) == richm.ERR_ARG
    assert h.value is None


def test_leja_order_matches_oracle_and_q1_stencil(clib):
    # host-only entries: the Leja permutation (bit-exact integers) and the Q1 stencil
    from oracle.iterations import chebyshev_weights, leja_order
    from oracle.operators import assemble_q1, gershgorin_max
    rng = np.random.default_rng(12)
    for m in (1, 3, 8, 16, 64):
        for w in (chebyshev_weights(3.0, 0.1, m), 1.0 / rng.uniform(0.05, 4.0, m),
                  rng.uniform(0.1, 1.0, m).astype(np.float32).astype(np.float64)):
            wa = (ctypes.c_double * m)(*w)
            perm = (ctypes.c_int * m)()
            assert clib.richm_leja_order(wa, m, perm) == 0
            assert list(perm) == list(leja_order(w))
    bad = (ctypes.c_double * 2)(1.0, 0.0)
    assert clib.richm_leja_order(bad, 2, (ctypes.c_int * 2)()) == 1
    clib.richm_q1_stencil.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    for eps, th in [(1e-2, math.pi / 6), (1.0, 0.0), (0.3, 2.2)]:
        q = (ctypes.c_double * 6)()
        assert clib.richm_q1_stencil(eps, th, q) == 0
        A = assemble_q1(5, eps, th).toarray()
        row = A[12].reshape(5, 5)  # interior unknown (2, 2): rows are y, columns x
        np.testing.assert_allclose([q[0], q[1], q[2], q[3], q[4]],
                                   [row[2, 2], row[2, 3], row[3, 2], row[3, 3], row[1, 3]], rtol=1e-13, atol=1e-15)
        assert abs(q[5] - gershgorin_max(assemble_q1(7, eps, th))) <= 1e-13 * q[5]
    assert clib.richm_q1_stencil(0.0, 0.0, (ctypes.c_double * 6)()) == 1
