"""Thin Python binding of librichm.so (the C ABI in include/richm.h).

Every function here marshals arguments and calls the library; no step of the
solver runs in Python. Tensors are PyTorch CUDA tensors (PyTorch supplies device
memory and the current stream); a missing or unbuilt library raises
``RichmError`` instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librichm.so")

# richm_status
OK, ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_NOT_CONVERGED, ERR_DIVERGED, ERR_UNSUPPORTED = range(7)
# richm_problem
ANISO_Q1, HELMHOLTZ_FD5_ABC, HELMHOLTZ_FD5_DIRICHLET, HELMHOLTZ_FD5_SPONGE = 0, 1, 2, 3
# richm_dtype
F64, F32, C64, C128, BF16 = 0, 1, 2, 3, 4
HEAD_NAG_SHARED, HEAD_RICHARDSON, HEAD_MOM, HEAD_NAG, HEAD_NAGEX, HEAD_RAW = 0, 1, 2, 3, 4, 5
HEAD_OUTPUTS = {HEAD_NAG_SHARED: lambda m: m + 1, HEAD_RICHARDSON: lambda m: m, HEAD_MOM: lambda m: 2 * m,
                HEAD_NAG: lambda m: 2 * m, HEAD_NAGEX: lambda m: 3 * m, HEAD_RAW: lambda m: m}

TORCH_DTYPE = {F64: torch.float64, F32: torch.float32, C64: torch.complex64, C128: torch.complex128,
               BF16: torch.bfloat16}
REAL_DTYPE = {F64: torch.float64, F32: torch.float32, C64: torch.float32, C128: torch.float64, BF16: torch.float32}
DTYPE_OF = {v: k for k, v in TORCH_DTYPE.items()}


class RichmError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


class richm_pde(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int), ("eps", C.c_double), ("theta", C.c_double), ("k", C.c_double)]


class richm_sweep_opts(C.Structure):
    _fields_ = [("m", C.c_int), ("k_start", C.c_int), ("precond", C.c_int), ("fuse", C.c_int),
                ("relax", C.c_double)]


class richm_solve_opts(C.Structure):
    _fields_ = [("m", C.c_int), ("tol", C.c_double), ("max_sweeps", C.c_longlong), ("refine_every", C.c_int),
                ("inner", C.c_int), ("precond", C.c_int), ("fuse", C.c_int), ("use_graph", C.c_int),
                ("relax", C.c_double), ("fp64_residual", C.c_int)]


class richm_solve_info(C.Structure):
    _fields_ = [("sweeps", C.c_longlong), ("rel_res", C.c_double), ("status", C.c_int)]


class richm_fgmres_opts(C.Structure):
    _fields_ = [("restart", C.c_int), ("tol", C.c_double), ("max_iters", C.c_int), ("m", C.c_int),
                ("sweeps", C.c_int), ("inner", C.c_int), ("precond", C.c_int), ("basis", C.c_int)]


class richm_fgmres_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_res", C.c_double), ("status", C.c_int)]


_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_SZ = C.c_size_t
_SIGS = {
    "richm_operator_create": (_I, [C.POINTER(richm_pde), _I, C.POINTER(_P)]),
    "richm_operator_destroy": (None, [_P]),
    "richm_operator_batch": (_I, [_P, C.POINTER(_I)]),
    "richm_stencil": (_I, [_P, _I, C.POINTER(_D)]),
    "richm_gershgorin": (_I, [_P, C.POINTER(_D)]),
    "richm_chebyshev_weights": (_I, [_D, _D, _I, C.POINTER(_D)]),
    "richm_q1_stencil": (_I, [_D, _D, C.POINTER(_D)]),
    "richm_fns_map_workspace": (_I, [C.POINTER(_SZ)]),
    "richm_symbol_from_stencil": (_I, [_I, C.POINTER(_D), _P, _P, _P]),
    "richm_symbol_from_stencil_vjp": (_I, [_I, C.POINTER(_D), _P, _P, _P, _P, _SZ, _P]),
    "richm_transition_from_band": (_I, [_I, _P, _P, _P]),
    "richm_transition_from_band_vjp": (_I, [_I, _P, _P, _P, _SZ, _P]),
    "richm_fourier_correction_t": (_I, [_P, _I, _P, _P, _P, _P, _P, _SZ, _P]),
    "richm_fourier_t_vjp_workspace": (_I, [_P, C.POINTER(_SZ)]),
    "richm_fourier_correction_t_vjp": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "richm_fgmres_workspace": (_I, [_P, C.POINTER(richm_fgmres_opts), C.POINTER(_SZ)]),
    "richm_fgmres": (_I, [_P, _P, _P, _P, _P, _P, C.POINTER(richm_fgmres_opts), C.POINTER(richm_fgmres_info), _P,
                          _SZ, _P]),
    "richm_leja_order": (_I, [C.POINTER(_D), _I, C.POINTER(_I)]),
    "richm_leja_permute": (_I, [_P, _I, _P, _P, _P, _I, _P, _P, _P, _P]),
    "richm_layout": (_I, [_P, _I, C.POINTER(_SZ), C.POINTER(_I), C.POINTER(_I)]),
    "richm_buffer_elems": (_I, [_P, C.POINTER(_SZ)]),
    "richm_pack": (_I, [_P, _I, _P, _P, _P]),
    "richm_unpack": (_I, [_P, _I, _P, _P, _P]),
    "richm_sweeps_workspace": (_I, [_P, _I, C.POINTER(_SZ)]),
    "richm_apply_sweeps": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _I, C.POINTER(richm_sweep_opts), _P, _SZ, _P]),
    "richm_residual_workspace": (_I, [_P, C.POINTER(_SZ)]),
    "richm_autotune_workspace": (_I, [_P, C.POINTER(_SZ)]),
    "richm_autotune": (_I, [_P, _I, _I, _P, _SZ, _P, C.POINTER(_I), C.POINTER(C.c_float)]),
    "richm_tuned": (_I, [_P, C.POINTER(_I), C.POINTER(_I)]),
    "richm_set_tuning": (_I, [_P, _I, _I]),
    "richm_residual_norm": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "richm_residual_norm_static": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P]),
    "richm_solve_workspace": (_I, [_P, C.POINTER(richm_solve_opts), C.POINTER(_SZ)]),
    "richm_solve": (_I, [_P, _P, _P, _P, _P, _P, C.POINTER(richm_solve_opts), C.POINTER(richm_solve_info), _P, _SZ,
                         _P]),
    "richm_solver_create": (_I, [_P, C.POINTER(richm_solve_opts), _P, _P, _P, _P, _SZ, C.POINTER(_P)]),
    "richm_solver_start": (_I, [_P, _P, _P, _P]),
    "richm_solver_start_zero": (_I, [_P, _P, _P, _P]),
    "richm_solve_host_workspace": (_I, [_P, C.POINTER(richm_solve_opts), C.POINTER(_SZ)]),
    "richm_solve_host": (_I, [_P, _P, _P, _P, _P, _P, C.POINTER(richm_solve_opts), C.POINTER(richm_solve_info), _P,
                              _SZ, _P]),
    "richm_solver_step": (_I, [_P, _I, C.POINTER(_I), _P]),
    "richm_solver_finish": (_I, [_P, C.POINTER(richm_solve_info), _P]),
    "richm_solver_state_bytes": (_I, [_P, C.POINTER(C.c_size_t)]),
    "richm_solver_save": (_I, [_P, _P, C.c_size_t, _P]),
    "richm_solver_resume": (_I, [_P, _P, _P, _P, C.c_size_t, _P]),
    "richm_solver_destroy": (None, [_P]),
    "richm_refine": (_I, [_P, _P, _P, _P, _P, _I, _P, _P, _P, _SZ, _P]),
    "richm_checkpoint_elems": (_I, [_P, _I, _I, C.POINTER(_SZ)]),
    "richm_forward_checkpointed": (_I, [_P, _I, _P, _P, _P, _P, _P, _I, _I, _I, _I, C.c_double, _P, _P, _P, _SZ,
                                        _P]),
    "richm_adjoint_workspace": (_I, [_P, _I, _I, C.POINTER(_SZ)]),
    "richm_loss_log_residual": (_I, [_P, _I, _P, _P, _P, _P, _P, _SZ, _P]),
    "richm_sweeps_adjoint": (_I, [_P, _I, _P, _I, _P, _P, _P, _P, _P, _I, _I, _I, C.c_double, _P, _P, _P, _P, _P,
                                  _SZ, _P]),
    "richm_meta_param_count": (_I, [_I, _I, C.POINTER(_I)]),
    "richm_meta_forward": (_I, [_P, _P, _P, _I, _I, _I, _P, _P, _P, _P, _P]),
    "richm_meta_backward": (_I, [_P, _P, _P, _P, _I, _I, _I, _P, _P, _P, _P, _P, _SZ, _P]),
    "richm_adam_step": (_I, [_P, _P, _P, _P, _I, _I, C.c_float, C.c_float, C.c_float, C.c_float, _P]),
    "richm_fourier_workspace": (_I, [_P, C.POINTER(_SZ)]),
    "richm_fourier_correction": (_I, [_P, _I, _P, _P, _P, _P, _SZ, _P]),
    "richm_fourier_vjp_workspace": (_I, [_P, C.POINTER(_SZ)]),
    "richm_fourier_correction_vjp": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "richm_selftest_conversions": (_I, [C.POINTER(C.c_longlong)]),
    "richm_fma_peak": (_I, [_I, C.POINTER(_D)]),
    "richm_last_error": (C.c_char_p, []),
    "richm_version": (C.c_char_p, []),
}

_lib = None


def load():
    """Load librichm.so (built by ``paper_2412_08076_gb300.build``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RichmError(-1, "load", f"{LIB_PATH} is missing: build it with "
                             "`python -m paper_2412_08076_gb300.build`")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int, where: str):
    if status != OK:
        raise RichmError(status, where, load().richm_last_error().decode())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream=None) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


def version() -> str:
    return load().richm_version().decode()


FMA_F32, FMA_F32X2, FMA_F64 = 0, 1, 2


def fma_peak(kind: int) -> float:
    """richm_fma_peak: measured FMA throughput in TFLOP/s (kind FMA_F32, FMA_F32X2 or FMA_F64)."""
    out = C.c_double()
    _check(load().richm_fma_peak(kind, C.byref(out)), "richm_fma_peak")
    return out.value


def selftest_conversions() -> tuple[int, int]:
    """richm_selftest_conversions: (widening, narrowing) mismatch counts against the
    hardware FP32 <-> FP64 conversions; (0, 0) when the integer-field versions agree."""
    out = (C.c_longlong * 2)()
    _check(load().richm_selftest_conversions(out), "richm_selftest_conversions")
    return int(out[0]), int(out[1])


def chebyshev_weights(lmax: float, lmin: float, m: int) -> list[float]:
    """richm_chebyshev_weights (eqs. 8-9), host."""
    out = (C.c_double * m)()
    _check(load().richm_chebyshev_weights(lmax, lmin, m, out), "richm_chebyshev_weights")
    return list(out)


def q1_stencil(eps: float, theta: float) -> list[float]:
    """richm_q1_stencil (Sec. 2.4), host: [centre, x-nbr, y-nbr, corner(+1,+1), corner(+1,-1), Gershgorin]."""
    out = (C.c_double * 6)()
    _check(load().richm_q1_stencil(eps, theta, out), "richm_q1_stencil")
    return list(out)


def leja_order(w) -> list[int]:
    """richm_leja_order, host: perm[s] = the step that runs at position s of the period."""
    m = len(w)
    wa = (C.c_double * m)(*[float(v) for v in w])
    out = (C.c_int * m)()
    _check(load().richm_leja_order(wa, m, out), "richm_leja_order")
    return list(out)


def _map_work():
    b = C.c_size_t()
    _check(load().richm_fns_map_workspace(C.byref(b)), "richm_fns_map_workspace")
    return torch.empty(b.value, dtype=torch.uint8, device="cuda")


def symbol_from_stencil(n: int, q, o, out=None, stream=None):
    """richm_symbol_from_stencil: the FNS symbol (complex64 [n][n]) from the base stencil q
    (6 values: the Q1 stencil and delta's base) and the network outputs o (FP32 [6] device)."""
    qa = (C.c_double * 6)(*[float(v) for v in q])
    if out is None:
        out = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    _check(load().richm_symbol_from_stencil(n, qa, _ptr(o), _ptr(out), _stream(stream)), "richm_symbol_from_stencil")
    return out


def symbol_from_stencil_vjp(n: int, q, o, dsymbol, d_o=None, stream=None):
    """richm_symbol_from_stencil_vjp: dL/do (FP32 [6] device) from dL/dS."""
    qa = (C.c_double * 6)(*[float(v) for v in q])
    if d_o is None:
        d_o = torch.empty(6, dtype=torch.float32, device="cuda")
    w = _map_work()
    _check(load().richm_symbol_from_stencil_vjp(n, qa, _ptr(o), _ptr(dsymbol), _ptr(d_o), _ptr(w), w.numel(),
                                                _stream(stream)), "richm_symbol_from_stencil_vjp")
    return d_o


def transition_from_band(n: int, tau, out=None, stream=None):
    """richm_transition_from_band: the transition field (FP32 [n][n]) of the band kernel tau (FP32 [9])."""
    if out is None:
        out = torch.empty((n, n), dtype=torch.float32, device="cuda")
    _check(load().richm_transition_from_band(n, _ptr(tau), _ptr(out), _stream(stream)), "richm_transition_from_band")
    return out


def transition_from_band_vjp(n: int, dtransition, dtau=None, stream=None):
    """richm_transition_from_band_vjp: dL/dtau (FP32 [9] device) from dL/dt."""
    if dtau is None:
        dtau = torch.empty(9, dtype=torch.float32, device="cuda")
    w = _map_work()
    _check(load().richm_transition_from_band_vjp(n, _ptr(dtransition), _ptr(dtau), _ptr(w), w.numel(),
                                                 _stream(stream)), "richm_transition_from_band_vjp")
    return dtau


def meta_param_count(m: int, head: int = HEAD_NAG_SHARED) -> int:
    c = C.c_int()
    _check(load().richm_meta_param_count(m, head, C.byref(c)), "richm_meta_param_count")
    return c.value


@dataclass
class Layout:
    offset: int
    pitch: int
    rows: int


class Operator:
    """Owner of a richm_operator handle plus marshalling helpers for its buffers."""

    def __init__(self, pdes):
        """pdes: list of (kind, n, eps, theta, k) tuples or richm_pde."""
        lib = load()
        arr = (richm_pde * len(pdes))()
        for i, p in enumerate(pdes):
            if isinstance(p, richm_pde):
                arr[i] = p
            else:
                kind, n, eps, theta, k = p
                arr[i] = richm_pde(int(kind), int(n), float(eps), float(theta), float(k))
        h = C.c_void_p()
        _check(lib.richm_operator_create(arr, len(pdes), C.byref(h)), "richm_operator_create")
        self.handle = h
        self.batch = len(pdes)
        self.ns = [int(arr[i].n) for i in range(len(pdes))]
        el = C.c_size_t()
        _check(lib.richm_buffer_elems(h, C.byref(el)), "richm_buffer_elems")
        self.elems = el.value
        self.layouts = [self.layout(i) for i in range(self.batch)]
        self._solve_ws = None  # workspace of solve / solve_host calls that pass none

    def _solve_workspace(self, nbytes: int) -> torch.Tensor:
        """A workspace kept for solve / solve_host calls without one (both synchronise
        before they return): the library keeps a one-call solve's session, graphs
        included, for the next call with the same workspace pointer."""
        if self._solve_ws is None or self._solve_ws.numel() < nbytes:
            self._solve_ws = None
            self._solve_ws = self.workspace(nbytes)
        return self._solve_ws

    def close(self):
        if getattr(self, "handle", None):
            load().richm_operator_destroy(self.handle)
            self.handle = None
        self._solve_ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- host queries
    def layout(self, i: int) -> Layout:
        off, pitch, rows = C.c_size_t(), C.c_int(), C.c_int()
        _check(load().richm_layout(self.handle, i, C.byref(off), C.byref(pitch), C.byref(rows)), "richm_layout")
        return Layout(off.value, pitch.value, rows.value)

    def stencil(self, i: int) -> list[float]:
        c = (C.c_double * 8)()
        _check(load().richm_stencil(self.handle, i, c), "richm_stencil")
        return list(c)

    def gershgorin(self) -> list[float]:
        out = (C.c_double * self.batch)()
        _check(load().richm_gershgorin(self.handle, out), "richm_gershgorin")
        return list(out)

    # -- buffers
    def zeros(self, dtype: int) -> torch.Tensor:
        """A zeroed padded buffer (caller-owned device memory from PyTorch)."""
        return torch.zeros(self.elems, dtype=TORCH_DTYPE[dtype], device="cuda")

    def dense_elems(self) -> int:
        return sum(n * n for n in self.ns)

    def pack(self, dense: torch.Tensor, dtype: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """richm_pack: dense concatenation (n_b*n_b each) -> padded buffer."""
        if out is None:
            out = torch.empty(self.elems, dtype=TORCH_DTYPE[dtype], device="cuda")
        _check(load().richm_pack(self.handle, dtype, _ptr(dense), _ptr(out), _stream(stream)), "richm_pack")
        return out

    def unpack(self, padded: torch.Tensor, dtype: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """richm_unpack: padded buffer -> dense concatenation."""
        if out is None:
            out = torch.empty(self.dense_elems(), dtype=TORCH_DTYPE[dtype], device="cuda")
        _check(load().richm_unpack(self.handle, dtype, _ptr(padded), _ptr(out), _stream(stream)), "richm_unpack")
        return out

    # -- workspaces
    def _ws(self, fn, *args) -> int:
        b = C.c_size_t()
        _check(getattr(load(), fn)(self.handle, *args, C.byref(b)), fn)
        return b.value

    def workspace(self, nbytes: int) -> torch.Tensor:
        return torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")

    # -- compute
    def apply_sweeps(self, dtype, x, x_prev, b, w, alpha=None, alpha_t=None, K=1, m=None, k_start=0, precond=0,
                     fuse=0, work=None, stream=None, relax=1.0):
        """richm_apply_sweeps (Table 1 iteration, eq. 17); x / x_prev updated in place.
        precond: 0 none, 1 Jacobi, 2 SSOR with relaxation factor `relax`."""
        m = m if m is not None else w.numel() // self.batch
        o = richm_sweep_opts(m, k_start, precond, fuse, relax)
        need = self._ws("richm_sweeps_workspace", dtype)
        if work is None:
            work = self.workspace(need)
        _check(load().richm_apply_sweeps(self.handle, dtype, _ptr(x), _ptr(x_prev), _ptr(b), _ptr(w), _ptr(alpha),
                                         _ptr(alpha_t), K, C.byref(o), _ptr(work), work.numel(), _stream(stream)),
               "richm_apply_sweeps")

    def fgmres(self, b, x, w=None, alpha=None, alpha_t=None, restart=20, tol=1e-6, max_iters=1000, m=None,
               sweeps=None, inner=C64, precond=0, work=None, stream=None, basis=C128):
        """richm_fgmres (Sec. 3.2, Table 9): b, x padded complex128 (x: guess in, solution
        out); the preconditioner is `sweeps` Table 1 sweeps with coefficients w, alpha,
        alpha_t ([batch][m], real type of `inner`); returns (status, [(iters, rel_res, status)])."""
        if m is None:
            m = w.numel() // self.batch if w is not None else 1
        if sweeps is None:
            sweeps = m if w is not None else 0
        o = richm_fgmres_opts(restart, tol, max_iters, m, sweeps, inner, precond, basis)
        need = C.c_size_t()
        _check(load().richm_fgmres_workspace(self.handle, C.byref(o), C.byref(need)), "richm_fgmres_workspace")
        if work is None:
            work = self.workspace(need.value)
        info = (richm_fgmres_info * self.batch)()
        st = load().richm_fgmres(self.handle, _ptr(b), _ptr(x), _ptr(w), _ptr(alpha), _ptr(alpha_t), C.byref(o), info,
                                 _ptr(work), work.numel(), _stream(stream))
        if st not in (OK, ERR_NOT_CONVERGED, ERR_DIVERGED):
            _check(st, "richm_fgmres")
        return st, [(info[i].iters, info[i].rel_res, info[i].status) for i in range(self.batch)]

    def leja_permute(self, dtype, w, alpha=None, alpha_t=None, stream=None):
        """richm_leja_permute: per-instance Leja reordering of the coefficient arrays
        [batch][m] (device); returns new tensors (w, alpha, alpha_t), None where not given."""
        m = w.numel() // self.batch
        outs = [None if t is None else torch.empty_like(t) for t in (w, alpha, alpha_t)]
        _check(load().richm_leja_permute(self.handle, dtype, _ptr(w), _ptr(alpha), _ptr(alpha_t), m, _ptr(outs[0]),
                                         _ptr(outs[1]), _ptr(outs[2]), _stream(stream)), "richm_leja_permute")
        return tuple(outs)

    def autotune(self, m=16, momentum=True, stream=None):
        """richm_autotune: pick sweeps per pass for FP32 sweeps; returns (fuse, ms per sweep)."""
        work = self.workspace(self._ws("richm_autotune_workspace"))
        best, ms = C.c_int(), C.c_float()
        _check(load().richm_autotune(self.handle, m, int(momentum), _ptr(work), work.numel(), _stream(stream),
                                     C.byref(best), C.byref(ms)), "richm_autotune")
        return best.value, ms.value

    def tuned(self):
        """richm_tuned: (sweeps per pass, fused tile rows) the operator uses."""
        f, r = C.c_int(), C.c_int()
        _check(load().richm_tuned(self.handle, C.byref(f), C.byref(r)), "richm_tuned")
        return f.value, r.value

    def set_tuning(self, fuse: int, rows: int):
        """richm_set_tuning: fix the pass length and the fused tile height."""
        _check(load().richm_set_tuning(self.handle, fuse, rows), "richm_set_tuning")

    def residual_norm(self, dtype, x, b, r_out=None, work=None, stream=None):
        """richm_residual_norm: returns (rnorm, bnorm, rel) as FP64 CUDA tensors [batch]."""
        rn = torch.empty(self.batch, dtype=torch.float64, device="cuda")
        bn = torch.empty_like(rn)
        rel = torch.empty_like(rn)
        if work is None:
            work = self.workspace(self._ws("richm_residual_workspace"))
        _check(load().richm_residual_norm(self.handle, dtype, _ptr(x), _ptr(b), _ptr(rn), _ptr(bn), _ptr(rel),
                                          _ptr(r_out), _ptr(work), work.numel(), _stream(stream)),
               "richm_residual_norm")
        return rn, bn, rel

    def refine(self, x, b, e, e_prev, inner, rhs_out, work=None, stream=None):
        """richm_refine: x += e, e_prev -= e, e = 0, rhs_out = b - A x; returns rel [batch]."""
        rel = torch.empty(self.batch, dtype=torch.float64, device="cuda")
        if work is None:
            work = self.workspace(self._ws("richm_residual_workspace"))
        _check(load().richm_refine(self.handle, _ptr(x), _ptr(b), _ptr(e), _ptr(e_prev), inner, _ptr(rhs_out),
                                   _ptr(rel), _ptr(work), work.numel(), _stream(stream)), "richm_refine")
        return rel

    def solve_opts(self, m, tol=1e-10, max_sweeps=10**7, refine_every=64, inner=F32, precond=0, fuse=0, use_graph=1,
                   relax=1.0, fp64_residual=0):
        return richm_solve_opts(m, tol, max_sweeps, refine_every, inner, precond, fuse, use_graph, relax,
                                fp64_residual)

    def solve(self, b, x, w, alpha=None, alpha_t=None, opts=None, work=None, stream=None):
        """richm_solve; returns (status, list of (sweeps, rel_res, status))."""
        need = C.c_size_t()
        _check(load().richm_solve_workspace(self.handle, C.byref(opts), C.byref(need)), "richm_solve_workspace")
        if work is None:
            work = self._solve_workspace(need.value)
        info = (richm_solve_info * self.batch)()
        st = load().richm_solve(self.handle, _ptr(b), _ptr(x), _ptr(w), _ptr(alpha), _ptr(alpha_t), C.byref(opts),
                                info, _ptr(work), work.numel(), _stream(stream))
        if st not in (OK, ERR_NOT_CONVERGED, ERR_DIVERGED):
            _check(st, "richm_solve")
        return st, [(info[i].sweeps, info[i].rel_res, info[i].status) for i in range(self.batch)]

    def solve_host(self, b_host, x_host, w, alpha=None, alpha_t=None, opts=None, work=None, stream=None):
        """richm_solve_host: b_host / x_host are CPU float64 tensors (dense concatenation;
        pinned for fast copies); returns (status, info)."""
        if b_host.is_cuda or x_host.is_cuda or b_host.dtype != torch.float64 or x_host.dtype != torch.float64:
            raise ValueError("b_host and x_host must be CPU float64 tensors")
        need = C.c_size_t()
        _check(load().richm_solve_host_workspace(self.handle, C.byref(opts), C.byref(need)),
               "richm_solve_host_workspace")
        if work is None:
            work = self._solve_workspace(need.value)
        info = (richm_solve_info * self.batch)()
        st = load().richm_solve_host(self.handle, b_host.data_ptr(), x_host.data_ptr(), _ptr(w), _ptr(alpha),
                                     _ptr(alpha_t), C.byref(opts), info, _ptr(work), work.numel(), _stream(stream))
        if st not in (OK, ERR_NOT_CONVERGED, ERR_DIVERGED):
            _check(st, "richm_solve_host")
        return st, [(info[i].sweeps, info[i].rel_res, info[i].status) for i in range(self.batch)]

    def loss_log_residual(self, dtype, x, b, g=None, work=None, stream=None):
        """richm_loss_log_residual: returns the loss (device FP64 scalar tensor); fills g."""
        loss = torch.empty(1, dtype=torch.float64, device="cuda")
        if work is None:
            work = self.workspace(self._ws("richm_adjoint_workspace", dtype, 1))
        _check(load().richm_loss_log_residual(self.handle, dtype, _ptr(x), _ptr(b), _ptr(loss), _ptr(g), _ptr(work),
                                              work.numel(), _stream(stream)), "richm_loss_log_residual")
        return loss

    def checkpoint_elems(self, K, every) -> int:
        e = C.c_size_t()
        _check(load().richm_checkpoint_elems(self.handle, K, every, C.byref(e)), "richm_checkpoint_elems")
        return e.value

    def forward_checkpointed(self, dtype, x0, b, w, alpha, alpha_t, m, K, every, precond, ckpts, xK, work=None,
                             stream=None, relax=1.0):
        """richm_forward_checkpointed (precond 2: SSOR with relaxation factor `relax`)."""
        if work is None:
            work = self.workspace(self._ws("richm_adjoint_workspace", dtype, every))
        _check(load().richm_forward_checkpointed(self.handle, dtype, _ptr(x0), _ptr(b), _ptr(w), _ptr(alpha),
                                                 _ptr(alpha_t), m, K, every, precond, float(relax), _ptr(ckpts),
                                                 _ptr(xK),
                                                 _ptr(work), work.numel(), _stream(stream)),
               "richm_forward_checkpointed")

    def sweeps_adjoint(self, dtype, ckpts, every, b, gK, w, alpha, alpha_t, m, K, precond, g_w=None, g_alpha=None,
                       g_alpha_t=None, g_x0=None, work=None, stream=None, relax=1.0):
        """richm_sweeps_adjoint (the same precond and relax as the forward)."""
        if work is None:
            work = self.workspace(self._ws("richm_adjoint_workspace", dtype, every))
        _check(load().richm_sweeps_adjoint(self.handle, dtype, _ptr(ckpts), every, _ptr(b), _ptr(gK), _ptr(w),
                                           _ptr(alpha), _ptr(alpha_t), m, K, precond, float(relax), _ptr(g_w),
                                           _ptr(g_alpha),
                                           _ptr(g_alpha_t), _ptr(g_x0), _ptr(work), work.numel(), _stream(stream)),
               "richm_sweeps_adjoint")

    def fourier_correction(self, x, b, symbol, work=None, stream=None, transition=None):
        """richm_fourier_correction(_t): x += t Re(IFFT2(S * FFT2(t (b - A x)))) (F32 state;
        transition t real [n][n], None for T = I)."""
        if work is None:
            work = self.workspace(self._ws("richm_fourier_workspace"))
        if transition is None:
            _check(load().richm_fourier_correction(self.handle, F32, _ptr(x), _ptr(b), _ptr(symbol), _ptr(work),
                                                   work.numel(), _stream(stream)), "richm_fourier_correction")
        else:
            _check(load().richm_fourier_correction_t(self.handle, F32, _ptr(x), _ptr(b), _ptr(symbol),
                                                     _ptr(transition), _ptr(work), work.numel(), _stream(stream)),
                   "richm_fourier_correction_t")

    def fourier_correction_t_vjp(self, x, b, g, symbol, transition, dsymbol=None, dtransition=None, g_x=None,
                                 work=None, stream=None):
        """richm_fourier_correction_t_vjp: dsymbol (complex64 [n][n]), dtransition (F32 [n][n]),
        g_x = g - A (t h) (padded F32; may be g itself); each output may be None."""
        if work is None:
            work = self.workspace(self._ws("richm_fourier_t_vjp_workspace"))
        _check(load().richm_fourier_correction_t_vjp(self.handle, F32, _ptr(x), _ptr(b), _ptr(g), _ptr(symbol),
                                                     _ptr(transition), _ptr(dsymbol), _ptr(dtransition), _ptr(g_x),
                                                     _ptr(work), work.numel(), _stream(stream)),
               "richm_fourier_correction_t_vjp")

    def fourier_correction_vjp(self, x, b, g, symbol, dsymbol=None, g_x=None, work=None, stream=None):
        """richm_fourier_correction_vjp: dsymbol = sum_b conj(R) G / n^2 (complex64 [n][n]),
        g_x = g - A Re(IFFT2(conj(S) * G)) (padded F32; may be g itself)."""
        if work is None:
            work = self.workspace(self._ws("richm_fourier_vjp_workspace"))
        _check(load().richm_fourier_correction_vjp(self.handle, F32, _ptr(x), _ptr(b), _ptr(g), _ptr(symbol),
                                                   _ptr(dsymbol), _ptr(g_x), _ptr(work), work.numel(),
                                                   _stream(stream)), "richm_fourier_correction_vjp")


class Solver:
    """richm_solver session (create / start / step / finish / destroy)."""

    def __init__(self, op: Operator, opts: richm_solve_opts, w, alpha=None, alpha_t=None, work=None):
        need = C.c_size_t()
        _check(load().richm_solve_workspace(op.handle, C.byref(opts), C.byref(need)), "richm_solve_workspace")
        self.work = work if work is not None else op.workspace(need.value)
        self.need = need.value
        self.opts = opts
        self.keep = (w, alpha, alpha_t)
        self.op = op
        h = C.c_void_p()
        _check(load().richm_solver_create(op.handle, C.byref(opts), _ptr(w), _ptr(alpha), _ptr(alpha_t),
                                          _ptr(self.work), self.work.numel(), C.byref(h)), "richm_solver_create")
        self.handle = h

    def views(self):
        """Views into the session's workspace (the layout richm_solve_workspace documents):
        (inner-state buffers [4], inner right-hand side, second FP64 solution buffer or None)."""
        o = self.opts
        el = self.op.elems
        es = {F64: 8, F32: 4, BF16: 2}[o.inner]
        E = (el * es + 255) // 256 * 256
        st = {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16}[o.inner]
        bufs = [self.work[j * E: j * E + el * es].view(st) for j in range(4)]
        rs = 8 if o.inner == F64 else 4
        rhs = self.work[4 * E: 4 * E + el * rs].view(torch.float64 if rs == 8 else torch.float32)
        x2 = None
        if o.inner != F64:
            X2 = (el * 8 + 255) // 256 * 256
            need = self.need
            x2 = self.work[need - X2: need - X2 + el * 8].view(torch.float64)
        return bufs, rhs, x2

    def start(self, b, x, stream=None, zero=False):
        self.bx = (b, x)
        fn = load().richm_solver_start_zero if zero else load().richm_solver_start
        _check(fn(self.handle, _ptr(b), _ptr(x), _stream(stream)), "richm_solver_start")

    def step(self, cycles: int, sync: bool = True, stream=None):
        act = C.c_int(-1)
        _check(load().richm_solver_step(self.handle, cycles, C.byref(act) if sync else None, _stream(stream)),
               "richm_solver_step")
        return act.value if sync else None

    def finish(self, stream=None):
        info = (richm_solve_info * self.op.batch)()
        st = load().richm_solver_finish(self.handle, info, _stream(stream))
        if st not in (OK, ERR_NOT_CONVERGED, ERR_DIVERGED):
            _check(st, "richm_solver_finish")
        return st, [(info[i].sweeps, info[i].rel_res, info[i].status) for i in range(self.op.batch)]

    def save(self, stream=None) -> bytes:
        """richm_solver_save: the session's image (between steps) as bytes."""
        n = C.c_size_t()
        _check(load().richm_solver_state_bytes(self.handle, C.byref(n)), "richm_solver_state_bytes")
        buf = (C.c_ubyte * n.value)()
        _check(load().richm_solver_save(self.handle, C.addressof(buf), n.value, _stream(stream)), "richm_solver_save")
        return bytes(buf)

    def resume(self, b, x, image: bytes, stream=None):
        """richm_solver_resume: bind b and x and restore a saved image."""
        self.bx = (b, x)
        buf = (C.c_ubyte * len(image)).from_buffer_copy(image)
        _check(load().richm_solver_resume(self.handle, _ptr(b), _ptr(x), C.addressof(buf), len(image),
                                          _stream(stream)), "richm_solver_resume")

    def close(self):
        if getattr(self, "handle", None):
            load().richm_solver_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- meta network

def meta_forward(params, inputs, G, m, acts=None, stream=None):
    """richm_meta_forward with the shared-momentum head: returns (w [B][m], alpha [B][m])
    FP32 CUDA tensors (the sweeps take at = alpha)."""
    w, a, _ = meta_forward_head(params, inputs, G, m, HEAD_NAG_SHARED, acts, stream)
    return w, a


def meta_forward_head(params, inputs, G, m, head, acts=None, stream=None):
    """richm_meta_forward with any head: returns (w, alpha, alpha_t), each [B][m] FP32 CUDA
    tensors or None, as the sweeps take them: alpha None for Richardson (no momentum),
    alpha_t None where at = alpha (NAG heads), zeros for MOM."""
    B = inputs.shape[0]
    w = torch.empty(B, m, dtype=torch.float32, device="cuda")
    a = None if head in (HEAD_RICHARDSON, HEAD_RAW) else torch.empty(B, m, dtype=torch.float32, device="cuda")
    at = torch.empty(B, m, dtype=torch.float32, device="cuda") if head in (HEAD_MOM, HEAD_NAGEX) else None
    _check(load().richm_meta_forward(_ptr(params), _ptr(inputs), _ptr(G), B, m, head, _ptr(w), _ptr(a), _ptr(at),
                                     _ptr(acts), _stream(stream)), "richm_meta_forward")
    return w, a, at


def meta_backward(params, inputs, G, acts, m, g_w, g_alpha, g_params=None, work=None, stream=None,
                  head=HEAD_NAG_SHARED, g_alpha_t=None):
    B = inputs.shape[0]
    cnt = meta_param_count(m, head)
    if g_params is None:
        g_params = torch.empty(cnt, dtype=torch.float32, device="cuda")
    if work is None:
        work = torch.empty(B * cnt * 4, dtype=torch.uint8, device="cuda")
    _check(load().richm_meta_backward(_ptr(params), _ptr(inputs), _ptr(G), _ptr(acts), B, m, head, _ptr(g_w),
                                      _ptr(g_alpha), _ptr(g_alpha_t), _ptr(g_params), _ptr(work), work.numel(),
                                      _stream(stream)),
           "richm_meta_backward")
    return g_params


def adam_step(params, grads, m1, m2, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().richm_adam_step(_ptr(params), _ptr(grads), _ptr(m1), _ptr(m2), params.numel(), t, lr, beta1, beta2,
                                  eps, _stream(stream)), "richm_adam_step")


def meta_acts_size(B: int, m: int, head: int = HEAD_NAG_SHARED) -> int:
    return B * (2 * 64 + HEAD_OUTPUTS[head](m))


def pack_mlp_params(layers) -> list[float]:
    """Flatten [(W1, b1), (W2, b2), (W3, b3)] (W[out][in]) into the library's order."""
    flat = []
    for W, b in layers:
        flat.extend(float(v) for v in W.reshape(-1))
        flat.extend(float(v) for v in b.reshape(-1))
    return flat
