"""GB300-native Richardson(m) / NAG-Richardson(m) stencil solver.

The compute path is the CUDA library ``librichm.so`` (sources in ``csrc/``, C ABI
in ``include/richm.h``); ``richm`` is its thin ctypes binding, ``autograd`` wraps
the forward / adjoint sweep pair as a ``torch.autograd.Function`` and ``train``
drives meta-network training through the library's kernels.
Build with ``python -m paper_2412_08076_gb300.build``.
"""
__all__ = ["richm", "build"]
