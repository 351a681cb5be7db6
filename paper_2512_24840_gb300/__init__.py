"""GB300-native grouped stellar-spectrum fitting (LASP-Adam hot path, arXiv 2512.24840).

`lasp` is the Python binding of the CUDA C-ABI library liblasp.so
(include/lasp.h); `autograd` wraps its forward model and hand-written
adjoint in a torch.autograd.Function; `server` runs continuous batching of
fit requests over device-resident slot state.
"""
from . import _build  # noqa: F401

__all__ = ["lasp", "autograd", "server"]
