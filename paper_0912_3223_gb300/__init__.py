"""GB300-native stochastic Lagrangian particle model (arXiv:0912.3223 method).

The compute path is the CUDA library ``liblpm.so`` (C ABI in include/lpm.h); ``lpm`` is
its Python binding. Build with ``paper_0912_3223_gb300.build.build()``.
"""
from . import lpm  # noqa: F401
from .lpm import Sim, LpmError  # noqa: F401

__all__ = ["lpm", "Sim", "LpmError"]
