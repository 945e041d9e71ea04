"""tcgemm: tensor-core GEMM with low-precision inputs, precision refinement,
batched/grouped GEMM and a serving queue, for one NVIDIA GB300 (sm_103a).

The product is the C-ABI library built from ``csrc/`` (declared in
``include/tcgemm.h``); ``paper_1803_04014_gb300.binding`` is its ctypes
binding with the same names.  Importing ``binding`` loads the library and
fails if it cannot be built or loaded.
"""
from .builder import build  # noqa: F401

__all__ = ["build"]
