"""GB300-native match-count top-k search (GENIE, arXiv 1603.08390).

The library proper is ``libgenie.so`` (CUDA, sm_103a) behind the C ABI in
``include/genie.h``; ``genie`` is its Python binding and ``runner`` drives it
from host or device arrays.  Build with ``paper_1603_08390_gb300._build.build()``.
"""
from . import genie  # noqa: F401

__all__ = ["genie"]
