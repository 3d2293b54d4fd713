"""GB300 (sm_103a) Fast Local Regression (arXiv 2410.11625).

The compute path is ``libflr.so`` (hand-written CUDA, C ABI in ``include/flr.h``);
``paper_2410_11625_gb300.flr`` only marshals arguments to it through ctypes.  There is
no CPU fallback: if the library is missing or no GPU is present, calls raise.
"""
from ._build import build  # noqa: F401

__all__ = ["build", "flr"]
