"""GB300-native CSR SpMV by speculative segmented sum (Liu & Vinter).

The compute path is ``libssspmv.so`` (CUDA for sm_103a, C ABI declared in
``include/ssspmv.h``); ``ssspmv`` is its ctypes binding and ``api`` a small
torch-facing convenience layer (device allocations and streams only,
imported on demand: ``from paper_1504_06474_gb300 import api``).
"""
from . import ssspmv  # noqa: F401

__all__ = ["ssspmv", "api"]
