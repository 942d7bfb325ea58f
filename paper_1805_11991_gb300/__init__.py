"""GB300 point counting of hyperelliptic curves over small finite fields.

The computation lives in the CUDA library libhwc.so (C ABI in include/hwc.h);
``paper_1805_11991_gb300.hwc`` is its ctypes binding.
"""
from . import build, hwc  # noqa: F401

__all__ = ["build", "hwc"]
