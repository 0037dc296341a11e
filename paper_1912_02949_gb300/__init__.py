"""GB300-native SketchyCGAL (Yurtsever et al., arXiv 1912.02949).

The solver is the CUDA library libscgal.so (sources in csrc/, C ABI in
include/scgal.h); ``scgal`` is its thin ctypes binding.  Build with
``python -m paper_1912_02949_gb300.build``.
"""
from . import scgal  # noqa: F401  (the shared library is loaded on first use)
