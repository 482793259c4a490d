"""Layered-media Laplace FMM (arXiv 1908.10863) for one GB300 (sm_103a).

``LayeredFMM`` wraps the C ABI of ``include/lfmm.h``; all work runs in the
CUDA library built from ``csrc/``.
"""
from .lfmm import LayeredFMM, LayeredFMMBatch, LfmmError, gauss_laguerre, load  # noqa: F401
