"""GB300-native fractional finite element assembly (arXiv 1811.03339 hot path).

The compute path is the CUDA library ``libfem3`` (``csrc/``, C ABI in ``include/fem3.h``);
``fem3`` is its thin Python binding and ``inputs`` the seeded synthetic workloads.
"""
from . import fem3, inputs  # noqa: F401

__all__ = ["inputs", "fem3"]
