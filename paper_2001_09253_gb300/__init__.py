"""GB300 (sm_103a) cubic-spline fit + evaluation, after Hornbeck, arXiv 2001.09253.

The compute path is the CUDA library ``libspl.so`` (C ABI in ``include/spl.h``);
``spl`` is its ctypes binding and ``synth`` the seeded input generator.
"""
from . import synth  # noqa: F401
