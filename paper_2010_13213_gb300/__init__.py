"""GB300 (sm_103a) multi-resolution lattice Green's function library.

The compute path lives in ``csrc/`` (CUDA kernels + the C ABI of ``include/lgf.h``), built into
``_build/liblgf.so`` by :mod:`paper_2010_13213_gb300.build`; :mod:`paper_2010_13213_gb300.lgf` is the ctypes
binding with the C names.  There is no CPU fallback: without the built library every call raises.
"""
from . import lgf  # noqa: F401
from .lgf import *  # noqa: F401,F403
