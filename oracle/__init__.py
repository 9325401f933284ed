"""CPU oracle for the multi-resolution lattice Green's function (LGF) Poisson and heat-kernel path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is a plain, slow, FP64 restatement of the method of
Yu, Dorschner & Colonius (2020), written for checking by eye against the paper, and it shares no
code, header, table or constant with the CUDA library in ``paper_2010_13213_gb300``.

Contents
--------
``core``   the LGF table (Sec. 2.2), scaled Bessel functions, direct and FFT lattice convolutions,
           the discrete heat kernel (Sec. 2.3) and the 7-point Laplacian.
``amr``    the multi-level FLGF-AMR algorithm (Sec. 3.4, Eqs. (eq:combine_S)-(eq:FLGF-AMR)) and the
           FIF-AMR heat apply (Sec. 3.5, Eq. (eq:FIF-AMR)) on dense per-level boxes.
``refresh`` the velocity refresh u = -C^T L_E^{-1} omega (Sec. 4.1, Eq. (eq:vel_update)).
``refine`` the refinement indicator from the combined source (Sec. 4.2, Eqs. (eq:refine1)-(eq:refine2)).
``projection`` the HERK stage projection L p = D r, u = H (r - G p) (Sec. 2.4, Sec. 3.6).

Parity status (which functions are pinned by something other than themselves) is listed in the
module docstrings; every function here is pinned except where a docstring says "parity unpinned".
"""
from .core import *  # noqa: F401,F403
from . import amr  # noqa: F401
from . import projection  # noqa: F401
from . import refine  # noqa: F401
from . import refresh  # noqa: F401
