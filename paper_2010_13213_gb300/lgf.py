"""ctypes binding of ``liblgf.so`` (include/lgf.h): argument marshalling only.

Every function keeps the C name.  Device buffers are passed as integer addresses (for instance
``torch.Tensor.data_ptr()``) and streams as integer handles (``torch.cuda.Stream.cuda_stream``, 0 for
the legacy default stream).  A non-zero status raises :class:`LgfError` carrying ``lgf_last_error()``.
The library must have been built (``paper_2010_13213_gb300.build``); a missing library raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_uint8, c_uint32, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblgf.so")

LGF_OK = 0
LGF_E_INVALID_ARG = -1
LGF_E_MESH = -2
LGF_E_TABLE_RANGE = -3
LGF_E_OOM = -4
LGF_E_CUDA = -5
LGF_E_TIMEOUT = -6
LGF_E_PRECISION = -7
LGF_E_UNSUPPORTED = -8
LGF_F64, LGF_F32 = 0, 1
LGF_PREC_FP64, LGF_PREC_FP32, LGF_PREC_DF32 = 0, 1, 2
LGF_MAC_AUTO, LGF_MAC_PAIR, LGF_MAC_BOX = 0, 1, 2
LGF_TBL_FP64, LGF_TBL_FP32, LGF_TBL_DF32, LGF_TBL_BOX_ONLY = 1, 2, 4, 8
LGF_SOLVE_NO_CORRECTION = 1
PHASES = ("restrict", "correction", "forward", "mac", "inverse", "interp", "residual", "heat")


class LgfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lgf status {status}: {msg}")
        self.status = status


class lgf_mesh(ctypes.Structure):
    _fields_ = [("nlevels", c_int32), ("block", c_int32), ("h0", c_double),
                ("nblocks", POINTER(c_int32)), ("block_ijk", POINTER(c_int32)),
                ("block_role", POINTER(c_uint8)), ("n_ext", c_int32)]


class lgf_solve_opts(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("mac_mode", c_int32), ("residual", c_int32),
                ("timing", c_int32), ("residual_tol", c_double), ("dft_slices", c_int32), ("flags", c_int32)]


class lgf_report(ctypes.Structure):
    _fields_ = [("ms_total", c_double), ("ms_phase", c_double * 8), ("residual_rel", c_double),
                ("target_cells", c_int64), ("source_blocks", c_int64), ("target_blocks", c_int64),
                ("pairs", c_int64), ("scratch_bytes", c_int64), ("kernel_launches", c_int64),
                ("mac_mode_used", c_int32), ("reserved", c_int32), ("alg_bytes", c_int64), ("alg_flops", c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("ms_phase", "reserved")}
        d["ms_phase"] = {p: self.ms_phase[i] for i, p in enumerate(PHASES)}
        return d


class lgf_indicator(ctypes.Structure):
    _fields_ = [("alpha", c_double), ("beta", c_double), ("n_levels_max", c_int32), ("reserved", c_int32),
                ("rms_dev", c_void_p), ("flags_dev", c_void_p), ("s_max_dev", c_void_p)]


_LIB = None


def load():
    """Load the in-tree ``liblgf.so``; raise if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2010_13213_gb300.build`"
                               " (the CUDA path has no fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        lib.lgf_table_create.argtypes = [POINTER(c_void_p), c_int32, POINTER(c_int32), c_uint32, c_void_p]
        lib.lgf_table_destroy.argtypes = [c_void_p]
        lib.lgf_table_lgf_values.argtypes = [c_void_p, c_int32, POINTER(c_double)]
        lib.lgf_poisson_solve.argtypes = [c_void_p, POINTER(lgf_mesh), c_int32, c_void_p, c_void_p, c_int32,
                                          POINTER(lgf_solve_opts), POINTER(lgf_report), c_void_p]
        lib.lgf_heat_apply.argtypes = [c_void_p, POINTER(lgf_mesh), c_int32, c_void_p, c_void_p, c_int32,
                                       c_double, POINTER(lgf_solve_opts), POINTER(lgf_report), c_void_p]
        lib.lgf_poisson_solve_static.argtypes = [c_void_p, POINTER(lgf_mesh), c_int32, c_void_p, c_void_p,
                                                 c_int32, c_int32, c_void_p]
        lib.lgf_velocity_refresh.argtypes = [c_void_p, POINTER(lgf_mesh), c_void_p, c_void_p, c_int32,
                                             POINTER(lgf_solve_opts), POINTER(lgf_report), c_void_p]
        lib.lgf_table_prepare.argtypes = [c_void_p, POINTER(lgf_mesh), c_int32, c_int32, POINTER(lgf_solve_opts),
                                          c_void_p]
        lib.lgf_stage_projection.argtypes = [c_void_p, POINTER(lgf_mesh), c_void_p, c_void_p, c_void_p, c_int32,
                                             c_double, POINTER(lgf_solve_opts), POINTER(lgf_report), c_void_p]
        lib.lgf_refinement_indicator.argtypes = [c_void_p, POINTER(lgf_mesh), c_int32, c_void_p, c_void_p, c_int32,
                                                 POINTER(lgf_solve_opts), POINTER(lgf_indicator),
                                                 POINTER(lgf_report), c_void_p]
        PP = POINTER(c_void_p)
        lib.lgf_batch_create.argtypes = [POINTER(c_void_p), c_void_p, c_int32, POINTER(lgf_mesh), c_int32, c_int32,
                                         POINTER(c_double), POINTER(lgf_solve_opts), c_int32]
        lib.lgf_batch_destroy.argtypes = [c_void_p]
        lib.lgf_batch_stage.argtypes = [c_void_p, PP, PP, PP, POINTER(c_double), c_void_p]
        lib.lgf_batch_graph_create.argtypes = [c_void_p, c_int32, PP, PP, PP, PP, POINTER(c_double), c_void_p]
        lib.lgf_batch_graph_launch.argtypes = [c_void_p, c_void_p]
        lib.lgf_batch_graph_create_io.argtypes = [c_void_p, PP, PP, PP, PP, c_void_p]
        lib.lgf_batch_graph_nodes.argtypes = [c_void_p, POINTER(c_int64)]
        lib.lgf_batch_autotune.argtypes = [c_void_p, PP, PP, c_void_p]
        lib.lgf_batch_tuning.argtypes = [c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_double)]
        lib.lgf_device_status.argtypes = [c_void_p]
        lib.lgf_selftest_wait_timeout.argtypes = [c_void_p, c_int32, c_void_p]
        lib.lgf_last_error.restype = c_char_p
        lib.lgf_version.restype = c_char_p
        for name in ("lgf_table_create", "lgf_table_destroy", "lgf_table_lgf_values", "lgf_poisson_solve",
                     "lgf_heat_apply", "lgf_poisson_solve_static", "lgf_velocity_refresh",
                     "lgf_refinement_indicator", "lgf_stage_projection", "lgf_table_prepare", "lgf_batch_create",
                     "lgf_batch_destroy",
                     "lgf_batch_stage", "lgf_batch_graph_create", "lgf_batch_graph_launch", "lgf_batch_graph_nodes",
                     "lgf_batch_graph_create_io",
                     "lgf_batch_autotune", "lgf_batch_tuning",
                     "lgf_device_status", "lgf_selftest_wait_timeout"):
            getattr(lib, name).restype = c_int32
        _LIB = lib
    return _LIB


def _check(status: int):
    if status != LGF_OK:
        raise LgfError(status, lgf_last_error())


def lgf_last_error() -> str:
    return load().lgf_last_error().decode()


def lgf_version() -> str:
    return load().lgf_version().decode()


class Mesh:
    """Owns the host arrays behind an ``lgf_mesh`` (they must outlive the C call)."""

    def __init__(self, levels, block: int, h0: float, n_ext: int = 16, roles=None):
        self.levels = [np.ascontiguousarray(np.asarray(b, dtype=np.int32).reshape(-1, 3)) for b in levels]
        self.nb = np.array([len(b) for b in self.levels], dtype=np.int32)
        self.ijk = np.ascontiguousarray(np.concatenate(self.levels), dtype=np.int32)
        self.roles = None if roles is None else np.ascontiguousarray(roles, dtype=np.uint8)
        self.block, self.h0, self.n_ext = int(block), float(h0), int(n_ext)
        self.c = lgf_mesh(len(self.levels), self.block, self.h0,
                          self.nb.ctypes.data_as(POINTER(c_int32)), self.ijk.ctypes.data_as(POINTER(c_int32)),
                          None if self.roles is None else self.roles.ctypes.data_as(POINTER(c_uint8)),
                          self.n_ext)

    @property
    def total_blocks(self) -> int:
        return int(self.nb.sum())


def lgf_table_create(block: int, max_block_offset, flags: int = LGF_TBL_FP64, cuda_stream: int = 0):
    """Returns the opaque table handle (an int)."""
    h = c_void_p()
    mo = (c_int32 * 3)(*[int(v) for v in max_block_offset])
    _check(load().lgf_table_create(ctypes.byref(h), int(block), mo, int(flags), c_void_p(cuda_stream or None)))
    return h.value


def lgf_table_prepare(table, mesh: Mesh, ncomp: int, dtype: int = LGF_F64, opts: lgf_solve_opts | None = None,
                      cuda_stream: int = 0) -> None:
    _check(load().lgf_table_prepare(c_void_p(table), ctypes.byref(mesh.c), int(ncomp), int(dtype),
                                    ctypes.byref(opts) if opts is not None else None, c_void_p(cuda_stream or None)))


def lgf_table_destroy(table) -> None:
    _check(load().lgf_table_destroy(c_void_p(table)))


def lgf_table_lgf_values(table, n: int) -> np.ndarray:
    out = np.zeros((n + 1) ** 3)
    _check(load().lgf_table_lgf_values(c_void_p(table), int(n), out.ctypes.data_as(POINTER(c_double))))
    return out.reshape(n + 1, n + 1, n + 1)


def _opts(precision=LGF_PREC_FP64, mac_mode=LGF_MAC_AUTO, residual=0, timing=0, residual_tol=0.0, dft_slices=0,
          flags=0):
    return lgf_solve_opts(int(precision), int(mac_mode), int(residual), int(timing), float(residual_tol),
                          int(dft_slices), int(flags))


def lgf_device_status(table) -> None:
    """Synchronise and raise LgfError(LGF_E_TIMEOUT) if a bounded device wait gave up since the last read."""
    _check(load().lgf_device_status(c_void_p(table)))


def lgf_selftest_wait_timeout(table, log2_cycles: int = 24, cuda_stream: int = 0) -> None:
    _check(load().lgf_selftest_wait_timeout(c_void_p(table), int(log2_cycles), c_void_p(cuda_stream or None)))


def lgf_poisson_solve(table, mesh: Mesh, ncomp: int, f_dev: int, phi_dev: int, dtype: int = LGF_F64,
                      opts: lgf_solve_opts | None = None, report: lgf_report | None = None,
                      cuda_stream: int = 0) -> None:
    _check(load().lgf_poisson_solve(c_void_p(table), ctypes.byref(mesh.c), int(ncomp), c_void_p(f_dev),
                                    c_void_p(phi_dev), int(dtype),
                                    ctypes.byref(opts) if opts is not None else None,
                                    ctypes.byref(report) if report is not None else None,
                                    c_void_p(cuda_stream or None)))


def lgf_refinement_indicator(table, mesh: Mesh, ncomp: int, f_dev: int, phi_dev: int, dtype: int,
                             opts: lgf_solve_opts | None, alpha: float, beta: float, n_levels_max: int,
                             rms_dev: int, flags_dev: int, s_max_dev: int, report: lgf_report | None = None,
                             cuda_stream: int = 0) -> None:
    """Poisson solve plus the refinement indicator; rms_dev / flags_dev / s_max_dev are device addresses."""
    ind = lgf_indicator(float(alpha), float(beta), int(n_levels_max), 0, c_void_p(rms_dev), c_void_p(flags_dev),
                        c_void_p(s_max_dev))
    _check(load().lgf_refinement_indicator(c_void_p(table), ctypes.byref(mesh.c), int(ncomp), c_void_p(f_dev),
                                           c_void_p(phi_dev), int(dtype),
                                           ctypes.byref(opts) if opts is not None else None, ctypes.byref(ind),
                                           ctypes.byref(report) if report is not None else None,
                                           c_void_p(cuda_stream or None)))


def lgf_stage_projection(table, mesh: Mesh, r_dev: int, u_dev: int, p_dev: int, dtype: int, alpha_finest: float,
                         opts: lgf_solve_opts | None = None, report: lgf_report | None = None,
                         cuda_stream: int = 0) -> None:
    """L_C p = D r, u = H(r - G p) on the AMR grid; p_dev may be 0 (pressure not returned)."""
    _check(load().lgf_stage_projection(c_void_p(table), ctypes.byref(mesh.c), c_void_p(r_dev), c_void_p(u_dev),
                                       c_void_p(p_dev or None), int(dtype), float(alpha_finest),
                                       ctypes.byref(opts) if opts is not None else None,
                                       ctypes.byref(report) if report is not None else None,
                                       c_void_p(cuda_stream or None)))


def lgf_heat_apply(table, mesh: Mesh, ncomp: int, f_dev: int, g_dev: int, dtype: int, alpha_finest: float,
                   opts: lgf_solve_opts | None = None, report: lgf_report | None = None,
                   cuda_stream: int = 0) -> None:
    _check(load().lgf_heat_apply(c_void_p(table or None), ctypes.byref(mesh.c), int(ncomp), c_void_p(f_dev),
                                 c_void_p(g_dev), int(dtype), float(alpha_finest),
                                 ctypes.byref(opts) if opts is not None else None,
                                 ctypes.byref(report) if report is not None else None,
                                 c_void_p(cuda_stream or None)))


def lgf_velocity_refresh(table, mesh: Mesh, omega_dev: int, u_dev: int, dtype: int,
                         opts: lgf_solve_opts | None = None, report: lgf_report | None = None,
                         cuda_stream: int = 0) -> None:
    """u = -C^T L_E^{-1} omega on one level: omega on the positive edges, u on the positive faces, both
    [3][nblocks][B^3] device fields in dtype (Sec. 4.1, Eq. (eq:vel_update))."""
    _check(load().lgf_velocity_refresh(c_void_p(table), ctypes.byref(mesh.c), c_void_p(omega_dev), c_void_p(u_dev),
                                       int(dtype), ctypes.byref(opts) if opts is not None else None,
                                       ctypes.byref(report) if report is not None else None,
                                       c_void_p(cuda_stream or None)))


def lgf_poisson_solve_static(table, mesh: Mesh, ncomp: int, f_dev: int, phi_dev: int, dtype: int = LGF_F64,
                             precision: int = LGF_PREC_FP64, cuda_stream: int = 0) -> None:
    """Single-level solve whose scratch is the library's fixed 32 MiB device array (no allocation)."""
    _check(load().lgf_poisson_solve_static(c_void_p(table), ctypes.byref(mesh.c), int(ncomp), c_void_p(f_dev),
                                           c_void_p(phi_dev), int(dtype), int(precision),
                                           c_void_p(cuda_stream or None)))


def _ptrs(lst):
    arr = (c_void_p * len(lst))(*[c_void_p(int(p)) if p else None for p in lst])
    return ctypes.cast(arr, POINTER(c_void_p)), arr


class Batch:
    """Owns an ``lgf_batch`` and the host meshes behind it."""

    def __init__(self, table, meshes, ncomp: int, dtype: int = LGF_F64, alpha=None, opts=None, nstreams: int = 8):
        self.meshes = list(meshes)
        carr = (lgf_mesh * len(self.meshes))(*[m.c for m in self.meshes])
        al = None if alpha is None else (c_double * len(self.meshes))(*[float(a) for a in alpha])
        h = c_void_p()
        _check(load().lgf_batch_create(ctypes.byref(h), c_void_p(table), len(self.meshes), carr, int(ncomp),
                                       int(dtype), al, ctypes.byref(opts) if opts is not None else None,
                                       int(nstreams)))
        self.h = h.value

    def stage(self, f_ptrs, phi_ptrs, g_ptrs=None, cuda_stream: int = 0, alpha=None):
        """alpha: per-instance integrating-factor arguments of this stage (None: the create-time values)."""
        f, _a = _ptrs(f_ptrs)
        p, _b = _ptrs(phi_ptrs)
        g, _c = _ptrs(g_ptrs) if g_ptrs is not None else (None, None)
        al = None if alpha is None else (c_double * len(self.meshes))(*[float(a) for a in alpha])
        _check(load().lgf_batch_stage(c_void_p(self.h), f, p, g, al, c_void_p(cuda_stream or None)))

    def graph_create(self, nstages, f_ptrs, phi_ptrs, g_ptrs, tmp_ptrs, cuda_stream: int, alpha_stages=None):
        """g_ptrs None: Poisson-only stages.  alpha_stages: [nstages][ninst] values, or None."""
        f, _a = _ptrs(f_ptrs)
        p, _b = _ptrs(phi_ptrs)
        g, _c = _ptrs(g_ptrs) if g_ptrs is not None else (None, None)
        t, _d = _ptrs(tmp_ptrs) if tmp_ptrs is not None else (None, None)
        al = None
        if alpha_stages is not None:
            flat = [float(a) for row in alpha_stages for a in row]
            al = (c_double * len(flat))(*flat)
        _check(load().lgf_batch_graph_create(c_void_p(self.h), int(nstages), f, p, g, t, al, c_void_p(cuda_stream)))

    def graph_create_io(self, f_host_ptrs, phi_host_ptrs, f_ptrs, phi_ptrs, cuda_stream: int):
        """One Poisson stage with the pinned host transfers inside the graph."""
        fh, _a = _ptrs(f_host_ptrs)
        ph, _b = _ptrs(phi_host_ptrs)
        f, _c = _ptrs(f_ptrs)
        p, _d = _ptrs(phi_ptrs)
        _check(load().lgf_batch_graph_create_io(c_void_p(self.h), fh, ph, f, p, c_void_p(cuda_stream)))

    def autotune(self, f_ptrs, phi_ptrs, cuda_stream: int = 0):
        f, _a = _ptrs(f_ptrs)
        p, _b = _ptrs(phi_ptrs)
        _check(load().lgf_batch_autotune(c_void_p(self.h), f, p, c_void_p(cuda_stream or None)))

    def tuning(self):
        """(stream count, per-instance digit slices, per-instance measured solve ms)."""
        n = len(self.meshes)
        ns = c_int32()
        sl = (c_int32 * n)()
        ms = (c_double * n)()
        _check(load().lgf_batch_tuning(c_void_p(self.h), ctypes.byref(ns), sl, ms))
        return ns.value, list(sl), list(ms)

    def graph_launch(self, cuda_stream: int):
        _check(load().lgf_batch_graph_launch(c_void_p(self.h), c_void_p(cuda_stream)))

    def graph_nodes(self) -> int:
        n = c_int64()
        _check(load().lgf_batch_graph_nodes(c_void_p(self.h), ctypes.byref(n)))
        return n.value

    def close(self):
        if self.h:
            load().lgf_batch_destroy(c_void_p(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


make_opts = _opts
