"""Single-level oracle: LGF table, Bessel functions, convolutions, heat kernel, Laplacian.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper: Yu, Dorschner & Colonius, "Multi-resolution lattice Green's function method for
incompressible flows" (2020).

* Sec. 2.2, Eqs. (eq:discrete_laplace)-(eq:lgf_convolution): the free-space solution of the
  7-point problem ``L phi = f, phi -> 0`` is the lattice convolution ``phi = G * f`` with the LGF G.
  On a lattice of spacing h, ``L_h = h^-2 L_1`` so ``phi = h^2 (G * f)``.
* The LGF itself is taken from its Bessel-product integral
  ``G(n) = -int_0^inf prod_i e^{-2t} I_{n_i}(2t) dt`` (C code in ``lgf_oracle.c``).
* Sec. 2.3, Eqs. (eq:heat)-(eq:IF-single): the integrating factor is the exact solution operator of
  ``df/dt = L_1 f`` after a scaled time alpha; its kernel is ``E_alpha(n) = prod_i e^{-2 alpha}
  I_{|n_i|}(2 alpha)`` (the product of three 1D discrete heat kernels).

Pins (tests/test_oracle_pins.py): G(0) = -W/6 with Watson's W in closed form; L G = delta; the
far-field expansion; 30-digit values of G at small n (mpmath); the exact inverse
``h^2 G * (L_h g) = g`` for compactly supported g; brute force against mpmath sums; heat-kernel
mass, semigroup, ``dE/d alpha = L E``, ``E_0 = delta`` and ``-int E dt = G``.
"""
from __future__ import annotations

import ctypes
import functools
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblgforacle.so")
_SRC = os.path.join(_HERE, "lgf_oracle.c")

__all__ = [
    "build_oracle", "num_threads", "ive_all", "lgf_value", "lgf_octant", "lgf_offsets",
    "direct_conv", "fft_conv_box", "solve_box_direct", "solve_box_fft", "laplacian",
    "heat_weights_1d", "heat_kernel_full", "heat_box", "box_cells",
]


def build_oracle(force: bool = False) -> str:
    """Compile ``lgf_oracle.c`` into ``oracle/_build/liblgforacle.so`` (gcc, -O2, OpenMP, no contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
            "-o", tmp, _SRC, "-lm",
        ])
        os.replace(tmp, _SO)
    return _SO


@functools.lru_cache(maxsize=1)
def _lib():
    lib = ctypes.CDLL(build_oracle())
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    lib.oracle_ive_all.argtypes = [ctypes.c_double, ctypes.c_int, dp]
    lib.oracle_ive_all.restype = None
    lib.oracle_lgf_table.argtypes = [ctypes.c_int, dp]
    lib.oracle_lgf_table.restype = ctypes.c_int
    lib.oracle_lgf_value.argtypes = [ctypes.c_int] * 3
    lib.oracle_lgf_value.restype = ctypes.c_double
    lib.oracle_direct_conv.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, dp, ctypes.c_int, ip,
                                       ctypes.c_int, ctypes.c_double, dp]
    lib.oracle_direct_conv.restype = None
    lib.oracle_box_stencil_conv.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, dp]
    lib.oracle_box_stencil_conv.restype = None
    lib.oracle_num_threads.restype = ctypes.c_int
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def num_threads() -> int:
    """OpenMP threads the oracle's C loops use."""
    return int(_lib().oracle_num_threads())


def ive_all(x: float, kmax: int) -> np.ndarray:
    """``e^{-x} I_k(x)`` for k = 0..kmax (Miller backward recurrence, normalised by
    ``e^{-x}(I_0 + 2 sum_k I_k) = 1``)."""
    out = np.zeros(kmax + 1)
    _lib().oracle_ive_all(float(x), int(kmax), _dp(out))
    return out


def lgf_value(n1: int, n2: int, n3: int) -> float:
    """One value G(n) of the unit-lattice LGF (``L_1 G = delta``, Sec. 2.2)."""
    return float(_lib().oracle_lgf_value(int(n1), int(n2), int(n3)))


_TABLE: dict = {"nmax": -1, "G": None}


def lgf_octant(nmax: int) -> np.ndarray:
    """Dense first-octant table ``T[c, b, a] = G(a, b, c)`` for ``0 <= a, b, c <= nmax``.

    Cached: a request at or below the largest table computed so far is a slice of it.
    """
    if _TABLE["nmax"] < nmax:
        G = np.zeros((nmax + 1) ** 3)
        _lib().oracle_lgf_table(int(nmax), _dp(G))
        _TABLE["nmax"], _TABLE["G"] = nmax, G.reshape(nmax + 1, nmax + 1, nmax + 1)
    return _TABLE["G"][: nmax + 1, : nmax + 1, : nmax + 1]


def lgf_offsets(dz, dy, dx) -> np.ndarray:
    """G at integer offsets (arrays broadcast), through the octant table and |n| symmetry."""
    dz, dy, dx = (np.abs(np.asarray(v)) for v in (dz, dy, dx))
    nmax = int(max(dz.max(initial=0), dy.max(initial=0), dx.max(initial=0)))
    T = lgf_octant(nmax)
    return T[dz, dy, dx]


def box_cells(shape, origin=(0, 0, 0)) -> np.ndarray:
    """Integer (x, y, z) coordinates of every cell of a [nz][ny][nx] box, C order, as int32 [N, 3]."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xyz = np.stack([x.ravel() + origin[0], y.ravel() + origin[1], z.ravel() + origin[2]], axis=1)
    return np.ascontiguousarray(xyz, dtype=np.int32)


def direct_conv(kernel_octant: np.ndarray, src_xyz: np.ndarray, src_val: np.ndarray,
                tgt_xyz: np.ndarray, scale: float) -> np.ndarray:
    """Direct lattice convolution ``out[c, i] = scale * sum_j K(tgt_i - src_j) src_val[c, j]``
    (Eq. (eq:lgf_convolution) with K = G), Neumaier-compensated FP64, O(N_t N_s).

    ``kernel_octant[|dz|, |dy|, |dx|]`` must cover every offset for the LGF; for the heat kernel
    entries beyond its extent are zero.
    """
    K = np.ascontiguousarray(kernel_octant, dtype=np.float64)
    assert K.shape[0] == K.shape[1] == K.shape[2]
    src_xyz = np.ascontiguousarray(src_xyz, dtype=np.int32)
    tgt_xyz = np.ascontiguousarray(tgt_xyz, dtype=np.int32)
    val = np.ascontiguousarray(np.atleast_2d(src_val), dtype=np.float64)
    ncomp, nsrc = val.shape
    assert src_xyz.shape == (nsrc, 3)
    out = np.zeros((ncomp, tgt_xyz.shape[0]))
    _lib().oracle_direct_conv(_dp(K), K.shape[0], nsrc, _ip(src_xyz), _dp(val), tgt_xyz.shape[0],
                              _ip(tgt_xyz), ncomp, float(scale), _dp(out))
    return out


def solve_box_direct(f: np.ndarray, h: float, tgt_xyz: np.ndarray | None = None) -> np.ndarray:
    """Free-space solution ``phi = h^2 G * f`` of ``L_h phi = f`` (Sec. 2.2) by the direct sum.

    ``f`` is [ncomp][nz][ny][nx] (or [nz][ny][nx]) on a box at the lattice origin; the result is
    [ncomp][ntgt] at ``tgt_xyz`` (default: every cell of the box, C order).
    """
    f4 = f if f.ndim == 4 else f[None]
    shape = f4.shape[1:]
    src = box_cells(shape)
    if tgt_xyz is None:
        tgt_xyz = src
    dmax = 0
    for a, n in zip(range(3), shape[::-1]):  # (x, y, z) columns against nx, ny, nz
        if len(tgt_xyz):
            dmax = max(dmax, int(tgt_xyz[:, a].max()), int(n - 1 - tgt_xyz[:, a].min()))
    T = lgf_octant(max(dmax, 1))
    return direct_conv(T, src, f4.reshape(f4.shape[0], -1), tgt_xyz, h * h)


def _embed_kernel(T: np.ndarray, pshape) -> np.ndarray:
    """Circular embedding of G on a padded grid: K[i] = G(d) with d = i for i < P/2, i - P above.

    The middle slot i = P/2 (never reached by differences of two points of a box of size <= P/2)
    carries G(P/2) so that the embedded array stays even.
    """
    idx = [np.where(np.arange(p) <= p // 2, np.arange(p), p - np.arange(p)) for p in pshape]
    return T[np.ix_(idx[0], idx[1], idx[2])]


def fft_conv_box(K_full_embed: np.ndarray, src: np.ndarray, scale: float) -> np.ndarray:
    """Linear convolution on a box via the convolution theorem with 2x zero padding (FP64 pocketfft)."""
    pshape = K_full_embed.shape
    Fk = np.fft.rfftn(K_full_embed)
    s = src if src.ndim == 4 else src[None]
    out = np.empty(s.shape)
    nz, ny, nx = s.shape[1:]
    for c in range(s.shape[0]):
        Fs = np.fft.rfftn(s[c], s=pshape, axes=(0, 1, 2))
        full = np.fft.irfftn(Fs * Fk, s=pshape, axes=(0, 1, 2))
        out[c] = scale * full[:nz, :ny, :nx]
    return out if src.ndim == 4 else out[0]


def solve_box_fft(f: np.ndarray, h: float) -> np.ndarray:
    """``phi = h^2 G * f`` on the same box as ``f`` by a zero-padded FFT convolution (FP64).

    Same definition as ``solve_box_direct``; the FFT is a library primitive standing for the
    convolution sum (exact up to rounding because the padding 2n exceeds every difference).
    """
    shape = f.shape[-3:]
    pshape = tuple(2 * n for n in shape)
    T = lgf_octant(max(shape))
    K = _embed_kernel(T, pshape)
    return fft_conv_box(K, f, h * h)


def laplacian(phi: np.ndarray, h: float) -> np.ndarray:
    """7-point Laplacian ``L_h phi = h^-2 (sum_{+-e_i} phi(n +- e_i) - 6 phi(n))`` on the interior of a
    [.., nz, ny, nx] box (Sec. 2.1, ``L_C = -G^T G``); boundary cells are set to NaN."""
    out = np.full(phi.shape, np.nan)
    c = phi[..., 1:-1, 1:-1, 1:-1]
    s = (phi[..., 2:, 1:-1, 1:-1] + phi[..., :-2, 1:-1, 1:-1] + phi[..., 1:-1, 2:, 1:-1]
         + phi[..., 1:-1, :-2, 1:-1] + phi[..., 1:-1, 1:-1, 2:] + phi[..., 1:-1, 1:-1, :-2])
    out[..., 1:-1, 1:-1, 1:-1] = (s - 6.0 * c) / (h * h)
    return out


def heat_weights_1d(alpha: float, tol: float = 1e-18) -> np.ndarray:
    """1D discrete heat kernel ``w[n] = e^{-2 alpha} I_n(2 alpha)``, n = 0..r, with r the first order at
    which w drops below ``tol`` (Sec. 2.3: the IF kernel decays exponentially)."""
    kmax = 16
    while True:
        w = ive_all(2.0 * alpha, kmax)
        small = np.nonzero(w < tol)[0]
        if len(small):
            r = int(small[0]) - 1
            return w[: max(r, 0) + 1].copy()
        kmax *= 2


def heat_kernel_full(alpha: float, r: int | None = None) -> np.ndarray:
    """``E_alpha(d) = prod_i e^{-2 alpha} I_{|d_i|}(2 alpha)`` on [-r, r]^3 (Sec. 2.3, Eq. (eq:IF-single))."""
    w = heat_weights_1d(alpha)
    if r is None:
        r = len(w) - 1
    w1 = np.zeros(2 * r + 1)
    for d in range(-r, r + 1):
        if abs(d) < len(w):
            w1[d + r] = w[abs(d)]
    return w1[:, None, None] * w1[None, :, None] * w1[None, None, :], r


def heat_box(f: np.ndarray, alpha: float, r: int | None = None) -> np.ndarray:
    """``E_alpha * f`` on a dense box (sources outside the box are zero), 3D direct stencil sum."""
    K, r = heat_kernel_full(alpha, r)
    K = np.ascontiguousarray(K)
    f4 = f if f.ndim == 4 else f[None]
    out = np.empty(f4.shape)
    for c in range(f4.shape[0]):
        src = np.ascontiguousarray(f4[c], dtype=np.float64)
        o = np.empty_like(src)
        _lib().oracle_box_stencil_conv(_dp(K), r, _dp(src), *src.shape, _dp(o))
        out[c] = o
    return out if f.ndim == 4 else out[0]
