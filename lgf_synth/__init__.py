"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds data generation and data layout only -- none of the method's arithmetic.  The
vortex-ring vorticity follows the Gaussian-core ring used for the paper's ring experiments
(Sec. 6.2: ``omega_theta = Gamma / (pi sigma^2) exp(-s^2 / sigma^2)``, ``s^2 = z^2 + (r - R)^2``);
the manufactured streamfunction is the compact bump of Sec. 3.4's convergence test.  Everything is
seeded with ``numpy.random.default_rng``; arrays are C ordered ``[z][y][x]`` and the block layout
is ``[ncomp][nblocks][B][B][B]`` with block ``(bx, by, bz)`` holding cells ``B*(bx, by, bz) + [0, B)^3``.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "random_box", "ring_vorticity", "two_ring_vorticity", "bump_streamfunction",
    "box_blocks", "box_to_blocks", "blocks_to_box", "single_level_random", "single_level_ring",
    "three_level_ring", "two_ring_single_level", "batch_instances", "blocks_with_support", "ring_instance",
]


def random_box(shape, seed: int, ncomp: int = 1) -> np.ndarray:
    """i.i.d. N(0, 1) values on a [ncomp][nz][ny][nx] box."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((ncomp,) + tuple(shape))


def _centres(n: int, h: float, origin: float) -> np.ndarray:
    return origin + (np.arange(n) + 0.5) * h


def ring_vorticity(nx, ny, nz, h, R=1.0, sigma=0.2, gamma=1.0, origin=None, z0=0.0):
    """Cartesian vorticity [3][nz][ny][nx] of a Gaussian-core ring of radius R about the z axis.

    Cell centres are ``origin + (i + 1/2) h``; the default origin centres the box on the ring
    (``-n_i h / 2``).  ``omega = omega_theta * (-y/r, x/r, 0)`` and 0 on the axis.
    """
    if origin is None:
        origin = (-nx * h / 2, -ny * h / 2, -nz * h / 2)
    x = _centres(nx, h, origin[0])
    y = _centres(ny, h, origin[1])
    z = _centres(nz, h, origin[2])
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    r = np.sqrt(X * X + Y * Y)
    s2 = (Z - z0) ** 2 + (r - R) ** 2
    wt = gamma / (math.pi * sigma * sigma) * np.exp(-s2 / (sigma * sigma))
    with np.errstate(invalid="ignore", divide="ignore"):
        ex = np.where(r > 0, -Y / r, 0.0)
        ey = np.where(r > 0, X / r, 0.0)
    return np.stack([wt * ex, wt * ey, np.zeros_like(wt)])


def two_ring_vorticity(nx, ny, nz, h, R=1.0, sigma=0.15, sep=2.0):
    """Two coaxial Gaussian-core rings centred at z = +-sep/2 (same circulation sign)."""
    a = ring_vorticity(nx, ny, nz, h, R, sigma, z0=-sep / 2)
    b = ring_vorticity(nx, ny, nz, h, R, sigma, z0=+sep / 2)
    return a + b


def bump_streamfunction(nx, ny, nz, h, R=0.125, c1=1e3, c2=10.0, origin=None):
    """Manufactured streamfunction of the paper's AMR test (Sec. 3.4):
    ``Psi = f(sqrt((r - R)^2 + z^2) / R) e_theta``, ``f(t) = c1 exp(-c2 / (1 - t^2))`` for |t| < 1.
    Returns the Cartesian components [3][nz][ny][nx] sampled at cell centres (compact support)."""
    if origin is None:
        origin = (-nx * h / 2, -ny * h / 2, -nz * h / 2)
    x = _centres(nx, h, origin[0])
    y = _centres(ny, h, origin[1])
    z = _centres(nz, h, origin[2])
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    r = np.sqrt(X * X + Y * Y)
    t = np.sqrt((r - R) ** 2 + Z * Z) / R
    with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
        f = np.where(t < 1.0, c1 * np.exp(-c2 / np.maximum(1.0 - t * t, 1e-300)), 0.0)
        ex = np.where(r > 0, -Y / r, 0.0)
        ey = np.where(r > 0, X / r, 0.0)
    return np.stack([f * ex, f * ey, np.zeros_like(f)])


def _bump_fields(X, Y, Z, R, c1, c2):
    """The bump streamfunction Psi = f(t) e_theta, t = sqrt((r - R)^2 + z^2) / R, and its vector Laplacian
    at points (X, Y, Z), both as Cartesian components [3][...].  With f = c1 exp(-c2 / (1 - t^2)) for |t| < 1:
    f' = f h t, f'' = f ((h t)^2 + g), h = -2 c2 / (1 - t^2)^2, g = -2 c2 (1 + 3 t^2) / (1 - t^2)^3, and in
    cylindrical coordinates (Psi_theta = f) the vector Laplacian is
    d^2f/dr^2 + (1/r) df/dr + d^2f/dz^2 - f / r^2 = (f'' + f h) / R^2 + f h (r - R) / (r R^2) - f / r^2."""
    r = np.sqrt(X * X + Y * Y)
    t2 = ((r - R) ** 2 + Z * Z) / (R * R)
    inside = t2 < 1.0
    q = np.where(inside, 1.0 - t2, 1.0)
    with np.errstate(divide="ignore", over="ignore", invalid="ignore", under="ignore"):
        f = np.where(inside, c1 * np.exp(-c2 / q), 0.0)
        h = -2.0 * c2 / q ** 2
        g = -2.0 * c2 * (1.0 + 3.0 * t2) / q ** 3
        lap = (f * (h * h * t2 + g) + f * h) / R ** 2 + np.where(r > 0, f * h * (r - R) / (r * R * R) - f / r ** 2,
                                                                 0.0)
        lap = np.where(inside, lap, 0.0)
        ex = np.where(r > 0, -Y / r, 0.0)
        ey = np.where(r > 0, X / r, 0.0)
    zero = np.zeros_like(f)
    return np.stack([f * ex, f * ey, zero]), np.stack([lap * ex, lap * ey, zero])


def bump_case(refinements, B=16, R=0.125, c1=1e3, c2=10.0, h0=None, alpha=1.0 / 6.0, n_ext=14):
    """The bump test of Sec. 3.4 on a composite mesh with `refinements` levels above the base (K =
    refinements + 1): level 0 covers the bump's support (r < 2R, |z| < R) at h0 (default R/8) dilated by
    one block; level k+1 holds the children of level-k blocks with a cell where |omega| >
    alpha^(refinements - k) max |omega| (the paper's criterion with L_R = refinements; taking children only
    keeps the levels nested).  omega = the vector Laplacian of Psi, both sampled at each level's cell
    centres.  Returns (mesh, omega_levels, psi_levels) with fields [3][nblk][B][B][B]."""
    if h0 is None:
        h0 = R / 8
    K = refinements + 1
    n0 = [int(math.ceil(4 * R / h0 / B)) * B + 2 * B] * 2 + [int(math.ceil(2 * R / h0 / B)) * B + 2 * B]
    origin = (-n0[0] * h0 / 2, -n0[1] * h0 / 2, -n0[2] * h0 / 2)

    def centres(blocks, k):
        h = h0 / 2 ** k
        loc = (np.arange(B) + 0.5) * h
        out = []
        for bx, by, bz in blocks:
            Z, Y, X = np.meshgrid(origin[2] + bz * B * h + loc, origin[1] + by * B * h + loc,
                                  origin[0] + bx * B * h + loc, indexing="ij")
            out.append((X, Y, Z))
        return out

    # max |omega| from a fine sample of the support
    xs = np.linspace(-2 * R, 2 * R, 401)
    zs = np.linspace(-R, R, 201)
    Zs, Xs = np.meshgrid(zs, xs, indexing="ij")
    wmax = float(np.abs(_bump_fields(Xs, np.zeros_like(Xs), Zs, R, c1, c2)[1][1]).max())
    levels = [box_blocks((n0[2], n0[1], n0[0]), B)]
    kids = np.array([(i, j, l) for l in (0, 1) for j in (0, 1) for i in (0, 1)], np.int32)
    for k in range(1, K):
        cand = (2 * levels[k - 1][:, None, :] + kids[None]).reshape(-1, 3)
        thr = alpha ** (refinements - (k - 1)) * wmax
        keep = [b for b, (X, Y, Z) in zip(cand, centres(cand, k))
                if np.abs(_bump_fields(X, Y, Z, R, c1, c2)[1]).max() > thr]
        levels.append(np.array(sorted(map(tuple, keep)), np.int32).reshape(-1, 3))
    om, ps = [], []
    for k in range(K):
        o = np.zeros((3, len(levels[k]), B, B, B))
        p = np.zeros_like(o)
        for i, (X, Y, Z) in enumerate(centres(levels[k], k)):
            p[:, i], o[:, i] = _bump_fields(X, Y, Z, R, c1, c2)
        om.append(o)
        ps.append(p)
    mesh = dict(B=B, h0=h0, n_ext=n_ext, levels=[np.ascontiguousarray(b, dtype=np.int32) for b in levels])
    return mesh, om, ps


def box_blocks(shape, B: int) -> np.ndarray:
    """Block coordinates (bx, by, bz) tiling a [nz][ny][nx] box whose sides are multiples of B."""
    nz, ny, nx = shape
    assert nz % B == 0 and ny % B == 0 and nx % B == 0
    bz, by, bx = np.meshgrid(np.arange(nz // B), np.arange(ny // B), np.arange(nx // B), indexing="ij")
    return np.ascontiguousarray(np.stack([bx.ravel(), by.ravel(), bz.ravel()], 1), dtype=np.int32)


def box_to_blocks(box: np.ndarray, blocks: np.ndarray, B: int, origin=(0, 0, 0)) -> np.ndarray:
    """Gather a [ncomp][nz][ny][nx] box (cell (x,y,z) at box index (z,y,x) - origin) into blocks."""
    ncomp = box.shape[0]
    out = np.zeros((ncomp, len(blocks), B, B, B), dtype=box.dtype)
    for i, (bx, by, bz) in enumerate(blocks):
        x0, y0, z0 = B * bx - origin[0], B * by - origin[1], B * bz - origin[2]
        out[:, i] = box[:, z0:z0 + B, y0:y0 + B, x0:x0 + B]
    return out


def blocks_to_box(data: np.ndarray, blocks: np.ndarray, B: int, shape, origin=(0, 0, 0),
                  fill=0.0) -> np.ndarray:
    """Scatter [ncomp][nblk][B][B][B] block data into a [ncomp][nz][ny][nx] box."""
    ncomp = data.shape[0]
    out = np.full((ncomp,) + tuple(shape), fill, dtype=np.float64)
    for i, (bx, by, bz) in enumerate(blocks):
        x0, y0, z0 = B * bx - origin[0], B * by - origin[1], B * bz - origin[2]
        out[:, z0:z0 + B, y0:y0 + B, x0:x0 + B] = data[:, i]
    return out


def blocks_with_support(field: np.ndarray, B: int, rel: float) -> np.ndarray:
    """Blocks of a [ncomp][nz][ny][nx] box holding a cell with |field| >= rel * max |field|."""
    mag = np.sqrt((field ** 2).sum(0))
    thr = rel * mag.max()
    nz, ny, nx = mag.shape
    m = mag.reshape(nz // B, B, ny // B, B, nx // B, B).max(axis=(1, 3, 5)) >= thr
    bz, by, bx = np.nonzero(m)
    return np.ascontiguousarray(np.stack([bx, by, bz], 1), dtype=np.int32)


def single_level_random(n=32, B=16, seed=0, ncomp=1):
    """f ~ N(0, 1) on an n^3 box tiled by B^3 blocks, h = 1 (the 32^3, 8-block FP64 case)."""
    shape = (n, n, n)
    box = random_box(shape, seed, ncomp)
    blocks = box_blocks(shape, B)
    return dict(B=B, h=1.0, shape=shape, blocks=blocks, box=box, f=box_to_blocks(box, blocks, B))


def single_level_ring(nx=96, ny=96, nz=48, B=16, R=1.0, sigma=0.2, h=None, drop=1e-6):
    """Gaussian-core ring R = 1, sigma = 0.2 R, h = R/32 on a 96x96x48 box of 16^3 blocks; source
    blocks are those with max |omega| >= drop * max |omega|; targets are all blocks of the box."""
    if h is None:
        h = R / 32
    shape = (nz, ny, nx)
    box = ring_vorticity(nx, ny, nz, h, R, sigma)
    blocks = box_blocks(shape, B)
    src = blocks_with_support(box, B, drop)
    return dict(B=B, h=h, shape=shape, blocks=blocks, src_blocks=src, box=box,
                f=box_to_blocks(box, blocks, B))


def two_ring_single_level(nx=96, ny=96, nz=112, B=16, R=1.0, sigma=0.15, sep=2.0, h=None):
    """Two coaxial rings (separation 2R, sigma = 0.15 R) at h = R/32 on 96x96x112 cells."""
    if h is None:
        h = R / 32
    shape = (nz, ny, nx)
    box = two_ring_vorticity(nx, ny, nz, h, R, sigma, sep)
    blocks = box_blocks(shape, B)
    return dict(B=B, h=h, shape=shape, blocks=blocks, box=box, f=box_to_blocks(box, blocks, B))


def _level_blocks_over(field_fn, nxyz, h, origin, B, rel, vmax):
    """Blocks of a level grid (cells nxyz, spacing h, physical origin) holding |omega| > rel*vmax."""
    nx, ny, nz = nxyz
    box = field_fn(nx, ny, nz, h, origin)
    mag = np.sqrt((box ** 2).sum(0))
    m = mag.reshape(nz // B, B, ny // B, B, nx // B, B).max(axis=(1, 3, 5)) > rel * vmax
    bz, by, bx = np.nonzero(m)
    return np.stack([bx, by, bz], 1).astype(np.int32)


def three_level_ring(R=1.0, sigma=0.2, B=16, thresholds=(1e-3, 1e-2), n_ext=16, h_fine=None,
                     support=(48, 48, 32), dilate0=1, ring_fn=None):
    """Three-level composite mesh of the Gaussian-core ring (refinement ratio 2, B^3 blocks).

    Level 0 (h0 = 4 h_fine) covers the support box (``support`` level-0 cells, rounded up to blocks)
    dilated by ``dilate0`` blocks; level 1 holds the blocks with |omega| > thresholds[0] max plus the
    parents of level-2 blocks; level 2 holds the blocks with |omega| > thresholds[1] max.  The field
    is sampled at each level's own cell centres.  Returns mesh + per-level block data.
    """
    if h_fine is None:
        h_fine = R / 64
    if ring_fn is None:
        def ring_fn(nx, ny, nz, h, origin):
            return ring_vorticity(nx, ny, nz, h, R, sigma, origin=origin)
    nlev = 3
    hs = [h_fine * 2 ** (nlev - 1 - k) for k in range(nlev)]
    sx, sy, sz = (int(math.ceil(s / B)) * B for s in support)
    # level-0 grid: support box centred on the ring, dilated by whole blocks
    n0 = (sx + 2 * dilate0 * B, sy + 2 * dilate0 * B, sz + 2 * dilate0 * B)
    origin = (-n0[0] * hs[0] / 2, -n0[1] * hs[0] / 2, -n0[2] * hs[0] / 2)
    n_lev = [tuple(n * 2 ** k for n in n0) for k in range(nlev)]
    vmax = np.sqrt((ring_fn(*n_lev[2], hs[2], origin) ** 2).sum(0)).max()
    blocks = [box_blocks((n0[2], n0[1], n0[0]), B)]
    lvl2 = _level_blocks_over(ring_fn, n_lev[2], hs[2], origin, B, thresholds[1], vmax)
    lvl1 = _level_blocks_over(ring_fn, n_lev[1], hs[1], origin, B, thresholds[0], vmax)
    parents = np.unique((lvl2 * B // 2) // B, axis=0)
    lvl1 = np.unique(np.concatenate([lvl1, parents]), axis=0).astype(np.int32)
    blocks += [lvl1, lvl2]
    f = []
    for k in range(nlev):
        nx, ny, nz = n_lev[k]
        box = ring_fn(nx, ny, nz, hs[k], origin)
        f.append(box_to_blocks(box, blocks[k], B))
    mesh = dict(B=B, h0=hs[0], n_ext=n_ext, levels=[np.ascontiguousarray(b) for b in blocks])
    return mesh, f


def _ring_s2_blockmin(nxyz, h, origin, B, R):
    """Per block of a level grid: min over its cell centres of s^2 = z^2 + (r - R)^2 (ring about z)."""
    nx, ny, nz = nxyz
    x = _centres(nx, h, origin[0])
    y = _centres(ny, h, origin[1])
    z = _centres(nz, h, origin[2])
    r = np.sqrt(x[None, :] ** 2 + y[:, None] ** 2)                      # [ny][nx]
    d2 = ((r - R) ** 2).reshape(ny // B, B, nx // B, B).min(axis=(1, 3))  # [by][bx]
    z2 = (z ** 2).reshape(nz // B, B).min(axis=1)                        # [bz]
    return z2[:, None, None] + d2[None, :, :]                            # [bz][by][bx]


def _ring_on_blocks(blocks, B, h, origin, R, sigma, gamma=1.0):
    """Gaussian-core ring vorticity sampled at the cells of the given blocks: [3][nblk][B][B][B]."""
    blocks = np.asarray(blocks)
    loc = (np.arange(B) + 0.5) * h
    out = np.zeros((3, len(blocks), B, B, B))
    for i, (bx, by, bz) in enumerate(blocks):
        x = origin[0] + bx * B * h + loc
        y = origin[1] + by * B * h + loc
        z = origin[2] + bz * B * h + loc
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        r = np.sqrt(X * X + Y * Y)
        wt = gamma / (math.pi * sigma * sigma) * np.exp(-(Z * Z + (r - R) ** 2) / (sigma * sigma))
        with np.errstate(invalid="ignore", divide="ignore"):
            out[0, i] = np.where(r > 0, -wt * Y / r, 0.0)
            out[1, i] = np.where(r > 0, wt * X / r, 0.0)
    return out


def ring_instance(p, B=16, n_ext=16, thresholds=(1e-3, 1e-2), drop=1e-6):
    """Composite mesh of one batch instance (dict from ``batch_instances``): K = p["levels"] levels,
    finest spacing p["h_fine"], finest box p["nxy"]^2 x p["nz"] cells centred on the ring.  Level 0 covers
    the box at its own spacing (rounded up to blocks) dilated by one block (K > 1); for K = 3 level 1
    holds the blocks with a cell where |omega| > thresholds[0] max plus the parents of level 2; the
    finest level (K >= 2) the blocks with |omega| > thresholds[1] max; for K = 1 the single level is the
    box, with source blocks those reaching drop * max.  max|omega| is the analytic peak Gamma/(pi sigma^2),
    so |omega| > rel max is the cell-centre test s^2 < -sigma^2 ln(rel).  Returns (mesh, f_levels, roles)."""
    K, R, sig = p["levels"], p["R"], p["sigma"]
    hf = p["h_fine"]
    hs = [hf * 2 ** (K - 1 - k) for k in range(K)]
    fine_n = (p["nxy"], p["nxy"], p["nz"])
    scale = 2 ** (K - 1)
    n0 = tuple(int(math.ceil(n / scale / B)) * B + (2 * B if K > 1 else 0) for n in fine_n)
    origin = (-n0[0] * hs[0] / 2, -n0[1] * hs[0] / 2, -n0[2] * hs[0] / 2)
    n_lev = [tuple(n * 2 ** k for n in n0) for k in range(K)]

    def above(k, rel):
        m = _ring_s2_blockmin(n_lev[k], hs[k], origin, B, R) < -sig * sig * math.log(rel)
        bz, by, bx = np.nonzero(m)
        return np.stack([bx, by, bz], 1).astype(np.int32)

    blocks = [box_blocks((n0[2], n0[1], n0[0]), B)]
    roles = None
    if K == 1:
        src = {tuple(b) for b in above(0, drop)}
        roles = np.array([2 + (1 if tuple(b) in src else 0) for b in blocks[0]], np.uint8)
    if K >= 2:
        fine = above(K - 1, thresholds[1])
        mid = []
        if K == 3:
            parents = np.unique((fine * B // 2) // B, axis=0)
            mid = [np.unique(np.concatenate([above(1, thresholds[0]), parents]), axis=0).astype(np.int32)]
        blocks += mid + [fine]
    f = [_ring_on_blocks(blocks[k], B, hs[k], origin, R, sig) for k in range(K)]
    mesh = dict(B=B, h0=hs[0], n_ext=n_ext, levels=[np.ascontiguousarray(b, dtype=np.int32) for b in blocks])
    return mesh, f, roles


def batch_instances(n=64, seed0=1000, B=16):
    """Uneven batch of ring problems: instance i draws R ~ U[0.5, 1.5], sigma/R ~ U[0.1, 0.25],
    levels ~ U{1, 2, 3}, finest box edge n_xy ~ U{32, 48, ..., 192}, n_z = max(32, 16 ceil(n_xy/32)),
    h_fine = (2R + 8 sigma)/n_xy, from ``default_rng(seed0 + i)``.  Returns a list of parameter dicts."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed0 + i)
        R = float(rng.uniform(0.5, 1.5))
        sig = float(rng.uniform(0.1, 0.25)) * R
        nlev = int(rng.integers(1, 4))
        nxy = int(rng.choice(np.arange(32, 193, 16)))
        nz = max(32, 16 * int(math.ceil(nxy / 32)))
        h_fine = (2 * R + 8 * sig) / nxy
        out.append(dict(R=R, sigma=sig, levels=nlev, nxy=nxy, nz=nz, h_fine=h_fine, B=B))
    return out
