"""Multi-level oracle: the FLGF-AMR Poisson solve and the FIF-AMR heat apply on dense level boxes.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper: Yu, Dorschner & Colonius (2020), Sec. 3.  The composite grid is a stack of unbounded
lattices with ``h_{k+1} = h_k / 2`` (Sec. 3.1); the AMR grid keeps level-k values on the region
Omega_k, and the Omega_k partition space (Eq. (eq:partition)).  Readings of the paper used here:

* Omega_k is every cell of a level-k block that no level-(k+1) block covers (blocks are nested).
* Coarsening P_{k+1->k} is the mean of the 8 children; interpolation P_{k-1->k} is cell-centred
  tensor-product linear (weights 3/4 on the parent, 1/4 on the parent's neighbour towards the
  child, per axis).  The paper leaves both open (Sec. 3.2, Eq. (eq:interp): order N_p unstated) and
  describes its own as simple second-order averaging.
* The extended correction region Omega_k^E (Eq. (eq:extended_regions)) uses the max-norm and whole
  cells: level-k cells within n_ext cells of Omega_k and not in Omega_k.
* The sums of Eqs. (eq:AMR-LGF-2)-(eq:combine_S) run over the levels that exist (0..N_l-1).

FLGF-AMR (Sec. 3.4, the three-step summary after Eq. (eq:AMR-LGF)):

1. fine to coarse: ``F_k = fhat_k + P_{k+1->k} F_{k+1}`` (cumulative coarsening);
2. coarse to fine: ``psi_0 = L_0^{-1} fhat_0``; for k >= 1
   ``c_k = P_{k-1->k} psi_{k-1}``,
   ``s_k = (P L_{k-1} - L_k P) psi_{k-1}`` kept on Omega_k and Omega_k^E (Eq. (eq:source_correct)),
   ``phi^k = c_k + L_k^{-1} (s_k + F_k)``  (Eq. (eq:combine_S)),
   ``psi_k = c_k + L_k^{-1} (s_k + fhat_k)``  (Eqs. (eq:partial_LGF)-(eq:Scorrection));
3. restriction: the output on level k is phi^k on Omega_k (Eq. (eq:FLGF-AMR)).

``L_k^{-1} = h_k^2 G *`` is evaluated with a zero-padded FFT convolution over each level's box
(a library primitive standing for the convolution sum of Sec. 2.2).

FIF-AMR (Sec. 3.5, Eq. (eq:FIF-AMR)): ``g_k = Gamma_k E_{alpha_k} * (P_k fhat)`` where ``P_k fhat`` is the
level-k reconstruction of the function the AMR data sample (Eq. (eq:interp): every region of the
partition supplies the cells it holds, ``reconstruct``) and ``alpha_k = alpha_finest 4^{-(K-1-k)}``
(Eq. (eq:composite-LGF-IF): the IF argument scales with 1/dx_k^2).  (In FLGF-AMR the coarse-to-fine
operator acts on the partial solution psi_{k-1}, a function defined on the whole level, and on the
sources only through the correction S, so its P is the plain interpolation of lattice functions.)

Parity: K = 1 reduces to the single-level solve (pinned in ``core``); ``s_k = 0`` for linear psi;
with n_ext -> infinity the result approaches the composite-grid definition
``phi^k = L_k^{-1} sum_i P_{i->k} fhat_i`` evaluated directly (tests/test_oracle_amr.py).  The
reconstruction reproduces linear functions exactly on every level (across level boundaries too);
FIF-AMR keeps constants on every Omega_k cell away from the grid's outer boundary, and reproduces the
lattice heat kernel's second moment ``E_a * |n|^2 = |n|^2 + 6a``: the same physical increment
``6 kappa dt`` on every level pins the ``4^{-(K-1-k)}`` scaling of alpha_k.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft

from . import core

__all__ = ["Level", "build_levels", "flgf_amr", "fif_amr", "composite_definition", "reconstruct", "interp_up",
           "coarsen", "dilate_maxnorm", "laplacian_box", "solve_level_box"]


class Level:
    """One level's dense box: origin (level-k cell index of box cell 0, as (x, y, z)) and shape
    [nz][ny][nx]; masks of the user blocks and of Omega_k; the level spacing h."""

    def __init__(self, k, origin, shape, h):
        self.k, self.origin, self.shape, self.h = k, tuple(int(v) for v in origin), tuple(shape), h
        self.user = np.zeros(shape, bool)
        self.omega = np.zeros(shape, bool)

    def block_slice(self, bijk, B):
        x0, y0, z0 = (B * int(bijk[a]) - self.origin[a] for a in range(3))
        return (slice(z0, z0 + B), slice(y0, y0 + B), slice(x0, x0 + B))


def build_levels(mesh, pad_extra: int = 0):
    """Dense boxes per level: the bounding box of the level's blocks grown by a margin that holds
    Omega_k^E, the interpolation/Laplacian halos and every coarse cell a finer level reads."""
    B, n_ext = mesh["B"], mesh.get("n_ext", 16)
    K = len(mesh["levels"])
    pads = [0] * K
    pads[K - 1] = n_ext + 8 + pad_extra
    for k in range(K - 2, -1, -1):
        pads[k] = max(n_ext + 8 + pad_extra, int(math.ceil(pads[k + 1] / 2)) + 6)
    levels = []
    for k in range(K):
        blk = np.asarray(mesh["levels"][k])
        lo = blk.min(0) * B - pads[k]
        hi = (blk.max(0) + 1) * B + pads[k]
        lo = lo - (lo % 2)  # even origins keep parent/child alignment simple to read
        hi = hi + (hi % 2)
        shape = (int(hi[2] - lo[2]), int(hi[1] - lo[1]), int(hi[0] - lo[0]))
        L = Level(k, lo, shape, mesh["h0"] / 2 ** k)
        for b in blk:
            L.user[L.block_slice(b, B)] = True
        levels.append(L)
    for k in range(K):
        levels[k].omega = levels[k].user.copy()
        if k + 1 < K:
            levels[k].omega &= ~coarsen_mask(levels[k + 1].user, levels[k + 1], levels[k])
    return levels


def _fine_window(fine_lv, coarse_lv):
    """Slices of a fine-resolution array aligned with the coarse box footprint."""
    off = [fine_lv.origin[a] - 2 * coarse_lv.origin[a] for a in range(3)]
    return off


def coarsen_mask(fmask, fine_lv, coarse_lv):
    """Level-k cells with any child inside the level-(k+1) mask."""
    cz, cy, cx = coarse_lv.shape
    big = np.zeros((2 * cz, 2 * cy, 2 * cx), bool)
    ox, oy, oz = _fine_window(fine_lv, coarse_lv)
    fz, fy, fx = fmask.shape
    big[oz:oz + fz, oy:oy + fy, ox:ox + fx] = fmask
    return big.reshape(cz, 2, cy, 2, cx, 2).any(axis=(1, 3, 5))


def coarsen(ffine, fine_lv, coarse_lv):
    """P_{k+1->k}: each coarse cell is the mean of its 8 children (children outside the fine box
    hold zero).  ``ffine`` is [ncomp][...] on the fine box; returns [ncomp][...] on the coarse box."""
    cz, cy, cx = coarse_lv.shape
    ox, oy, oz = _fine_window(fine_lv, coarse_lv)
    fz, fy, fx = fine_lv.shape
    assert ox >= 0 and oy >= 0 and oz >= 0 and oz + fz <= 2 * cz and oy + fy <= 2 * cy and ox + fx <= 2 * cx
    out = np.zeros((ffine.shape[0], cz, cy, cx))
    for c in range(ffine.shape[0]):
        big = np.zeros((2 * cz, 2 * cy, 2 * cx))
        big[oz:oz + fz, oy:oy + fy, ox:ox + fx] = ffine[c]
        out[c] = big.reshape(cz, 2, cy, 2, cx, 2).sum(axis=(1, 3, 5)) / 8.0
    return out


def interp_up(fcoarse, coarse_lv, fine_lv):
    """P_{k-1->k}: cell-centred tensor-product linear interpolation.  Fine cell g (global index per
    axis) has parent p = floor(g/2) and neighbour q = p - 1 (g even) or p + 1 (g odd); its value is
    sum over the 8 corners of prod_axis (3/4 if parent else 1/4) * coarse value.  Cells whose
    stencil leaves the coarse box are NaN."""
    idx, wts = [], []
    for a, n in zip(range(3), fine_lv.shape[::-1]):  # x, y, z
        g = fine_lv.origin[a] + np.arange(n)
        p = g // 2
        q = np.where(g % 2 == 0, p - 1, p + 1)
        idx.append((p - coarse_lv.origin[a], q - coarse_lv.origin[a]))
    nzc, nyc, nxc = coarse_lv.shape
    lim = (nxc, nyc, nzc)
    out = np.zeros((fcoarse.shape[0],) + fine_lv.shape)
    valid = np.ones(fine_lv.shape, bool)
    for sx, wx in ((0, 0.75), (1, 0.25)):
        for sy, wy in ((0, 0.75), (1, 0.25)):
            for sz, wz in ((0, 0.75), (1, 0.25)):
                ix, iy, iz = idx[0][sx], idx[1][sy], idx[2][sz]
                okx = (ix >= 0) & (ix < lim[0])
                oky = (iy >= 0) & (iy < lim[1])
                okz = (iz >= 0) & (iz < lim[2])
                ok = okz[:, None, None] & oky[None, :, None] & okx[None, None, :]
                valid &= ok
                cx_ = np.clip(ix, 0, lim[0] - 1)
                cy_ = np.clip(iy, 0, lim[1] - 1)
                cz_ = np.clip(iz, 0, lim[2] - 1)
                w = wx * wy * wz
                out += w * fcoarse[:, cz_[:, None, None], cy_[None, :, None], cx_[None, None, :]]
    out[:, ~valid] = np.nan
    return out


def dilate_maxnorm(mask, r):
    """Cells within max-norm distance r of the mask."""
    out = mask.copy()
    if r <= 0:
        return out
    for axis in range(3):
        m = out.copy()
        for s in range(1, r + 1):
            m |= np.roll(out, s, axis) & _shift_valid(out.shape, axis, s)
            m |= np.roll(out, -s, axis) & _shift_valid(out.shape, axis, -s)
        out = m
    return out


def _shift_valid(shape, axis, s):
    v = np.ones(shape, bool)
    sl = [slice(None)] * 3
    if s > 0:
        sl[axis] = slice(0, s)
    else:
        sl[axis] = slice(shape[axis] + s, shape[axis])
    v[tuple(sl)] = False
    return v


def laplacian_box(phi, h):
    """7-point Laplacian on a [ncomp][...] box (NaN on the box boundary)."""
    return core.laplacian(phi, h)


def solve_level_box(src, lv):
    """``L_k^{-1} src = h_k^2 G * src`` on the level box (zero-padded FFT convolution, FP64)."""
    shape = lv.shape
    pshape = tuple(2 * n for n in shape)
    T = core.lgf_octant(max(shape))
    K = core._embed_kernel(T, pshape)
    Fk = sfft.rfftn(K, workers=-1)
    out = np.empty(src.shape)
    nz, ny, nx = shape
    for c in range(src.shape[0]):
        Fs = sfft.rfftn(src[c], s=pshape, workers=-1)
        out[c] = (lv.h * lv.h) * sfft.irfftn(Fs * Fk, s=pshape, workers=-1)[:nz, :ny, :nx]
    return out


def _user_field(lv, blocks, data, B):
    """User block data [ncomp][nblk][B]^3 placed on the level box, zero off Omega_k."""
    out = np.zeros((data.shape[0],) + lv.shape)
    for i, b in enumerate(blocks):
        out[(slice(None),) + lv.block_slice(b, B)] = data[:, i]
    out[:, ~lv.omega] = 0.0
    return out


def _to_blocks(lv, blocks, box, B):
    out = np.zeros((box.shape[0], len(blocks), B, B, B))
    for i, b in enumerate(blocks):
        out[:, i] = box[(slice(None),) + lv.block_slice(b, B)]
    return out


def flgf_amr(mesh, f_levels, return_internals=False, correction=True):
    """FLGF-AMR solve (Sec. 3.4).  ``f_levels[k]`` is [ncomp][nblk_k][B]^3 user data of level k.

    Returns per level [ncomp][nblk_k][B]^3 arrays holding phi^k on Omega_k and 0 elsewhere, and the
    Omega_k masks in the same block layout.  ``correction=False`` drops the source correction
    (``s_k = 0``): the uncorrected composite solve ``phi^k = P psi_{k-1} + L_k^{-1} sum_i P_{i->k} fhat_i``
    that the bump test of Sec. 3.4 (Fig. fig:source_correction_convergence) compares against.
    """
    B, n_ext = mesh["B"], mesh.get("n_ext", 16)
    blocks = mesh["levels"]
    K = len(blocks)
    lv = build_levels(mesh)
    fhat = [_user_field(lv[k], blocks[k], f_levels[k], B) for k in range(K)]
    # Step 1: F_k = fhat_k + P_{k+1->k} F_{k+1}
    F = [None] * K
    F[K - 1] = fhat[K - 1]
    for k in range(K - 2, -1, -1):
        F[k] = fhat[k] + coarsen(F[k + 1], lv[k + 1], lv[k])
    # Step 2: coarse to fine
    phi, psi, internals = [None] * K, [None] * K, []
    psi[0] = solve_level_box(fhat[0], lv[0])
    phi[0] = solve_level_box(F[0], lv[0])
    for k in range(1, K):
        c = interp_up(psi[k - 1], lv[k - 1], lv[k])
        lap_coarse = laplacian_box(psi[k - 1], lv[k - 1].h)
        s = interp_up(lap_coarse, lv[k - 1], lv[k]) - laplacian_box(c, lv[k].h)
        ext = dilate_maxnorm(lv[k].omega, n_ext) & ~lv[k].omega
        region = lv[k].omega | ext
        assert np.all(np.isfinite(s[:, region])), "level box too small for the correction region"
        s = np.where(region[None], s, 0.0) if correction else np.zeros_like(c)
        A = s + fhat[k]
        phi[k] = c + solve_level_box(A + (F[k] - fhat[k]), lv[k])
        psi[k] = c + solve_level_box(A, lv[k])
        internals.append(dict(c=c, s=s, ext=ext))
    # Step 3: restriction to Omega_k
    out, masks = [], []
    for k in range(K):
        assert np.all(np.isfinite(phi[k][:, lv[k].omega]))
        p = np.where(lv[k].omega[None], phi[k], 0.0)
        out.append(_to_blocks(lv[k], blocks[k], p, B))
        masks.append(_to_blocks(lv[k], blocks[k], lv[k].omega[None].astype(float), B)[0] > 0.5)
    if return_internals:
        return out, masks, dict(levels=lv, phi=phi, psi=psi, F=F, fhat=fhat, steps=internals)
    return out, masks


def composite_definition(mesh, f_levels):
    """The composite-grid definition the algorithm approximates (Eqs. (eq:interp), (eq:AMR-LGF-2)):
    ``phi^k = L_k^{-1} sum_i P_{i->k} fhat_i`` with every P applied to the whole (compact) field,
    restricted to Omega_k.  Finite and directly computable on small cases."""
    B = mesh["B"]
    blocks = mesh["levels"]
    K = len(blocks)
    lv = build_levels(mesh, pad_extra=8)
    fhat = [_user_field(lv[k], blocks[k], f_levels[k], B) for k in range(K)]
    out = []
    for k in range(K):
        tot = fhat[k].copy()
        # coarser levels: interpolate up level by level (composition, Eq. (eq:P_composition))
        for i in range(k):
            u = fhat[i]
            for j in range(i + 1, k + 1):
                u = interp_up(u, lv[j - 1], lv[j])
                u = np.nan_to_num(u, nan=0.0)
            tot = tot + u
        # finer levels: coarsen level by level
        for i in range(k + 1, K):
            u = fhat[i]
            for j in range(i - 1, k - 1, -1):
                u = coarsen(u, lv[j + 1], lv[j])
            tot = tot + u
        phi = solve_level_box(tot, lv[k])
        p = np.where(lv[k].omega[None], phi, 0.0)
        out.append(_to_blocks(lv[k], blocks[k], p, B))
    return out


def reconstruct(lv, fhat):
    """P_k fhat on every level box (Sec. 3.2, Eq. (eq:interp)): the level-k information of the function the
    AMR data sample.  ``fhat[k]`` is [ncomp][box_k], zero off Omega_k.  The regions partition space
    (Eq. (eq:partition)), so every level-k cell takes its value from the one region that holds it:
    * cells of the level-k blocks: F_k = fhat_k + P_{k+1->k} F_{k+1}, i.e. own values on Omega_k and the
      8-child means of the finer levels on covered cells (cumulative coarsening);
    * every other cell: P_{k-1->k} of the level-(k-1) reconstruction, which itself holds the coarsened
      level-k data on its covered cells, so the interpolation near a level boundary reads values of the
      same function on both sides.
    Constants and linear functions are reproduced exactly wherever the stencils stay inside the grid."""
    K = len(lv)
    F = [None] * K
    F[K - 1] = fhat[K - 1]
    for k in range(K - 2, -1, -1):
        F[k] = fhat[k] + coarsen(F[k + 1], lv[k + 1], lv[k])
    T = [F[0]]
    for k in range(1, K):
        up = interp_up(T[k - 1], lv[k - 1], lv[k])
        T.append(np.where(lv[k].user[None], F[k], up))
    return T


def fif_amr(mesh, f_levels, alpha_finest, r=None):
    """FIF-AMR heat apply (Sec. 3.5, Eq. (eq:FIF-AMR)): ``g_k = Gamma_k E_{alpha_k} * (P_k fhat)``.

    ``P_k fhat`` is the level-k reconstruction of the AMR data (``reconstruct``: own values on Omega_k,
    8-child means of the finer levels on covered cells, interpolation of the coarser level's reconstruction
    elsewhere).  The level-k kernel argument is ``alpha_k = alpha_finest * 4^{-(K-1-k)}``.
    """
    B = mesh["B"]
    blocks = mesh["levels"]
    K = len(blocks)
    lv = build_levels(mesh)
    fhat = [_user_field(lv[k], blocks[k], f_levels[k], B) for k in range(K)]
    T = reconstruct(lv, fhat)
    out = []
    for k in range(K):
        Pf = T[k]
        alpha_k = alpha_finest * 4.0 ** (-(K - 1 - k))
        Kh, rr = core.heat_kernel_full(alpha_k, r)
        region = dilate_maxnorm(lv[k].omega, rr)
        assert np.all(np.isfinite(Pf[:, region])), "level box too small for the heat stencil"
        src = np.where(region[None], Pf, 0.0)
        g = core.heat_box(src, alpha_k, rr)
        g = np.where(lv[k].omega[None], g, 0.0)
        out.append(_to_blocks(lv[k], blocks[k], g, B))
    return out
