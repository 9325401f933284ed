"""The HERK stage projection (Sec. 2.4, Eqs. (eq:projection-1), (eq:projection-2)) on one level and on the
AMR grid (Sec. 3.6, Eqs. (eq:approx0)-(eq:approx4)).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Staggered lattice (Sec. 2.1): the velocity-like fields r and u live on the positive faces (component a of
cell n at n + (1/2, 1/2, 1/2) + e_a / 2, stored at array index n), the pressure p at cell centres.  With
    (D r)(n)   = sum_a (r_a[n] - r_a[n - e_a]) / h          (divergence, faces -> cells)
    (G p)_a[n] = (p[n + e_a] - p[n]) / h                     (gradient, cells -> faces)
D = -G^T and D G = L_C, the 7-point Laplacian (Eq. (eq:mimetic)).  A stage solves
    L_C p = D r,    u = H (r - G p),                         H = E_alpha, the integrating factor.

On the AMR grid (readings of Sec. 3.6, which leaves the transfer of face data open):
* r^ is given on the caller's blocks of every level; only its values on Omega_k are used;
* D^r on Omega_k is D applied to the level-k reconstruction P_k r^ (``amr.reconstruct``: own values on
  Omega_k, 8-child means of the finer levels on covered cells, interpolation of the coarser level's
  reconstruction elsewhere; every component treated as a cell-centred scalar); the faces just outside
  Omega_k take their values from the neighbouring regions through it (the one-cell-larger restriction of
  Sec. 3.6);
* p^ = FLGF-AMR(D^r) on Omega_k (``amr.flgf_amr``);
* G^p on the faces of the Omega_k cells is G applied to the reconstruction P_k p^;
* u^ = FIF-AMR(r^ - G^p) (``amr.fif_amr``) with the caller's alpha for the finest level.
Outside the AMR grid every field is zero (the truncation of the computational domain, Sec. 4.1).

Pins (tests/test_oracle_projection.py): on one level D u = 0 on every cell at least the integrating
factor's radius + 2 cells inside the blocks (D H = H D and D G = L_C, with D and G written out in the
test); a divergence-free r (r = C^T psi of a compact edge field) passes unchanged through the projection
(p = 0, u = H r); with alpha = 0 the result is r - G p with D u = 0 two cells inside; on two levels the
divergence left on the cells deep inside each level is orders of magnitude below that of r.
"""
import numpy as np

from . import amr, core


def divergence(r, h):
    """D r on a box: r [3][nz][ny][nx] face components -> [nz][ny][nx]; faces outside the box are zero."""
    d = np.zeros(r.shape[1:])
    for a in range(3):
        ax = 2 - a  # array axis of component a ([z][y][x])
        back = np.zeros_like(r[a])
        sl_dst = [slice(None)] * 3
        sl_src = [slice(None)] * 3
        sl_dst[ax] = slice(1, None)
        sl_src[ax] = slice(0, -1)
        back[tuple(sl_dst)] = r[a][tuple(sl_src)]
        d += r[a] - back
    return d / h


def gradient(p, h):
    """G p on a box: p [nz][ny][nx] -> [3][nz][ny][nx] faces; cells outside the box are zero."""
    out = np.zeros((3,) + p.shape)
    for a in range(3):
        ax = 2 - a
        fwd = np.zeros_like(p)
        sl_dst = [slice(None)] * 3
        sl_src = [slice(None)] * 3
        sl_dst[ax] = slice(0, -1)
        sl_src[ax] = slice(1, None)
        fwd[tuple(sl_dst)] = p[tuple(sl_src)]
        out[a] = (fwd - p) / h
    return out


def _to_box(lv, blocks, data, B):
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


def project_amr(mesh, r_levels, alpha_finest, return_internals=False):
    """The stage projection on the AMR grid; ``r_levels[k]`` is [3][nblk_k][B]^3.  Returns (u^ per level on
    Omega_k, zero elsewhere, as [3][nblk_k][B]^3; p^ per level as [1][nblk_k][B]^3)."""
    B = mesh["B"]
    blocks = mesh["levels"]
    K = len(blocks)
    lv = amr.build_levels(mesh)
    rr = amr.reconstruct(lv, [_to_box(lv[k], blocks[k], r_levels[k], B) for k in range(K)])
    d = [np.where(lv[k].omega, divergence(rr[k], lv[k].h), 0.0)[None] for k in range(K)]
    d_blk = [_to_blocks(lv[k], blocks[k], d[k], B) for k in range(K)]
    p_blk, _ = amr.flgf_amr(mesh, d_blk)
    pp = amr.reconstruct(lv, [_to_box(lv[k], blocks[k], p_blk[k], B) for k in range(K)])
    w_blk = []
    for k in range(K):
        w = np.where(lv[k].omega[None], rr[k] - gradient(pp[k][0], lv[k].h), 0.0)
        w_blk.append(_to_blocks(lv[k], blocks[k], w, B))
    u_blk = amr.fif_amr(mesh, w_blk, alpha_finest)
    if return_internals:
        return u_blk, p_blk, dict(levels=lv, d=d_blk, w=w_blk)
    return u_blk, p_blk
