"""Pins of the multi-level oracle (FLGF-AMR, Sec. 3.4; FIF-AMR, Sec. 3.5) against limits and identities
that the paper and the mathematics fix, not against the oracle itself."""
import numpy as np
import pytest

import lgf_synth as S
import oracle
from oracle import amr, core


def _two_level_mesh(B=8, n_ext=4, h0=1.0):
    lvl0 = S.box_blocks((24, 24, 24), B)
    lvl1 = np.array([[2, 2, 2], [3, 2, 2], [2, 3, 2], [3, 3, 2], [2, 2, 3]], np.int32)
    return dict(B=B, h0=h0, n_ext=n_ext, levels=[lvl0, lvl1])


def _gaussian_levels(mesh, sigma=3.0, centre=(12.0, 12.0, 12.0)):
    """Smooth source sampled at each level's cell centres (level-0 cell units for the geometry)."""
    B = mesh["B"]
    out = []
    for k, blk in enumerate(mesh["levels"]):
        h = 0.5 ** k
        data = np.zeros((1, len(blk), B, B, B))
        for i, (bx, by, bz) in enumerate(blk):
            z, y, x = np.meshgrid(*[(B * b + np.arange(B) + 0.5) * h for b in (bz, by, bx)], indexing="ij")
            r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
            data[0, i] = np.exp(-r2 / sigma ** 2)
        out.append(data)
    return out


def test_single_level_reduces_to_lgf_solve():
    rng = np.random.default_rng(2)
    B = 8
    blk = S.box_blocks((16, 24, 16), B)
    f = rng.standard_normal((2, len(blk), B, B, B))
    mesh = dict(B=B, h0=0.25, n_ext=4, levels=[blk])
    out, masks = amr.flgf_amr(mesh, [f])
    box = S.blocks_to_box(f, blk, B, (16, 24, 16))
    ref = oracle.solve_box_fft(box, 0.25)
    got = S.blocks_to_box(out[0], blk, B, (16, 24, 16))
    assert masks[0].all()
    assert np.abs(got - ref).max() < 1e-14 * np.abs(ref).max()


def test_fine_only_sources_match_composite_definition_exactly():
    # with fhat_0 = 0, psi_0 = 0 and the correction vanishes: steps 1-3 reduce to the definition
    rng = np.random.default_rng(3)
    mesh = _two_level_mesh()
    B = mesh["B"]
    f0 = np.zeros((1, len(mesh["levels"][0]), B, B, B))
    f1 = rng.standard_normal((1, len(mesh["levels"][1]), B, B, B))
    out, masks = amr.flgf_amr(mesh, [f0, f1])
    comp = amr.composite_definition(mesh, [f0, f1])
    for k in range(2):
        scale = np.abs(comp[k][:, masks[k]]).max()
        assert np.abs(out[k] - comp[k])[:, masks[k]].max() < 1e-13 * scale


def test_interpolation_and_coarsening_on_linear_fields():
    lc = amr.Level(0, (-3, -4, -2), (10, 12, 14), 1.0)
    lf = amr.Level(1, (0, 0, 2), (8, 10, 12), 0.5)
    z, y, x = np.meshgrid(*[lc.origin[a] + np.arange(n) + 0.5 for a, n in zip((2, 1, 0), lc.shape)],
                          indexing="ij")
    lin = (0.3 * x - 1.1 * y + 0.7 * z + 2.0)[None]
    up = amr.interp_up(lin, lc, lf)
    zf, yf, xf = np.meshgrid(*[(lf.origin[a] + np.arange(n) + 0.5) / 2 for a, n in zip((2, 1, 0), lf.shape)],
                             indexing="ij")
    ref = 0.3 * xf - 1.1 * yf + 0.7 * zf + 2.0
    assert np.nanmax(np.abs(up[0] - ref)) < 1e-13 and np.isfinite(up).all()
    # coarsening a fine linear field gives the linear field at the parent centres
    down = amr.coarsen(ref[None], lf, lc)
    cover = amr.coarsen_mask(np.ones(lf.shape, bool), lf, lc)
    assert np.abs(down[0][cover] - lin[0][cover]).max() < 1e-13


def test_correction_source_vanishes_for_linear_psi():
    # S = P L_{k-1} - L_k P annihilates linear fields (P exact on them, both Laplacians zero)
    lc = amr.Level(0, (0, 0, 0), (10, 10, 10), 1.0)
    lf = amr.Level(1, (4, 4, 4), (8, 8, 8), 0.5)
    z, y, x = np.meshgrid(*[np.arange(n) + 0.5 for n in lc.shape], indexing="ij")
    psi = (2.0 * x - 0.5 * y + 0.25 * z)[None]
    s = amr.interp_up(amr.laplacian_box(psi, 1.0), lc, lf) - amr.laplacian_box(amr.interp_up(psi, lc, lf), 0.5)
    assert np.nanmax(np.abs(s)) < 1e-12


def test_converges_to_composite_definition_as_extension_grows():
    mesh = _two_level_mesh(n_ext=0)
    f = _gaussian_levels(mesh)
    errs = []
    for ne in (0, 2, 6, 14):
        mesh["n_ext"] = ne
        out, masks = amr.flgf_amr(mesh, f)
        comp = amr.composite_definition(mesh, f)
        errs.append(np.abs(out[1] - comp[1])[:, masks[1]].max() / np.abs(comp[1][:, masks[1]]).max())
    assert errs[-1] < errs[0] / 100 and errs[2] < errs[0]
    assert errs[-1] < 3e-4  # the order of the paper's ~1e-4 cut-off at N_E = 14 (Sec. 3.4)


def test_residual_identity_on_extended_region():
    # L_k phi^k = F_k + P L_{k-1} psi_{k-1} wherever the correction source is kept (Eq. (eq:combine_S))
    mesh = _two_level_mesh(n_ext=4)
    f = _gaussian_levels(mesh)
    rng = np.random.default_rng(8)
    f[1] = f[1] + 0.1 * rng.standard_normal(f[1].shape)
    out, masks, I = amr.flgf_amr(mesh, f, return_internals=True)
    lv, phi, psi, F = I["levels"], I["phi"], I["psi"], I["F"]
    lhs = amr.laplacian_box(phi[1], lv[1].h)
    rhs = F[1] + amr.interp_up(amr.laplacian_box(psi[0], lv[0].h), lv[0], lv[1])
    region = lv[1].omega | I["steps"][0]["ext"]
    inner = region & ~amr.dilate_maxnorm(~region, 1)
    d = np.abs(lhs - rhs)[:, inner]
    assert np.isfinite(d).all() and d.max() < 1e-10 * np.abs(rhs[:, inner]).max()


def test_heat_single_level_reduces_to_heat_kernel():
    rng = np.random.default_rng(6)
    B = 8
    blk = S.box_blocks((16, 16, 24), B)
    f = rng.standard_normal((1, len(blk), B, B, B))
    mesh = dict(B=B, h0=1.0, n_ext=4, levels=[blk])
    g = amr.fif_amr(mesh, [f], 0.1)[0]
    box = S.blocks_to_box(f, blk, B, (16, 16, 24))
    ref = oracle.heat_box(box, 0.1)
    assert np.abs(S.blocks_to_box(g, blk, B, (16, 16, 24)) - ref).max() < 1e-15 * np.abs(ref).max() + 1e-300


def test_heat_preserves_constants_away_from_level_boundaries():
    B = 8
    mesh = dict(B=B, h0=1.0, n_ext=4, levels=[S.box_blocks((40, 40, 40), B),
                                              np.array([[4, 4, 4], [5, 4, 4], [4, 5, 5]], np.int32)])
    f = [np.ones((1, len(b), B, B, B)) for b in mesh["levels"]]
    g = amr.fif_amr(mesh, f, 0.1)
    lv = amr.build_levels(mesh)
    # P_0 fhat = 1 on every level-0 user cell (own values on Omega_0, 8-child means of 1 under
    # level 1), so the kernel returns 1 on Omega_0 cells more than its radius from the user boundary
    om = lv[0].omega
    w = core.heat_weights_1d(0.1 / 4)
    deep = om & ~amr.dilate_maxnorm(~lv[0].user, len(w) + 1)
    box = np.zeros((1,) + lv[0].shape)
    for i, b in enumerate(mesh["levels"][0]):
        box[(slice(None),) + lv[0].block_slice(b, B)] = g[0][:, i]
    assert deep.sum() > 100
    assert np.abs(box[0][deep] - 1.0).max() < 1e-14


def _nested_mesh(B, shapes_and_offsets, h0=1.0, n_ext=4):
    """Nested levels: level 0 tiles a box; level k >= 1 tiles a box of level-k blocks starting at the
    given level-k block offset (every level-k block inside a level-(k-1) block)."""
    levels = []
    for k, (shape, off) in enumerate(shapes_and_offsets):
        levels.append(S.box_blocks(shape, B) + np.asarray(off, np.int32))
    return dict(B=B, h0=h0, n_ext=n_ext, levels=levels)


def _centre_field(mesh, fn):
    """fn(x, y, z) at every user cell centre of every level, x in level-0 spacing units."""
    B = mesh["B"]
    out = []
    for k, blk in enumerate(mesh["levels"]):
        h = mesh["h0"] / 2 ** k
        data = np.zeros((1, len(blk), B, B, B))
        for i, (bx, by, bz) in enumerate(blk):
            z, y, x = np.meshgrid(*[(B * b + np.arange(B) + 0.5) * h for b in (bz, by, bx)], indexing="ij")
            data[0, i] = fn(x, y, z)
        out.append(data)
    return out


@pytest.mark.parametrize("K", [2, 3])
def test_reconstruction_reproduces_linear_functions_across_levels(K):
    # Sec. 3.2, Eq. (eq:interp): P_k fhat estimates the function the AMR data sample on level k, to the
    # order of the interpolant; with 8-child means and tensor-product linear interpolation a linear
    # function is reproduced exactly on every level-k cell, at level boundaries included, wherever the
    # stencils stay inside the grid (here: cells two coarse cells inside the level-0 blocks)
    B = 8
    spec = [((24, 24, 24), (0, 0, 0)), ((16, 16, 32), (1, 2, 1)), ((16, 16, 16), (3, 5, 3))][:K]
    mesh = _nested_mesh(B, spec)
    lin = lambda x, y, z: 0.7 * x - 1.3 * y + 0.4 * z + 2.0
    f = _centre_field(mesh, lin)
    lv = amr.build_levels(mesh)
    fh = [amr._user_field(lv[k], mesh["levels"][k], f[k], B) for k in range(K)]
    T = amr.reconstruct(lv, fh)
    inside0 = lv[0].user & ~amr.dilate_maxnorm(~lv[0].user, 2)
    for k in range(K):
        z, y, x = np.meshgrid(*[(lv[k].origin[a] + np.arange(n) + 0.5) * mesh["h0"] / 2 ** k
                                for a, n in zip((2, 1, 0), lv[k].shape)], indexing="ij")
        # level-k cells whose level-0 ancestor lies two cells inside the level-0 blocks
        anc = [((lv[k].origin[a] + np.arange(n)) // 2 ** k) - lv[0].origin[a] for a, n in zip((2, 1, 0), lv[k].shape)]
        ok = np.zeros(lv[k].shape, bool)
        vz, vy, vx = [(a >= 0) & (a < m) for a, m in zip(anc, lv[0].shape)]
        sub = inside0[np.clip(anc[0], 0, lv[0].shape[0] - 1)][:, np.clip(anc[1], 0, lv[0].shape[1] - 1)][
            :, :, np.clip(anc[2], 0, lv[0].shape[2] - 1)]
        ok = sub & vz[:, None, None] & vy[None, :, None] & vx[None, None, :]
        assert ok.sum() > 1000
        err = np.abs(T[k][0] - lin(x, y, z))[ok]
        assert np.isfinite(err).all() and err.max() < 1e-12, (k, err.max())


@pytest.mark.parametrize("K", [2, 3])
def test_heat_keeps_constants_on_every_omega_cell(K):
    # E_alpha has unit mass, so FIF-AMR of a constant returns it on every Omega_k cell whose heat stencil
    # stays inside the grid, next to level boundaries too
    B = 8
    spec = [((48, 48, 48), (0, 0, 0)), ((32, 32, 32), (2, 2, 2)), ((16, 16, 16), (5, 5, 5))][:K]
    mesh = _nested_mesh(B, spec)
    f = [np.ones((1, len(b), B, B, B)) for b in mesh["levels"]]
    g = amr.fif_amr(mesh, f, 0.1)
    lv = amr.build_levels(mesh)
    for k in range(K):
        r = len(core.heat_weights_1d(0.1 / 4 ** (K - 1 - k))) - 1
        box = np.zeros(lv[k].shape)
        for i, b in enumerate(mesh["levels"][k]):
            box[lv[k].block_slice(b, B)] = g[k][0, i]
        far = lv[k].omega & (~amr.dilate_maxnorm(~lv[k].user, r + 1) if k == 0 else lv[k].omega)
        assert far.sum() > 100
        assert np.abs(box[far] - 1.0).max() < 1e-14, (k, np.abs(box[far] - 1.0).max())


def test_heat_second_moment_gives_the_same_physical_increment_on_every_level():
    # E_a * |n|^2 = |n|^2 + 6a on the unit lattice (zero mean, variance 2a per axis of the lattice heat
    # kernel), so for q = |x - c|^2 in physical units E_{alpha_k} * q = q + 6 alpha_k h_k^2 on cells
    # where the reconstruction P_k fhat is q itself.  One time step diffuses by the same kappa dt on
    # every level: the increment must equal 6 alpha_finest h_finest^2 on each of them.
    B = 8
    mesh = _nested_mesh(B, [((64, 64, 64), (0, 0, 0)), ((48, 48, 48), (1, 1, 1))], h0=1.0, n_ext=4)
    c = (32.0, 32.0, 32.0)
    q = _centre_field(mesh, lambda x, y, z: (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    alpha = 0.1
    g = amr.fif_amr(mesh, q, alpha)
    lv = amr.build_levels(mesh)
    expected = 6.0 * alpha * (mesh["h0"] / 2) ** 2
    for k in range(2):
        r = len(core.heat_weights_1d(alpha / 4 ** (1 - k))) - 1
        deep_box = lv[k].omega & ~amr.dilate_maxnorm(~lv[k].omega, r + 3)
        deep = amr._to_blocks(lv[k], mesh["levels"][k], deep_box[None].astype(float), B)[0] > 0.5
        assert deep.sum() > 200, k
        inc = (g[k] - q[k])[0][deep]
        assert np.abs(inc - expected).max() < 1e-10 * expected, (k, inc.min(), inc.max(), expected)


def test_uncorrected_solve_satisfies_its_own_identity():
    # without the source correction phi^k = c_k + L_k^{-1} F_k, so L_k (phi^k - c_k) = F_k on the level box
    # interior, while the corrected identity L_k phi^k = F_k + P L_{k-1} psi_{k-1} fails by the correction
    mesh = _two_level_mesh(n_ext=4)
    f = _gaussian_levels(mesh)
    out, masks, I = amr.flgf_amr(mesh, f, return_internals=True, correction=False)
    lv, phi, psi, F = I["levels"], I["phi"], I["psi"], I["F"]
    c = I["steps"][0]["c"]
    assert np.abs(I["steps"][0]["s"]).max() == 0.0
    inner = lv[1].omega & ~amr.dilate_maxnorm(~lv[1].omega, 1)
    lhs = amr.laplacian_box(phi[1] - c, lv[1].h)
    d = np.abs(lhs - F[1])[:, inner]
    assert np.isfinite(d).all() and d.max() < 1e-10 * np.abs(F[1][:, inner]).max()
    corrected = F[1] + amr.interp_up(amr.laplacian_box(psi[0], lv[0].h), lv[0], lv[1])
    miss = np.abs(amr.laplacian_box(phi[1], lv[1].h) - corrected)[:, inner].max()
    assert miss > 1e-6 * np.abs(corrected[:, inner]).max()
    # and it differs from the corrected solve by more than rounding
    ref, _ = amr.flgf_amr(mesh, f)
    assert np.abs(out[1] - ref[1])[:, masks[1]].max() > 1e-6 * np.abs(ref[1][:, masks[1]]).max()
