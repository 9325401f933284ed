"""Pins of the stage-projection oracle (Sec. 2.4, Eqs. (eq:projection-1), (eq:projection-2); Sec. 3.6) against
identities of the staggered operators, with the divergence written out here (not the oracle's):
D H = H D and D G = L_C make the projected field divergence-free wherever the integrating factor's stencil
stays inside the blocks, a divergence-free r passes through unchanged (p = 0, u = H r), and on two levels
the divergence left deep inside each level is orders of magnitude below that of r."""
import numpy as np

import lgf_synth as S
from oracle import amr, core, projection


def _div(r, h):
    """Divergence of a face field [3][nz][ny][nx] on the cells that have all six faces: [nz-1][ny-1][nx-1]."""
    return ((r[0][1:, 1:, 1:] - r[0][1:, 1:, :-1]) + (r[1][1:, 1:, 1:] - r[1][1:, :-1, 1:]) +
            (r[2][1:, 1:, 1:] - r[2][:-1, 1:, 1:])) / h


def _one_level(shape=(32, 32, 40), B=8, h=0.5):
    return dict(B=B, h0=h, n_ext=4, levels=[S.box_blocks(shape, B)]), shape


def _bump(shape, h, rng, ncomp=3):
    z, y, x = np.meshgrid(*[(np.arange(n) + 0.5 - n / 2) * h for n in shape], indexing="ij")
    env = np.exp(-(x ** 2 + y ** 2 + z ** 2) / (0.15 * (min(shape) * h) ** 2))
    return env[None] * rng.standard_normal((ncomp,) + shape)


def test_single_level_projection_is_divergence_free_inside():
    mesh, shape = _one_level()
    h, B = mesh["h0"], mesh["B"]
    rng = np.random.default_rng(41)
    rbox = _bump(shape, h, rng)
    r = S.box_to_blocks(rbox, mesh["levels"][0], B)
    for alpha, margin in ((0.1, len(core.heat_weights_1d(0.1)) + 1), (0.0, 2)):
        u, p = projection.project_amr(mesh, [r], alpha)
        ubox = S.blocks_to_box(u[0], mesh["levels"][0], B, shape)
        du = _div(ubox, h)[margin:-margin, margin:-margin, margin:-margin]
        dr = np.abs(_div(rbox, h)).max()
        assert du.size > 300 and np.abs(du).max() < 1e-11 * dr, (alpha, np.abs(du).max() / dr)
        assert np.abs(p[0]).max() > 1e-3 * dr * h * h


def test_divergence_free_field_passes_unchanged():
    mesh, shape = _one_level()
    h, B = mesh["h0"], mesh["B"]
    rng = np.random.default_rng(42)
    psi = _bump(shape, h, rng)  # compact edge field; r = C^T psi is divergence-free on the lattice
    pz, py, px = psi[2], psi[1], psi[0]

    def back(a, ax):  # a[n] - a[n - e_ax] (zero outside), ax = 0 for x
        out = a.copy()
        sl_d, sl_s = [slice(None)] * 3, [slice(None)] * 3
        sl_d[2 - ax], sl_s[2 - ax] = slice(1, None), slice(0, -1)
        out[tuple(sl_d)] -= a[tuple(sl_s)]
        return out

    rbox = np.stack([back(pz, 1) - back(py, 2), back(px, 2) - back(pz, 0), back(py, 0) - back(px, 1)]) / h
    assert np.abs(_div(rbox, h)).max() < 1e-12 * np.abs(rbox).max() / h
    r = S.box_to_blocks(rbox, mesh["levels"][0], B)
    u, p = projection.project_amr(mesh, [r], 0.05)
    assert np.abs(p[0]).max() < 1e-12 * np.abs(rbox).max() * h
    want = core.heat_box(rbox, 0.05)
    got = S.blocks_to_box(u[0], mesh["levels"][0], B, shape)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_two_level_projection_removes_the_divergence():
    B = 8
    mesh = dict(B=B, h0=0.5, n_ext=4, levels=[S.box_blocks((40, 40, 40), B),
                                              np.array([[x, y, z] for x in (3, 4, 5, 6) for y in (3, 4, 5, 6)
                                                        for z in (4, 5)], np.int32)])
    rng = np.random.default_rng(43)
    lv = amr.build_levels(mesh)
    r = []
    for k, blk in enumerate(mesh["levels"]):
        h = mesh["h0"] / 2 ** k
        data = np.zeros((3, len(blk), B, B, B))
        coef = rng.standard_normal((3, 3))
        for i, (bx, by, bz) in enumerate(blk):
            z, y, x = np.meshgrid(*[(B * b + np.arange(B) + 0.5) * h - 10.0 for b in (bz, by, bx)], indexing="ij")
            env = np.exp(-(x ** 2 + y ** 2 + z ** 2) / 16.0)
            for c in range(3):
                data[c, i] = env * (coef[c, 0] * x + coef[c, 1] * y + coef[c, 2] * z)
        r.append(data)
    u, p = projection.project_amr(mesh, r, 0.0)
    for k in range(2):
        box_u = projection._to_box(lv[k], mesh["levels"][k], u[k], B)
        box_r = projection._to_box(lv[k], mesh["levels"][k], r[k], B)
        deep = lv[k].omega & ~amr.dilate_maxnorm(~lv[k].omega, 3)
        du = np.abs(_div(box_u, lv[k].h))[deep[1:, 1:, 1:]]
        dr = np.abs(_div(box_r, lv[k].h))[deep[1:, 1:, 1:]]
        assert deep.sum() > 500 and du.max() < 1e-2 * dr.max(), (k, du.max() / dr.max())


def test_interface_faces_come_from_the_neighbouring_levels():
    # r = C^T psi of a smooth edge field is divergence-free on each level's lattice; at the cells next to a
    # level boundary the divergence source D^r needs faces of the other level, which the reconstruction
    # P_k r^ supplies (interpolation / coarsening).  Leaving those faces at zero instead makes D^r as large
    # as |r| / h there; with the reconstruction it stays a fraction of that.
    B = 8
    mesh = dict(B=B, h0=0.5, n_ext=4, levels=[S.box_blocks((40, 40, 40), B),
                                              np.array([[x, y, z] for x in (3, 4, 5, 6) for y in (3, 4, 5, 6)
                                                        for z in (4, 5)], np.int32)])
    r = []
    for k, blk in enumerate(mesh["levels"]):
        h = mesh["h0"] / 2 ** k
        data = np.zeros((3, len(blk), B, B, B))
        for i, (bx, by, bz) in enumerate(blk):
            idx = [B * b + np.arange(B) for b in (bx, by, bz)]
            Zc, Yc, Xc = np.meshgrid(idx[2], idx[1], idx[0], indexing="ij")

            def psi(a, dx=0, dy=0, dz=0):  # edge component a at n + (1, 1, 1) - e_a / 2, physical units
                p = [Xc + dx + 1.0, Yc + dy + 1.0, Zc + dz + 1.0]
                p[a] = p[a] - 0.5
                X, Y, Z = (q * h for q in p)
                return np.exp(-((X - 10) ** 2 + (Y - 10) ** 2 + (Z - 10) ** 2) / 9.0) * (1.0 + 0.3 * a)

            ux = (psi(2) - psi(2, 0, -1, 0)) - (psi(1) - psi(1, 0, 0, -1))
            uy = (psi(0) - psi(0, 0, 0, -1)) - (psi(2) - psi(2, -1, 0, 0))
            uz = (psi(1) - psi(1, -1, 0, 0)) - (psi(0) - psi(0, 0, -1, 0))
            data[:, i] = np.stack([ux, uy, uz]) / h
        r.append(data)
    _, _, I = projection.project_amr(mesh, r, 0.0, return_internals=True)
    rel = [np.abs(I["d"][k]).max() * (mesh["h0"] / 2 ** k) / np.abs(r[k]).max() for k in range(2)]
    assert rel[0] < 0.1 and rel[1] < 0.35, rel  # without the reconstruction both are about 0.5
