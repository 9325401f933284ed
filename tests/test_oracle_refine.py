"""Pins of the oracle's refinement indicator (Sec. 4.2, Eqs. (eq:refine1)-(eq:refine2)) from the combined
source of Eq. (eq:combined_source).  The block RMS is checked against sums over the caller's input arrays
written out here (one level: S_0 = the source; two levels with no level-0 source: S_1 = the level-1
source, since psi_0 = 0 makes the correction vanish, and S_0 = its 8-child mean on the covered cells),
and the flags against the properties the criteria fix (dimensionless, S_max carried over time, refine
and coarsen exclusive)."""
import numpy as np

import lgf_synth as S
from oracle import refine


def _two_level(B=8):
    lvl0 = S.box_blocks((24, 24, 24), B)
    lvl1 = np.array([[2, 2, 2], [3, 2, 2], [2, 3, 2], [3, 3, 2]], np.int32)
    return dict(B=B, h0=1.0, n_ext=4, levels=[lvl0, lvl1])


def _rms(x):  # x: [ncomp][...] -> sqrt(mean over cells of sum over components)
    return float(np.sqrt((x ** 2).sum(axis=0).mean()))


def test_single_level_rms_is_the_source_rms():
    B = 8
    blocks = S.box_blocks((16, 16, 24), B)
    f = np.random.default_rng(3).standard_normal((3, len(blocks), B, B, B))
    out = refine.refinement_indicator(dict(B=B, h0=1.0, n_ext=4, levels=[blocks]), [f], 0.5, 0.5, 2)
    want = np.array([_rms(f[:, i]) for i in range(len(blocks))])
    assert np.allclose(out["rms"][0], want, rtol=1e-13, atol=0)
    assert out["s_max"] == max(want)


def test_two_levels_without_coarse_source():
    mesh = _two_level()
    B = mesh["B"]
    rng = np.random.default_rng(4)
    f0 = np.zeros((2, len(mesh["levels"][0]), B, B, B))
    f1 = rng.standard_normal((2, len(mesh["levels"][1]), B, B, B))
    out = refine.refinement_indicator(mesh, [f0, f1], 0.5, 0.5, 2)
    # level 1: S_1 = fhat_1 on its blocks (the only fine level: every cell is in Omega_1)
    assert np.allclose(out["rms"][1], [_rms(f1[:, i]) for i in range(len(f1[0]))], rtol=1e-12, atol=0)
    # level 0: S_0 = the 8-child mean of the level-1 source on the covered cells, 0 elsewhere
    fine = S.blocks_to_box(f1, mesh["levels"][1], B, (32, 64, 64))  # level-1 cells [z][y][x] from 0
    coarse = fine.reshape(2, 16, 2, 32, 2, 32, 2).mean(axis=(2, 4, 6))  # level-0 cells 0..15, 0..31
    want = []
    for bx, by, bz in mesh["levels"][0]:
        blk = np.zeros((2, B, B, B))
        z0, y0, x0 = B * bz, B * by, B * bx
        sub = coarse[:, z0:z0 + B, y0:y0 + B, x0:x0 + B]
        blk[:, :sub.shape[1], :sub.shape[2], :sub.shape[3]] = sub
        want.append(_rms(blk))
    assert np.allclose(out["rms"][0], want, rtol=1e-12, atol=1e-15)


def test_flags_are_dimensionless_and_exclusive():
    mesh = _two_level()
    B = mesh["B"]
    rng = np.random.default_rng(5)
    f = [rng.standard_normal((3, len(b), B, B, B)) for b in mesh["levels"]]
    a = refine.refinement_indicator(mesh, f, 0.3, 0.4, 2)
    b = refine.refinement_indicator(mesh, [1e3 * x for x in f], 0.3, 0.4, 2)
    assert np.isclose(b["s_max"], 1e3 * a["s_max"], rtol=1e-12)
    for k in range(2):
        assert np.allclose(b["rms"][k], 1e3 * a["rms"][k], rtol=1e-12)
        assert (a["refine"][k] == b["refine"][k]).all() and (a["coarsen"][k] == b["coarsen"][k]).all()
        assert not (a["refine"][k] & a["coarsen"][k]).any()
    assert any(r.any() for r in a["refine"])


def test_smax_carried_over_time_raises_the_thresholds():
    mesh = _two_level()
    B = mesh["B"]
    rng = np.random.default_rng(6)
    f = [rng.standard_normal((3, len(b), B, B, B)) for b in mesh["levels"]]
    now = refine.refinement_indicator(mesh, f, 0.3, 0.4, 2)
    later = refine.refinement_indicator(mesh, f, 0.3, 0.4, 2, s_max_prev=10 * now["s_max"])
    assert later["s_max"] == 10 * now["s_max"]
    for k in range(2):
        assert (later["refine"][k] <= now["refine"][k]).all()   # higher threshold: never more refinement
        assert (later["coarsen"][k] >= now["coarsen"][k]).all()


def test_extended_region_flags_the_coarse_blocks_under_it():
    # Level-0 blocks with no source of their own are flagged for refinement exactly when a level-1
    # extended-region cell with a correction source above the level-1 threshold lies in them (Sec. 4.2:
    # points of Omega_1^E outside the level-1 blocks).  The only source is a level-0 block far from
    # level 1, so the correction s = (P L_0 - L_1 P) psi_0 is the whole of S_1; alpha = 0.01 with
    # N_l = 5 puts the level-1 threshold at 1e-8 S_max, far below s on the extended region.
    B = 8
    lvl0 = S.box_blocks((48, 48, 48), B)                    # level-0 blocks 0..5 per axis
    lvl1 = S.box_blocks((16, 16, 16), B) + np.int32(4)      # covers level-0 block (2, 2, 2) exactly
    mesh = dict(B=B, h0=1.0, n_ext=8, levels=[lvl0, lvl1])  # N_E = 8 fine cells = 4 coarse cells < B
    f0 = np.zeros((1, len(lvl0), B, B, B))
    src = [i for i, b in enumerate(lvl0) if tuple(b) == (5, 5, 5)][0]
    z, y, x = np.meshgrid(*[np.arange(B) - 3.5] * 3, indexing="ij")
    f0[0, src] = np.exp(-(x ** 2 + y ** 2 + z ** 2) / 8.0)
    f1 = np.zeros((1, len(lvl1), B, B, B))
    out = refine.refinement_indicator(mesh, [f0, f1], 0.01, 0.5, 5)
    want = {(5, 5, 5)}
    want |= {(2 + dx, 2 + dy, 2 + dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)}
    want.discard((2, 2, 2))  # covered by level 1: its own S_0 is the (zero) coarsened level-1 source
    got = {tuple(int(v) for v in b) for b, r in zip(lvl0, out["refine"][0]) if r}
    assert got == want
