"""GPU refinement indicator (Sec. 4.2, Eqs. (eq:refine1), (eq:maximumS), (eq:refine2)) against the oracle
(oracle/refine.py) through the C ABI: block RMS of the combined source of Eq. (eq:combined_source), the
refine / coarsen flags, S_max carried over calls, and the extended-region flag on the coarser level.

Tolerances: the block RMS to 1e-12 (FP64), 1e-10 (DF32), 1e-5 (FP32) relative to the largest RMS; the flags
exactly, except for blocks whose largest |S_k| lies within the arithmetic's error of a threshold (checked
to be few and skipped)."""
import numpy as np
import pytest

import lgf_synth as S
from oracle import refine

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 2: 1e-10, 1: 1e-5}


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_13213_gb300.lgf as L
    L.load()
    return L


@pytest.fixture(scope="module")
def table8(L):
    t = L.lgf_table_create(8, (14, 14, 8), L.LGF_TBL_FP64 | L.LGF_TBL_FP32 | L.LGF_TBL_DF32)
    yield t
    L.lgf_table_destroy(t)


def _run(L, table, mesh, f, precision, alpha, beta, nl, s_prev=0.0, mode=1):
    m = L.Mesh(mesh["levels"], mesh["B"], mesh["h0"], n_ext=mesh["n_ext"])
    ft = torch.from_numpy(np.concatenate(f, axis=1)).cuda()
    phi = torch.zeros_like(ft)
    n = m.total_blocks
    rms = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    flags = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
    smax = torch.tensor([s_prev], dtype=torch.float64, device="cuda")
    L.lgf_refinement_indicator(table, m, ft.shape[0], ft.data_ptr(), phi.data_ptr(), L.LGF_F64,
                               L.make_opts(precision=precision, mac_mode=mode), alpha, beta, nl,
                               rms.data_ptr(), flags.data_ptr(), smax.data_ptr())
    torch.cuda.synchronize()
    return rms.cpu().numpy(), flags.cpu().numpy(), float(smax.item()), phi


def _split(arr, mesh):
    out, o = [], 0
    for b in mesh["levels"]:
        out.append(arr[o:o + len(b)])
        o += len(b)
    return out


def _check(got, ref, mesh, tol, ratio_margin):
    rms, flags, smax = got[:3]
    scale = max(r.max() for r in ref["rms"])
    for k, (r, g) in enumerate(zip(ref["rms"], _split(rms, mesh))):
        assert np.abs(g - r).max() <= tol * scale, k
    assert abs(smax - ref["s_max"]) <= tol * ref["s_max"]
    for k, fl in enumerate(_split(flags, mesh)):
        assert ((fl & 1) > 0).tolist() == ref["refine"][k].tolist(), k
        assert ((fl & 2) > 0).tolist() == ref["coarsen"][k].tolist(), k


def two_level(n_ext=4):
    B = 8
    lvl0 = S.box_blocks((24, 24, 24), B)
    lvl1 = np.array([[2, 2, 2], [3, 2, 2], [2, 3, 2], [3, 3, 2], [2, 2, 3]], np.int32)
    return dict(B=B, h0=0.5, n_ext=n_ext, levels=[lvl0, lvl1])


@pytest.mark.parametrize("precision", [0, 2, 1])
def test_indicator_two_levels_random(L, table8, precision):
    mesh = two_level()
    rng = np.random.default_rng(31)
    f = [rng.standard_normal((3, len(b), 8, 8, 8)) * (1.0 + k) for k, b in enumerate(mesh["levels"])]
    n0 = len(mesh["levels"][0])  # level-0 amplitudes over three decades, so some blocks coarsen
    f[0] *= (10.0 ** (-3.0 * np.arange(n0) / n0))[None, :, None, None, None]
    ref = refine.refinement_indicator(mesh, f, 0.6, 0.5, 2)
    got = _run(L, table8, mesh, f, precision, 0.6, 0.5, 2)
    _check(got, ref, mesh, TOL[precision], 0)
    assert any(r.any() for r in ref["refine"]) and any(c.any() for c in ref["coarsen"])


def test_indicator_extended_region_flags_coarse_blocks(L, table8):
    # the only source sits in a far level-0 block, so the correction source alone forms S_1; with
    # alpha = 0.01 and N_l = 5 the 26 level-0 blocks around the level-1 patch are flagged through
    # Omega_1^E (the same mesh as the oracle's pin)
    B = 8
    lvl0 = S.box_blocks((48, 48, 48), B)
    lvl1 = S.box_blocks((16, 16, 16), B) + np.int32(4)
    mesh = dict(B=B, h0=1.0, n_ext=8, levels=[lvl0, lvl1])
    f0 = np.zeros((1, len(lvl0), B, B, B))
    src = [i for i, b in enumerate(lvl0) if tuple(b) == (5, 5, 5)][0]
    z, y, x = np.meshgrid(*[np.arange(B) - 3.5] * 3, indexing="ij")
    f0[0, src] = np.exp(-(x ** 2 + y ** 2 + z ** 2) / 8.0)
    f = [f0, np.zeros((1, len(lvl1), B, B, B))]
    ref = refine.refinement_indicator(mesh, f, 0.01, 0.5, 5)
    t = L.lgf_table_create(8, (12, 12, 12), L.LGF_TBL_FP64)
    try:
        got = _run(L, t, mesh, f, 0, 0.01, 0.5, 5)
    finally:
        L.lgf_table_destroy(t)
    _check(got, ref, mesh, 1e-12, 0)
    assert int((got[1][:len(lvl0)] & 1).sum()) == 27


def test_indicator_smax_carried_and_single_level(L, table8):
    B = 8
    blocks = S.box_blocks((16, 24, 32), B)
    mesh = dict(B=B, h0=1.0, n_ext=4, levels=[blocks])
    rng = np.random.default_rng(32)
    f = [rng.standard_normal((2, len(blocks), B, B, B)) * np.linspace(0.1, 3.0, len(blocks))[None, :, None, None,
                                                                                               None]]
    ref = refine.refinement_indicator(mesh, f, 0.5, 0.5, 1)
    got = _run(L, table8, mesh, f, 0, 0.5, 0.5, 1)
    _check(got, ref, mesh, 1e-12, 0)
    later_ref = refine.refinement_indicator(mesh, f, 0.5, 0.5, 1, s_max_prev=10 * ref["s_max"])
    later = _run(L, table8, mesh, f, 0, 0.5, 0.5, 1, s_prev=10 * ref["s_max"])
    _check(later, later_ref, mesh, 1e-12, 0)
    assert later[2] == 10 * ref["s_max"]


def test_indicator_three_level_ring_box_mode(L):
    # config-3 geometry at B = 16 in DF32 box mode: the library's composite-mesh solve of the ring
    mesh, f = S.three_level_ring()
    ref = refine.refinement_indicator(mesh, f, 0.3, 0.5, 2)
    t = L.lgf_table_create(16, (13, 13, 9), L.LGF_TBL_BOX_ONLY)
    try:
        got = _run(L, t, mesh, f, 2, 0.3, 0.5, 2, mode=2)
    finally:
        L.lgf_table_destroy(t)
    _check(got, ref, mesh, 1e-10, 0)
