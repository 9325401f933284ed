"""GPU parity of the composite-mesh Poisson solve (FLGF-AMR, Sec. 3.4) and heat apply (FIF-AMR,
Sec. 3.5) against the CPU oracle (oracle/amr.py), through the C ABI.

Tolerances (relative L-infinity over the Omega_k cells of each level): 1e-12 for FP64, 1e-10 for
DF32, 2e-5 for plain FP32.  The FP64 residual L_k phi - F_k - P L_{k-1} psi_{k-1} reported by the
library is zero in exact arithmetic; its bound scales with 12/h^2 times phi's own rounding.
"""
import numpy as np
import pytest

import lgf_synth as S
from oracle import amr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 2: 1e-10, 1: 2e-5}


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


def two_level(n_ext=4):
    B = 8
    lvl0 = S.box_blocks((24, 24, 24), B)
    lvl1 = np.array([[2, 2, 2], [3, 2, 2], [2, 3, 2], [3, 3, 2], [2, 2, 3]], np.int32)
    return dict(B=B, h0=0.5, n_ext=n_ext, levels=[lvl0, lvl1])


def flat(f_levels):
    return np.concatenate(f_levels, axis=1)


def split(arr, mesh):
    out, o = [], 0
    for b in mesh["levels"]:
        out.append(arr[:, o:o + len(b)])
        o += len(b)
    return out


def rel_err_levels(got, ref, masks):
    errs = []
    for g, r, m in zip(got, ref, masks):
        if m.sum() == 0:
            continue
        scale = np.abs(r[:, m]).max()
        errs.append(np.abs(g[:, m] - r[:, m]).max() / scale)
    return max(errs)


def gpu_solve(L, table, mesh, f_levels, precision, residual=0):
    m = L.Mesh(mesh["levels"], mesh["B"], mesh["h0"], n_ext=mesh["n_ext"])
    f = torch.from_numpy(flat(f_levels)).cuda()
    phi = torch.full_like(f, float("nan"))
    rep = L.lgf_report()
    L.lgf_poisson_solve(table, m, f.shape[0], f.data_ptr(), phi.data_ptr(), L.LGF_F64,
                        L.make_opts(precision=precision, mac_mode=L.LGF_MAC_PAIR, residual=residual), rep)
    torch.cuda.synchronize()
    return split(phi.cpu().numpy(), mesh), rep


@pytest.mark.parametrize("precision", [0, 2, 1])
def test_two_level_random_sources(L, table8, precision):
    mesh = two_level()
    rng = np.random.default_rng(12)
    f = [rng.standard_normal((2, len(b), 8, 8, 8)) for b in mesh["levels"]]
    ref, masks = amr.flgf_amr(mesh, f)
    got, rep = gpu_solve(L, table8, mesh, f, precision, residual=1)
    err = rel_err_levels(got, ref, masks)
    assert err <= TOL[precision], f"precision {precision}: {err:.3e}"
    # cells outside Omega_k are left untouched
    for g, msk in zip(got, masks):
        assert np.isnan(g[:, ~msk]).all()
    if precision == 0:
        assert rep.residual_rel < 1e-11
    assert rep.target_cells == sum(int(m.sum()) for m in masks)


@pytest.mark.parametrize("n_ext", [0, 3, 9])
def test_two_level_extension_widths(L, table8, n_ext):
    mesh = two_level(n_ext)
    rng = np.random.default_rng(100 + n_ext)
    f = [rng.standard_normal((1, len(b), 8, 8, 8)) for b in mesh["levels"]]
    ref, masks = amr.flgf_amr(mesh, f)
    got, _ = gpu_solve(L, table8, mesh, f, 0)
    assert rel_err_levels(got, ref, masks) <= 1e-12


@pytest.fixture(scope="module")
def ring3():
    mesh, f = S.three_level_ring(R=1.0, sigma=0.2, B=8, n_ext=6, h_fine=1 / 32, support=(24, 24, 16), dilate0=1)
    ref, masks = amr.flgf_amr(mesh, f)
    return mesh, f, ref, masks


@pytest.mark.parametrize("precision", [0, 2])
def test_three_level_ring(L, table8, ring3, precision):
    mesh, f, ref, masks = ring3
    got, rep = gpu_solve(L, table8, mesh, f, precision, residual=1)
    for c in range(2):
        err = rel_err_levels([g[c:c + 1] for g in got], [r[c:c + 1] for r in ref], masks)
        assert err <= TOL[precision], f"component {c}: {err:.3e}"
    assert np.abs(np.concatenate([g[2][m] for g, m in zip(got, masks)])).max() == 0.0
    # L_k amplifies phi's own rounding by ~12/h_k^2 (h = 1/32 on the finest level): a phi accurate to
    # ~3e-14 relative gives a residual of ~1e-10 of max|source|; DF32 carries ~100x that
    assert rep.residual_rel < (5e-9 if precision == 0 else 5e-7)


def gpu_heat(L, mesh, f_levels, alpha, precision, table=None, rep=None):
    m = L.Mesh(mesh["levels"], mesh["B"], mesh["h0"], n_ext=mesh["n_ext"])
    f = torch.from_numpy(flat(f_levels)).cuda()
    g = torch.full_like(f, float("nan"))
    L.lgf_heat_apply(table, m, f.shape[0], f.data_ptr(), g.data_ptr(), L.LGF_F64, alpha,
                     L.make_opts(precision=precision), rep)
    torch.cuda.synchronize()
    return split(g.cpu().numpy(), mesh)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (2, 1e-12), (1, 1e-6)])
def test_heat_two_level(L, precision, tol):
    mesh = two_level()
    rng = np.random.default_rng(31)
    f = [rng.standard_normal((2, len(b), 8, 8, 8)) for b in mesh["levels"]]
    ref = amr.fif_amr(mesh, f, 0.1)
    lv = amr.build_levels(mesh)
    masks = [amr._to_blocks(lv[k], mesh["levels"][k], lv[k].omega[None].astype(float), 8)[0] > 0.5
             for k in range(2)]
    rep = L.lgf_report()
    got = gpu_heat(L, mesh, f, 0.1, precision, rep=rep)
    assert rel_err_levels(got, ref, masks) <= tol
    # restriction (2) + coarsening (1) + per level (reconstruction, 3 passes, store)
    assert rep.kernel_launches == 13


def test_heat_single_level_with_table_workspace(L, table8):
    rng = np.random.default_rng(8)
    B = 8
    blk = S.box_blocks((16, 24, 16), B)
    mesh = dict(B=B, h0=1.0, n_ext=4, levels=[blk])
    f = [rng.standard_normal((1, len(blk), B, B, B))]
    ref = amr.fif_amr(mesh, f, 0.37)
    got = gpu_heat(L, mesh, f, 0.37, 0, table=table8)
    assert np.abs(got[0] - ref[0]).max() <= 1e-12 * np.abs(ref[0]).max()


def test_mesh_errors(L, table8):
    mesh = two_level()
    bad = dict(mesh)
    bad["levels"] = [mesh["levels"][0], np.array([[9, 9, 9]], np.int32)]  # not nested
    with pytest.raises(L.LgfError) as e:
        gpu_solve(L, table8, bad, [np.zeros((1, 27, 8, 8, 8)), np.zeros((1, 1, 8, 8, 8))], 0)
    assert e.value.status == L.LGF_E_MESH
    small = L.lgf_table_create(8, (1, 1, 1), L.LGF_TBL_FP64)
    try:
        with pytest.raises(L.LgfError) as e:
            gpu_solve(L, small, mesh, [np.zeros((1, 27, 8, 8, 8)), np.zeros((1, 5, 8, 8, 8))], 0)
        assert e.value.status == L.LGF_E_TABLE_RANGE
    finally:
        L.lgf_table_destroy(small)


def _reblock(mesh16, fields16):
    """The same composite mesh with 8^3 blocks: block (bx, by, bz) of 16^3 cells -> its eight 8^3 sub-blocks;
    fields [ncomp][nblk][16][16][16] -> [ncomp][8 nblk][8][8][8] in the matching order."""
    sub = [(i, j, l) for l in (0, 1) for j in (0, 1) for i in (0, 1)]
    levels8, f8 = [], []
    for blk, f in zip(mesh16["levels"], fields16):
        levels8.append(np.array([[2 * bx + i, 2 * by + j, 2 * bz + l] for bx, by, bz in blk for i, j, l in sub],
                                np.int32))
        out = np.zeros((f.shape[0], 8 * len(blk), 8, 8, 8))
        for n in range(len(blk)):
            for s, (i, j, l) in enumerate(sub):
                out[:, 8 * n + s] = f[:, n, 8 * l:8 * l + 8, 8 * j:8 * j + 8, 8 * i:8 * i + 8]
        f8.append(out)
    return dict(B=8, h0=mesh16["h0"], n_ext=mesh16["n_ext"], levels=levels8), f8


@pytest.mark.parametrize("precision", [0, 2])
def test_results_do_not_depend_on_the_block_size(L, table8, precision):
    # the regions Omega_k, Omega_k^E and the correction are defined on cells (n_ext in cells, whole-cell
    # masks), so re-blocking the same composite mesh from 16^3 into 8^3 blocks changes only rounding
    B = 16
    lvl0 = S.box_blocks((48, 48, 32), B)
    lvl1 = np.array([[2, 2, 1], [3, 2, 1], [2, 3, 1], [3, 3, 1], [2, 2, 2]], np.int32)
    mesh16 = dict(B=B, h0=0.5, n_ext=6, levels=[lvl0, lvl1])
    rng = np.random.default_rng(61)
    f16 = [rng.standard_normal((2, len(b), B, B, B)) for b in mesh16["levels"]]
    mesh8, f8 = _reblock(mesh16, f16)
    t16 = L.lgf_table_create(16, (6, 6, 6), L.LGF_TBL_FP64 | L.LGF_TBL_DF32)
    try:
        got16, _ = gpu_solve(L, t16, mesh16, f16, precision)
    finally:
        L.lgf_table_destroy(t16)
    got8, _ = gpu_solve(L, table8, mesh8, f8, precision)
    _, back = _reblock(mesh16, got16)  # express the B = 16 result in the 8^3 layout
    for k in range(2):
        a, b = back[k], got8[k]
        m = np.isfinite(b)
        assert (np.isfinite(a) == m).all()  # the same cells (Omega_k) written
        scale = np.abs(b[m]).max()
        assert np.abs(a[m] - b[m]).max() <= TOL[precision] * scale, k
